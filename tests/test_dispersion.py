"""Dispersion analysis (Sec. 6.3) with the oracle step: pins the probing and the
eigenvalue bookkeeping on the CPU.

The propagator of U <- Re sum_k beta_k (alpha_k + tau L)^{-1} U is f(tau L) with the
scalar REXI response f; so its eigenvalues are f(tau omega) on the exact frequencies
omega of L, computed here independently from the dense operator.
"""
import numpy as np
import pytest

from dispersion_util import exact_frequencies, fsphere_frequencies
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts
from paper_1812_03431_gb300 import dispersion

C = Consts()


@pytest.fixture(scope="module")
def case():
    N, M, h, dt = 6, 64, 0.2, 400.0
    al, be, _ = rc.rexi_coefficients(M, h)
    out = ostep.rexi_step_spectral(dispersion.probe_states(N), N, al, be, dt, C)
    om, re_max = exact_frequencies(N, C)
    return dict(N=N, M=M, h=h, dt=dt, al=al, be=be, E=dispersion.assemble(out, N), om=om, re_max=re_max)


def test_coordinates_count():
    for N in (1, 6, 16):
        K = (N + 1) * (N + 2) // 2
        # 3 fields of K complex coefficients, m = 0 ones real, minus zeta_0^0 and delta_0^0
        assert len(dispersion.real_coordinates(N)) == 3 * (2 * K - (N + 1)) - 2


def test_L_is_neutral_with_zero_modes(case):
    # Eq. (1) linearised about rest conserves energy: no growth or decay
    assert case["re_max"] < 1e-12 * np.abs(case["om"]).max()
    # the m = 0 geostrophic modes are steady: one per zonal degree n >= 1 plus Phi_0^0
    assert np.sum(np.abs(case["om"]) < 1e-12 * np.abs(case["om"]).max()) == case["N"] + 1


def test_propagator_is_the_rexi_symbol(case):
    lam = dispersion.eigenvalues_by_phase(case["E"])
    pred = rc.response(case["al"], case["be"], case["dt"] * case["om"])
    pred = pred[np.argsort(np.angle(pred), kind="stable")]
    assert np.abs(lam - pred).max() < 1e-12


def test_phase_error_is_flat_and_bounded(case):
    w, amp = dispersion.dispersion_relation(case["E"], case["dt"])
    we, rel = dispersion.relative_phase_error(w, case["om"])
    # the relative error of the numerical frequency does not grow with the frequency
    # (Sec. 6.3): it stays at the symbol's slope error near zero
    assert np.ptp(rel) < 0.1 * np.abs(rel).max()
    assert np.abs(rel).max() <= rc.imag_tail_bound(1.0, case["M"], case["h"])
    # Re f = cos to fit accuracy, so |f|^2 - 1 = Im(f)^2 - sin^2: the amplitude error of a
    # mode is at most about rel * sin^2(omega dt), i.e. vanishes for the slow modes
    s2 = np.sin(np.sort(case["om"]) * case["dt"]) ** 2
    assert np.all(np.abs(amp - 1.0) <= 1.1 * np.abs(rel).max() * s2 + 1e-11)


def test_fsphere_propagator_matches_closed_form_frequencies():
    # on the f-sphere the frequencies are known in closed form (Sec. 4, Sec. 6.3)
    N, M, dt = 6, 64, 400.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    om = fsphere_frequencies(N, C)
    om_dense, _ = exact_frequencies(N, C, fsphere=True)
    np.testing.assert_allclose(np.sort(om_dense), np.sort(om), rtol=0, atol=1e-12 * om.max())
    out = ostep.rexi_step_spectral(dispersion.probe_states(N), N, al, be, dt, C, fsphere=True)
    lam = dispersion.eigenvalues_by_phase(dispersion.assemble(out, N))
    pred = rc.response(al, be, dt * om)
    pred = pred[np.argsort(np.angle(pred), kind="stable")]
    assert np.abs(lam - pred).max() < 1e-12
