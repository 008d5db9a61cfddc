"""Dispersion analysis by column probing (Sec. 6.3) through the C-ABI at T16, dt = 400 s.

All 865 real coordinates are stepped as one batch; the eigenvalues of the assembled
propagator must be the REXI response f(dt omega) on the exact frequencies of L.
"""
import numpy as np
import pytest

from dispersion_util import exact_frequencies, fsphere_frequencies
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.swe import Consts

pytestmark = pytest.mark.gpu
C = Consts()


@pytest.mark.parametrize("M", [64, 256])
def test_propagator_eigenvalues_are_the_rexi_symbol(M):
    from paper_1812_03431_gb300 import dispersion, rexi
    N, dt, h = 16, 400.0, 0.2
    al, be, _ = rc.rexi_coefficients(M, h)
    n = len(dispersion.real_coordinates(N))
    plan = rexi.Plan(N, 18, 36, tau=dt, max_batch=n, layout="spectral", alpha=al, beta=be)
    E = dispersion.propagator(plan, N)
    plan.close()
    # the whole propagator against the oracle's, column by column
    ref = dispersion.assemble(ostep.rexi_step_spectral(dispersion.probe_states(N), N, al, be, dt, C), N)
    # columns mix units (Phi in m^2/s^2, zeta and delta in 1/s), so compare column by column
    colerr = np.linalg.norm(E - ref, axis=0) / np.linalg.norm(ref, axis=0)
    assert colerr.max() < 1e-12
    om, _ = exact_frequencies(N, C)
    lam = dispersion.eigenvalues_by_phase(E)
    pred = rc.response(al, be, dt * om)
    pred = pred[np.argsort(np.angle(pred), kind="stable")]
    assert np.abs(lam - pred).max() < 1e-11
    w, amp = dispersion.dispersion_relation(E, dt)
    we, rel = dispersion.relative_phase_error(w, om)
    assert np.abs(rel).max() <= rc.imag_tail_bound(1.0, M, h)
    assert np.ptp(rel) < 0.1 * np.abs(rel).max()  # flat across the spectrum (within 10 %)


def test_fsphere_dispersion_closed_form():
    """The paper's eigenvalue study runs on the f-sphere, where the frequencies are known
    in closed form: the propagator's eigenvalues are f(dt omega) on them."""
    from paper_1812_03431_gb300 import dispersion, rexi
    N, dt, M = 16, 400.0, 128
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    n = len(dispersion.real_coordinates(N))
    plan = rexi.Plan(N, 18, 36, tau=dt, max_batch=n, layout="spectral", alpha=al, beta=be, fsphere=True)
    E = dispersion.propagator(plan, N)
    plan.close()
    om = fsphere_frequencies(N, C)
    lam = dispersion.eigenvalues_by_phase(E)
    pred = rc.response(al, be, dt * om)
    pred = pred[np.argsort(np.angle(pred), kind="stable")]
    assert np.abs(lam - pred).max() < 1e-11
    w, _ = dispersion.dispersion_relation(E, dt)
    _, rel = dispersion.relative_phase_error(w, om)
    assert np.abs(rel).max() <= rc.imag_tail_bound(1.0, M, 0.2)
