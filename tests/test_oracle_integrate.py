"""Pins of the reference integrators (oracle/integrate.py) used by the Gaussian-bump study."""
import numpy as np
import pytest

from oracle import integrate
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.sphere import idx, nspec
from oracle.swe import Consts, operator_m
from paper_1812_03431_gb300 import inputs

C = Consts()


def test_exact_fsphere_single_degree_closed_form():
    # f-sphere (constant f = 2 Omega): one degree n is a closed 3x3 system.  From
    # Phi(0) = Phi0, zeta(0) = delta(0) = 0, with G = n(n+1)/a^2, w^2 = f^2 + Phibar G:
    #   Phi = Phi0 (1 - Phibar G (1 - cos wt) / w^2), zeta = -f G Phi0 (1 - cos wt) / w^2,
    #   delta = G Phi0 sin(wt) / w
    N, m, n, t = 12, 3, 7, 5000.0
    f, G = 2 * C.omega, n * (n + 1) / C.radius ** 2
    w = np.sqrt(f * f + C.phibar * G)
    p0 = 1.0e3 * (0.6 - 0.8j)
    U = np.zeros((3, nspec(N)), complex)
    U[0, idx(m, n, N)] = p0
    got = integrate.exact(U, N, t, C, fsphere=True)
    i = idx(m, n, N)
    ref = [p0 * (1 - C.phibar * G * (1 - np.cos(w * t)) / w ** 2), -f * G * p0 * (1 - np.cos(w * t)) / w ** 2,
           G * p0 * np.sin(w * t) / w]
    np.testing.assert_allclose(got[:, i], ref, rtol=1e-12, atol=1e-12 * abs(p0) * G / w)
    rest = np.ones(got.shape, bool)
    rest[:, i] = False
    assert np.all(got[rest] == 0)


def test_exact_keeps_geostrophic_state_and_energy():
    N = 31
    U = inputs.balanced_zonal_flow(N)
    V = integrate.exact(U, N, 1.5 * 86400.0, C)
    assert np.linalg.norm(V - U) < 1e-12 * np.linalg.norm(U)
    R = inputs.random_spectral(N, 2, 11)
    e0 = integrate.energy(R, N, C)
    e1 = integrate.energy(integrate.exact(R, N, 1.5 * 86400.0, C), N, C)
    np.testing.assert_allclose(e1, e0, rtol=1e-13)


def test_exact_matches_matrix_exponential():
    # exp(tL) = W^(-1/2) exp(tS) W^(1/2) with S = W^(1/2) L W^(-1/2) is exact algebra; scipy's
    # expm of the well-scaled S (|tS| ~ 5, while |tL| ~ 3e8) gives the reference
    import scipy.linalg
    N, t = 17, 3000.0
    U = inputs.random_spectral(N, 1, 12)[0]
    got = integrate.exact(U, N, t, C)
    for m in (0, 1, 9, 17):
        rows = integrate._rows(m, N)
        sw = np.sqrt(integrate.energy_weights(m, N, C))
        S = sw[:, None] * operator_m(m, N, C) / sw[None, :]
        ref = (scipy.linalg.expm(t * S) @ (sw * U.reshape(-1)[rows])) / sw
        g = got.reshape(-1)[rows]
        # compare in the energy norm, where both are well conditioned
        assert np.linalg.norm(sw * (g - ref)) < 1e-12 * np.linalg.norm(sw * ref)
        # and the unscaled exponential agrees to its own conditioning
        ref2 = scipy.linalg.expm(t * operator_m(m, N, C)) @ U.reshape(-1)[rows]
        assert np.linalg.norm(sw * (g - ref2)) < 1e-8 * np.linalg.norm(sw * ref2)


def test_sparse_operator_matches_blocks():
    N = 9
    L = integrate.sparse_operator(N, C).toarray()
    for m in (0, 4, 9):
        rows = integrate._rows(m, N)
        np.testing.assert_array_equal(L[np.ix_(rows, rows)], operator_m(m, N, C))
    # nothing couples different orders
    blocks = np.zeros_like(L, dtype=bool)
    for m in range(N + 1):
        rows = integrate._rows(m, N)
        blocks[np.ix_(rows, rows)] = True
    assert np.all(L[~blocks] == 0)


def test_rk4_energy_decay_per_mode_closed_form():
    # on an eigenvector (L v = i w v) one RK4 step multiplies by R(i w dt) with
    # |R(iy)|^2 = 1 - y^6/72 + y^8/576, so energy decays by that factor per step
    N, m, n, dt, K = 48, 5, 40, 300.0, 20
    A = operator_m(m, N, C, fsphere=True)
    i = n - m
    blk = A[3 * i:3 * i + 3, 3 * i:3 * i + 3]
    lam, vec = np.linalg.eig(blk)
    j = int(np.argmax(lam.imag))
    w = np.sqrt((2 * C.omega) ** 2 + C.phibar * n * (n + 1) / C.radius ** 2)
    assert abs(lam[j].imag - w) < 1e-12 * w
    U = np.zeros((3, nspec(N)), complex)
    U[:, idx(m, n, N)] = vec[:, j] * 1e3
    y = w * dt
    amp2 = 1 - y ** 6 / 72 + y ** 8 / 576
    e0 = integrate.energy(U, N, C)
    e1 = integrate.energy(integrate.rk4(U, N, dt, K, C, fsphere=True), N, C)
    np.testing.assert_allclose(e1 / e0, amp2 ** K, rtol=1e-10)
    assert e1 / e0 < 0.99  # the decay is visible at this step


def test_rk4_is_fourth_order():
    N, t = 21, 7200.0
    U = inputs.random_spectral(N, 1, 3)
    ref = integrate.exact(U, N, t, C)
    errs = [np.linalg.norm(integrate.rk4(U, N, t / k, k, C) - ref) for k in (8, 16)]
    assert 14.0 < errs[0] / errs[1] < 18.0


def test_rexi_modal_is_the_shifted_solve_step():
    N, M, tau = 21, 64, 3600.0
    al, be, _ = rc.rexi_coefficients(M, 0.2)
    U = inputs.random_spectral(N, 2, 13)
    ref = ostep.rexi_step_spectral(U, N, al, be, tau, C)
    got = integrate.rexi_modal(U, N, al, be, tau, 1, C)
    for f in range(3):
        assert np.linalg.norm(got[:, f] - ref[:, f]) < 1e-12 * np.linalg.norm(ref[:, f])
    # two steps are the step applied twice
    ref2 = ostep.rexi_step_spectral(ref, N, al, be, tau, C)
    got2 = integrate.rexi_modal(U, N, al, be, tau, 2, C)
    assert np.linalg.norm(got2 - ref2) < 1e-12 * np.linalg.norm(ref2)


def test_rexi_modal_converges_to_exact():
    # within the covered range |tau omega| < h M the response is e^{i tau omega} up to the
    # approximation error, so K steps approach exp(K tau L)
    N, tau, K = 21, 1800.0, 4
    U = inputs.random_spectral(N, 1, 14)
    ref = integrate.exact(U, N, K * tau, C)
    errs = []
    for M in (64, 1024):
        al, be, _ = rc.rexi_coefficients(M, 0.2)
        errs.append(np.linalg.norm(integrate.rexi_modal(U, N, al, be, tau, K, C) - ref) / np.linalg.norm(ref))
    assert errs[1] < 1e-4 and errs[1] < 0.1 * errs[0]
