"""Pins for oracle.swe and oracle.step (Eq. (1), Sec. 4.2-4.3, Algorithm 1, Sec. 6.1)."""
import math

import numpy as np
import pytest
from scipy.linalg import expm
from scipy.special import lpmv

from oracle import rexi_coeffs as rc
from oracle import sphere, swe
from oracle.step import GridStep, rexi_step_spectral
from paper_1812_03431_gb300 import inputs

C = swe.Consts()


def pbar(m, n, mu):
    norm = math.sqrt((2 * n + 1) / 2.0 * math.factorial(n - m) / math.factorial(n + m))
    return (-1) ** m * norm * lpmv(m, n, mu)


def hbar(m, n, mu):
    out = -n * mu * pbar(m, n, mu)
    if n > m:
        out = out + math.sqrt((2 * n + 1) * (n * n - m * m) / (2 * n - 1.0)) * pbar(m, n - 1, mu)
    return out


def rand_state(N, rng, batch=()):
    n, m = inputs.degree_order(N)
    S = rng.standard_normal(batch + (3, n.size)) + 1j * rng.standard_normal(batch + (3, n.size))
    S[..., m == 0] = S[..., m == 0].real
    S[..., 1:, 0] = 0.0  # zeta_0^0 = delta_0^0 = 0
    scale = np.array([C.phibar, 1e-5, 1e-5])[:, None]
    return S * scale


def test_operator_matches_grid_evaluation():
    """L from the spectral derivation == Eq. (1) evaluated pointwise on a grid and projected."""
    N, nlat, nlon = 7, 12, 32
    a, om = C.radius, C.omega
    S = rand_state(N, np.random.default_rng(5))
    x, w = np.polynomial.legendre.leggauss(nlat)
    mu = x[:, None]
    lam = 2 * np.pi * np.arange(nlon)[None, :] / nlon
    cosl = np.sqrt(1 - mu * mu)
    fld = {k: np.zeros((nlat, nlon)) for k in ("Phi", "zeta", "delta", "U", "V", "lapPhi")}
    for mm in range(N + 1):
        cm = 1.0 if mm == 0 else 2.0
        for n in range(mm, N + 1):
            k = sphere.idx(mm, n, N)
            e = np.exp(1j * mm * lam)
            Y = pbar(mm, n, mu) * e
            HY = hbar(mm, n, mu) * e  # (1-mu^2) d/dmu of Y
            Phi, zeta, delta = S[:, k]
            psi = -a * a * zeta / (n * (n + 1)) if n > 0 else 0.0
            chi = -a * a * delta / (n * (n + 1)) if n > 0 else 0.0
            fld["Phi"] += cm * np.real(Phi * Y)
            fld["zeta"] += cm * np.real(zeta * Y)
            fld["delta"] += cm * np.real(delta * Y)
            fld["lapPhi"] += cm * np.real(-n * (n + 1) / a ** 2 * Phi * Y)
            # U = u cos(phi) = -(1/a)(1-mu^2) dpsi/dmu + (1/a) dchi/dlambda
            fld["U"] += cm * np.real((-psi * HY + 1j * mm * chi * Y) / a)
            # V = v cos(phi) = (1/a) dpsi/dlambda + (1/a)(1-mu^2) dchi/dmu
            fld["V"] += cm * np.real((1j * mm * psi * Y + chi * HY) / a)
    f = 2 * om * mu
    zeta_t = -f * fld["delta"] - (2 * om / a) * fld["V"]           # -f delta - V.grad f
    delta_t = f * fld["zeta"] - (2 * om / a) * fld["U"] - fld["lapPhi"]  # f zeta + k.(grad f x V) - lap Phi
    Phi_t = -C.phibar * fld["delta"]
    ref = np.zeros_like(S)
    for i, F in enumerate((Phi_t, zeta_t, delta_t)):
        Fm = np.fft.rfft(F, axis=1) / nlon
        for mm in range(N + 1):
            for n in range(mm, N + 1):
                ref[i, sphere.idx(mm, n, N)] = np.sum(w * pbar(mm, n, x) * Fm[:, mm])
    ref[1:, 0] = 0
    got = swe.apply_L(S, N, C)
    for i in range(3):
        np.testing.assert_allclose(got[i], ref[i], rtol=0, atol=1e-12 * np.abs(ref[i]).max())


def test_energy_weighted_operator_is_anti_hermitian():
    # the linear SWE conserve int (Phi'^2 + Phibar |V|^2)/2, so L is anti-Hermitian in that norm
    N = 12
    L = swe.dense_operator(N, C)
    n, m = inputs.degree_order(N)
    wz = np.where(n > 0, C.radius * np.sqrt(C.phibar / np.maximum(n * (n + 1), 1)), 1.0)
    d = np.concatenate([np.ones(n.size), wz, wz])
    A = d[:, None] * L / d[None, :]
    assert np.abs(A + A.conj().T).max() < 1e-13 * np.abs(A).max()


def test_geostrophic_balance_is_steady():
    # Sec. 6.1: the balanced zonal flow has zero time derivative; a normalised REXI step
    # keeps it to O(1e-12).
    N = 63
    U = inputs.balanced_zonal_flow(N)
    LU = swe.apply_L(U, N, C)
    Uz = U.copy()
    Uz[0] = 0
    scale = np.abs(swe.apply_L(Uz, N, C)).max()
    assert np.abs(LU).max() < 1e-13 * scale
    al, be, _ = rc.rexi_coefficients(128, 0.2)
    out = rexi_step_spectral(U, N, al, be, 3600.0, C)
    assert np.linalg.norm(out - U) / np.linalg.norm(U) < 1e-12


def test_grid_layout_round_trip_and_balance():
    N, nlat, nlon = 31, 48, 96
    al, be, _ = rc.rexi_coefficients(16, 0.2)
    gs = GridStep(N, nlat, nlon, al, be, 600.0, C)
    S = inputs.balanced_zonal_flow(N)
    x = inputs.balanced_grid(gs.g.mu, nlon)
    A = gs.analyse(x)
    for i in range(3):
        assert np.abs(A[i] - S[i]).max() <= 1e-13 * np.abs(S).max(axis=1)[i] + 1e-30
    y = gs(x)
    assert np.abs(y - x).max() < 1e-13 * np.abs(x).max()
    R = rand_state(N, np.random.default_rng(3))
    R2 = gs.analyse(gs.synthesise(R))
    for i in range(3):
        assert np.abs(R2[i] - R[i]).max() <= 1e-13 * np.abs(R[i]).max()


def _dense_rexi(S, N, al, be, tau):
    L = swe.dense_operator(N, C)
    u = S.reshape(-1)
    I = np.eye(L.shape[0])
    out = sum(b * np.linalg.solve(a * I + tau * L, u) for a, b in zip(al, be))
    out = out.reshape(S.shape)
    out[:, : N + 1] = out[:, : N + 1].real
    out[1:, 0] = 0
    return out


def test_banded_equals_dense_solve():
    N, tau = 8, 3600.0
    al, be, _ = rc.rexi_coefficients(16, 0.2)
    S = rand_state(N, np.random.default_rng(7))
    got = rexi_step_spectral(S, N, al, be, tau, C)
    ref = _dense_rexi(S, N, al, be, tau)
    for i in range(3):
        np.testing.assert_allclose(got[i], ref[i], rtol=0, atol=1e-13 * np.abs(ref[i]).max())


def _eigen(N):
    L = swe.dense_operator(N, C)
    n, m = inputs.degree_order(N)
    wz = np.where(n > 0, C.radius * np.sqrt(C.phibar / np.maximum(n * (n + 1), 1)), 1.0)
    d = np.concatenate([np.ones(n.size), wz, wz])
    A = d[:, None] * L / d[None, :]
    om, Q = np.linalg.eigh(1j * A)  # A = -i H, eigenvalues of L are -i om
    return d, -om, Q


def test_step_equals_rational_function_of_eigenvalues():
    N, tau = 10, 3600.0
    al, be, _ = rc.rexi_coefficients(64, 0.2)
    S = rand_state(N, np.random.default_rng(11))
    d, om, Q = _eigen(N)
    fx = rc.response(al, be, tau * om)
    ref = (Q @ (fx * (Q.conj().T @ (d * S.reshape(-1))))) / d
    ref = ref.reshape(S.shape)
    ref[:, : N + 1] = ref[:, : N + 1].real
    ref[1:, 0] = 0
    got = rexi_step_spectral(S, N, al, be, tau, C)
    for i in range(3):
        np.testing.assert_allclose(got[i], ref[i], rtol=0, atol=1e-12 * np.abs(ref[i]).max())


def test_step_approximates_exponential_within_scalar_error():
    N, tau = 10, 3600.0
    M, h = 128, 0.2
    al, be, _ = rc.rexi_coefficients(M, h)
    S = rand_state(N, np.random.default_rng(13))
    d, om, Q = _eigen(N)
    x = tau * om
    assert np.abs(x).max() < h * M / 2
    scal = np.abs(rc.response(al, be, x) - np.exp(1j * x)).max()
    bound = np.abs(rc.response(al, be, x).real - np.cos(x)).max() + rc.imag_tail_bound(np.abs(x).max(), M, h)
    assert scal <= bound + 1e-10
    L = swe.dense_operator(N, C)
    ref = expm(tau * L) @ S.reshape(-1)
    got = rexi_step_spectral(S, N, al, be, tau, C).reshape(-1)
    # energy norm: Q is unitary there
    err = np.linalg.norm(d * (got - ref)) / np.linalg.norm(d * S.reshape(-1))
    assert err <= 1.01 * scal + 1e-12


def test_fsphere_closed_form_projectors():
    # f-sphere (constant f, Sec. 4.3): per (m, n) a 3x3 block with eigenvalues 0, +-i w,
    # w = sqrt(f^2 + Phibar n(n+1)/a^2).  f(tau L) = sum_k f(lambda_k) Pi_k with the
    # Lagrange projectors Pi_k = prod_{j != k} (A - lambda_j)/(lambda_k - lambda_j).
    N, tau, f0 = 9, 1800.0, 2 * C.omega
    al, be, _ = rc.rexi_coefficients(64, 0.2)
    S = rand_state(N, np.random.default_rng(17))
    ref = np.zeros_like(S)
    for mm in range(N + 1):
        for n in range(max(mm, 1), N + 1):
            k = sphere.idx(mm, n, N)
            G = n * (n + 1) / C.radius ** 2
            A = np.array([[0, 0, -C.phibar], [0, 0, -f0], [G, f0, 0]], dtype=complex)
            w = math.sqrt(f0 * f0 + C.phibar * G)
            lams = [0.0, 1j * w, -1j * w]
            acc = np.zeros((3, 3), dtype=complex)
            for i, lk in enumerate(lams):
                Pi = np.eye(3, dtype=complex)
                for j, lj in enumerate(lams):
                    if j != i:
                        Pi = Pi @ (A - lj * np.eye(3)) / (lk - lj)
                acc += rc.response(al, be, np.array([tau * lk.imag if isinstance(lk, complex) else 0.0]))[0] * Pi
            ref[:, k] = acc @ S[:, k]
        if mm == 0:
            ref[0, 0] = np.sum(be / al) * S[0, 0]
    ref[:, : N + 1] = ref[:, : N + 1].real
    out = rexi_step_spectral(S, N, al, be, tau, C, fsphere=True)
    for i in range(3):
        np.testing.assert_allclose(out[i], ref[i], rtol=0, atol=1e-12 * np.abs(ref[i]).max())


def test_adjoint_dot_product_spectral():
    N, tau = 16, 3600.0
    al, be, _ = rc.rexi_coefficients(32, 0.2)
    rng = np.random.default_rng(19)
    x = rand_state(N, rng)
    y = rand_state(N, rng)
    Gx = rexi_step_spectral(x, N, al, be, tau, C)
    GTy = rexi_step_spectral(y, N, al, be, tau, C, adjoint=True)
    lhs = np.real(np.vdot(y, Gx))
    rhs = np.real(np.vdot(GTy, x))
    assert abs(lhs - rhs) < 1e-13 * np.linalg.norm(y) * np.linalg.norm(Gx)


def test_adjoint_dot_product_grid():
    N, nlat, nlon = 21, 32, 64
    al, be, _ = rc.rexi_coefficients(32, 0.2)
    gs = GridStep(N, nlat, nlon, al, be, 3600.0, C)
    rng = np.random.default_rng(23)
    x = inputs.random_grid(2, nlat, nlon, 1)
    y = inputs.random_grid(2, nlat, nlon, 2)
    lhs = np.sum(y * gs(x))
    rhs = np.sum(gs.adjoint(y) * x)
    assert abs(lhs - rhs) < 1e-12 * np.sqrt(np.sum(y * y) * np.sum(gs(x) ** 2))


def test_adjoint_equals_dense_jacobian_transpose():
    N, nlat, nlon = 4, 8, 16
    al, be, _ = rc.rexi_coefficients(8, 0.2)
    gs = GridStep(N, nlat, nlon, al, be, 3600.0, C)
    n = 3 * nlat * nlon
    E = np.eye(n).reshape(n, 3, nlat, nlon)
    J = gs(E).reshape(n, n).T  # column k = step(e_k)
    y = inputs.random_grid(1, nlat, nlon, 3)[0]
    np.testing.assert_allclose(gs.adjoint(y).reshape(-1), J.T @ y.reshape(-1), rtol=0,
                               atol=1e-12 * np.abs(J.T @ y.reshape(-1)).max())
