"""Pins for oracle.sphere (paper Sec. 3) against library routines and closed forms."""
import math

import numpy as np
import pytest
from scipy.special import lpmv

from oracle import sphere
from oracle.swe import Consts

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def pbar_scipy(m, n, mu):
    """Orthonormal Pbar_n^m without Condon-Shortley phase, from scipy's lpmv."""
    norm = math.sqrt((2 * n + 1) / 2.0 * math.factorial(n - m) / math.factorial(n + m))
    return (-1) ** m * norm * lpmv(m, n, mu)


@pytest.mark.parametrize("nlat", [8, 96, 512])
def test_gauss_nodes_match_numpy(nlat):
    mu, w = sphere.gauss_legendre(nlat)
    x, wx = np.polynomial.legendre.leggauss(nlat)
    assert np.all(np.diff(mu) < 0)
    np.testing.assert_allclose(mu, x[::-1], rtol=0, atol=2e-15)
    # both weight formulas amplify node rounding by ~nlat^2 near the poles; numpy's
    # are the less accurate ones at large nlat (see the orthonormality test)
    np.testing.assert_allclose(w, wx[::-1], rtol=1e-15 * nlat * nlat, atol=0)
    assert abs(w.sum() - 2.0) < 1e-14


def test_alp_match_scipy():
    mu = np.linspace(-0.99, 0.99, 37)
    N = 20
    for m in range(0, N + 1, 3):
        P, _ = sphere.alp(m, N, mu)
        for n in range(m, N + 1):
            ref = pbar_scipy(m, n, mu)
            np.testing.assert_allclose(P[n - m], ref, rtol=1e-11, atol=1e-13)


def test_H_independent_identity():
    # (1-mu^2) dPbar_n/dmu = -n mu Pbar_n + sqrt((2n+1)(n^2-m^2)/(2n-1)) Pbar_{n-1}  (unnormalised
    # identity (1-x^2) P' = -n x P_n + (n+m) P_{n-1} rescaled), evaluated with scipy values.
    mu = np.linspace(-0.97, 0.97, 29)
    N = 18
    for m in range(0, N + 1, 2):
        _, H = sphere.alp(m, N, mu)
        for n in range(m, N + 1):
            ref = -n * mu * pbar_scipy(m, n, mu)
            if n > m:
                ref = ref + math.sqrt((2 * n + 1) * (n * n - m * m) / (2 * n - 1.0)) * pbar_scipy(m, n - 1, mu)
            np.testing.assert_allclose(H[n - m], ref, rtol=1e-10, atol=1e-12)


def test_H_finite_difference():
    mu = np.linspace(-0.9, 0.9, 11)
    d = 1e-6
    N = 12
    for m in (0, 3, 7):
        _, H = sphere.alp(m, N, mu)
        Pp, _ = sphere.alp(m, N, mu + d)
        Pm, _ = sphere.alp(m, N, mu - d)
        fd = (1 - mu ** 2) * (Pp - Pm) / (2 * d)
        np.testing.assert_allclose(H, fd, rtol=0, atol=1e-7)


@pytest.mark.parametrize("N,nlat", [(31, 48), (341, 512)])
def test_quadrature_orthonormality(N, nlat):
    mu, w = sphere.gauss_legendre(nlat)
    for m in (0, 1, 5, 17, 31, N // 2, N):
        P, _ = sphere.alp(m, N, mu)
        G = (P * w) @ P.T
        np.testing.assert_allclose(G, np.eye(N - m + 1), atol=1e-16 * nlat)


def _rand_spec(N, rng, zero_n0=False):
    n, m = [], []
    for mm in range(N + 1):
        for nn in range(mm, N + 1):
            n.append(nn)
            m.append(mm)
    n, m = np.array(n), np.array(m)
    x = rng.standard_normal(n.size) + 1j * rng.standard_normal(n.size)
    x[m == 0] = x[m == 0].real
    if zero_n0:
        x[n == 0] = 0
    return x


def test_scalar_round_trip():
    N, nlat, nlon = 21, 33, 64
    g = sphere.Grid(N, nlat, nlon)
    x = _rand_spec(N, np.random.default_rng(1))
    np.testing.assert_allclose(g.analysis(g.synthesis(x)), x, atol=1e-13)


def test_vector_round_trip():
    N, nlat, nlon = 21, 33, 64
    g = sphere.Grid(N, nlat, nlon)
    rng = np.random.default_rng(2)
    z = _rand_spec(N, rng, zero_n0=True) * 1e-5
    d = _rand_spec(N, rng, zero_n0=True) * 1e-5
    U, V = g.vortdiv_to_uv(z, d, 6.37e6)
    z2, d2 = g.uv_to_vortdiv(U, V, 6.37e6)
    np.testing.assert_allclose(z2, z, atol=1e-18)
    np.testing.assert_allclose(d2, d, atol=1e-18)


def test_solid_body_rotation_closed_form():
    # u = u0 cos(phi), v = 0  ->  zeta = 2 u0 sin(phi) / a, delta = 0
    N, nlat, nlon = 15, 24, 48
    a, u0 = 6.37122e6, 20.0
    g = sphere.Grid(N, nlat, nlon)
    U = u0 * (1 - g.mu ** 2)[:, None] * np.ones((1, nlon))
    z, d = g.uv_to_vortdiv(U, np.zeros_like(U), a)
    ref = np.zeros_like(z)
    ref[sphere.idx(0, 1, N)] = 2 * u0 / a * math.sqrt(2.0 / 3.0)
    tol = 1e-14 * np.abs(ref).max()
    np.testing.assert_allclose(z, ref, atol=tol)
    np.testing.assert_allclose(d, 0, atol=tol)


def test_balanced_state_closed_form_matches_synthesis():
    from paper_1812_03431_gb300 import inputs
    N, nlat, nlon = 31, 48, 96
    c = Consts()
    g = sphere.Grid(N, nlat, nlon)
    S = inputs.balanced_zonal_flow(N)
    ref = inputs.balanced_grid(g.mu, nlon)
    Phi = g.synthesis(S[0])
    np.testing.assert_allclose(Phi / c.gravity, ref[0], rtol=0, atol=1e-9)
    U, V = g.vortdiv_to_uv(S[1], S[2], c.radius)
    np.testing.assert_allclose(U / g.coslat[:, None], ref[1], atol=1e-11)
    np.testing.assert_allclose(V, 0, atol=1e-12)
