"""Pins of the paper's geopotential-only solver (oracle/phi_solver.py, Sec. 4.3 and 5)."""
import numpy as np
import pytest

from oracle import phi_solver
from oracle import rexi_coeffs as rc
from oracle import step as ostep
from oracle.sphere import gauss_legendre, idx
from oracle.swe import Consts
from paper_1812_03431_gb300 import inputs

C = Consts()


def relerr(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def embed(S, L, N):
    out = np.zeros(S.shape[:-1] + ((N + 1) * (N + 2) // 2,), complex)
    for m in range(L + 1):
        for n in range(m, L + 1):
            out[..., idx(m, n, N)] = S[..., idx(m, n, L)]
    return out


def restrict(S, N, L):
    out = np.zeros(S.shape[:-1] + ((L + 1) * (L + 2) // 2,), complex)
    for m in range(L + 1):
        for n in range(m, L + 1):
            out[..., idx(m, n, L)] = S[..., idx(m, n, N)]
    return out


@pytest.mark.parametrize("recover", ["physical", "spectral"])
@pytest.mark.parametrize("consts,fsphere", [(C, True), (Consts(omega=0.0), False)])
def test_equals_delta_elimination_where_truncation_does_not_act(consts, fsphere, recover):
    # constant f (f-sphere) or no rotation: D is a constant, multiplying through by it
    # commutes with truncation, and both solvers solve the same truncated system
    N, tau = 21, 3600.0
    al, be, _ = rc.rexi_coefficients(16, 0.2)
    S = inputs.random_spectral(N, 2, 3)
    a = phi_solver.rexi_step_phi(S, N, 32, al, be, tau, consts, fsphere=fsphere, recover=recover)
    b = ostep.rexi_step_spectral(S, N, al, be, tau, consts, fsphere=fsphere)
    for f in range(3):
        assert relerr(a[:, f], b[:, f]) < 1e-12


@pytest.mark.parametrize("recover", ["physical", "spectral"])
def test_agrees_in_low_degrees_on_the_rotating_sphere(recover):
    # a band-limited state (n <= 10): both discretisations converge to the same solution,
    # so the degrees n <= 10 agree once N is large enough.  A sign slip in any of the
    # grad f terms would leave an O(1) difference here.
    L, N, tau = 10, 21, 3600.0
    al, be, _ = rc.rexi_coefficients(16, 0.2)
    S = embed(inputs.random_spectral(L, 1, 5), L, N)
    a = restrict(phi_solver.rexi_step_phi(S, N, 30, al, be, tau, C, recover=recover), N, L)
    b = restrict(ostep.rexi_step_spectral(S, N, al, be, tau, C), N, L)
    assert relerr(a, b) < 1e-13
    # and with full-spectrum input they differ at the truncation edge only
    R = inputs.random_spectral(N, 1, 6)
    a = phi_solver.rexi_step_phi(R, N, 30, al, be, tau, C, recover=recover)
    b = ostep.rexi_step_spectral(R, N, al, be, tau, C)
    d = relerr(a, b)
    assert 1e-9 < d < 1e-3
    low = relerr(restrict(a, N, 10), restrict(b, N, 10))
    assert low < 0.1 * d


def test_matrix_is_banded_and_exactly_projected():
    # the multiplied-through operator has coefficients up to mu^4: degrees couple at
    # offsets 0, +-2, +-4 only; the quadrature is exact once nlat >= N + 3
    N, m, tau = 24, 3, 3600.0
    al, _, _ = rc.rexi_coefficients(16, 0.2)
    K = N - m + 1
    U_m = np.zeros((3, K), complex)
    mats = []
    for nlat in (28, 60):
        mu, w = gauss_legendre(nlat)
        Bm, _, _ = phi_solver.phi_matrix_and_rhs(m, N, mu, w, al[10], tau, C, U_m)
        mats.append(Bm)
    np.testing.assert_allclose(mats[0], mats[1], rtol=0, atol=1e-13 * np.abs(mats[1]).max())
    i, j = np.indices((K, K))
    outside = (np.abs(i - j) > 4) | ((i - j) % 2 == 1)
    assert np.abs(mats[1][outside]).max() < 1e-13 * np.abs(mats[1]).max()
    assert np.abs(np.diag(mats[1], 4)).min() > 0  # the mu^4 coupling is really there
