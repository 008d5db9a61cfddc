"""One T-REXI time step (paper Sec. 4.2 and Algorithm 1) and its adjoint -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

    U(t + tau) ~ Re sum_n beta_n (alpha_n + tau L)^{-1} U(t)

(the operator at the start of Sec. 4.3 is alpha I + L with the step scaled to
one; here tau is kept explicit).  L is block-diagonal in the zonal order m, so
every (pole, m) pair is an independent banded system in the degree n; each is
solved here with LAPACK's banded LU with partial pivoting on the full
interleaved (Phi, zeta, delta) unknowns (``scipy.linalg.solve_banded``), and
the beta-weighted sum runs over the poles in ascending n.  A real state is
stored as m >= 0 coefficients; with the conjugate-symmetric pole set the
m >= 0 sum is the real-field result, and the paper's Re(.) becomes "take the
real part of the m = 0 coefficients".

Grid layout (h', u, v on the Gaussian grid) wraps the spectral step in the
forward and inverse transforms of ``oracle.sphere``:  Phi = g h',
U = u cos(phi), V = v cos(phi) -> (Phi, zeta, delta) -> step -> back.

The adjoint is the transpose of this real-linear map for the Euclidean inner
products (sum x y on the grid, Re sum conj(x) y on coefficients):
G^T = sum_n conj(beta_n) (conj(alpha_n) + tau L^H)^{-1} per m, and the
transforms are transposed stage by stage.

Pins: dense numpy.linalg.solve of the same sum; Q f(tau Lambda) Q^{-1} from the
dense eigendecomposition; geostrophic steady state; dot-product and dense
Jacobian-transpose checks of the adjoint.
"""

import numpy as np
from scipy.linalg import solve_banded

from .sphere import Grid, idx, nspec
from .swe import Consts, deinterleave, interleave, operator_m

_BW = 4  # lower = upper bandwidth of (alpha + tau L_m) in interleaved order


def _to_banded(A, l=_BW, u=_BW):
    n = A.shape[0]
    ab = np.zeros((l + u + 1, n), dtype=np.complex128)
    for d in range(-l, u + 1):
        if abs(d) >= n:
            continue
        diag = np.diagonal(A, offset=d)
        if d >= 0:
            ab[u - d, d:] = diag
        else:
            ab[u - d, : n + d] = diag
    return ab


def _state_mask(m, N):
    """1 for unknowns that are part of the state, 0 for zeta_0^0 / delta_0^0."""
    K = N - m + 1
    mask = np.ones(3 * K)
    if m == 0:
        mask[1] = mask[2] = 0.0
    return mask


def _check_band(A):
    n = A.shape[0]
    i, j = np.nonzero(A)
    assert np.all(np.abs(i - j) <= _BW), "operator wider than the assumed band"
    return n


def rexi_step_spectral(U, N, alpha, beta, tau, c=Consts(), adjoint=False, ms=None, real_m0=True,
                       fsphere=False):
    """Apply sum_n beta_n (alpha_n + tau L)^{-1} to spectral states.

    U: [..., 3, nspec] complex (Phi, zeta, delta).  With ``adjoint`` the
    transposed map sum_n conj(beta_n) (conj(alpha_n) + tau L^H)^{-1} is applied.
    ``ms`` restricts the work to a subset of zonal orders (other m left zero).
    ``real_m0=False`` keeps the m = 0 result complex (a single pole is not a
    conjugate-symmetric set, so its m = 0 response is complex).
    ``fsphere`` uses the constant-f operator of Sec. 4 (eigenvalue analysis).
    """
    U = np.asarray(U, dtype=np.complex128)
    out = np.zeros_like(U)
    lead = U.shape[:-2]
    ms = range(N + 1) if ms is None else ms
    for m in ms:
        A = tau * operator_m(m, N, c, fsphere)
        if adjoint:
            A = A.conj().T
        _check_band(A)
        ab0 = _to_banded(A)
        mask = _state_mask(m, N)
        rhs = (interleave(U, m, N) * mask).reshape(-1, 3 * (N - m + 1)).T  # [3K, nrhs]
        acc = np.zeros_like(rhs)
        for a_n, b_n in zip(alpha, beta):
            if adjoint:
                a_n, b_n = np.conj(a_n), np.conj(b_n)
            ab = ab0.copy()
            ab[_BW, :] += a_n
            acc += b_n * solve_banded((_BW, _BW), ab, rhs)
        res = (acc * mask[:, None]).T.reshape(lead + (-1,))
        if m == 0 and real_m0:
            res = res.real.astype(np.complex128)
        deinterleave(res, out, m, N)
    return out


class GridStep:
    """REXI step in grid layout: (h', u, v) on an nlat x nlon Gaussian grid."""

    def __init__(self, N, nlat, nlon, alpha, beta, tau, c=Consts(), fsphere=False):
        self.N, self.g = N, Grid(N, nlat, nlon)
        self.alpha, self.beta, self.tau, self.c = alpha, beta, tau, c
        self.fsphere = fsphere

    # grid (h', u, v) -> spectral (Phi, zeta, delta)
    def analyse(self, x):
        g, c = self.g, self.c
        cl = g.coslat[:, None]
        Phi = g.analysis(c.gravity * x[..., 0, :, :])
        zeta, delta = g.uv_to_vortdiv(x[..., 1, :, :] * cl, x[..., 2, :, :] * cl, c.radius)
        return np.stack([Phi, zeta, delta], axis=-2)

    # spectral (Phi, zeta, delta) -> grid (h', u, v)
    def synthesise(self, S):
        g, c = self.g, self.c
        cl = g.coslat[:, None]
        h = g.synthesis(S[..., 0, :]) / c.gravity
        U, V = g.vortdiv_to_uv(S[..., 1, :], S[..., 2, :], c.radius)
        return np.stack([h, U / cl, V / cl], axis=-3)

    def __call__(self, x):
        S = self.analyse(np.asarray(x, dtype=np.float64))
        S = rexi_step_spectral(S, self.N, self.alpha, self.beta, self.tau, self.c, fsphere=self.fsphere)
        return self.synthesise(S)

    # ---- transposes of the grid-layout stages --------------------------------
    def synthesise_T(self, y):
        """Transpose of ``synthesise``: grid cotangent -> spectral cotangent."""
        g, c, N = self.g, self.c, self.N
        cl = g.coslat[:, None]
        cm = np.full(N + 1, 2.0)
        cm[0] = 1.0
        # inverse-FFT transpose: Fbar_m = c_m sum_i xbar_i e^{-i m lambda_i}
        def fft_T(xb):
            return np.fft.rfft(xb, axis=-1)[..., : N + 1] * cm
        FP = fft_T(y[..., 0, :, :] / c.gravity)
        FU = fft_T(y[..., 1, :, :] / cl)
        FV = fft_T(y[..., 2, :, :] / cl)
        out = np.zeros(y.shape[:-3] + (3, nspec(N)), dtype=np.complex128)
        for m in range(N + 1):
            P, H = g.tables(m)
            ns = np.arange(m, N + 1)
            inv = np.zeros(ns.size)
            inv[ns > 0] = -c.radius / (ns[ns > 0] * (ns[ns > 0] + 1.0))
            sl = slice(idx(m, m, N), idx(m, N, N) + 1)
            fp, fu, fv = FP[..., :, m], FU[..., :, m], FV[..., :, m]
            out[..., 0, sl] = np.einsum("nj,...j->...n", P, fp)
            # U = -H psi' + i m P chi',  V = i m P psi' + H chi'   (psi' = inv * zeta)
            psib = -np.einsum("nj,...j->...n", H, fu) - 1j * m * np.einsum("nj,...j->...n", P, fv)
            chib = -1j * m * np.einsum("nj,...j->...n", P, fu) + np.einsum("nj,...j->...n", H, fv)
            out[..., 1, sl] = psib * inv
            out[..., 2, sl] = chib * inv
        return out

    def analyse_T(self, S):
        """Transpose of ``analyse``: spectral cotangent -> grid cotangent."""
        g, c, N = self.g, self.c, self.N
        cl = g.coslat[:, None]
        FP = np.zeros(S.shape[:-2] + (g.nlat, N + 1), dtype=np.complex128)
        FU = np.zeros_like(FP)
        FV = np.zeros_like(FP)
        sc = g.w / (1.0 - g.mu ** 2) / c.radius
        for m in range(N + 1):
            P, H = g.tables(m)
            sl = slice(idx(m, m, N), idx(m, N, N) + 1)
            zb, db = S[..., 1, sl], S[..., 2, sl]
            FP[..., :, m] = np.einsum("nj,...n->...j", P * g.w, S[..., 0, sl])
            # zeta = sc [i m P F^V + H F^U],  delta = sc [i m P F^U - H F^V]
            FU[..., :, m] = sc * (np.einsum("nj,...n->...j", H, zb)
                                  - 1j * m * np.einsum("nj,...n->...j", P, db))
            FV[..., :, m] = sc * (-1j * m * np.einsum("nj,...n->...j", P, zb)
                                  - np.einsum("nj,...n->...j", H, db))
        # forward-FFT transpose: xbar_i = (1/nlon) sum_{m=0}^{N} Re(Fbar_m e^{i m lambda_i})
        half = np.full(N + 1, 0.5)
        half[0] = 1.0

        def fft_T(F):
            return g.fourier_inv(F * half) / g.nlon
        hb = c.gravity * fft_T(FP)
        ub = cl * fft_T(FU)
        vb = cl * fft_T(FV)
        return np.stack([hb, ub, vb], axis=-3)

    def adjoint(self, y):
        y = np.asarray(y, dtype=np.float64)
        S = self.synthesise_T(y)
        m0 = slice(0, self.N + 1)
        S[..., m0] = S[..., m0].real  # m = 0 cotangents of a real field are real
        S = rexi_step_spectral(S, self.N, self.alpha, self.beta, self.tau, self.c, adjoint=True,
                               fsphere=self.fsphere)
        return self.analyse_T(S)
