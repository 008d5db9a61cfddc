"""Reference time integrators for the Gaussian-bump study of Sec. 6.2 -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* ``rk4``       -- the classical fourth-order Runge-Kutta method with a fixed step,
                   which the paper uses (dt = 50 s) as its reference solution for
                   the 1.5-day bump propagation (Sec. 6.2, Sec. 6.4).
* ``exact``     -- exp(t L) U, per zonal order m from the Hermitian eigenproblem of
                   L in the energy inner product: the exact solution of the linear
                   system dU/dt = L U, which the RK4 reference only approximates.
* ``rexi_modal`` -- K T-REXI steps through the scalar REXI response on L's modes, for
                   long runs that the shifted-solve oracle (``step``) is too slow for.
* ``energy``    -- the quadratic invariant of the linearised equations (total
                   energy about the state of rest), used to pin both.

L is the spectral operator of ``swe`` (Eq. (1)), held as a scipy sparse matrix
over the field-major [3, nspec] state so that an RK4 stage is one sparse product.

Pins (tests/test_oracle_integrate.py): the f-sphere closed-form solution of a
single degree, the steady geostrophic state of Sec. 6.1, agreement of ``exact``
with scipy's matrix exponential, conservation of ``energy`` by ``exact`` and its
closed-form decay per mode under ``rk4``, RK4's fourth-order convergence to
``exact``, and ``rexi_modal`` against ``step.rexi_step_spectral`` (one step) and
against ``exact`` (many poles).
"""

import numpy as np
import scipy.linalg
import scipy.sparse

from .sphere import idx, nspec
from .swe import operator_m


def _rows(m, N):
    """Field-major positions of the interleaved (Phi, zeta, delta) rows of order m."""
    ns_ = nspec(N)
    return np.array([f * ns_ + idx(m, n, N) for n in range(m, N + 1) for f in range(3)])


def sparse_operator(N, c, fsphere=False):
    """L over the flattened field-major state [3 * nspec] as a CSR matrix."""
    ri, ci, vals = [], [], []
    for m in range(N + 1):
        A = operator_m(m, N, c, fsphere)
        r, q = np.nonzero(A)
        rows = _rows(m, N)
        ri.append(rows[r])
        ci.append(rows[q])
        vals.append(A[r, q])
    n = 3 * nspec(N)
    return scipy.sparse.csr_matrix((np.concatenate(vals), (np.concatenate(ri), np.concatenate(ci))), shape=(n, n))


def rk4(U, N, dt, nsteps, c, fsphere=False, L=None):
    """nsteps classical RK4 steps of dU/dt = L U from the spectral state U [..., 3, nspec]."""
    L = sparse_operator(N, c, fsphere) if L is None else L
    shape = U.shape
    x = np.asarray(U, dtype=np.complex128).reshape(-1, 3 * nspec(N)).T.copy()
    for _ in range(nsteps):
        k1 = L @ x
        k2 = L @ (x + 0.5 * dt * k1)
        k3 = L @ (x + 0.5 * dt * k2)
        k4 = L @ (x + dt * k3)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
    return x.T.reshape(shape)


def energy_weights(m, N, c):
    """Diagonal W of the energy x^H W x over order m's interleaved (Phi_n, zeta_n, delta_n)
    rows: 1 for Phi, Phibar a^2 / (n(n+1)) for zeta and delta (1 on the unused n = 0 rows)."""
    w = []
    for n in range(m, N + 1):
        k = c.phibar * c.radius ** 2 / (n * (n + 1)) if n > 0 else 1.0
        w.extend([1.0, k, k])
    return np.array(w)


def exact(U, N, t, c, fsphere=False):
    """exp(t L) U for the spectral state U [..., 3, nspec], per zonal order m.

    L conserves the energy x^H W x, so S = W^(1/2) L W^(-1/2) is skew-Hermitian; with the
    Hermitian eigendecomposition -i S = V diag(lam) V^H,
        exp(t L) = W^(-1/2) V diag(exp(i lam t)) V^H W^(1/2),
    which stays exactly norm-preserving for any t (no scaling and squaring)."""
    U = np.asarray(U, dtype=np.complex128)
    flat = U.reshape(-1, 3 * nspec(N))
    out = np.zeros_like(flat)
    for m in range(N + 1):
        rows = _rows(m, N)
        sw = np.sqrt(energy_weights(m, N, c))
        S = (sw[:, None] * operator_m(m, N, c, fsphere)) / sw[None, :]
        H = -0.5j * (S - S.conj().T)  # -i S, symmetrised against rounding
        lam, V = np.linalg.eigh(H)
        E = (V * np.exp(1j * lam * t)[None, :]) @ V.conj().T
        E = E / sw[:, None] * sw[None, :]
        out[:, rows] = flat[:, rows] @ E.T
    return out.reshape(U.shape)


def rexi_modal(U, N, alpha, beta, tau, nsteps, c, fsphere=False):
    """nsteps REXI steps evaluated mode by mode: U <- f(tau L)^nsteps U with the scalar
    response f(x) = sum_k beta_k / (alpha_k + i x) applied to the eigenvalues i lam of L
    (Hermitian eigenproblem in the energy inner product, as in ``exact``).

    A different algorithm from ``step.rexi_step_spectral`` (no shifted solves): the two
    agree because (alpha + tau L)^{-1} has the eigenvectors of L.  For m = 0 the real part
    of Sec. 4.2's sum is implied: the poles come in conjugate pairs, so f(-x) = conj f(x)
    and f(tau L) maps the real m = 0 coefficients to real ones."""
    U = np.asarray(U, dtype=np.complex128)
    flat = U.reshape(-1, 3 * nspec(N))
    out = np.zeros_like(flat)
    alpha = np.asarray(alpha)[:, None]
    beta = np.asarray(beta)[:, None]
    for m in range(N + 1):
        rows = _rows(m, N)
        sw = np.sqrt(energy_weights(m, N, c))
        S = (sw[:, None] * operator_m(m, N, c, fsphere)) / sw[None, :]
        lam, V = np.linalg.eigh(-0.5j * (S - S.conj().T))
        f = np.sum(beta / (alpha + 1j * tau * lam[None, :]), axis=0)
        E = (V * (f ** nsteps)[None, :]) @ V.conj().T
        E = E / sw[:, None] * sw[None, :]
        out[:, rows] = flat[:, rows] @ E.T
    return out.reshape(U.shape)


def energy(U, N, c):
    """Total energy of the linear SWE about rest, up to a constant factor:
    sum over m = -N..N and n of |Phi|^2 + Phibar a^2 / (n(n+1)) (|zeta|^2 + |delta|^2)
    (potential plus kinetic, with |V|^2 from zeta and delta by Parseval)."""
    U = np.asarray(U)
    e = np.zeros(U.shape[:-2])
    for m in range(N + 1):
        mult = 1.0 if m == 0 else 2.0
        for n in range(max(m, 1), N + 1):
            i = idx(m, n, N)
            w = c.phibar * c.radius ** 2 / (n * (n + 1))
            e = e + mult * (np.abs(U[..., 0, i]) ** 2 + w * (np.abs(U[..., 1, i]) ** 2 + np.abs(U[..., 2, i]) ** 2))
        if m == 0:
            e = e + np.abs(U[..., 0, idx(0, 0, N)]) ** 2
    return e
