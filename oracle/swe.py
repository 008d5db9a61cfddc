"""Linear SWE operator of the paper's Eq. (1) in spherical-harmonic space -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Eq. (1), vorticity-divergence form, linearised about rest with mean
geopotential Phibar = g Hbar and f = 2 Omega mu:
    zeta_t  = -f delta - V . grad f
    delta_t =  f zeta + k . (grad f x V) - lap Phi
    Phi_t   = -Phibar delta,        V = k x grad psi + grad chi.
With grad f = (2 Omega cos(phi)/a) e_phi this is
    zeta_t = -f delta - (2 Omega / a) V,   delta_t = f zeta - (2 Omega / a) U - lap Phi
in Robert's U = u cos(phi), V = v cos(phi).  Projecting on orthonormal
spherical harmonics with  mu Pbar_n = eps_{n+1} Pbar_{n+1} + eps_n Pbar_{n-1}  and
(1-mu^2) dPbar_n/dmu = -n eps_{n+1} Pbar_{n+1} + (n+1) eps_n Pbar_{n-1}  gives, per m,
    (L Phi)_n   = -Phibar delta_n
    (L zeta)_n  = i sigma_n zeta_n - 2 Omega [c_n delta_{n-1} + d_n delta_{n+1}]
    (L delta)_n = i sigma_n delta_n + 2 Omega [c_n zeta_{n-1} + d_n zeta_{n+1}] + n(n+1)/a^2 Phi_n
    sigma_n = 2 Omega m / (n(n+1)),  c_n = eps_n (n+1)/n,  d_n = eps_{n+1} n/(n+1).
Truncation (reading: the paper is silent): couplings to degree N+1 are
dropped; zeta_0^0 and delta_0^0 are not state variables (the global means of
vorticity and divergence vanish) and are held at zero.

The derivation is the builder's; it is pinned by a brute-force grid
evaluation of Eq. (1) built on scipy's Legendre functions, by the
geostrophic-balance steady state of Sec. 6.1, and by the eigenvalues of L
being purely imaginary.  ``fsphere=True`` replaces f by the constant 2 Omega
(the paper's f-sphere, Sec. 4.3), used only as an extra closed-form pin.
"""

from dataclasses import dataclass

import numpy as np

from .sphere import eps, idx, nspec


@dataclass(frozen=True)
class Consts:
    radius: float = 6.37122e6      # a   (Sec. 6)
    omega: float = 7.292e-5        # Omega
    gravity: float = 9.80616       # g
    mean_depth: float = 1.0e4      # Hbar

    @property
    def phibar(self):
        return self.gravity * self.mean_depth


def coupling(m, N, c):
    """Per-degree coefficients (n, sigma_n, ct_n, dt_n, G_n) for n = m..N.

    ct/dt are c_n/d_n with the couplings that leave the state set to zero:
    ct_n = 0 when n-1 < max(m,1), dt_n = 0 when n+1 > N.
    """
    ns = np.arange(m, N + 1)
    nf = ns.astype(np.float64)
    sig = np.zeros(ns.size)
    ct = np.zeros(ns.size)
    dt = np.zeros(ns.size)
    pos = ns > 0
    sig[pos] = 2.0 * c.omega * m / (nf[pos] * (nf[pos] + 1.0))
    nmin = max(m, 1)
    e_n = eps(ns, m)
    e_np1 = eps(ns + 1, m)
    okc = (ns - 1 >= nmin) & pos
    ct[okc] = e_n[okc] * (nf[okc] + 1.0) / nf[okc]
    okd = (ns + 1 <= N) & pos
    dt[okd] = e_np1[okd] * nf[okd] / (nf[okd] + 1.0)
    G = nf * (nf + 1.0) / c.radius ** 2
    return ns, sig, ct, dt, G


def operator_m(m, N, c, fsphere=False):
    """Dense L_m in the interleaved ordering (Phi_n, zeta_n, delta_n), n = m..N."""
    ns, sig, ct, dt, G = coupling(m, N, c)
    K = ns.size
    A = np.zeros((3 * K, 3 * K), dtype=np.complex128)
    tw = 2.0 * c.omega
    for i, n in enumerate(ns):
        P, Z, D = 3 * i, 3 * i + 1, 3 * i + 2
        if n == 0:
            continue  # Phi_0^0 is constant under L; zeta_0^0, delta_0^0 are not state
        A[P, D] = -c.phibar
        A[D, P] = G[i]
        if fsphere:
            A[Z, D] = -tw
            A[D, Z] = tw
            continue
        A[Z, Z] = 1j * sig[i]
        A[D, D] = 1j * sig[i]
        if ct[i] != 0.0:
            A[Z, 3 * (i - 1) + 2] = -tw * ct[i]
            A[D, 3 * (i - 1) + 1] = tw * ct[i]
        if dt[i] != 0.0:
            A[Z, 3 * (i + 1) + 2] = -tw * dt[i]
            A[D, 3 * (i + 1) + 1] = tw * dt[i]
    return A


def interleave(U, m, N):
    """[..., 3, nspec] spectral state -> [..., 3K] interleaved vector for order m."""
    sl = slice(idx(m, m, N), idx(m, N, N) + 1)
    x = np.stack([U[..., 0, sl], U[..., 1, sl], U[..., 2, sl]], axis=-1)
    return x.reshape(x.shape[:-2] + (-1,))


def deinterleave(x, out, m, N):
    sl = slice(idx(m, m, N), idx(m, N, N) + 1)
    y = x.reshape(x.shape[:-1] + (-1, 3))
    out[..., 0, sl] = y[..., 0]
    out[..., 1, sl] = y[..., 1]
    out[..., 2, sl] = y[..., 2]


def apply_L(U, N, c, fsphere=False):
    """L U for a spectral state U [..., 3, nspec]."""
    out = np.zeros_like(U, dtype=np.complex128)
    for m in range(N + 1):
        deinterleave(interleave(U, m, N) @ operator_m(m, N, c, fsphere).T, out, m, N)
    return out


def dense_operator(N, c, fsphere=False):
    """Block-diagonal L over all m as one dense matrix in [3, nspec] (field-major) order."""
    ns_ = nspec(N)
    L = np.zeros((3 * ns_, 3 * ns_), dtype=np.complex128)
    for m in range(N + 1):
        A = operator_m(m, N, c, fsphere)
        K = N - m + 1
        rows = np.array([f * ns_ + idx(m, m + i, N) for i in range(K) for f in range(3)])
        L[np.ix_(rows, rows)] = A
    return L
