"""Spherical harmonics on a Gaussian grid (paper Sec. 3) -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Conventions (the paper defers to SHTns defaults and fixes none of them, so these
are readings):

* Triangular truncation at degree N: coefficients xi_n^m for 0 <= m <= n <= N,
  stored m-major, ``idx(m, n) = m(2N+3-m)/2 + (n-m)``, ``nspec=(N+1)(N+2)/2``.
* Orthonormal associated Legendre functions without Condon-Shortley phase,
  int_{-1}^{1} Pbar_n^m(mu)^2 dmu = 1, so that a real field is
  xi(lambda, mu) = sum_{m=-N}^{N} sum_n xi_n^m Pbar_n^m(mu) e^{i m lambda}
  with xi_n^{-m} = conj(xi_n^m), and the analysis integral of Sec. 3
  xi_n^m = int (1/2pi) int xi e^{-i m lambda} dlambda Pbar_n^m dmu holds as printed.
* Gaussian grid: mu_j = sin(phi_j) are the nlat Gauss-Legendre nodes ordered
  north to south (mu descending); lambda_i = 2 pi i / nlon.
* Velocities enter through Robert's cos(phi) scaling (Sec. 3):
  U = u cos(phi), V = v cos(phi).

Pins: Gauss nodes/weights vs numpy.polynomial.legendre.leggauss; Pbar vs
scipy.special.lpmv with the normalisation written out; H = (1-mu^2) dPbar/dmu
vs an independent derivative identity and vs finite differences; transform
round trips on band-limited fields; solid-body rotation closed form.
"""

import numpy as np


def nspec(N):
    return (N + 1) * (N + 2) // 2


def idx(m, n, N):
    """Position of xi_n^m in the m-major triangular array."""
    return m * (2 * N + 3 - m) // 2 + (n - m)


def gauss_legendre(nlat):
    """Gauss-Legendre nodes (descending) and weights by Newton iteration on P_nlat.

    P_nlat and its derivative come from the Bonnet three-term recurrence; the
    weights are 2 / ((1 - mu^2) P'_nlat(mu)^2).
    """
    k = np.arange(1, nlat + 1)
    x = np.cos(np.pi * (k - 0.25) / (nlat + 0.5))  # descending initial guesses
    for _ in range(100):
        p0 = np.ones_like(x)
        p1 = x.copy()
        for n in range(2, nlat + 1):
            p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
        dp = nlat * (x * p1 - p0) / (x * x - 1.0)
        dx = p1 / dp
        x = x - dx
        if np.max(np.abs(dx)) < 1e-16:
            break
    p0 = np.ones_like(x)
    p1 = x.copy()
    for n in range(2, nlat + 1):
        p0, p1 = p1, ((2 * n - 1) * x * p1 - (n - 1) * p0) / n
    dp = nlat * (x * p1 - p0) / (x * x - 1.0)
    w = 2.0 / ((1.0 - x * x) * dp * dp)
    return x, w


def eps(n, m):
    """epsilon_n^m = sqrt((n^2 - m^2) / (4 n^2 - 1)); 0 for n <= m."""
    n = np.asarray(n, dtype=np.float64)
    out = np.zeros_like(n)
    ok = n > m
    out[ok] = np.sqrt((n[ok] ** 2 - m * m) / (4.0 * n[ok] ** 2 - 1.0))
    return out


def alp(m, N, mu):
    """Pbar_n^m(mu) and H_n^m(mu) = (1-mu^2) dPbar_n^m/dmu for n = m..N.

    Returns two arrays of shape [N-m+1, len(mu)].  Seed
    Pbar_0^0 = 1/sqrt(2), Pbar_m^m = sqrt((2m+1)/(2m)) sqrt(1-mu^2) Pbar_{m-1}^{m-1};
    then mu Pbar_{n} = eps_{n+1} Pbar_{n+1} + eps_n Pbar_{n-1} upwards in n.
    H follows from (1-mu^2) dPbar_n/dmu = -n eps_{n+1} Pbar_{n+1} + (n+1) eps_n Pbar_{n-1}.
    """
    mu = np.asarray(mu, dtype=np.float64)
    s = np.sqrt(1.0 - mu * mu)
    pmm = np.full_like(mu, 1.0 / np.sqrt(2.0))
    for k in range(1, m + 1):
        pmm = pmm * np.sqrt((2.0 * k + 1.0) / (2.0 * k)) * s
    # one extra degree (N+1) is needed for H_N
    P = np.zeros((N - m + 2, mu.size))
    P[0] = pmm
    if N + 1 > m:
        P[1] = np.sqrt(2.0 * m + 3.0) * mu * pmm
    for n in range(m + 2, N + 2):
        e_n = eps(np.array([n]), m)[0]
        e_nm1 = eps(np.array([n - 1]), m)[0]
        P[n - m] = (mu * P[n - m - 1] - e_nm1 * P[n - m - 2]) / e_n
    ns = np.arange(m, N + 1)
    H = np.zeros((N - m + 1, mu.size))
    e_np1 = eps(ns + 1, m)
    e_n = eps(ns, m)
    for i, n in enumerate(ns):
        H[i] = -n * e_np1[i] * P[i + 1]
        if i > 0:
            H[i] += (n + 1) * e_n[i] * P[i - 1]
    return P[: N - m + 1], H


class Grid:
    """Gaussian grid plus the per-m Legendre tables for truncation N."""

    def __init__(self, N, nlat, nlon):
        if nlon < 2 * N + 1 or nlat < N + 1:
            raise ValueError("grid too coarse for truncation")
        self.N, self.nlat, self.nlon = N, nlat, nlon
        self.mu, self.w = gauss_legendre(nlat)
        self.coslat = np.sqrt(1.0 - self.mu ** 2)
        self.lam = 2.0 * np.pi * np.arange(nlon) / nlon
        self._tab = {}

    def tables(self, m):
        if m not in self._tab:
            self._tab[m] = alp(m, self.N, self.mu)
        return self._tab[m]

    # ---- longitude transforms ------------------------------------------------
    def fourier(self, x):
        """F_m(mu_j) = (1/nlon) sum_i x(lambda_i, mu_j) e^{-i m lambda_i}, m = 0..N."""
        return np.fft.rfft(x, axis=-1)[..., : self.N + 1] / self.nlon

    def fourier_inv(self, F):
        """x(lambda_i) = sum_{m=-N}^{N} F_m e^{i m lambda_i} with F_{-m} = conj(F_m)."""
        G = np.zeros(F.shape[:-1] + (self.nlon // 2 + 1,), dtype=np.complex128)
        G[..., : self.N + 1] = F * self.nlon
        return np.fft.irfft(G, n=self.nlon, axis=-1)

    # ---- scalar transforms (Sec. 3) -----------------------------------------
    def analysis(self, x):
        """Grid [..., nlat, nlon] -> spectral [..., nspec] by Gaussian quadrature."""
        N = self.N
        F = self.fourier(x)  # [..., nlat, N+1]
        out = np.zeros(x.shape[:-2] + (nspec(N),), dtype=np.complex128)
        for m in range(N + 1):
            P, _ = self.tables(m)
            out[..., idx(m, m, N): idx(m, N, N) + 1] = np.einsum(
                "nj,...j->...n", P * self.w, F[..., :, m])
        return out

    def synthesis(self, xi):
        """Spectral [..., nspec] -> grid [..., nlat, nlon]."""
        N = self.N
        F = np.zeros(xi.shape[:-1] + (self.nlat, N + 1), dtype=np.complex128)
        for m in range(N + 1):
            P, _ = self.tables(m)
            F[..., :, m] = np.einsum("nj,...n->...j", P, xi[..., idx(m, m, N): idx(m, N, N) + 1])
        return self.fourier_inv(F)

    # ---- vector transforms (Sec. 2: V = k x grad psi + grad chi) -------------
    def uv_to_vortdiv(self, U, V, radius):
        """Robert-scaled winds U = u cos(phi), V = v cos(phi) -> (zeta, delta) spectral.

        zeta_n^m = (1/a) sum_j w_j/(1-mu_j^2) [ i m Pbar F^V + H F^U ]
        delta_n^m = (1/a) sum_j w_j/(1-mu_j^2) [ i m Pbar F^U - H F^V ]
        (curl and divergence on the sphere, integrated by parts in mu).
        """
        N = self.N
        FU = self.fourier(U)
        FV = self.fourier(V)
        sc = self.w / (1.0 - self.mu ** 2) / radius
        zeta = np.zeros(U.shape[:-2] + (nspec(N),), dtype=np.complex128)
        delta = np.zeros_like(zeta)
        for m in range(N + 1):
            P, H = self.tables(m)
            sl = slice(idx(m, m, N), idx(m, N, N) + 1)
            fu = FU[..., :, m]
            fv = FV[..., :, m]
            zeta[..., sl] = (1j * m * np.einsum("nj,...j->...n", P * sc, fv)
                             + np.einsum("nj,...j->...n", H * sc, fu))
            delta[..., sl] = (1j * m * np.einsum("nj,...j->...n", P * sc, fu)
                              - np.einsum("nj,...j->...n", H * sc, fv))
        return zeta, delta

    def vortdiv_to_uv(self, zeta, delta, radius):
        """(zeta, delta) spectral -> Robert-scaled U = u cos(phi), V = v cos(phi) on the grid.

        psi_n = -a^2 zeta_n / (n(n+1)), chi_n = -a^2 delta_n / (n(n+1)) (zero for n = 0),
        U = (1/a) sum_n [ -H psi_n + i m Pbar chi_n ],  V = (1/a) sum_n [ i m Pbar psi_n + H chi_n ].
        """
        N = self.N
        FU = np.zeros(zeta.shape[:-1] + (self.nlat, N + 1), dtype=np.complex128)
        FV = np.zeros_like(FU)
        for m in range(N + 1):
            P, H = self.tables(m)
            ns = np.arange(m, N + 1)
            inv = np.zeros(ns.size)
            inv[ns > 0] = -radius / (ns[ns > 0] * (ns[ns > 0] + 1.0))  # psi/a
            sl = slice(idx(m, m, N), idx(m, N, N) + 1)
            ps = zeta[..., sl] * inv
            ch = delta[..., sl] * inv
            FU[..., :, m] = (-np.einsum("nj,...n->...j", H, ps)
                             + 1j * m * np.einsum("nj,...n->...j", P, ch))
            FV[..., :, m] = (1j * m * np.einsum("nj,...n->...j", P, ps)
                             + np.einsum("nj,...n->...j", H, ch))
        return self.fourier_inv(FU), self.fourier_inv(FV)
