"""Seeded synthetic inputs shared by the tests, the oracle runs and ``bench.py``.

This module draws random numbers and writes down closed-form initial states;
it contains none of the REXI method's arithmetic (no transforms, no operator,
no solves), so both the CUDA path and the oracle can take their inputs from it.

States are spectral (Phi, zeta, delta) in the library's layout
``[B, 3, nspec]`` complex128, m-major triangular order
``idx(m, n) = m(2N+3-m)/2 + (n-m)``, orthonormal Legendre functions
(int_{-1}^{1} Pbar^2 dmu = 1, no Condon-Shortley phase).  Parseval for that
normalisation gives the sphere mean square of a real field as
1/2 * sum_{m=-N}^{N} sum_n |xi_n^m|^2, and the mean kinetic energy of
V = k x grad psi + grad chi as 1/2 * sum a^2/(n(n+1)) (|zeta_n^m|^2 + |delta_n^m|^2).
"""

import numpy as np

EARTH = dict(radius=6.37122e6, omega=7.292e-5, gravity=9.80616, mean_depth=1.0e4)


def nspec(N):
    return (N + 1) * (N + 2) // 2


def degree_order(N):
    """Arrays (n, m) for every coefficient in m-major order."""
    ms, ns = [], []
    for m in range(N + 1):
        ns.extend(range(m, N + 1))
        ms.extend([m] * (N - m + 1))
    return np.array(ns), np.array(ms)


def _mean_square(coef, mvec, weight=None):
    mult = np.where(mvec == 0, 1.0, 2.0)
    w = 1.0 if weight is None else weight
    return 0.5 * np.sum(mult * w * np.abs(coef) ** 2, axis=-1)


def random_spectral(N, batch, seed, h_std=50.0, uv_std=5.0, slope=-3.0, consts=EARTH):
    """Complex-normal spectra with amplitude ~ n^slope, rescaled per state so that
    std(h') = h_std and std(u) = std(v) = uv_std (in expectation).

    Returns [batch, 3, nspec] complex128 (Phi = g h', zeta, delta); the n = 0
    coefficients are zero and m = 0 coefficients are real.
    """
    rng = np.random.default_rng(seed)
    n, m = degree_order(N)
    ns_ = nspec(N)
    amp = np.zeros(ns_)
    amp[n > 0] = n[n > 0].astype(np.float64) ** slope
    z = (rng.standard_normal((batch, 3, ns_)) + 1j * rng.standard_normal((batch, 3, ns_))) / np.sqrt(2.0)
    z[..., m == 0] = z[..., m == 0].real * np.sqrt(2.0)
    S = z * amp
    a = consts["radius"]
    g = consts["gravity"]
    inv_lap = np.zeros(ns_)
    inv_lap[n > 0] = a * a / (n[n > 0] * (n[n > 0] + 1.0))
    for b in range(batch):
        hs = S[b, 0] / 1.0
        S[b, 0] *= g * h_std / np.sqrt(_mean_square(hs, m))
        ke = _mean_square(S[b, 1], m, inv_lap) + _mean_square(S[b, 2], m, inv_lap)
        S[b, 1:] *= uv_std * np.sqrt(2.0) / np.sqrt(ke)
    return S


def balanced_zonal_flow(N, u0=20.0, consts=EARTH):
    """Spectral state of the linearised geostrophically balanced zonal flow (Sec. 6.1):
    u = u0 cos(phi), v = 0, Phi' = u0 a Omega cos^2(phi).

    Closed-form projections: zeta = 2 u0 mu / a = (2 u0 / a) sqrt(2/3) Pbar_1^0;
    1 - mu^2 = (2 sqrt(2)/3) Pbar_0^0 - (2/3) sqrt(2/5) Pbar_2^0.
    Returns [3, nspec] complex128.
    """
    if N < 2:
        raise ValueError("N >= 2 needed")
    a, om = consts["radius"], consts["omega"]
    S = np.zeros((3, nspec(N)), dtype=np.complex128)
    amp = u0 * a * om
    S[0, 0] = amp * 2.0 * np.sqrt(2.0) / 3.0          # (m,n) = (0,0)
    S[0, 2] = -amp * (2.0 / 3.0) * np.sqrt(2.0 / 5.0)  # (0,2)
    S[1, 1] = 2.0 * u0 / a * np.sqrt(2.0 / 3.0)        # (0,1)
    return S


def balanced_grid(mu, nlon, u0=20.0, consts=EARTH):
    """The same balanced flow evaluated on a grid with latitudes mu: (h', u, v) [3, nlat, nlon]."""
    a, om, g = consts["radius"], consts["omega"], consts["gravity"]
    cos2 = (1.0 - mu * mu)[:, None] * np.ones((1, nlon))
    h = u0 * a * om * cos2 / g
    u = u0 * np.sqrt(cos2)
    return np.stack([h, u, np.zeros_like(u)])


def noisy_balanced(N, seed, u0=20.0, noise_std=1e-3, consts=EARTH):
    """Balanced zonal flow plus seeded n^-3 noise with std(h') = noise_std m and
    std(u,v) = noise_std m/s.  Returns [1, 3, nspec]."""
    noise = random_spectral(N, 1, seed, h_std=noise_std, uv_std=noise_std, consts=consts)
    return balanced_zonal_flow(N, u0, consts)[None] + noise


def random_grid(batch, nlat, nlon, seed, scale=(50.0, 5.0, 5.0)):
    """White-noise grid fields (h', u, v) [batch, 3, nlat, nlon] float64 (not band-limited)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((batch, 3, nlat, nlon))
    return x * np.asarray(scale)[None, :, None, None]


BUMPS = ((0.2 * np.pi, np.pi / 3.0, 20.0), (1.2 * np.pi, -np.pi / 5.0, 80.0), (1.6 * np.pi, -np.pi / 4.0, 360.0))


def gaussian_bumps(mu, nlon, consts=EARTH, bumps=BUMPS):
    """The three-bump initial state of Sec. 6.2 on a grid with latitudes mu: (h', u, v)
    [3, nlat, nlon], at rest, h' = sum of 0.1 Hbar exp(-p d^2) with d the great-circle
    angle to the bump centre (lambda_c, phi_c)."""
    phi = np.arcsin(np.asarray(mu))[:, None]
    lam = 2.0 * np.pi * np.arange(nlon)[None, :] / nlon
    h = np.zeros((phi.shape[0], nlon))
    for lc, pc, p in bumps:
        c = np.sin(pc) * np.sin(phi) + np.cos(pc) * np.cos(phi) * np.cos(lam - lc)
        d = np.arccos(np.clip(c, -1.0, 1.0))
        h += 0.1 * consts["mean_depth"] * np.exp(-d * d * p)
    return np.stack([h, np.zeros_like(h), np.zeros_like(h)])
