"""The paper's own T-REXI solver: a geopotential-only system per pole (Sec. 4.3 and
Sec. 5) -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Per pole alpha and time step tau, with f = 2 Omega mu, the shifted system
(alpha + tau L) X = X0 of Eq. (1) is, in (Phi, V):
    alpha Phi - tau Phibar div V = Phi0,        A V = V0 + tau grad Phi,
    A = [[alpha, tau f], [-tau f, alpha]],      A^{-1} = M / D,
    M = [[alpha, -tau f], [tau f, alpha]],      D = alpha^2 + tau^2 f^2
(Sec. 4.3, the 3x3 operator and the velocity equation).  Substituting V and
multiplying by D^2 (the paper multiplies through by alpha^2 + f^2 so that no
1/(alpha^2 + f^2) is left to expand in spherical harmonics, Sec. 5) gives a
geopotential-only equation whose coefficients are polynomials in mu:
    alpha D^2 Phi - tau^2 Phibar [ D (alpha lap Phi + tau (2 Omega/a^2) dPhi/dlambda)
        - 2 tau^2 f (2 Omega/a^2) (alpha (1-mu^2) dPhi/dmu + tau f dPhi/dlambda) ]
  = D^2 Phi0 + tau Phibar [ D (alpha delta0 - tau f zeta0 + tau (2 Omega/a) U0)
        - 2 tau^2 f (2 Omega/a) (alpha V0 + tau f U0) ],
with Robert's U0 = u0 cos(phi), V0 = v0 cos(phi).  (The derivation is the builder's;
the paper prints the same structure as its Z_1 ... Z_8 decomposition, with the sign
slips noted in the design notes.)  Its coefficients reach mu^4, so in degree n the
matrix couples n, n +- 2, n +- 4.

This oracle follows the paper's steps per zonal order m and pole: the matrix is
the Galerkin projection of that operator onto degrees m..N (each basis function is
evaluated on the Gaussian latitudes and projected back by quadrature, which is
exact for these polynomial degrees when nlat >= N + 3), the right-hand side is
assembled on the latitudes from the synthesised (Phi0, zeta0, delta0, U0, V0) and
projected, the system is solved, the velocities are recovered pointwise in
latitude from V = A^{-1} (V0 + tau grad Phi), and zeta, delta are their curl and
divergence projected back; beta_k times the result is summed over the poles.
A second recovery, in spectral space from the Phi and zeta rows of the system, is
the GPU path's form (``recover="spectral"``).

Truncating the multiplied-through equation is a different discretisation from
truncating L itself, so this result equals ``step.rexi_step_spectral`` only where
truncation does not act: exactly on the f-sphere (constant f, D constant) and
without rotation, and in the low degrees otherwise.  Those are its pins
(tests/test_oracle_phi_solver.py), together with the band structure of the matrix.
"""

import numpy as np

from .sphere import alp, gauss_legendre, idx
from .swe import Consts, coupling


def phi_matrix_and_rhs(m, N, mu, w, alpha, tau, c, U_m, fsphere=False):
    """Galerkin matrix B_m [K, K] and right-hand sides [..., K] of the geopotential
    equation at order m for one pole, from the input coefficients U_m = (Phi0, zeta0,
    delta0) [..., 3, K] of that order."""
    a, om, pb = c.radius, c.omega, c.phibar
    P, H = alp(m, N, mu)  # [K, nlat]; H = (1 - mu^2) dP/dmu
    ns = np.arange(m, N + 1)
    f = 2.0 * om * (np.ones_like(mu) if fsphere else mu)
    g = 0.0 if fsphere else 2.0 * om / a  # d f / d y times 1/cos(phi): grad f = (0, g cos(phi))
    D = alpha * alpha + tau * tau * f * f
    im = 1j * m
    lap = np.zeros(ns.size)
    lap[ns > 0] = -ns[ns > 0] * (ns[ns > 0] + 1.0) / a ** 2
    # operator applied to every basis function, on the latitudes: [K (basis), nlat]
    BP = (alpha * D * D * P
          - tau * tau * pb * (D * (alpha * lap[:, None] * P + tau * (g / a) * im * P)
                              - 2.0 * tau * tau * f * (g / a) * (alpha * H + tau * f * im * P)))
    Bm = (BP * w) @ P.T  # Bm[n', n] = sum_j P_n'(mu_j) w_j (B P_n)(mu_j); row = test degree
    Bm = Bm.T.copy()     # rows: projected degree, columns: basis degree
    # right-hand side on the latitudes
    Phi0, zeta0, delta0 = U_m[..., 0, :], U_m[..., 1, :], U_m[..., 2, :]
    inv = np.zeros(ns.size)
    inv[ns > 0] = -a * a / (ns[ns > 0] * (ns[ns > 0] + 1.0))
    psi, chi = zeta0 * inv, delta0 * inv
    U0 = (-(psi @ H) + im * (chi @ P)) / a
    V0 = (im * (psi @ P) + (chi @ H)) / a
    Phg, zg, dg = Phi0 @ P, zeta0 @ P, delta0 @ P
    rhs_g = (D * D * Phg
             + tau * pb * (D * (alpha * dg - tau * f * zg + tau * g * U0)
                           - 2.0 * tau * tau * f * g * (alpha * V0 + tau * f * U0)))
    rhs = rhs_g @ (P * w).T
    return Bm, rhs, (P, H, f, D, U0, V0)


def rexi_step_phi(U, N, nlat, alpha, beta, tau, c=Consts(), fsphere=False, ms=None, recover="physical"):
    """sum_k beta_k (alpha_k + tau L)^{-1} U through the geopotential-only system, for
    spectral states U [..., 3, nspec]; the m = 0 result is made real.

    ``recover="physical"`` follows the paper: velocities V = A^{-1}(V0 + tau grad Phi)
    pointwise in latitude, then their curl and divergence.  ``recover="spectral"`` takes
    delta from the Phi row of the system, delta = (alpha Phi - Phi0) / (tau Phibar), and
    zeta from its zeta row, zeta_n = (zeta0_n + 2 Omega tau (c_n delta_{n-1} + d_n delta_{n+1}))
    / (alpha + i tau sigma_n) (the spectral operator of Eq. (1)); this is the form the GPU
    path uses, with no per-pole transforms."""
    U = np.asarray(U, dtype=np.complex128)
    mu, w = gauss_legendre(nlat)
    a = c.radius
    out = np.zeros_like(U)
    ms = range(N + 1) if ms is None else ms
    sc = w / (1.0 - mu * mu) / a
    q = 2.0 * c.omega * tau
    for m in ms:
        sl = slice(idx(m, m, N), idx(m, N, N) + 1)
        U_m = U[..., :, sl]
        acc = np.zeros_like(U_m)
        ns, sig, ct, dt, _ = coupling(m, N, c)
        if fsphere:
            sig = np.zeros_like(sig)
        for al, be in zip(alpha, beta):
            Bm, rhs, (P, H, f, D, U0, V0) = phi_matrix_and_rhs(m, N, mu, w, al, tau, c, U_m, fsphere)
            Phi = np.linalg.solve(Bm, rhs.reshape(-1, rhs.shape[-1]).T).T.reshape(rhs.shape)
            if recover == "physical":
                # velocities pointwise in latitude: V = A^{-1} (V0 + tau grad Phi), Robert-scaled
                Phg = Phi @ P
                Wu = U0 + tau * (1j * m) * Phg / a
                Wv = V0 + tau * (Phi @ H) / a
                Uk = (al * Wu - tau * f * Wv) / D
                Vk = (tau * f * Wu + al * Wv) / D
                zeta = 1j * m * (Vk @ (P * sc).T) + Uk @ (H * sc).T
                delta = 1j * m * (Uk @ (P * sc).T) - Vk @ (H * sc).T
            else:
                delta = (al * Phi - U_m[..., 0, :]) / (tau * c.phibar)
                delta[..., ns == 0] = 0.0
                dm = np.zeros_like(delta)
                dp = np.zeros_like(delta)
                dm[..., 1:] = delta[..., :-1]
                dp[..., :-1] = delta[..., 1:]
                if fsphere:
                    zeta = (U_m[..., 1, :] + q * delta) / al
                else:
                    zeta = (U_m[..., 1, :] + q * (ct * dm + dt * dp)) / (al + 1j * tau * sig)
                zeta[..., ns == 0] = 0.0
            acc[..., 0, :] += be * Phi
            acc[..., 1, :] += be * zeta
            acc[..., 2, :] += be * delta
        if m == 0:
            acc = acc.real.astype(np.complex128)
            acc[..., 1:, 0] = 0.0  # zeta_0^0, delta_0^0 are not state
        out[..., :, sl] = acc
    return out
