"""Exact frequencies of L over the real coordinates of the dispersion analysis."""
import numpy as np

from oracle import swe


def exact_frequencies(N, consts, fsphere=False):
    """omega for the eigenvalues i*omega of L, as a real map on ``real_coordinates(N)``."""
    from paper_1812_03431_gb300.dispersion import assemble, probe_states
    L = swe.dense_operator(N, consts, fsphere)  # complex, field-major [3 nspec]
    P = probe_states(N)
    nspec = P.shape[2]
    LP = (L @ P.reshape(len(P), 3 * nspec).T).T.reshape(P.shape)
    lam = np.linalg.eigvals(assemble(LP, N))
    return lam.imag, np.abs(lam.real).max()


def fsphere_frequencies(N, consts):
    """Closed-form frequencies on the f-sphere over the same real coordinates: degree n
    carries a steady mode and the gravity pair +-sqrt(f^2 + Phibar n(n+1)/a^2), f = 2 Omega;
    each m > 0 coefficient counts twice (real and imaginary parts); Phi_0^0 is steady."""
    f = 2.0 * consts.omega
    out = [0.0]
    for m in range(N + 1):
        for n in range(max(m, 1), N + 1):
            w = np.sqrt(f * f + consts.phibar * n * (n + 1) / consts.radius ** 2)
            out += [0.0, w, -w] * (1 if m == 0 else 2)
    return np.array(out)
