"""T-REXI coefficients (paper Sec. 4.1 and Sec. 6.1) -- oracle, FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Construction, in the paper's order and notation:

1. Gaussian rational approximation (Sec. 4.1, first block):
   psi_h(x) = (4 pi)^{-1/2} exp(-x^2/(4h^2)) ~ Re sum_{l=-K}^{K} a_l / (i x/h + mu + i l), K = 11.
   The paper takes mu and a_l from Haut et al., Table 1, which is not available
   here; they are refitted: for fixed mu the fit is linear least squares in
   (Re a_l, Im a_l) on dense samples of y = x/h, and mu < 0 is chosen by a
   golden-section search on the sup error (a reading: the table is missing).
2. Gaussian-basis expansion of the exponential (Sec. 4.1, second block):
   exp(i x) ~ sum_{m=-M}^{M} b_m psi_h(x + m h).  The paper prints no b_m;
   Poisson summation of the Gaussian gives b_m = exp(h^2) exp(-i m h)
   (error O(exp(-(2 pi - h)^2)) for |x| well inside [-hM, hM]).
3. Real part: Re(e^{ix}) ~ sum_m Re(b_m psi_h(x + m h))
   ~ sum_n Re( beta^Re_n / (i x + alpha_n) ) with
   alpha_n = h (mu + i n),  beta^Re_n = h sum_{l+m=n} Re(b_m) a_l,
   n = -(M+K) .. (M+K); the imaginary-part set beta^Im uses Im(b_m).
4. Merge (a reading of "merged"): the linear SWE operator and state are real, and
   for a real operator the conjugate-symmetric imaginary-part terms contribute
   exactly zero to Re(sum beta X); the coefficient set applied in Algorithm 1
   is beta_n = beta^Re_n.  With it the x = 0 residual
   eps = 1 - sum beta/alpha is O(1e-12), the order the paper prints for
   M = 128 (Sec. 6.1: -1.559352647e-11 with Haut's table at h = 0.15).
5. Renormalisation (Sec. 6.1): beta_n <- beta_n / (1 - eps) so the response at
   x = 0 is exactly one.

Pins: symmetry a_{-l} = conj(a_l) and the fit's sup error; the real part of
the response equals cos(x) to the fit level on |x| <= h(M-10); the x = 0
residual is of the printed order; the imaginary part obeys the closed-form
truncation bound derived from the Hilbert-transform tail of the b_m sum; and
conjugate symmetry alpha_{-n} = conj(alpha_n), beta_{-n} = conj(beta_n).
"""

import functools

import numpy as np

K_GAUSS = 11  # rational terms per side (the paper's K)


def psi(y):
    """Gaussian of Sec. 4.1 in the scaled variable y = x/h."""
    return np.exp(-0.25 * y * y) / np.sqrt(4.0 * np.pi)


def _design(mu, y):
    l = np.arange(-K_GAUSS, K_GAUSS + 1)
    t = y[:, None] + l[None, :]
    den = mu * mu + t * t
    # Re[(ar + i ai) / (i y + mu + i l)] = (ar mu + ai (y + l)) / (mu^2 + (y + l)^2)
    return np.hstack([mu / den, t / den])


_Y_FIT = np.linspace(-60.0, 60.0, 6001)


def _fit_fixed_mu(mu):
    A = _design(mu, _Y_FIT)
    c, *_ = np.linalg.lstsq(A, psi(_Y_FIT), rcond=None)
    a = c[: 2 * K_GAUSS + 1] + 1j * c[2 * K_GAUSS + 1:]
    return 0.5 * (a + np.conj(a[::-1]))  # the LS solution is symmetric up to rounding


def gaussian_rational(y, mu, a):
    """R(y) = sum_l a_l / (i y + mu + i l)."""
    l = np.arange(-K_GAUSS, K_GAUSS + 1)
    y = np.atleast_1d(np.asarray(y, dtype=np.float64))
    return (a[None, :] / (1j * y[:, None] + mu + 1j * l[None, :])).sum(axis=1)


def _sup_err(mu):
    a = _fit_fixed_mu(mu)
    return np.max(np.abs(gaussian_rational(_Y_FIT, mu, a).real - psi(_Y_FIT)))


@functools.lru_cache(maxsize=None)
def gaussian_fit():
    """Return (mu, a_l for l=-K..K, sup error on the fit samples)."""
    lo, hi = -8.0, -2.0
    g = (np.sqrt(5.0) - 1.0) / 2.0
    x1 = hi - g * (hi - lo)
    x2 = lo + g * (hi - lo)
    f1, f2 = _sup_err(x1), _sup_err(x2)
    for _ in range(48):
        if f1 < f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - g * (hi - lo)
            f1 = _sup_err(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + g * (hi - lo)
            f2 = _sup_err(x2)
    mu = 0.5 * (lo + hi)
    a = _fit_fixed_mu(mu)
    return mu, a, _sup_err(mu)


def b_coeffs(M, h):
    """b_m, m = -M..M, of exp(i x) ~ sum_m b_m psi_h(x + m h) (Poisson summation)."""
    m = np.arange(-M, M + 1)
    return np.exp(h * h) * np.exp(-1j * m * h)


def rexi_parts(M, h):
    """Return (alpha, beta_re, beta_im), each indexed n = -(M+K)..(M+K) ascending."""
    mu, a, _ = gaussian_fit()
    b = b_coeffs(M, h)
    J = M + K_GAUSS
    beta_re = np.zeros(2 * J + 1, dtype=np.complex128)
    beta_im = np.zeros(2 * J + 1, dtype=np.complex128)
    m = np.arange(-M, M + 1)
    for li, l in enumerate(range(-K_GAUSS, K_GAUSS + 1)):
        beta_re[l + m + J] += h * b.real * a[li]
        beta_im[l + m + J] += h * b.imag * a[li]
    n = np.arange(-J, J + 1)
    alpha = h * (mu + 1j * n)
    return alpha, beta_re, beta_im


def rexi_coefficients(M, h, normalize=True):
    """(alpha_n, beta_n) applied in Algorithm 1, n ascending; P = 2(M+K)+1 terms.

    Also returns eps = 1 - sum beta/alpha before renormalisation.
    """
    alpha, beta, _ = rexi_parts(M, h)
    eps = 1.0 - np.sum(beta / alpha)
    if normalize:
        beta = beta / np.sum(beta / alpha)
    return alpha, beta, eps


def response(alpha, beta, x):
    """Scalar REXI symbol  f(x) = sum_n beta_n / (i x + alpha_n)  (approximates e^{ix})."""
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    return (beta[None, :] / (1j * x[:, None] + alpha[None, :])).sum(axis=1)


def imag_tail_bound(x, M, h):
    """Closed-form bound on |Im f(x) - sin x| from truncating sum_m at |m| = M.

    For a one-sided rational function Im f is the Hilbert transform of Re f; the
    terms |m| > M dropped from sum_m Re(b_m) psi_h(x + m h) leave, paired as
    m and -m, e^{h^2} (2 y / pi) sum_{m>M} cos(m h) / (m^2 - y^2) with y = x/h,
    and |sum_{m>M} cos(m h)/m^2| <= 1 / (M^2 sin(h/2)) by Abel summation.
    Valid for |y| <= M/2; the factor 4/3 covers m^2 - y^2 >= 3 m^2/4.
    """
    y = np.abs(np.asarray(x, dtype=np.float64)) / h
    return np.exp(h * h) * (2.0 * y / np.pi) * (4.0 / 3.0) / (M * M * np.sin(0.5 * h))
