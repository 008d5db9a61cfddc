// Host-side plan math of librexi: Gauss-Legendre nodes and the T-REXI
// coefficients (paper Sec. 4.1, renormalisation of Sec. 6.1).
//
// The paper takes mu and a_l of the Gaussian rational approximation
//   psi(y) = (4 pi)^{-1/2} exp(-y^2/4) ~ Re sum_{l=-K}^{K} a_l / (i y + mu + i l),  K = 11,
// from Haut et al.'s Table 1, which is not available; they are refitted here:
// for a fixed mu the fit is linear least squares in (Re a_l, Im a_l), solved by
// Householder QR on dense samples y in [-60, 60], and mu < 0 minimises the
// sampled sup error by golden-section search.  The exponential is expanded in
// shifted Gaussians with b_m = e^{h^2} e^{-i m h} (Poisson summation of the
// Gaussian), and the poles applied to the real SWE are the real-part set
//   alpha_n = h (mu + i n),  beta_n = h sum_{l+m=n} Re(b_m) a_l,
// n = -(M+K)..(M+K), optionally renormalised so that sum beta/alpha = 1.
#include <cmath>
#include <mutex>

#include "rexi_internal.h"

namespace rexi {

void gauss_legendre_host(int nlat, std::vector<double> &mu, std::vector<double> &w) {
  // Newton iteration on the Legendre polynomial P_nlat from the three-term
  // recurrence; nodes descending (north to south), weights 2/((1-x^2) P'^2).
  mu.assign(nlat, 0.0);
  w.assign(nlat, 0.0);
  for (int k = 0; k < nlat; ++k) {
    double x = std::cos(M_PI * (k + 0.75) / (nlat + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int n = 2; n <= nlat; ++n) {
        double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
        p0 = p1;
        p1 = p2;
      }
      dp = nlat * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double p0 = 1.0, p1 = x;
    for (int n = 2; n <= nlat; ++n) {
      double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
      p0 = p1;
      p1 = p2;
    }
    dp = nlat * (x * p1 - p0) / (x * x - 1.0);
    mu[k] = x;
    w[k] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

namespace {

constexpr int kNl = 2 * kGaussTerms + 1;  // 23 complex unknowns
constexpr int kNc = 2 * kNl;              // 46 real unknowns
constexpr int kNs = 6001;                 // samples on [-60, 60]

double psi(double y) { return std::exp(-0.25 * y * y) / std::sqrt(4.0 * M_PI); }
double ysample(int s) { return -60.0 + 120.0 * s / (kNs - 1); }

// Least-squares fit for fixed mu by Householder QR of the kNs x kNc design matrix
// with columns Re[1/(i y + mu + i l)] and Re[i/(i y + mu + i l)].
void fit_fixed(double mu, cplx *a, double *sup) {
  std::vector<double> A((size_t)kNs * kNc), b(kNs);
  for (int s = 0; s < kNs; ++s) {
    double y = ysample(s);
    for (int li = 0; li < kNl; ++li) {
      double t = y + (li - kGaussTerms);
      double den = mu * mu + t * t;
      A[(size_t)li * kNs + s] = mu / den;
      A[(size_t)(li + kNl) * kNs + s] = t / den;
    }
    b[s] = psi(y);
  }
  // Householder QR, column-major A.
  for (int k = 0; k < kNc; ++k) {
    double *col = &A[(size_t)k * kNs];
    double nrm = 0.0;
    for (int s = k; s < kNs; ++s) nrm += col[s] * col[s];
    nrm = std::sqrt(nrm);
    double alpha = col[k] > 0 ? -nrm : nrm;
    double v0 = col[k] - alpha;
    // v = (v0, col[k+1:]); H = I - 2 v v^T / (v^T v)
    double vtv = v0 * v0;
    for (int s = k + 1; s < kNs; ++s) vtv += col[s] * col[s];
    if (vtv == 0.0) continue;
    auto apply = [&](double *x) {
      double d = v0 * x[k];
      for (int s = k + 1; s < kNs; ++s) d += col[s] * x[s];
      double f = 2.0 * d / vtv;
      x[k] -= f * v0;
      for (int s = k + 1; s < kNs; ++s) x[s] -= f * col[s];
    };
    for (int j = k + 1; j < kNc; ++j) apply(&A[(size_t)j * kNs]);
    apply(b.data());
    col[k] = alpha;
  }
  double c[kNc];
  for (int k = kNc - 1; k >= 0; --k) {
    double acc = b[k];
    for (int j = k + 1; j < kNc; ++j) acc -= A[(size_t)j * kNs + k] * c[j];
    c[k] = acc / A[(size_t)k * kNs + k];
  }
  for (int li = 0; li < kNl; ++li) a[li] = cplx(c[li], c[li + kNl]);
  // the least-squares solution is conjugate-symmetric in l up to rounding
  cplx sym[kNl];
  for (int li = 0; li < kNl; ++li) sym[li] = 0.5 * (a[li] + std::conj(a[kNl - 1 - li]));
  for (int li = 0; li < kNl; ++li) a[li] = sym[li];
  double e = 0.0;
  for (int s = 0; s < kNs; ++s) {
    double y = ysample(s);
    double re = 0.0;
    for (int li = 0; li < kNl; ++li) {
      cplx d(mu, y + (li - kGaussTerms));
      re += (a[li] / d).real();
    }
    e = std::fmax(e, std::fabs(re - psi(y)));
  }
  *sup = e;
}

GaussFit compute_fit() {
  GaussFit f{};
  cplx a[kNl];
  double lo = -8.0, hi = -2.0, e1, e2;
  const double g = (std::sqrt(5.0) - 1.0) / 2.0;
  double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
  fit_fixed(x1, a, &e1);
  fit_fixed(x2, a, &e2);
  for (int it = 0; it < 48; ++it) {
    if (e1 < e2) {
      hi = x2; x2 = x1; e2 = e1;
      x1 = hi - g * (hi - lo);
      fit_fixed(x1, a, &e1);
    } else {
      lo = x1; x1 = x2; e1 = e2;
      x2 = lo + g * (hi - lo);
      fit_fixed(x2, a, &e2);
    }
  }
  f.mu = 0.5 * (lo + hi);
  fit_fixed(f.mu, f.a, &f.sup_err);
  return f;
}

}  // namespace

const GaussFit &gauss_fit() {
  static GaussFit fit;
  static std::once_flag once;
  std::call_once(once, [] { fit = compute_fit(); });
  return fit;
}

void rexi_coeffs_host(int M, double h, bool normalize, std::vector<cplx> &alpha,
                      std::vector<cplx> &beta, double *eps) {
  const GaussFit &f = gauss_fit();
  const int J = M + kGaussTerms, P = 2 * J + 1;
  alpha.assign(P, cplx(0, 0));
  beta.assign(P, cplx(0, 0));
  const double eh = std::exp(h * h);
  for (int m = -M; m <= M; ++m) {
    const double rb = eh * std::cos(m * h);  // Re(b_m)
    for (int l = -kGaussTerms; l <= kGaussTerms; ++l) beta[l + m + J] += h * rb * f.a[l + kGaussTerms];
  }
  for (int n = -J; n <= J; ++n) alpha[n + J] = cplx(h * f.mu, h * n);
  cplx s(0, 0);
  for (int k = 0; k < P; ++k) s += beta[k] / alpha[k];
  if (eps) *eps = 1.0 - s.real();
  if (normalize)
    for (int k = 0; k < P; ++k) beta[k] /= s;
}

}  // namespace rexi
