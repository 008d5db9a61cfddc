// The paper's geopotential-only solver (Sec. 4.3 and 5) as an alternative to the
// delta elimination, in binary64 or (REXI_SOLVE_FP32X2) float-float arithmetic.
//
// Per pole alpha (tau kept explicit, f = F mu with F = 2 Omega, g = 2 Omega / a):
//   alpha Phi - tau Phibar div V = Phi0,   A V = V0 + tau grad Phi,   D = alpha^2 + tau^2 f^2.
// Eliminating V and multiplying by D^2 gives an equation for Phi whose coefficients are
// polynomials in mu.  Galerkin-truncated to degrees m..N it is, per zonal order m,
//   B = b1 I + b2 Z2 + b3 Z3 + b4 lap + b5 Z2 lap + b6 Z6,
//   Z2 = P mu^2 P, Z3 = P mu^4 P, Z6 = P mu (1 - mu^2) d/dmu P, lap = -n(n+1)/a^2,
//   b1 = alpha^5 - tau^3 Phibar (g/a) i m alpha^2,  b2 = 2 tau^2 F^2 alpha^3 + tau^5 Phibar F^2 (g/a) i m,
//   b3 = tau^4 F^4 alpha,  b4 = -tau^2 Phibar alpha^3,  b5 = -tau^4 Phibar F^2 alpha,
//   b6 = 2 tau^4 Phibar F (g/a) alpha
// (the paper's Z_1 ... Z_8 split).  Z2, Z3, Z6 are real, pole-independent and couple
// n with n +- 2, n +- 4: a pentadiagonal complex system per (pole, m, parity of n - m),
// factorised per plan (banded LU, no pivoting).  The right-hand side is a polynomial in
// alpha with pole-independent coefficients,
//   rhs = Q4 alpha^4 + Q3 alpha^3 + Q2 alpha^2 + Q1 alpha + Q0,
//   Q4 = Phi0,  Q3 = tau Phibar delta0,
//   Q2 = 2 tau^2 F^2 mu^2 Phi0 - tau^2 Phibar F mu zeta0 + tau^2 Phibar g U0,
//   Q1 = tau^3 Phibar (F^2 mu^2 delta0 - 2 F g mu V0),
//   Q0 = tau^4 (F^4 mu^4 Phi0 - Phibar F^3 mu^3 zeta0 - Phibar F^2 g mu^2 U0),
// every product projected exactly with the Legendre recurrences (U0, V0 Robert winds
// from zeta0, delta0).  phi_rhs_kernel forms the Q_p once per step; per pole the
// solve evaluates rhs by Horner's rule.  delta and zeta come from the Phi and zeta rows
// of the system in spectral space, delta = (alpha Phi - Phi0) / (tau Phibar),
// zeta_n = (zeta0_n + 2 Omega tau (c_n delta_{n-1} + d_n delta_{n+1})) / (alpha + i tau sigma_n),
// so the beta-weighted sums need sum beta Phi, sum beta alpha Phi and the zeta couplings.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <type_traits>

#include "ff.h"
#include "rexi_internal.h"

namespace rexi {

namespace {

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double2 cscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {
  double re = fma(a.x, b.x, acc.x);
  re = fma(-a.y, b.y, re);
  double im = fma(a.x, b.y, acc.y);
  im = fma(a.y, b.x, im);
  return make_double2(re, im);
}
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b) {
  double re = fma(-a.x, b.x, acc.x);
  re = fma(a.y, b.y, re);
  double im = fma(-a.x, b.y, acc.y);
  im = fma(-a.y, b.x, im);
  return make_double2(re, im);
}
__device__ __forceinline__ double2 ld(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ int64_t base_of(int N, int m) { return (int64_t)m * (2 * N + 3 - m) / 2 - m; }

struct PhiConsts {
  double tau, phibar, F, g, radius, q;  // F = 2 Omega, g = 2 Omega / a, q = 2 Omega tau
};

// ---- plan time: B per (pole, system), banded LU, zeta coupling weights ----------------
struct PhiSetupArgs {
  const double *coef;  // [nspec][4] sigma, ct, dt, G
  const double *zc;    // [nspec][12] Z2(-2, 0, +2), Z3(-4 .. +4), Z6(-2, 0, +2)
  const double2 *alpha, *beta;
  double2 *fac;        // [7][nrows][P]: l1, l2, u1, u2, 1/u0, zeta weights zp, zm
                       // (float-float plans: [nrows][P][7], converted after this kernel)
  const int4 *sys;     // per (m, p): {m, n0, len, row0}
  int nsys, P, N;
  int64_t nrows;
  PhiConsts c;
  int interleaved;
};

__global__ void phi_factor_kernel(PhiSetupArgs a) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)a.P * a.nsys) return;
  const int k = (int)(t % a.P);
  const int4 sy = a.sys[t / a.P];
  const int m = sy.x, n0 = sy.y, len = sy.z;
  const int64_t row0 = sy.w;
  if (len <= 0) return;
  const int N = a.N;
  const PhiConsts c = a.c;
  const double2 al = a.alpha[k], be = a.beta[k];
  const double t2 = c.tau * c.tau, t3 = t2 * c.tau, t4 = t3 * c.tau, t5 = t4 * c.tau;
  const double F = c.F, F2 = F * F, pb = c.phibar, ga = c.g / c.radius;
  const double2 al2 = cmul(al, al), al3 = cmul(al2, al), al5 = cmul(cmul(al3, al), al);
  const double2 im = make_double2(0.0, (double)m);
  const double2 b1 = csub(al5, cscale(cmul(im, al2), t3 * pb * ga));
  const double2 b2 = cadd(cscale(al3, 2.0 * t2 * F2), cscale(im, t5 * pb * F2 * ga));
  const double2 b3 = cscale(al, t4 * F2 * F2);
  const double2 b4 = cscale(al3, -t2 * pb);
  const double2 b5 = cscale(al, -t4 * pb * F2);
  const double2 b6 = cscale(al, 2.0 * t4 * pb * F * ga);
  const double a2 = c.radius * c.radius;
  auto lap = [&](int n) { return -(double)n * (n + 1.0) / a2; };
  const int64_t base = base_of(N, m);
  const int64_t NR = a.nrows, P = a.P;
  auto put = [&](int comp, int64_t row, double2 v) {
    a.fac[a.interleaved ? (row * P + k) * 7 + comp : ((int64_t)comp * NR + row) * P + k] = v;
  };
  const double2 zero = make_double2(0, 0), one = make_double2(1, 0);
  const double2 bal = cmul(be, al);
  const double wz = c.q / (c.tau * pb);
  // rolling U entries of the two previous rows
  double2 u0m2 = one, u1m2 = zero, u2m2 = zero, u0m1 = one, u1m1 = zero, u2m1 = zero;
  for (int i = 0; i < len; ++i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base + n;
    const double *z = a.zc + 12 * ix;
    // B[i][i + d], d = -2 .. 2 (degree offsets 2d)
    double2 Bd[5];
    Bd[0] = cscale(b3, z[3]);
    Bd[1] = cadd(cadd(cscale(b2, z[0]), cscale(b3, z[4])), cadd(cscale(b5, z[0] * lap(n - 2)), cscale(b6, z[8])));
    Bd[2] = cadd(cadd(cadd(b1, cscale(b4, lap(n))), cadd(cscale(b2, z[1]), cscale(b3, z[5]))),
                 cadd(cscale(b5, z[1] * lap(n)), cscale(b6, z[9])));
    Bd[3] = cadd(cadd(cscale(b2, z[2]), cscale(b3, z[6])), cadd(cscale(b5, z[2] * lap(n + 2)), cscale(b6, z[10])));
    Bd[4] = cscale(b3, z[7]);
    // Doolittle on the band: L unit lower with two subdiagonals, U with two superdiagonals
    const double2 l2 = i >= 2 ? cdiv(Bd[0], u0m2) : zero;
    const double2 l1 = i >= 1 ? cdiv(csub(Bd[1], cmul(l2, u1m2)), u0m1) : zero;
    const double2 u0 = csub(csub(Bd[2], cmul(l1, u1m1)), cmul(l2, u2m2));
    const double2 u1 = csub(Bd[3], cmul(l1, u2m1));
    const double2 u2 = Bd[4];
    const int64_t row = row0 + i;
    put(0, row, l1);
    put(1, row, l2);
    put(2, row, u1);
    put(3, row, u2);
    put(4, row, cdiv(one, u0));
    // zeta_{n+1} (coupling c_{n+1} delta_n) and zeta_{n-1} (coupling d_{n-1} delta_n),
    // delta_n = (alpha Phi_n - Phi0_n) / (tau Phibar): the Phi_n weights
    double2 zp = zero, zm = zero;
    if (n + 1 <= N) {
      const double sg = a.coef[4 * (ix + 1) + 0], ct = a.coef[4 * (ix + 1) + 1];
      zp = cscale(cdiv(bal, make_double2(al.x, al.y + c.tau * sg)), wz * ct);
    }
    if (n - 1 >= m) {
      const double sg = a.coef[4 * (ix - 1) + 0], dt = a.coef[4 * (ix - 1) + 2];
      zm = cscale(cdiv(bal, make_double2(al.x, al.y + c.tau * sg)), wz * dt);
    }
    put(5, row, zp);
    put(6, row, zm);
    u0m2 = u0m1; u1m2 = u1m1; u2m2 = u2m1;
    u0m1 = u0; u1m1 = u1; u2m1 = u2;
  }
}

// ---- per step: the pole-independent right-hand-side coefficients Q_p -------------------
struct PhiRhsArgs {
  const double2 *sin;  // [3][nspec][B]
  double2 *q;          // [5][nspec][B]  Q0 .. Q4 (float-float plans: float-float values)
  const int32_t *m_of;
  int N, B;
  int64_t nspec;
  PhiConsts c;
  int ff;
  int *err;            // device error word (DEV_ERR_RANGE)
};

__device__ __forceinline__ double eps_nm(int n, int m) {
  return n > m ? sqrt(((double)n * n - (double)m * m) / (4.0 * n * n - 1.0)) : 0.0;
}

// (mu x)_n = eps_n x_{n-1} + eps_{n+1} x_{n+1} on a window around degree k: in[j] holds
// degree k - O + j, out[j] degree k - O + 1 + j (j < L - 2); ew[i] = eps at degree k - 5 + i
template <int L, int O>
__device__ __forceinline__ void mu_apply(const double2 (&in)[L], double2 (&out)[L - 2], const double (&ew)[11]) {
#pragma unroll
  for (int j = 0; j < L - 2; ++j) {
    // degree n = k - O + 1 + j: eps_n = ew[6 - O + j], eps_{n+1} = ew[7 - O + j]
    out[j] = cadd(cscale(in[j], ew[6 - O + j]), cscale(in[j + 2], ew[7 - O + j]));
  }
}

__global__ void phi_rhs_kernel(PhiRhsArgs a) {
  const int64_t total = a.nspec * a.B;
  const int N = a.N, B = a.B;
  const PhiConsts c = a.c;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % B);
    const int64_t ix = t / B;
    const int m = a.m_of[ix];
    const int64_t base = base_of(N, m);
    const int k = (int)(ix - base);
    auto X = [&](int f, int n) -> double2 {
      return (n >= m && n <= N) ? a.sin[((int64_t)f * a.nspec + base + n) * B + b] : make_double2(0, 0);
    };
    const double rad = c.radius;
    auto stream_fn = [&](int f, int n) -> double2 {  // psi_n (f = 1) or chi_n (f = 2) = -a^2 x_n / (n(n+1))
      if (n < m || n > N || n == 0) return make_double2(0, 0);
      return cscale(X(f, n), -rad * rad / ((double)n * (n + 1.0)));
    };
    // eps at degrees k - 5 .. k + 5, once per output
    double ew[11];
#pragma unroll
    for (int i = 0; i < 11; ++i) ew[i] = eps_nm(k - 5 + i, m);
    // Phi0 at k-4 .. k+4 -> mu^2 Phi0, mu^4 Phi0 at k
    double2 p9[9], p7[7], p5[5], p3[3], p1[1];
#pragma unroll
    for (int j = 0; j < 9; ++j) p9[j] = X(0, k - 4 + j);
    mu_apply<9, 4>(p9, p7, ew);
    mu_apply<7, 3>(p7, p5, ew);
    mu_apply<5, 2>(p5, p3, ew);
    mu_apply<3, 1>(p3, p1, ew);
    const double2 m2p = p5[2], m4p = p1[0];
    // zeta0 at k-3 .. k+3 -> mu zeta0, mu^3 zeta0 at k
    double2 z7[7], z5[5], z3[3], z1[1];
#pragma unroll
    for (int j = 0; j < 7; ++j) z7[j] = X(1, k - 3 + j);
    mu_apply<7, 3>(z7, z5, ew);
    mu_apply<5, 2>(z5, z3, ew);
    mu_apply<3, 1>(z3, z1, ew);
    const double2 mz = z5[2], m3z = z1[0];
    // delta0 at k-2 .. k+2 -> mu^2 delta0 at k
    double2 d5[5], d3[3], d1[1];
#pragma unroll
    for (int j = 0; j < 5; ++j) d5[j] = X(2, k - 2 + j);
    mu_apply<5, 2>(d5, d3, ew);
    mu_apply<3, 1>(d3, d1, ew);
    const double2 m2d = d1[0];
    // Robert winds: U_n = (1/a)[(n-1) eps_n psi_{n-1} - (n+2) eps_{n+1} psi_{n+1} + i m chi_n],
    //               V_n = (1/a)[i m psi_n - (n-1) eps_n chi_{n-1} + (n+2) eps_{n+1} chi_{n+1}]
    double2 ps[7], ch[7];
#pragma unroll
    for (int j = 0; j < 7; ++j) {
      ps[j] = stream_fn(1, k - 3 + j);
      ch[j] = stream_fn(2, k - 3 + j);
    }
    const double fm = (double)m;
    double2 u5[5], u3[3], u1[1];
#pragma unroll
    for (int j = 0; j < 5; ++j) {
      const int n = k - 2 + j;
      const double e0 = ew[3 + j], e1 = ew[4 + j];  // eps_n, eps_{n+1}
      double2 v = cadd(cscale(ps[j], (n - 1.0) * e0), cscale(ps[j + 2], -(n + 2.0) * e1));
      v = cadd(v, make_double2(-fm * ch[j + 1].y, fm * ch[j + 1].x));
      u5[j] = cscale(v, 1.0 / rad);
    }
    mu_apply<5, 2>(u5, u3, ew);
    mu_apply<3, 1>(u3, u1, ew);
    const double2 U0 = u5[2], m2U = u1[0];
    double2 v3[3], v1[1];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      const int n = k - 1 + j;
      const double e0 = ew[4 + j], e1 = ew[5 + j];  // eps_n, eps_{n+1}
      double2 v = make_double2(-fm * ps[j + 2].y, fm * ps[j + 2].x);
      v = cadd(v, cadd(cscale(ch[j + 1], -(n - 1.0) * e0), cscale(ch[j + 3], (n + 2.0) * e1)));
      v3[j] = cscale(v, 1.0 / rad);
    }
    mu_apply<3, 1>(v3, v1, ew);
    const double2 mV = v1[0];
    const double tau = c.tau, pb = c.phibar, F = c.F, g = c.g;
    const double t2 = tau * tau, t3 = t2 * tau, t4 = t3 * tau;
    double2 Q[5];
    Q[4] = p9[4];
    Q[3] = cscale(d5[2], tau * pb);
    Q[2] = cadd(cadd(cscale(m2p, 2.0 * t2 * F * F), cscale(mz, -t2 * pb * F)), cscale(U0, t2 * pb * g));
    Q[1] = cadd(cscale(m2d, t3 * pb * F * F), cscale(mV, -2.0 * t3 * pb * F * g));
    Q[0] = cadd(cadd(cscale(m4p, t4 * F * F * F * F), cscale(m3z, -t4 * pb * F * F * F)),
                cscale(m2U, -t4 * pb * F * F * g));
#pragma unroll
    for (int p = 0; p < 5; ++p) {
      const int64_t o = ((int64_t)p * a.nspec + ix) * B + b;
      if (a.ff) {
        const float4 f = ff::csplit(Q[p]);
        if (ff::split_overflow(Q[p], f)) atomicOr(a.err, DEV_ERR_RANGE);
        reinterpret_cast<float4 *>(a.q)[o] = f;
      } else {
        a.q[o] = Q[p];
      }
    }
  }
}

// ---- per step: the pentadiagonal solves and the beta-weighted sums --------------------
struct PhiSolveArgs {
  const double2 *fac, *q, *alpha, *beta;
  const float4 *abf;  // float-float plans: alpha, beta, beta alpha per pole ([3][P])
  int ffil;           // float-float factors interleaved ([nrows][P][7]) or pole-fastest ([7][nrows][P])
  double2 *part;  // [3][nspec][slots][B]: (sum beta Phi, zeta couplings, sum beta alpha Phi)
  const int4 *sys;
  double2 *ybuf;
  const WorkItem *items;
  const int32_t *slots_m;  // per zonal order slot count (<= slots, the partial stride)
  unsigned *counter;
  int nitems, lmax, P, N, B, bw, kk, slots;
  int64_t nspec, nrows;
};

template <int KC>
__device__ __forceinline__ void phi_sweep(const PhiSolveArgs &a, const int (&k)[KC], int m, int n0, int len,
                                          int64_t row0, int64_t base, const double2 *qb, double2 *pP, double2 *pZ,
                                          double2 *pD, int64_t rstride, bool first, double2 *ybuf) {
  const int64_t NR = a.nrows, P = a.P, NS = a.nspec;
  const int N = a.N, B = a.B;
  double2 al[KC], be[KC], bal[KC];
  const double2 *fL1[KC], *fL2[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    al[c] = ld(a.alpha + k[c]);
    be[c] = ld(a.beta + k[c]);
    bal[c] = cmul(be[c], al[c]);
    fL1[c] = a.fac + (0 * NR + row0) * P + k[c];
    fL2[c] = a.fac + (1 * NR + row0) * P + k[c];
  }
  // forward: y_i = rhs_i - l1 y_{i-1} - l2 y_{i-2},  rhs = (((Q4 a + Q3) a + Q2) a + Q1) a + Q0
  double2 y1[KC], y2[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) y1[c] = y2[c] = make_double2(0, 0);
  for (int i = 0; i < len; ++i) {
    const int64_t ix = base + n0 + 2 * i;
    double2 Q[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) Q[p] = ld(qb + ((int64_t)p * NS + ix) * B);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      double2 r = cfma(Q[3], Q[4], al[c]);
      r = cfma(Q[2], r, al[c]);
      r = cfma(Q[1], r, al[c]);
      r = cfma(Q[0], r, al[c]);
      r = cfms(r, ld(fL1[c] + (int64_t)i * P), y1[c]);
      r = cfms(r, ld(fL2[c] + (int64_t)i * P), y2[c]);
      ybuf[((int64_t)i * KC + c) * 32] = r;
      y2[c] = y1[c];
      y1[c] = r;
    }
  }
  // backward: x_i = (y_i - u1 x_{i+1} - u2 x_{i+2}) / u0, with the sums
  const double2 *fU1[KC], *fU2[KC], *fIU[KC], *fZP[KC], *fZM[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    fU1[c] = a.fac + (2 * NR + row0) * P + k[c];
    fU2[c] = a.fac + (3 * NR + row0) * P + k[c];
    fIU[c] = a.fac + (4 * NR + row0) * P + k[c];
    fZP[c] = a.fac + (5 * NR + row0) * P + k[c];
    fZM[c] = a.fac + (6 * NR + row0) * P + k[c];
  }
  double2 x1[KC], x2[KC], zmn[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) x1[c] = x2[c] = zmn[c] = make_double2(0, 0);
  for (int i = len - 1; i >= 0; --i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base + n;
    double2 xv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      double2 r = ybuf[((int64_t)i * KC + c) * 32];
      r = cfms(r, ld(fU1[c] + (int64_t)i * P), x1[c]);
      r = cfms(r, ld(fU2[c] + (int64_t)i * P), x2[c]);
      xv[c] = cmul(r, ld(fIU[c] + (int64_t)i * P));
    }
    double2 accP = first ? make_double2(0, 0) : pP[ix * rstride];
    double2 accD = first ? make_double2(0, 0) : pD[ix * rstride];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      accP = cfma(accP, be[c], xv[c]);
      accD = cfma(accD, bal[c], xv[c]);
    }
    pP[ix * rstride] = accP;
    pD[ix * rstride] = accD;
    if (n + 1 <= N) {
      double2 accZ = first ? make_double2(0, 0) : pZ[(ix + 1) * rstride];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        accZ = cfma(accZ, ld(fZP[c] + (int64_t)i * P), xv[c]);
        accZ = cfma(accZ, zmn[c], x1[c]);
      }
      pZ[(ix + 1) * rstride] = accZ;
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      zmn[c] = ld(fZM[c] + (int64_t)i * P);
      x2[c] = x1[c];
      x1[c] = xv[c];
    }
  }
  if (n0 - 1 >= m) {
    const int64_t ix = base + n0 - 1;
    double2 accZ = first ? make_double2(0, 0) : pZ[ix * rstride];
#pragma unroll
    for (int c = 0; c < KC; ++c) accZ = cfma(accZ, zmn[c], x1[c]);
    pZ[ix * rstride] = accZ;
  }
}

// The same sweeps in float-float arithmetic (ff.h) on the FP32 pipes: factors
// [nrows][P][7], right-hand-side coefficients, sweep intermediates and slot partials
// hold float-float values in their double2 slots; each row's data is prefetched into
// L2 three rows ahead.
__device__ __forceinline__ void l2_prefetch(const void *p) { asm volatile("prefetch.global.L2 [%0];" : : "l"(p)); }

template <int KC, bool IL>
__device__ __forceinline__ void phi_sweep_ff(const PhiSolveArgs &a, const int (&k)[KC], int m, int n0, int len,
                                             int64_t row0, int64_t base, const float4 *qb, float4 *pP, float4 *pZ,
                                             float4 *pD, int64_t rstride, bool first, float4 *ybuf) {
  constexpr int D = 3;  // rows prefetched ahead into L2
  // factor (comp, row i, pole c) at fk[c] + i RS + comp CS: interleaved (IL) rows of P x 7
  // values, or the pole-fastest layout [7][nrows][P]
  const int64_t NS = a.nspec, RS = IL ? (int64_t)a.P * 7 : (int64_t)a.P, CS = IL ? 1 : a.nrows * a.P;
  const int N = a.N, B = a.B;
  float4 al[KC], be[KC], bal[KC];
  const float4 *fk[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    al[c] = a.abf[k[c]];
    be[c] = a.abf[a.P + k[c]];
    bal[c] = a.abf[2 * a.P + k[c]];
    fk[c] = reinterpret_cast<const float4 *>(a.fac) + (IL ? (row0 * a.P + k[c]) * 7 : row0 * a.P + k[c]);
  }
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  auto pf_fwd = [&](int i) {
    const int64_t ix = base + n0 + 2 * i;
#pragma unroll
    for (int p = 0; p < 5; ++p) l2_prefetch(qb + ((int64_t)p * NS + ix) * B);
#pragma unroll
    for (int c = 0; c < KC; ++c) {  // factors 0 and 1
      l2_prefetch(fk[c] + (int64_t)i * RS);
      l2_prefetch(fk[c] + (int64_t)i * RS + CS);
    }
  };
  auto pf_bwd = [&](int i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base + n;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;  // factors 2..6
      if (IL) {
        l2_prefetch(f + 2);
        l2_prefetch(f + 6);
      } else {
#pragma unroll
        for (int q = 2; q <= 6; ++q) l2_prefetch(f + q * CS);
      }
      l2_prefetch(ybuf + ((int64_t)i * KC + c) * 32);
    }
    if (!first) {
      l2_prefetch(pP + ix * rstride);
      l2_prefetch(pD + ix * rstride);
      if (n + 1 <= N) l2_prefetch(pZ + (ix + 1) * rstride);
    }
  };
  // forward: y_i = rhs_i - l1 y_{i-1} - l2 y_{i-2},  rhs = (((Q4 a + Q3) a + Q2) a + Q1) a + Q0
  float4 y1[KC], y2[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) y1[c] = y2[c] = zero;
  for (int j = 1; j <= D && j < len; ++j) pf_fwd(j);
  for (int i = 0; i < len; ++i) {
    if (i + D < len) pf_fwd(i + D);
    const int64_t ix = base + n0 + 2 * i;
    float4 Q[5];
#pragma unroll
    for (int p = 0; p < 5; ++p) Q[p] = __ldg(qb + ((int64_t)p * NS + ix) * B);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;
      ff::CAcc r = ff::cacc(Q[3]);
      ff::cmac(r, Q[4], al[c]);
#pragma unroll
      for (int p = 2; p >= 0; --p) {
        ff::CAcc r2 = ff::cacc(Q[p]);
        ff::cmac(r2, ff::raw(r), al[c]);
        r = r2;
      }
      ff::cmsub(r, __ldg(f + 0 * CS), y1[c]);
      ff::cmsub(r, __ldg(f + 1 * CS), y2[c]);
      const float4 yv = ff::raw(r);
      ybuf[((int64_t)i * KC + c) * 32] = yv;
      y2[c] = y1[c];
      y1[c] = yv;
    }
  }
  // backward: x_i = (y_i - u1 x_{i+1} - u2 x_{i+2}) / u0, with the sums
  float4 x1[KC], x2[KC], zmn[KC];
#pragma unroll
  for (int c = 0; c < KC; ++c) x1[c] = x2[c] = zmn[c] = zero;
  for (int j = len - 2; j >= 0 && j >= len - 1 - D; --j) pf_bwd(j);
  for (int i = len - 1; i >= 0; --i) {
    if (i - D >= 0) pf_bwd(i - D);
    const int n = n0 + 2 * i;
    const int64_t ix = base + n;
    float4 xv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;
      ff::CAcc r = ff::cacc(ybuf[((int64_t)i * KC + c) * 32]);
      ff::cmsub(r, __ldg(f + 2 * CS), x1[c]);
      ff::cmsub(r, __ldg(f + 3 * CS), x2[c]);
      ff::CAcc x = ff::czero();
      ff::cmac(x, ff::raw(r), __ldg(f + 4 * CS));
      xv[c] = ff::raw(x);
    }
    ff::CAcc accP = first ? ff::czero() : ff::cacc(pP[ix * rstride]);
    ff::CAcc accD = first ? ff::czero() : ff::cacc(pD[ix * rstride]);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      ff::cmac(accP, be[c], xv[c]);
      ff::cmac(accD, bal[c], xv[c]);
    }
    pP[ix * rstride] = ff::raw(accP);
    pD[ix * rstride] = ff::raw(accD);
    if (n + 1 <= N) {
      ff::CAcc accZ = first ? ff::czero() : ff::cacc(pZ[(ix + 1) * rstride]);
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        ff::cmac(accZ, __ldg(fk[c] + (int64_t)i * RS + 5 * CS), xv[c]);
        ff::cmac(accZ, zmn[c], x1[c]);
      }
      pZ[(ix + 1) * rstride] = ff::raw(accZ);
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      zmn[c] = __ldg(fk[c] + (int64_t)i * RS + 6 * CS);
      x2[c] = x1[c];
      x1[c] = xv[c];
    }
  }
  if (n0 - 1 >= m) {
    const int64_t ix = base + n0 - 1;
    ff::CAcc accZ = first ? ff::czero() : ff::cacc(pZ[ix * rstride]);
#pragma unroll
    for (int c = 0; c < KC; ++c) ff::cmac(accZ, zmn[c], x1[c]);
    pZ[ix * rstride] = ff::raw(accZ);
  }
}

// float-float: capped at 128 registers (four CTAs per SM); a few spilled bytes cost less
// than the fourth CTA gains (14.5 against 15.3 ms at T341 with 16 states)
template <bool FF>
__global__ void __launch_bounds__(128, FF ? 4 : 1) phi_solve_kernel(PhiSolveArgs a) {
  const int lane = threadIdx.x & 31;
  const int wslot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double2 *ybuf = a.ybuf + (int64_t)wslot * a.lmax * 2 * 32 + lane;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(a.counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)a.nitems) break;
    const WorkItem w = a.items[it];
    const int bl = lane % a.bw;
    const int p = (lane / a.bw) & 1;
    const int kk = lane / (2 * a.bw);
    const int b = w.b0 + bl;
    const int4 sy = a.sys[2 * w.m + p];
    const int m = sy.x, n0 = sy.y, len = sy.z;
    const int slot = w.g * a.kk + kk;
    const int Sm = a.slots_m[m];
    if (kk >= a.kk || b >= a.B || len <= 0 || slot >= Sm) continue;
    const int64_t NS = a.nspec, S = a.slots, B = a.B;
    const int64_t base = base_of(a.N, m);
    double2 *pP = a.part + (int64_t)slot * B + b;
    double2 *pZ = pP + NS * S * B;
    double2 *pD = pP + 2 * NS * S * B;
    const int64_t rstride = S * B;
    const double2 *qb = a.q + b;
    bool first = true;
    int k0 = slot;
    if constexpr (FF) {
      const float4 *fq = reinterpret_cast<const float4 *>(qb);
      float4 *fP = reinterpret_cast<float4 *>(pP), *fZ = reinterpret_cast<float4 *>(pZ),
             *fD = reinterpret_cast<float4 *>(pD), *fy = reinterpret_cast<float4 *>(ybuf);
      auto sweeps = [&](auto il) {
        constexpr bool IL = decltype(il)::value;
        for (; k0 + Sm < a.P; k0 += 2 * Sm) {
          const int kp[2] = {k0, k0 + Sm};
          phi_sweep_ff<2, IL>(a, kp, m, n0, len, sy.w, base, fq, fP, fZ, fD, rstride, first, fy);
          first = false;
        }
        if (k0 < a.P) {
          const int kp[1] = {k0};
          phi_sweep_ff<1, IL>(a, kp, m, n0, len, sy.w, base, fq, fP, fZ, fD, rstride, first, fy);
        }
      };
      if (a.ffil) sweeps(std::true_type{});
      else sweeps(std::false_type{});
    } else {
      for (; k0 + Sm < a.P; k0 += 2 * Sm) {
        const int kp[2] = {k0, k0 + Sm};
        phi_sweep<2>(a, kp, m, n0, len, sy.w, base, qb, pP, pZ, pD, rstride, first, ybuf);
        first = false;
      }
      if (k0 < a.P) {
        const int kp[1] = {k0};
        phi_sweep<1>(a, kp, m, n0, len, sy.w, base, qb, pP, pZ, pD, rstride, first, ybuf);
      }
    }
  }
}

// ---- per step: ordered slot sums and the pole-independent terms ------------------------
struct PhiReduceArgs {
  const double2 *part, *sin;
  double2 *sout;
  const uint8_t *rflags;  // [3][nspec]: bit0 partials present, bit1 forced zero
  const double2 *w;       // [nspec] sum_k beta_k / (alpha_k + i tau sigma_n)
  const double *coef;     // [nspec][4]
  const int32_t *m_of;
  const int32_t *slots_m; // per zonal order slot count (<= slots, the partial stride)
  double2 sumb;           // sum_k beta_k
  int slots, B, N;
  int64_t nspec;
  double inv_tp, qz;      // 1 / (tau Phibar), 2 Omega tau / (tau Phibar)
};

template <bool FF>
__global__ void phi_reduce_kernel(PhiReduceArgs a) {
  const int64_t total = 3 * a.nspec * a.B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % a.B);
    const int64_t fi = t / a.B;
    const int f = (int)(fi / a.nspec);
    const int64_t ix = fi - (int64_t)f * a.nspec;
    const uint8_t fl = a.rflags[fi];
    double2 acc = make_double2(0, 0);
    if (!(fl & 2)) {
      if (fl & 1) {
        const int Sm = a.slots_m[a.m_of[ix]];
        if constexpr (FF) {  // float-float partials added in slot order, rounded once
          const float4 *p = reinterpret_cast<const float4 *>(a.part) + fi * a.slots * a.B + b;
          ff::CAcc fa = ff::czero();
          for (int s = 0; s < Sm; ++s) ff::cadd(fa, __ldcs(p + (int64_t)s * a.B));
          acc = make_double2(f32_to_f64(fa.re.s) + f32_to_f64(fa.re.e), f32_to_f64(fa.im.s) + f32_to_f64(fa.im.e));
        } else {
          const double2 *p = a.part + fi * a.slots * a.B + b;
          int s = 0;
          for (; s + 8 <= Sm; s += 8) {
            double2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(p + (int64_t)(s + u) * a.B);
#pragma unroll
            for (int u = 0; u < 8; ++u) acc = cadd(acc, v[u]);
          }
          for (; s < Sm; ++s) acc = cadd(acc, p[(int64_t)s * a.B]);
        }
      }
      const int64_t NB = a.nspec * a.B;
      const int64_t sb = ix * a.B + b;
      if (f == 2) {  // delta = (sum beta alpha Phi - sum beta Phi0) / (tau Phibar)
        acc = cscale(csub(acc, cmul(a.sumb, a.sin[sb])), a.inv_tp);
      } else if (f == 1) {  // zeta: W zeta0 - (q / (tau Phibar)) W (c_n Phi0_{n-1} + d_n Phi0_{n+1})
        const double ct = a.coef[4 * ix + 1], dt = a.coef[4 * ix + 2];
        double2 ph = make_double2(0, 0);
        if (ct != 0.0) ph = cadd(ph, cscale(a.sin[sb - a.B], ct));
        if (dt != 0.0) ph = cadd(ph, cscale(a.sin[sb + a.B], dt));
        const double2 wv = a.w[ix];
        acc = cadd(acc, cmul(wv, a.sin[NB + sb]));
        acc = csub(acc, cscale(cmul(wv, ph), a.qz));
      }
      if (a.m_of[ix] == 0) acc.y = 0.0;
    }
    a.sout[t] = acc;
  }
}

}  // namespace

namespace {
PhiConsts phi_consts(const Plan &pl) {
  return PhiConsts{pl.prm.tau, pl.prm.gravity * pl.prm.mean_depth, 2.0 * pl.prm.omega,
                   2.0 * pl.prm.omega / pl.prm.radius, pl.prm.radius, 2.0 * pl.prm.omega * pl.prm.tau};
}
}  // namespace

cudaError_t launch_phi_factor(Plan &pl, cudaStream_t st) {
  PhiSetupArgs a;
  a.coef = pl.coef_dev;
  a.zc = pl.phi_zc;
  a.alpha = pl.alpha_dev;
  a.beta = pl.beta_dev;
  a.fac = pl.fac_fwd;
  a.sys = pl.sys_dev;
  a.nsys = (int)pl.sys.size();
  a.P = pl.P;
  a.N = pl.N;
  a.nrows = pl.nrows;
  a.c = phi_consts(pl);
  a.interleaved = pl.ffil ? 1 : 0;
  const int64_t total = (int64_t)a.P * a.nsys;
  phi_factor_kernel<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && pl.ff) e = launch_to_ff(pl, pl.fac_fwd, (int64_t)7 * pl.nrows * pl.P, st);
  return e;
}

// right-hand sides Q_p, then the persistent pentadiagonal solve into the slot partials
cudaError_t launch_phi_solve(Plan &pl, const SolveLayout &lay, const double2 *sin, int B, cudaStream_t st) {
  const PhiConsts c = phi_consts(pl);
  {
    PhiRhsArgs r{sin, pl.phi_q, pl.m_of_dev, pl.N, B, pl.nspec, c, pl.ff ? 1 : 0, pl.dev_err};
    const int64_t total = pl.nspec * B;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, (int64_t)pl.num_sms * 16));
    phi_rhs_kernel<<<blocks, 128, 0, st>>>(r);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  {
    PhiSolveArgs s;
    s.fac = pl.fac_fwd;
    s.q = pl.phi_q;
    s.alpha = pl.alpha_dev;
    s.beta = pl.beta_dev;
    s.abf = reinterpret_cast<const float4 *>(pl.phi_abf);
    s.ffil = pl.ffil ? 1 : 0;
    s.part = pl.partial;
    s.sys = pl.sys_dev;
    s.ybuf = pl.yscratch;
    s.items = lay.items_dev;
    s.slots_m = lay.slots_m_dev;
    s.counter = pl.counter;
    s.nitems = lay.nitems;
    s.lmax = pl.lmax;
    s.P = pl.P;
    s.N = pl.N;
    s.B = B;
    s.bw = lay.bw;
    s.kk = lay.kk;
    s.slots = lay.slots;
    s.nspec = pl.nspec;
    s.nrows = pl.nrows;
    cudaError_t e = cudaMemsetAsync(pl.counter, 0, sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    if (pl.ff) phi_solve_kernel<true><<<pl.resident_warps / 4, 128, 0, st>>>(s);
    else phi_solve_kernel<false><<<pl.resident_warps / 4, 128, 0, st>>>(s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_phi_reduce(Plan &pl, const SolveLayout &lay, const double2 *sin, double2 *sout, int B,
                              cudaStream_t st) {
  const PhiConsts c = phi_consts(pl);
  PhiReduceArgs r;
  r.part = pl.partial;
  r.sin = sin;
  r.sout = sout;
  r.rflags = pl.rflags_dev;
  r.w = pl.w_fwd;
  r.coef = pl.coef_dev;
  r.m_of = pl.m_of_dev;
  r.slots_m = lay.slots_m_dev;
  r.sumb = pl.sumb;
  r.slots = lay.slots;
  r.B = B;
  r.N = pl.N;
  r.nspec = pl.nspec;
  r.inv_tp = 1.0 / (c.tau * c.phibar);
  r.qz = c.q / (c.tau * c.phibar);
  const int64_t total = 3 * pl.nspec * B;
  const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)pl.num_sms * 8);
  if (pl.ff) phi_reduce_kernel<true><<<blocks, 256, 0, st>>>(r);
  else phi_reduce_kernel<false><<<blocks, 256, 0, st>>>(r);
  return cudaGetLastError();
}

}  // namespace rexi
