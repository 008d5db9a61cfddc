// Banded shifted solves and the beta-weighted pole sum (paper Sec. 4.2, Sec. 5,
// Algorithm 1), in binary64 or in float-float arithmetic (ff.h) on the FP32 pipes.
//
// Per zonal order m, (alpha + tau L_m) X = U couples (Phi_n, zeta_n, delta_n)
// with L_m of Eq. (1) in spectral form:
//   (L Phi)_n = -Phibar delta_n
//   (L zeta)_n = i sigma_n zeta_n - 2 Omega [c_n delta_{n-1} + d_n delta_{n+1}]
//   (L delta)_n = i sigma_n delta_n + 2 Omega [c_n zeta_{n-1} + d_n zeta_{n+1}] + G_n Phi_n
// Eliminating Phi_n (Phi row) and zeta_{n+-1} (zeta rows) leaves, for each
// parity of n - m, a complex tridiagonal system in delta over n, n +- 2.  This
// is the paper's banded matrix B of Sec. 5 reached by a different elimination
// (the paper multiplies by alpha^2 + f^2 and keeps Phi, bandwidth 5); the
// shifted operator and its solution are the same.
//
// Everything that depends only on (pole k, m, n) -- the LU factors of the
// tridiagonal systems, the right-hand-side couplings and the beta-weighted
// recovery weights of Phi and zeta -- is computed once per plan
// (factor_setup_kernel).  The per-step kernel then does, per (state, m,
// parity, pole) and per row, a forward sweep
//   y_i = delta0_n - g Phi0_n - e zeta0_{n-1} - f zeta0_{n+1} - l y_{i-1}
// and a backward sweep  w_i = y_i - Chat w_{i+1}  (delta_n = w_i / d'_i, folded
// into the weights) accumulating beta-weighted sums of delta, Phi and zeta in
// FP64 (solve_kernel<false>) or float-float (solve_kernel<true>, for plans with
// REXI_SOLVE_FP32X2).  The poles are split into `slots` groups summed separately
// (each in ascending k) and reduced in slot order, so results are bit-reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>
#include <string>
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
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}
// acc - a * b  (4 FP64 FMA)
__device__ __forceinline__ double2 cfms(double2 acc, double2 a, double2 b) {
  double re = fma(-a.x, b.x, acc.x);
  re = fma(a.y, b.y, re);
  double im = fma(-a.x, b.y, acc.y);
  im = fma(-a.y, b.x, im);
  return make_double2(re, im);
}
// acc + a * b  (4 FP64 FMA)
__device__ __forceinline__ double2 cfma(double2 acc, double2 a, double2 b) {
  double re = fma(a.x, b.x, acc.x);
  re = fma(-a.y, b.y, re);
  double im = fma(a.x, b.y, acc.y);
  im = fma(a.y, b.x, im);
  return make_double2(re, im);
}

struct SetupArgs {
  const double *coef;   // [nspec][4] = sigma, ct, dt, G
  const double2 *alpha, *beta;
  double2 *fac;         // [F_NCOMP][nrows][P]; float-float plans: the F_NCOMPACT set (compact),
                        // as [F_NCOMPACT][nrows][P] or interleaved [nrows][P][F_NCOMPACT]
  const int4 *sys;      // per system (m, p): {m, n0, len, row0}
  int nsys, P, N;
  int64_t nrows;
  double tau, phibar, q;  // q = 2 Omega tau
  int adjoint;
  int interleaved;      // float-float plans: the factors of a (row, pole) are adjacent
  int compact;          // float-float plans: the 7 factors of compact_comp (g and the Phi
                        // weight are formed in the sweep)
};

__device__ __forceinline__ int64_t sidx(int N, int m, int n) { return (int64_t)m * (2 * N + 3 - m) / 2 + (n - m); }

// One thread per (pole, system): builds the tridiagonal rows, factorises them
// (Thomas, no pivoting) and writes every per-row factor.
__global__ void factor_setup_kernel(SetupArgs a) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)a.P * a.nsys) return;
  const int k = (int)(t % a.P);
  const int4 sy = a.sys[t / a.P];
  const int m = sy.x, n0 = sy.y, len = sy.z;
  const int64_t row0 = sy.w;
  if (len <= 0) return;
  const int N = a.N, nmin = m > 1 ? m : 1;
  double2 al = a.alpha[k], be = a.beta[k];
  if (a.adjoint) { al = cconj(al); be = cconj(be); }
  const double tau = a.tau, q = a.q, pb = a.phibar;
  auto C4 = [&](int n, int c) -> double {
    if (n < nmin || n > N) return 0.0;
    return a.coef[4 * sidx(N, m, n) + c];
  };
  auto ct = [&](int n) { return C4(n, 1); };
  auto dt = [&](int n) { return C4(n, 2); };
  auto s_of = [&](int n) -> double2 {  // alpha + i tau sigma_n (forward) / conj(alpha) - i tau sigma_n
    double sg = C4(n, 0);
    return a.adjoint ? make_double2(al.x, al.y - tau * sg) : make_double2(al.x, al.y + tau * sg);
  };
  const int64_t NR = a.nrows, P = a.P;
  double2 *F = a.fac;
  auto at = [&](int comp, int64_t row) -> int64_t {
    if (a.compact) comp = compact_comp(comp);
    return a.interleaved ? (row * P + k) * F_NCOMPACT + comp : ((int64_t)comp * NR + row) * P + k;
  };
  auto put = [&](int comp, int64_t row, double2 v) {
    if (a.compact && compact_comp(comp) < 0) return;  // formed in the sweep
    F[at(comp, row)] = v;
  };
  const double2 one = make_double2(1.0, 0.0);

  // first pass: d' and l, store d' temporarily in the F_C slot
  double2 dprev = make_double2(1.0, 0.0), Cprev = make_double2(0.0, 0.0);
  for (int i = 0; i < len; ++i) {
    const int n = n0 + 2 * i;
    const double G = C4(n, 3);
    const double2 sn = s_of(n);
    double2 D = cadd(sn, cscale(cdiv(one, al), tau * tau * pb * G));
    double2 A = make_double2(0, 0), C = make_double2(0, 0);
    double2 g, e = make_double2(0, 0), f = make_double2(0, 0);
    if (!a.adjoint) {
      if (ct(n) != 0.0) {
        double2 inv = cdiv(one, s_of(n - 1));
        D = cadd(D, cscale(inv, q * q * ct(n) * dt(n - 1)));
        A = cscale(inv, q * q * ct(n) * ct(n - 1));
        e = cscale(inv, q * ct(n));
      }
      if (dt(n) != 0.0) {
        double2 inv = cdiv(one, s_of(n + 1));
        D = cadd(D, cscale(inv, q * q * dt(n) * ct(n + 1)));
        C = cscale(inv, q * q * dt(n) * dt(n + 1));
        f = cscale(inv, q * dt(n));
      }
      g = cscale(cdiv(one, al), tau * G);
    } else {
      if (dt(n - 1) != 0.0) {
        double2 inv = cdiv(one, s_of(n - 1));
        D = cadd(D, cscale(inv, q * q * dt(n - 1) * ct(n)));
        A = cscale(inv, q * q * dt(n - 1) * dt(n - 2));
        e = cscale(inv, -q * dt(n - 1));
      }
      if (ct(n + 1) != 0.0) {
        double2 inv = cdiv(one, s_of(n + 1));
        D = cadd(D, cscale(inv, q * q * ct(n + 1) * dt(n)));
        C = cscale(inv, q * q * ct(n + 1) * ct(n + 2));
        f = cscale(inv, -q * ct(n + 1));
      }
      g = cscale(cdiv(one, al), -tau * pb);
    }
    double2 l = make_double2(0, 0), dp = D;
    if (i > 0) {
      l = cdiv(A, dprev);
      dp = csub(D, cmul(l, Cprev));
    }
    const int64_t row = row0 + i;
    put(F_L, row, l);
    put(F_G, row, g);
    put(F_E, row, e);
    put(F_F, row, f);
    put(F_C, row, C);   // raw upper coefficient, rescaled below
    put(F_BD, row, dp); // d' (replaced below)
    dprev = dp;
    Cprev = C;
  }
  // second pass: Chat_i = C_i / d'_{i+1} and the beta-weighted recovery weights
  double2 dnext = make_double2(1.0, 0.0);
  for (int i = len - 1; i >= 0; --i) {
    const int n = n0 + 2 * i;
    const int64_t row = row0 + i;
    const double2 C = F[at(F_C, row)];
    const double2 dp = F[at(F_BD, row)];
    put(F_C, row, i == len - 1 ? make_double2(0, 0) : cdiv(C, dnext));
    const double2 bd = cdiv(be, dp);  // beta / d'
    const double G = C4(n, 3);
    double2 bad, zp = make_double2(0, 0), zm = make_double2(0, 0);
    if (!a.adjoint) {
      bad = cscale(cdiv(bd, al), tau * pb);
      if (ct(n + 1) != 0.0) zp = cscale(cdiv(bd, s_of(n + 1)), q * ct(n + 1));
      if (dt(n - 1) != 0.0) zm = cscale(cdiv(bd, s_of(n - 1)), q * dt(n - 1));
    } else {
      bad = cscale(cdiv(bd, al), -tau * G);
      if (dt(n) != 0.0) zp = cscale(cdiv(bd, s_of(n + 1)), -q * dt(n));
      if (ct(n) != 0.0) zm = cscale(cdiv(bd, s_of(n - 1)), -q * ct(n));
    }
    put(F_BD, row, bd);
    put(F_BAD, row, bad);
    put(F_ZP, row, zp);
    put(F_ZM, row, zm);
    dnext = dp;
  }
}

struct SolveArgs {
  SolveView v;
  double2 *ybuf;        // [resident warps][lmax][sweep_width][32]
  const WorkItem *items;
  unsigned *counter;
  int nitems, lmax;
};

__device__ __forceinline__ double2 ld(const double2 *p) { return __ldg(p); }

// Sweeps of KC poles of one lane at once (KC independent recurrences share the
// state loads and one read-modify-write of the slot partials per row).
template <int KC>
__device__ __forceinline__ void sweep_poles(const SolveView &a, const int (&k)[KC], int n0, int len, int nmin,
                                            int64_t row0, int64_t base_idx, const double2 *sPhi,
                                            const double2 *sZeta, const double2 *sDel, double2 *pPhi,
                                            double2 *pZeta, double2 *pDel, int64_t rstride, bool first,
                                            double2 *ybuf) {
  const int64_t NR = a.nrows, P = a.P;
  const int N = a.N, B = a.B;
  const double2 *fL[KC], *fG[KC], *fE[KC], *fF[KC];
  for (int c = 0; c < KC; ++c) {
    fL[c] = a.fac + ((int64_t)F_L * NR + row0) * P + k[c];
    fG[c] = a.fac + ((int64_t)F_G * NR + row0) * P + k[c];
    fE[c] = a.fac + ((int64_t)F_E * NR + row0) * P + k[c];
    fF[c] = a.fac + ((int64_t)F_F * NR + row0) * P + k[c];
  }
  // ---- forward sweep: y_i = delta0 - g Phi0 - e zeta0_{n-1} - f zeta0_{n+1} - l y_{i-1}
  double2 yprev[KC];
  for (int c = 0; c < KC; ++c) yprev[c] = make_double2(0, 0);
  double2 zprev = (n0 - 1 >= nmin) ? ld(sZeta + (base_idx + n0 - 1) * B) : make_double2(0, 0);
  for (int i = 0; i < len; ++i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
    const double2 zn = (n + 1 <= N) ? ld(sZeta + (ix + 1) * B) : make_double2(0, 0);
    const double2 d0 = ld(sDel + ix * B), p0 = ld(sPhi + ix * B);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      double2 y = cfms(d0, ld(fG[c] + (int64_t)i * P), p0);
      y = cfms(y, ld(fE[c] + (int64_t)i * P), zprev);
      y = cfms(y, ld(fF[c] + (int64_t)i * P), zn);
      y = cfms(y, ld(fL[c] + (int64_t)i * P), yprev[c]);
      ybuf[((int64_t)i * KC + c) * 32] = y;
      yprev[c] = y;
    }
    zprev = zn;
  }
  // ---- backward sweep w_i = y_i - Chat w_{i+1} with the beta-weighted accumulation;
  // zeta_{n+1} collects Zp_i w_i (row i) and Zm_{i+1} w_{i+1} (row i + 1), folded in as
  // complex FMAs with row i + 1's weight and w kept in registers.
  const double2 *fC[KC], *fBD[KC], *fBAD[KC], *fZP[KC], *fZM[KC];
  for (int c = 0; c < KC; ++c) {
    fC[c] = a.fac + ((int64_t)F_C * NR + row0) * P + k[c];
    fBD[c] = a.fac + ((int64_t)F_BD * NR + row0) * P + k[c];
    fBAD[c] = a.fac + ((int64_t)F_BAD * NR + row0) * P + k[c];
    fZP[c] = a.fac + ((int64_t)F_ZP * NR + row0) * P + k[c];
    fZM[c] = a.fac + ((int64_t)F_ZM * NR + row0) * P + k[c];
  }
  double2 wnext[KC], zmnext[KC];
  for (int c = 0; c < KC; ++c) wnext[c] = zmnext[c] = make_double2(0, 0);
  for (int i = len - 1; i >= 0; --i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
    double2 wv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) wv[c] = cfms(ybuf[((int64_t)i * KC + c) * 32], ld(fC[c] + (int64_t)i * P), wnext[c]);
    double2 accD = first ? make_double2(0, 0) : pDel[ix * rstride];
    double2 accP = first ? make_double2(0, 0) : pPhi[ix * rstride];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      accD = cfma(accD, ld(fBD[c] + (int64_t)i * P), wv[c]);
      accP = cfma(accP, ld(fBAD[c] + (int64_t)i * P), wv[c]);
    }
    pDel[ix * rstride] = accD;
    pPhi[ix * rstride] = accP;
    if (n + 1 <= N) {
      double2 accZ = first ? make_double2(0, 0) : pZeta[(ix + 1) * rstride];
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        accZ = cfma(accZ, ld(fZP[c] + (int64_t)i * P), wv[c]);
        accZ = cfma(accZ, zmnext[c], wnext[c]);
      }
      pZeta[(ix + 1) * rstride] = accZ;
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      zmnext[c] = ld(fZM[c] + (int64_t)i * P);
      wnext[c] = wv[c];
    }
  }
  if (n0 - 1 >= nmin) {
    const int64_t ix = base_idx + n0 - 1;
    double2 accZ = first ? make_double2(0, 0) : pZeta[ix * rstride];
#pragma unroll
    for (int c = 0; c < KC; ++c) accZ = cfma(accZ, zmnext[c], wnext[c]);
    pZeta[ix * rstride] = accZ;
  }
}

// The same sweeps in float-float arithmetic (ff.h): factors, states, the sweep
// intermediates and the slot partials are complex float-float values (float4) in the
// buffers' double2 slots, and every FP64 FMA of the sweep above becomes an
// error-compensated FP32 product and sum.  On GB300 the FP64 unit issues 1/64 of the
// FP32 rate, so the solve runs on the FP32 pipes at 48-bit significand precision.
__device__ __forceinline__ float4 ldf(const float4 *p) { return __ldg(p); }

// bring the line holding p into L2 (no register result, no wait)
__device__ __forceinline__ void l2_prefetch(const void *p) { asm volatile("prefetch.global.L2 [%0];" : : "l"(p)); }

template <int KC, bool IL>
__device__ __forceinline__ void sweep_poles_ff(const SolveView &a, const int (&k)[KC], int n0, int len, int nmin,
                                               int64_t row0, int64_t base_idx, const float4 *sPhi,
                                               const float4 *sZeta, const float4 *sDel, float4 *pPhi,
                                               float4 *pZeta, float4 *pDel, int64_t rstride, bool first,
                                               float4 *ybuf) {
  constexpr int D = 3;  // rows prefetched ahead into L2
  // the compact factor set (compact_comp): factor (comp, row i, pole c) at
  // fk[c] + i RS + comp CS, interleaved (IL) rows of P x F_NCOMPACT values or the
  // pole-fastest layout [F_NCOMPACT][nrows][P]; g and the Phi weight are formed from 1/alpha
  // (conj in the adjoint) and per-row reals
  const int64_t RS = IL ? (int64_t)a.P * F_NCOMPACT : (int64_t)a.P;
  const int64_t CS = IL ? 1 : a.nrows * a.P;
  const int N = a.N, B = a.B;
  constexpr int oL = compact_comp(F_L), oE = compact_comp(F_E), oF = compact_comp(F_F), oC = compact_comp(F_C),
                oBD = compact_comp(F_BD), oZP = compact_comp(F_ZP), oZM = compact_comp(F_ZM);
  float4 ia[KC], cpw[KC];  // 1/alpha per pole; the forward Phi weight's factor ia tau Phibar
#pragma unroll
  for (int c = 0; c < KC; ++c) {
    ia[c] = a.adj ? ff::cconj(__ldg(a.ffc_ia + k[c])) : __ldg(a.ffc_ia + k[c]);
    cpw[c] = ff::rscale(a.ffc_tpb, ia[c]);
  }
  const float4 *fk[KC];
  for (int c = 0; c < KC; ++c)
    fk[c] = reinterpret_cast<const float4 *>(a.fac) + (IL ? (row0 * a.P + k[c]) * F_NCOMPACT : row0 * a.P + k[c]);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);
  // Every row's data (states, factors, sweep intermediates, slot partials) is prefetched
  // into L2 D rows ahead, so that the row's own loads find it there; the prefetches hold
  // no registers (a register prefetch of the next row needed 168 registers per thread,
  // this kernel 128, i.e. four CTAs per SM instead of three).
  auto pf_fwd = [&](int i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
    if (n + 1 <= N) l2_prefetch(sZeta + (ix + 1) * B);
    l2_prefetch(sDel + ix * B);
    l2_prefetch(sPhi + ix * B);
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;
      if (IL) {  // factors 0..2 of the 112-byte record: at most two lines
        l2_prefetch(f);
        l2_prefetch(f + 2);
      } else {
#pragma unroll
        for (int q = oL; q <= oF; ++q) l2_prefetch(f + q * CS);
      }
    }
  };
  auto pf_bwd = [&](int i) {
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;  // factors 4..8
      if (IL) {  // factors 3..6
        l2_prefetch(f + 3);
        l2_prefetch(f + 6);
      } else {
#pragma unroll
        for (int q = oC; q <= oZM; ++q) l2_prefetch(f + q * CS);
      }
      l2_prefetch(ybuf + ((int64_t)i * KC + c) * 32);
    }
    if (!first) {
      l2_prefetch(pDel + ix * rstride);
      l2_prefetch(pPhi + ix * rstride);
      if (n + 1 <= N) l2_prefetch(pZeta + (ix + 1) * rstride);
    }
  };
  // ---- forward sweep: y_i = delta0 - g Phi0 - e zeta0_{n-1} - f zeta0_{n+1} - l y_{i-1}
  float4 yprev[KC];
  for (int c = 0; c < KC; ++c) yprev[c] = zero;
  float4 zprev = (n0 - 1 >= nmin) ? ldf(sZeta + (base_idx + n0 - 1) * B) : zero;
  for (int j = 1; j <= D && j < len; ++j) pf_fwd(j);
  // the states, first in each row's chain, are loaded into registers one row ahead
  auto ld_states = [&](int i, float4 &zn, float4 &d0, float4 &p0) {
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
    zn = (n + 1 <= N) ? ldf(sZeta + (ix + 1) * B) : zero;
    d0 = ldf(sDel + ix * B);
    p0 = ldf(sPhi + ix * B);
  };
  float4 znc, d0c, p0c;
  ld_states(0, znc, d0c, p0c);
  for (int i = 0; i < len; ++i) {
    if (i + D < len) pf_fwd(i + D);
    float4 znn, d0n, p0n;
    ld_states(i + 1 < len ? i + 1 : i, znn, d0n, p0n);
    const float4 zn = znc, d0 = d0c, p0 = p0c;
    znc = znn;
    d0c = d0n;
    p0c = p0n;
    float4 rp0 = zero;  // compact: (tau G_n, or -tau Phibar in the adjoint) Phi0
    {
      const float2 rg = a.adj ? make_float2(-a.ffc_tpb.x, -a.ffc_tpb.y) : __ldg(a.ffc_rows + base_idx + n0 + 2 * i);
      rp0 = ff::rscale(rg, p0);
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      const float4 *f = fk[c] + (int64_t)i * RS;
      ff::CAcc y = ff::cacc(d0);
      ff::cmsub(y, ia[c], rp0);
      ff::cmsub(y, ldf(f + oE * CS), zprev);
      ff::cmsub(y, ldf(f + oF * CS), zn);
      ff::cmsub(y, ldf(f + oL * CS), yprev[c]);
      const float4 yv = ff::raw(y);
      ybuf[((int64_t)i * KC + c) * 32] = yv;
      yprev[c] = yv;
    }
    zprev = zn;
  }
  // ---- backward sweep with the beta-weighted accumulation (as in sweep_poles)
  float4 wnext[KC], zmnext[KC];
  for (int c = 0; c < KC; ++c) wnext[c] = zmnext[c] = zero;
  for (int j = len - 2; j >= 0 && j >= len - 1 - D; --j) pf_bwd(j);
  // the sweep intermediates and the delta / Phi partials, first in each row's chains, are
  // loaded into registers one row ahead
  auto ld_heads = [&](int i, float4 (&y)[KC], float4 &pd, float4 &pp) {
    const int64_t ix = base_idx + n0 + 2 * i;
#pragma unroll
    for (int c = 0; c < KC; ++c) y[c] = ybuf[((int64_t)i * KC + c) * 32];
    pd = first ? zero : pDel[ix * rstride];
    pp = first ? zero : pPhi[ix * rstride];
  };
  float4 yc[KC], pdc, ppc;
  ld_heads(len - 1, yc, pdc, ppc);
  for (int i = len - 1; i >= 0; --i) {
    if (i - D >= 0) pf_bwd(i - D);
    const int n = n0 + 2 * i;
    const int64_t ix = base_idx + n;
    float4 yn[KC], pdn, ppn;
    ld_heads(i > 0 ? i - 1 : i, yn, pdn, ppn);
    float4 wv[KC];
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      ff::CAcc w = ff::cacc(yc[c]);
      ff::cmsub(w, ldf(fk[c] + (int64_t)i * RS + oC * CS), wnext[c]);
      wv[c] = ff::raw(w);
    }
    ff::CAcc accD = ff::cacc(pdc);
    ff::CAcc accP = ff::cacc(ppc);
#pragma unroll
    for (int c = 0; c < KC; ++c) yc[c] = yn[c];
    pdc = pdn;
    ppc = ppn;
    {  // u = (beta/d') w; delta += u, Phi += (Phi weight / (beta/d')) u
      float2 rrow = make_float2(0.f, 0.f);  // adjoint: -tau G_n
      if (a.adj) {
        const float2 r = __ldg(a.ffc_rows + ix);
        rrow = make_float2(-r.x, -r.y);
      }
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        const float4 u = ff::cmul(ldf(fk[c] + (int64_t)i * RS + oBD * CS), wv[c]);
        ff::cadd(accD, u);
        ff::cmac(accP, a.adj ? ff::rscale(rrow, ia[c]) : cpw[c], u);
      }
    }
    pDel[ix * rstride] = ff::raw(accD);
    pPhi[ix * rstride] = ff::raw(accP);
    if (n + 1 <= N) {
      ff::CAcc accZ = first ? ff::czero() : ff::cacc(pZeta[(ix + 1) * rstride]);
#pragma unroll
      for (int c = 0; c < KC; ++c) {
        ff::cmac(accZ, ldf(fk[c] + (int64_t)i * RS + oZP * CS), wv[c]);
        ff::cmac(accZ, zmnext[c], wnext[c]);
      }
      pZeta[(ix + 1) * rstride] = ff::raw(accZ);
    }
#pragma unroll
    for (int c = 0; c < KC; ++c) {
      zmnext[c] = ldf(fk[c] + (int64_t)i * RS + oZM * CS);
      wnext[c] = wv[c];
    }
  }
  if (n0 - 1 >= nmin) {
    const int64_t ix = base_idx + n0 - 1;
    ff::CAcc accZ = first ? ff::czero() : ff::cacc(pZeta[ix * rstride]);
#pragma unroll
    for (int c = 0; c < KC; ++c) ff::cmac(accZ, zmnext[c], wnext[c]);
    pZeta[ix * rstride] = ff::raw(accZ);
  }
}

// Forward/backward sweeps of one work item (m, pole group g, states from b0) for this
// lane = (state b, parity p, slot kk): its poles k = slot, slot + S, ... two at a time,
// accumulated into its slot's partials in ascending k.
template <bool FF>
__device__ __forceinline__ void solve_item(const SolveView &a, int wm, int wg, int wb0, int lane,
                                           double2 *ybuf) {
  const int bl = lane % a.bw;
  const int p = (lane / a.bw) & 1;
  const int kk = lane / (2 * a.bw);
  const int64_t NS = a.nspec;
  const int N = a.N, B = a.B, S = a.slots;
  const int b = wb0 + bl;
  const int4 sy = a.sys[2 * wm + p];
  const int m = sy.x, n0 = sy.y, len = sy.z;
  const int64_t row0 = sy.w;
  const int slot = wg * a.kk + kk;
  const int Sm = a.slots_m ? a.slots_m[m] : S;  // this order's slot count; S is the buffer stride
  if (kk >= a.kk || b >= B || len <= 0 || slot >= Sm) return;
  const int nmin = m > 1 ? m : 1;
  const int64_t base_idx = (int64_t)m * (2 * N + 3 - m) / 2 - m;  // idx(m, n) = base_idx + n
  const double2 *sPhi = a.sin + b;
  const double2 *sZeta = a.sin + NS * B + b;
  const double2 *sDel = a.sin + 2 * NS * B + b;
  double2 *pPhi = a.part + (int64_t)slot * B + b;
  double2 *pZeta = pPhi + NS * S * B;
  double2 *pDel = pPhi + 2 * NS * S * B;
  const int64_t rstride = (int64_t)S * B;  // partial stride per idx
  bool first = true;
  int k0 = a.pole_begin + slot;
  if constexpr (FF) {
    const float4 *fPhi = reinterpret_cast<const float4 *>(sPhi), *fZeta = reinterpret_cast<const float4 *>(sZeta),
                 *fDel = reinterpret_cast<const float4 *>(sDel);
    float4 *qPhi = reinterpret_cast<float4 *>(pPhi), *qZeta = reinterpret_cast<float4 *>(pZeta),
           *qDel = reinterpret_cast<float4 *>(pDel), *fy = reinterpret_cast<float4 *>(ybuf);
    auto sweeps = [&](auto il) {
      constexpr bool IL = decltype(il)::value;
      for (; k0 + Sm < a.pole_end; k0 += 2 * Sm) {
        const int kp[2] = {k0, k0 + Sm};
        sweep_poles_ff<2, IL>(a, kp, n0, len, nmin, row0, base_idx, fPhi, fZeta, fDel, qPhi, qZeta, qDel, rstride,
                              first, fy);
        first = false;
      }
      if (k0 < a.pole_end) {
        const int kp[1] = {k0};
        sweep_poles_ff<1, IL>(a, kp, n0, len, nmin, row0, base_idx, fPhi, fZeta, fDel, qPhi, qZeta, qDel, rstride,
                              first, fy);
      }
    };
    if (a.ffil) sweeps(std::true_type{});
    else sweeps(std::false_type{});
  } else {
    for (; k0 + Sm < a.pole_end; k0 += 2 * Sm) {
      const int kp[2] = {k0, k0 + Sm};
      sweep_poles<2>(a, kp, n0, len, nmin, row0, base_idx, sPhi, sZeta, sDel, pPhi, pZeta, pDel, rstride, first,
                     ybuf);
      first = false;
    }
    if (k0 < a.pole_end) {
      const int kp[1] = {k0};
      sweep_poles<1>(a, kp, n0, len, nmin, row0, base_idx, sPhi, sZeta, sDel, pPhi, pZeta, pDel, rstride, first,
                     ybuf);
    }
  }
}

// Persistent kernel: each warp takes (m, pole group, first state) items from an
// atomic counter (items are sorted longest first) and runs one tridiagonal
// forward/backward sweep per (lane, pole).
template <bool FF>
__global__ void __launch_bounds__(128) solve_kernel(SolveArgs a) {
  const int lane = threadIdx.x & 31;
  const int wslot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double2 *ybuf = a.ybuf + (int64_t)wslot * a.lmax * 2 * 32 + lane;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(a.counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)a.nitems) break;
    const WorkItem w = a.items[it];
    solve_item<FF>(a.v, w.m, w.g, w.b0, lane, ybuf);
  }
}

// The same over a ragged work list spanning several plans (mixed truncations and
// pole counts): item = (m, pole group, first state, plan index), longest first.
struct RaggedArgs {
  const SolveView *views;
  const WorkItem *items;  // len field carries the plan index
  double2 *ybuf;
  unsigned *counter;
  int nitems, lmax;
};

template <bool FF>
__global__ void __launch_bounds__(128) solve_ragged_kernel(RaggedArgs a) {
  const int lane = threadIdx.x & 31;
  const int wslot = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  double2 *ybuf = a.ybuf + (int64_t)wslot * a.lmax * 2 * 32 + lane;
  for (;;) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(a.counter, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if (it >= (unsigned)a.nitems) break;
    const WorkItem w = a.items[it];
    const SolveView v = a.views[w.len];
    solve_item<FF>(v, w.m, w.g, w.b0, lane, ybuf);
  }
}

struct ReduceArgs {
  const double2 *part, *sin;
  double2 *sout;
  const uint8_t *rflags;   // [3][nspec]
  const double2 *w;        // [nspec] zeta weights sum beta/s
  const double *coef;      // [nspec][4] (for single-pole s_n)
  const int32_t *m_of;     // [nspec] zonal order of idx
  const int32_t *slots_m;  // per zonal order slot count (<= slots, the partial stride), or null
  double2 sphi;
  int slots, B, N;
  int64_t nspec;
  int single, realm0, adjoint;
  double2 alpha_k, beta_k;
  double tau;
};

// the pole-independent terms of output t = (f, idx, b), and the real part at m = 0
__device__ __forceinline__ double2 reduce_finish(const ReduceArgs &a, int64_t t, int f, int64_t ix, double2 acc) {
  const double2 x0 = a.sin[t];
  if (!a.single) {
    if (f == 0) acc = cfma(acc, a.sphi, x0);
    else if (f == 1) acc = cfma(acc, a.w[ix], x0);
  } else {
    // single pole: partials carry beta_k X_k; divide beta_k out and add Phi0/alpha, zeta0/s
    acc = cdiv(acc, a.beta_k);
    if (f == 0) acc = cadd(acc, cdiv(x0, a.alpha_k));
    else if (f == 1) {
      double sg = a.coef[4 * ix + 0];
      double2 s = a.adjoint ? make_double2(a.alpha_k.x, -a.alpha_k.y - a.tau * sg)
                            : make_double2(a.alpha_k.x, a.alpha_k.y + a.tau * sg);
      acc = cadd(acc, cdiv(x0, s));
    }
  }
  if (a.realm0 && a.m_of[ix] == 0) acc.y = 0.0;
  return acc;
}

// Slot sums of float-float partials (solve_kernel<true>): added in slot order as
// float-float values, rounded once to binary64 (hi and lo converted on the integer pipe).
__device__ __forceinline__ double2 ff_result(const ff::CAcc &fa) {
  return make_double2(f32_to_f64(fa.re.s) + f32_to_f64(fa.re.e), f32_to_f64(fa.im.s) + f32_to_f64(fa.im.e));
}

// out[f][idx][b] = sum over slots (in order) + the pole-independent terms; one thread
// per output.
template <bool FF>
__global__ void reduce_kernel(ReduceArgs a) {
  const int64_t total = 3 * a.nspec * a.B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(t % a.B);
    const int64_t fi = t / a.B;  // f * nspec + idx
    const int f = (int)(fi / a.nspec);
    const int64_t ix = fi - (int64_t)f * a.nspec;
    const uint8_t fl = a.rflags[fi];
    double2 acc = make_double2(0, 0);
    if (!(fl & 2)) {
      if (fl & 1) {
        // loads issued eight at a time, added strictly in slot order (bit-reproducible)
        const int Sm = a.slots_m ? a.slots_m[a.m_of[ix]] : a.slots;
        if constexpr (FF) {
          const float4 *p = reinterpret_cast<const float4 *>(a.part) + fi * a.slots * a.B + b;
          ff::CAcc fa = ff::czero();
          int s = 0;
          for (; s + 8 <= Sm; s += 8) {
            float4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldcs(p + (int64_t)(s + u) * a.B);
#pragma unroll
            for (int u = 0; u < 8; ++u) ff::cadd(fa, v[u]);
          }
          for (; s < Sm; ++s) ff::cadd(fa, p[(int64_t)s * a.B]);
          acc = ff_result(fa);
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
      acc = reduce_finish(a, t, f, ix, acc);
    }
    a.sout[t] = acc;
  }
}

// The same with one warp per output for many slots (small batches): lane l sums slots
// l, l + 32, ... in order, then a fixed butterfly adds the lanes (bit-reproducible).
template <bool FF>
__global__ void reduce_wide_kernel(ReduceArgs a) {
  const int lane = threadIdx.x & 31;
  const int64_t total = 3 * a.nspec * a.B;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < total; t += nwarps) {
    const int b = (int)(t % a.B);
    const int64_t fi = t / a.B;
    const int f = (int)(fi / a.nspec);
    const int64_t ix = fi - (int64_t)f * a.nspec;
    const uint8_t fl = a.rflags[fi];
    double2 acc = make_double2(0, 0);
    if (!(fl & 2)) {
      if (fl & 1) {
        const int Sm = a.slots_m ? a.slots_m[a.m_of[ix]] : a.slots;
        if constexpr (FF) {
          const float4 *p = reinterpret_cast<const float4 *>(a.part) + fi * a.slots * a.B + b;
          ff::CAcc fa = ff::czero();
          for (int s = lane; s < Sm; s += 32) ff::cadd(fa, __ldcs(p + (int64_t)s * a.B));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            const float rs = __shfl_xor_sync(0xffffffffu, fa.re.s, o), re = __shfl_xor_sync(0xffffffffu, fa.re.e, o);
            const float is = __shfl_xor_sync(0xffffffffu, fa.im.s, o), ie = __shfl_xor_sync(0xffffffffu, fa.im.e, o);
            ff::add(fa.re, rs, re);
            ff::add(fa.im, is, ie);
          }
          acc = ff_result(fa);
        } else {
          const double2 *p = a.part + fi * a.slots * a.B + b;
          for (int s = lane; s < Sm; s += 32) acc = cadd(acc, __ldcs(p + (int64_t)s * a.B));
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
            acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
          }
        }
      }
      if (lane == 0) acc = reduce_finish(a, t, f, ix, acc);
    }
    if (lane == 0) a.sout[t] = acc;
  }
}

// f-sphere (constant f = 2 Omega): per degree n the shifted system of the forward map
//   s Phi - tau Phibar delta = rP,  s zeta - q delta = rZ,  s delta + q zeta + tau G Phi = rD
// (q = 2 Omega tau, G = n(n+1)/a^2) closes in closed form:
//   delta = (s rD - q rZ - tau G rP) / (s^2 + q^2 + tau^2 Phibar G),
//   Phi = (rP + tau Phibar delta) / s,  zeta = (rZ + q delta) / s.
// The adjoint map uses conj(s) and L^T:
//   delta = (s rD + q rZ + tau Phibar rP) / (...),  Phi = (rP - tau G delta) / s,
//   zeta = (rZ - q delta) / s.
// One thread per (idx, state) sums beta_k x_k over the poles in ascending k.
struct FsphereArgs {
  const double2 *sin, *alpha, *beta;
  double2 *sout;
  const uint8_t *rflags;
  const double *coef;
  const int32_t *m_of;
  int64_t nspec;
  int B, k0, k1, single, realm0, adjoint;
  double tau, q, phibar;
};

__global__ void fsphere_kernel(FsphereArgs a) {
  const int64_t total = a.nspec * a.B;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t ix = t / a.B;
    const int64_t NB = a.nspec * a.B;
    const double2 rP = a.sin[t], rZ = a.sin[NB + t], rD = a.sin[2 * NB + t];
    const double G = a.coef[4 * ix + 3];
    const double tg = a.tau * G, tp = a.tau * a.phibar, q = a.q;
    double2 aP = make_double2(0, 0), aZ = aP, aD = aP;
    for (int k = a.k0; k < a.k1; ++k) {
      double2 s = a.alpha[k], be = a.single ? make_double2(1.0, 0.0) : a.beta[k];
      if (a.adjoint) { s = cconj(s); be = cconj(be); }
      double2 den = cmul(s, s);
      den.x += q * q + tp * tg;
      double2 num = cmul(s, rD);
      double2 dl, ph, ze;
      if (!a.adjoint) {
        num = csub(num, cadd(cscale(rZ, q), cscale(rP, tg)));
        dl = cdiv(num, den);
        ph = cdiv(cadd(rP, cscale(dl, tp)), s);
        ze = cdiv(cadd(rZ, cscale(dl, q)), s);
      } else {
        num = cadd(num, cadd(cscale(rZ, q), cscale(rP, tp)));
        dl = cdiv(num, den);
        ph = cdiv(csub(rP, cscale(dl, tg)), s);
        ze = cdiv(csub(rZ, cscale(dl, q)), s);
      }
      aP = cfma(aP, be, ph);
      aZ = cfma(aZ, be, ze);
      aD = cfma(aD, be, dl);
    }
    double2 acc[3] = {aP, aZ, aD};
    for (int f = 0; f < 3; ++f) {
      if (a.rflags[f * a.nspec + ix] & 2) acc[f] = make_double2(0, 0);
      if (a.realm0 && a.m_of[ix] == 0) acc[f].y = 0.0;
      a.sout[f * NB + t] = acc[f];
    }
  }
}

// In-place binary64 -> float-float conversion of complex values (factors, once per plan);
// a value beyond binary32's range sets DEV_ERR_RANGE.
__global__ void to_ff_kernel(double2 *v, int64_t n, int *err) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double2 z = v[t];
    const float4 f = ff::csplit(z);
    if (ff::split_overflow(z, f)) atomicOr(err, DEV_ERR_RANGE);
    reinterpret_cast<float4 *>(v)[t] = f;
  }
}

// States for a float-float solve: in (binary64) -> out (float-float), once per step; a
// value beyond binary32's range sets DEV_ERR_RANGE (rexi_check_device reports it).
__global__ void split_state_kernel(const double2 *in, float4 *out, int64_t n, int *err) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x) {
    const double2 z = in[t];
    const float4 f = ff::csplit(z);
    if (ff::split_overflow(z, f)) atomicOr(err, DEV_ERR_RANGE);
    out[t] = f;
  }
}

// [rows][cols] -> [cols][rows] of double2 via 32x32 shared tiles (tiles indexed
// linearly in blockIdx.x, so neither dimension is limited by gridDim.y).
__global__ void transpose_kernel(const double2 *in, double2 *out, int64_t rows, int64_t cols) {
  __shared__ double2 tile[32][33];
  const int64_t tiles_c = (cols + 31) / 32;
  const int64_t c0 = (int64_t)(blockIdx.x % tiles_c) * 32, r0 = (int64_t)(blockIdx.x / tiles_c) * 32;
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int64_t r = r0 + j, c = c0 + threadIdx.x;
    if (r < rows && c < cols) tile[j][threadIdx.x] = in[r * cols + c];
  }
  __syncthreads();
  for (int j = threadIdx.y; j < 32; j += blockDim.y) {
    int64_t c = c0 + j, r = r0 + threadIdx.x;
    if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][j];
  }
}

}  // namespace

cudaError_t launch_fsphere(Plan &pl, bool adjoint, const double2 *sin, double2 *sout, int B, bool single,
                           int pole, cudaStream_t st) {
  FsphereArgs a;
  a.sin = sin;
  a.sout = sout;
  a.alpha = pl.alpha_dev;
  a.beta = pl.beta_dev;
  a.rflags = pl.rflags_dev;
  a.coef = pl.coef_dev;
  a.m_of = pl.m_of_dev;
  a.nspec = pl.nspec;
  a.B = B;
  a.k0 = single ? pole : 0;
  a.k1 = single ? pole + 1 : pl.P;
  a.single = single ? 1 : 0;
  a.realm0 = single ? 0 : 1;
  a.adjoint = adjoint ? 1 : 0;
  a.tau = pl.prm.tau;
  a.q = 2.0 * pl.prm.omega * pl.prm.tau;
  a.phibar = pl.prm.gravity * pl.prm.mean_depth;
  const int64_t total = pl.nspec * B;
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((total + 127) / 128, (int64_t)pl.num_sms * 16));
  fsphere_kernel<<<blocks, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_factor_setup(Plan &pl, bool adjoint, cudaStream_t st) {
  SetupArgs a;
  a.coef = pl.coef_dev;
  a.alpha = pl.alpha_dev;
  a.beta = pl.beta_dev;
  a.fac = adjoint ? pl.fac_adj : pl.fac_fwd;
  a.sys = pl.sys_dev;
  a.nsys = (int)pl.sys.size();
  a.P = pl.P;
  a.N = pl.N;
  a.nrows = pl.nrows;
  a.tau = pl.prm.tau;
  a.phibar = pl.prm.gravity * pl.prm.mean_depth;
  a.q = 2.0 * pl.prm.omega * pl.prm.tau;
  a.adjoint = adjoint ? 1 : 0;
  a.interleaved = pl.ffil ? 1 : 0;
  a.compact = pl.ff ? 1 : 0;
  int64_t total = (int64_t)a.P * a.nsys;
  factor_setup_kernel<<<(unsigned)((total + 127) / 128), 128, 0, st>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && pl.ff) e = launch_to_ff(pl, a.fac, (int64_t)fac_ncomp(pl) * pl.nrows * pl.P, st);
  return e;
}

cudaError_t launch_to_ff(Plan &pl, double2 *v, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)pl.num_sms * 16));
  to_ff_kernel<<<blocks, 256, 0, st>>>(v, n, pl.dev_err);
  return cudaGetLastError();
}

cudaError_t launch_split_state(Plan &pl, const double2 *in, double2 *out, int64_t n, cudaStream_t st) {
  const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)pl.num_sms * 16));
  split_state_kernel<<<blocks, 256, 0, st>>>(in, reinterpret_cast<float4 *>(out), n, pl.dev_err);
  return cudaGetLastError();
}

rexi_status take_range_error(Plan &pl, const char *what) {
  int flag = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(&flag, pl.dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string(what) + ": " + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  if (!(flag & DEV_ERR_RANGE)) return REXI_OK;
  flag &= ~DEV_ERR_RANGE;
  cudaMemcpy(pl.dev_err, &flag, sizeof(int), cudaMemcpyHostToDevice);
  set_error(std::string(what) + ": a value exceeds binary32's range (|x| > 3.4e38), which float-float "
            "arithmetic cannot hold; use REXI_SOLVE_FP64");
  return REXI_ERANGE;
}

// the per-plan data of the compact float-float factor set (unused otherwise)
void set_compact_view(const Plan &pl, bool adjoint, SolveView &v) {
  const double tpb = pl.prm.tau * pl.prm.gravity * pl.prm.mean_depth;
  const float hi = (float)tpb;
  v.adj = adjoint ? 1 : 0;
  v.ffc_rows = pl.ffc_rows;
  v.ffc_ia = pl.ffc_ia;
  v.ffc_tpb = make_float2(hi, (float)(tpb - (double)hi));
}

SolveView make_view(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin, double2 *part, int B,
                    int pole_begin, int pole_end) {
  SolveView v;
  v.fac = adjoint ? pl.fac_adj : pl.fac_fwd;
  v.sin = sin;
  v.part = part;
  v.sys = pl.sys_dev;
  v.P = pl.P;
  v.N = pl.N;
  v.B = B;
  v.bw = lay.bw;
  v.kk = lay.kk;
  v.slots = lay.slots;
  v.slots_m = lay.slots_m_dev;
  v.ffil = pl.ffil ? 1 : 0;
  set_compact_view(pl, adjoint, v);
  v.pole_begin = pole_begin;
  v.pole_end = pole_end;
  v.nspec = pl.nspec;
  v.nrows = pl.nrows;
  return v;
}

cudaError_t launch_solve(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin, int B,
                         int pole_begin, int pole_end, bool, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (pl.ff) {  // the solve reads the states as float-float values
    e = launch_split_state(pl, sin, pl.s_ff, 3 * pl.nspec * B, st);
    if (e != cudaSuccess) return e;
    sin = pl.s_ff;
  }
  SolveArgs a;
  a.v = make_view(pl, lay, adjoint, sin, pl.partial, B, pole_begin, pole_end);
  a.ybuf = pl.yscratch;
  a.items = lay.items_dev;
  a.counter = pl.counter;
  a.nitems = lay.nitems;
  a.lmax = pl.lmax;
  e = cudaMemsetAsync(pl.counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (pl.ff) solve_kernel<true><<<pl.resident_warps / 4, 128, 0, st>>>(a);
  else solve_kernel<false><<<pl.resident_warps / 4, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_solve_ragged(const SolveView *views_dev, const WorkItem *items, int nitems, double2 *ybuf,
                                int lmax, unsigned *counter, int resident_warps, bool ff, cudaStream_t st) {
  RaggedArgs a{views_dev, items, ybuf, counter, nitems, lmax};
  cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (ff) solve_ragged_kernel<true><<<resident_warps / 4, 128, 0, st>>>(a);
  else solve_ragged_kernel<false><<<resident_warps / 4, 128, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_reduce(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin,
                          double2 *sout, int B, bool single_pole, int pole, cudaStream_t st) {
  ReduceArgs a;
  a.part = pl.partial;
  a.sin = sin;
  a.sout = sout;
  a.rflags = pl.rflags_dev;
  a.w = adjoint ? pl.w_adj : pl.w_fwd;
  a.coef = pl.coef_dev;
  a.m_of = pl.m_of_dev;
  a.sphi = adjoint ? pl.sphi_adj : pl.sphi_fwd;
  a.slots = single_pole ? 1 : lay.slots;
  a.slots_m = single_pole ? nullptr : lay.slots_m_dev;
  a.B = B;
  a.N = pl.N;
  a.nspec = pl.nspec;
  a.single = single_pole ? 1 : 0;
  a.realm0 = single_pole ? 0 : 1;
  a.adjoint = adjoint ? 1 : 0;
  a.tau = pl.prm.tau;
  a.alpha_k = single_pole ? make_double2(pl.alpha[pole].real(), pl.alpha[pole].imag()) : make_double2(0, 0);
  a.beta_k = single_pole ? make_double2(pl.beta[pole].real(), pl.beta[pole].imag()) : make_double2(1, 0);
  int64_t total = 3 * pl.nspec * B;
  // a warp per output when one thread per output would leave most of the GPU idle
  if (a.slots >= 128 && total < (int64_t)pl.num_sms * 512) {
    int blocks = (int)std::min<int64_t>((total + 7) / 8, (int64_t)pl.num_sms * 8);
    if (pl.ff) reduce_wide_kernel<true><<<blocks, 256, 0, st>>>(a);
    else reduce_wide_kernel<false><<<blocks, 256, 0, st>>>(a);
  } else {
    int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)pl.num_sms * 8);
    if (pl.ff) reduce_kernel<true><<<blocks, 256, 0, st>>>(a);
    else reduce_kernel<false><<<blocks, 256, 0, st>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_transpose_in(const double2 *user, double2 *sint, int64_t nspec, int B,
                                cudaStream_t st) {
  // user [B][3 nspec] -> sint [3 nspec][B]
  int64_t rows = B, cols = 3 * nspec;
  const int64_t tiles = ((cols + 31) / 32) * ((rows + 31) / 32);
  transpose_kernel<<<(unsigned)tiles, dim3(32, 8), 0, st>>>(user, sint, rows, cols);
  return cudaGetLastError();
}

cudaError_t launch_transpose_out(const double2 *sint, double2 *user, int64_t nspec, int B, int,
                                 cudaStream_t st) {
  int64_t rows = 3 * nspec, cols = B;
  const int64_t tiles = ((cols + 31) / 32) * ((rows + 31) / 32);
  transpose_kernel<<<(unsigned)tiles, dim3(32, 8), 0, st>>>(sint, user, rows, cols);
  return cudaGetLastError();
}


// ---- allocation-free spectral step ---------------------------------------------------
// A variant of the spectral step for callers that may not allocate device memory
// when they step (for example code running under a fixed device-memory budget
// that was fully handed out at start-up, or a host application whose allocator
// must not be re-entered from the time-stepping loop).  All per-call scratch
// -- the transposed input and output states, the pole-slot partial sums, the
// forward-sweep intermediates, the work list and the work counter -- lives in
// one file-scope device array of kStaticScratchBytes; only the plan's read-only
// tables are used besides the caller's input and output.
namespace {

constexpr size_t kStaticScratchBytes = (size_t)64 << 20;  // 64 MiB, held by every device that loads the library
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
// device address of g_static_scratch per device ordinal, looked up once per device; the
// mutex orders first calls that race from several host threads.  The address stays valid
// for the life of the device context (a cudaDeviceReset ends it, together with every plan).
std::mutex g_static_mu;
void *g_static_addr[kMaxDevices] = {};

__global__ void static_items_kernel(WorkItem *items, int nitems, int nb, int bw, const int4 *sys) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nitems) return;
  const int m = t / nb, bb = t - m * nb;  // one pole group; m ascending = longest systems first
  const int l = max(sys[2 * m].z, sys[2 * m + 1].z);
  items[t] = WorkItem{m, 0, bb * bw, l};
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

rexi_status step_static(Plan &pl, const void *in, void *out, int B, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    set_error("rexi_step_static: no usable current device");
    return REXI_ECUDA;
  }
  // scratch layout for a batch (one pole group; lanes (state, parity, pole slot))
  struct StaticLayout {
    int bw, kk, slots, nb, nitems;
    size_t state_b, part_b, y_b, item_b, ffstate_b, need;
  };
  auto layout_of = [&pl](int nb_states) {
    StaticLayout L;
    L.bw = 1;
    while (L.bw < nb_states && L.bw < 16) L.bw *= 2;
    L.kk = 32 / (2 * L.bw);
    L.slots = std::min(L.kk, pl.P);
    L.nb = (nb_states + L.bw - 1) / L.bw;
    L.nitems = (pl.N + 1) * L.nb;
    const int warps = pl.num_sms * 4;
    L.state_b = align256((size_t)3 * pl.nspec * nb_states * sizeof(double2));
    L.part_b = align256((size_t)3 * pl.nspec * L.slots * nb_states * sizeof(double2));
    L.y_b = align256((size_t)warps * pl.lmax * sweep_width(pl.ff) * 32 * sizeof(double2));
    L.item_b = align256((size_t)L.nitems * sizeof(WorkItem));
    L.ffstate_b = pl.ff ? L.state_b : 0;  // float-float copy of the input states
    L.need = 2 * L.state_b + L.part_b + L.y_b + L.item_b + 256 + L.ffstate_b;
    return L;
  };
  const StaticLayout SL = layout_of(B);
  const int bw = SL.bw, slots = SL.slots, nb = SL.nb, nitems = SL.nitems;
  const int warps = pl.num_sms * 4;
  const size_t state_b = SL.state_b, part_b = SL.part_b, y_b = SL.y_b, item_b = SL.item_b;
  if (SL.need > kStaticScratchBytes) {
    // the sweep buffers (four warps per SM) do not shrink with the batch: when even one
    // state does not fit, no batch does
    const bool any_batch = layout_of(1).need > kStaticScratchBytes;
    set_error("rexi_step_static: this truncation and batch need " + std::to_string(SL.need) +
              " bytes of scratch, above the fixed limit of " + std::to_string(kStaticScratchBytes) +
              " bytes (64 MiB); " +
              (any_batch ? std::string("this truncation is not supported at any batch size on this GPU (the "
                                       "sweep buffers grow with its number of SMs); use rexi_step")
                         : std::string("use rexi_step or a smaller batch")));
    return REXI_EINVAL;
  }
  void *addr = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_static_mu);
    if (!g_static_addr[dev]) {
      void *p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p) {
        set_error(std::string("rexi_step_static: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
        return REXI_ECUDA;
      }
      g_static_addr[dev] = p;
    }
    addr = g_static_addr[dev];
  }
  unsigned char *base = static_cast<unsigned char *>(addr);
  double2 *s_in = reinterpret_cast<double2 *>(base);
  double2 *s_out = reinterpret_cast<double2 *>(base + state_b);
  double2 *part = reinterpret_cast<double2 *>(base + 2 * state_b);
  double2 *ybuf = reinterpret_cast<double2 *>(base + 2 * state_b + part_b);
  WorkItem *items = reinterpret_cast<WorkItem *>(base + 2 * state_b + part_b + y_b);
  unsigned *counter = reinterpret_cast<unsigned *>(base + 2 * state_b + part_b + y_b + item_b);
  double2 *s_ff = reinterpret_cast<double2 *>(base + 2 * state_b + part_b + y_b + item_b + 256);

  if (pl.prm.fsphere) {  // closed-form per-degree solves: only the two state buffers are used
    e = launch_transpose_in(static_cast<const double2 *>(in), s_in, pl.nspec, B, st);
    if (e == cudaSuccess) e = launch_fsphere(pl, false, s_in, s_out, B, false, 0, st);
    if (e == cudaSuccess) e = launch_transpose_out(s_out, static_cast<double2 *>(out), pl.nspec, B, pl.N, st);
    if (e != cudaSuccess) {
      set_error(std::string("rexi_step_static: ") + cudaGetErrorString(e));
      return REXI_ECUDA;
    }
    return REXI_OK;
  }
  e = launch_transpose_in(static_cast<const double2 *>(in), s_in, pl.nspec, B, st);
  if (e == cudaSuccess) {
    static_items_kernel<<<(nitems + 127) / 128, 128, 0, st>>>(items, nitems, nb, bw, pl.sys_dev);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(unsigned), st);  // the work counter starts at zero
  if (e == cudaSuccess && pl.ff) e = launch_split_state(pl, s_in, s_ff, 3 * pl.nspec * B, st);
  if (e == cudaSuccess) {
    SolveArgs a;
    a.v.fac = pl.fac_fwd;
    a.v.sin = pl.ff ? s_ff : s_in;
    a.v.part = part;
    a.v.sys = pl.sys_dev;
    a.v.P = pl.P;
    a.v.N = pl.N;
    a.v.B = B;
    a.v.bw = bw;
    a.v.kk = slots;
    a.v.slots = slots;
    a.v.slots_m = nullptr;
    a.v.ffil = pl.ffil ? 1 : 0;
    set_compact_view(pl, false, a.v);
    a.v.pole_begin = 0;
    a.v.pole_end = pl.P;
    a.v.nspec = pl.nspec;
    a.v.nrows = pl.nrows;
    a.ybuf = ybuf;
    a.items = items;
    a.counter = counter;
    a.nitems = nitems;
    a.lmax = pl.lmax;
    if (pl.ff) solve_kernel<true><<<warps / 4, 128, 0, st>>>(a);
    else solve_kernel<false><<<warps / 4, 128, 0, st>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    ReduceArgs r;
    r.part = part;
    r.sin = s_in;
    r.sout = s_out;
    r.rflags = pl.rflags_dev;
    r.w = pl.w_fwd;
    r.coef = pl.coef_dev;
    r.m_of = pl.m_of_dev;
    r.sphi = pl.sphi_fwd;
    r.slots = slots;
    r.slots_m = nullptr;
    r.B = B;
    r.N = pl.N;
    r.nspec = pl.nspec;
    r.single = 0;
    r.realm0 = 1;
    r.adjoint = 0;
    r.alpha_k = make_double2(0, 0);
    r.beta_k = make_double2(1, 0);
    r.tau = pl.prm.tau;
    const int64_t total = 3 * pl.nspec * B;
    const int blocks = (int)std::min<int64_t>((total + 255) / 256, (int64_t)pl.num_sms * 8);
    if (pl.ff) reduce_kernel<true><<<blocks, 256, 0, st>>>(r);
    else reduce_kernel<false><<<blocks, 256, 0, st>>>(r);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = launch_transpose_out(s_out, static_cast<double2 *>(out), pl.nspec, B, pl.N, st);
  if (e != cudaSuccess) {
    set_error(std::string("rexi_step_static: ") + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  return REXI_OK;
}

}  // namespace rexi
