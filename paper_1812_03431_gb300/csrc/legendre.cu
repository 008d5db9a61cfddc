// Legendre transforms per zonal order m on the Gaussian grid (paper Sec. 3), FP64.
//
// Analysis (Fourier data already scaled per latitude by the FFT: g w_j for
// Phi, cos(lat) w_j / (a (1 - mu_j^2)) for U = u cos, V = v cos):
//   Phi_n   = sum_j Pbar_n(mu_j) F^Phi_j
//   zeta_n  = sum_j [ i m Pbar_n F^V_j + H_n F^U_j ]
//   delta_n = sum_j [ i m Pbar_n F^U_j - H_n F^V_j ]        (times zdscale[idx])
// Synthesis:  with psi'_n = zdscale[idx] zeta_n, chi'_n = zdscale[idx] delta_n,
//   F^Phi_j = sum_n Pbar_n Phi_n
//   F^U_j   = sum_n [ -H_n psi'_n + i m Pbar_n chi'_n ]
//   F^V_j   = sum_n [ i m Pbar_n psi'_n + H_n chi'_n ]
// H_n = (1 - mu^2) dPbar_n/dmu.  Pbar_n(-mu) = (-1)^{n-m} Pbar_n(mu) and H has the
// opposite parity, so both sums run over the northern latitudes only, on
// symmetric (E = F(mu) + F(-mu)) and antisymmetric (O = F(mu) - F(-mu)) parts.
// The same kernels with other zdscale arrays give the transposed transforms of
// the adjoint step.
//
// Tables Pbar, H: [nspec][J] (J = nlat / 2 northern latitudes), FP64.
#include <cuda_runtime.h>

#include <algorithm>

#include "rexi_internal.h"

namespace rexi {

namespace {

constexpr int kJC = 32;  // latitudes per staged chunk (analysis)
constexpr int kNC = 32;  // degrees per staged chunk (synthesis)

struct LegArgs {
  const double *tabP, *tabH;
  double2 *four;        // [nlat][N+1][3B]
  double2 *sint;        // [3][nspec][B]
  const double *zd;     // [nspec]
  int N, nlat, J, B, TB, TN;
  int64_t nspec;
};

__device__ __forceinline__ double2 zmad(double2 acc, double t, double2 x) {
  return make_double2(fma(t, x.x, acc.x), fma(t, x.y, acc.y));
}

// grid: (row tiles, m, b tiles); block = TN * TB threads (TN rows x TB states)
__global__ void __launch_bounds__(256) leg_ana_kernel(LegArgs a) {
  extern __shared__ double smem[];
  const int m = blockIdx.y;
  const int nrows = a.N - m + 1;
  const int r0 = blockIdx.x * a.TN;
  if (r0 >= nrows) return;
  const int b0 = blockIdx.z * a.TB;
  const int TB = a.TB, TN = a.TN;
  const int ncolT = 3 * TB;
  double2 *xe = reinterpret_cast<double2 *>(smem);       // [kJC][3 TB]
  double2 *xo = xe + kJC * ncolT;                         // [kJC][3 TB]
  double *tp = reinterpret_cast<double *>(xo + kJC * ncolT);  // [TN][kJC]
  double *th = tp + TN * kJC;
  const int tid = threadIdx.x;
  const int rl = tid / TB, bl = tid - rl * TB;
  const int n = m + r0 + rl;
  const bool live = (r0 + rl) < nrows && (b0 + bl) < a.B;
  const int par = (n - m) & 1;
  const int64_t idx0 = (int64_t)m * (2 * a.N + 3 - m) / 2;  // idx(m, m)
  const int M1 = a.N + 1, ncol = 3 * a.B;
  double2 aPhi = make_double2(0, 0), aPV = aPhi, aPU = aPhi, aHU = aPhi, aHV = aPhi;
  for (int j0 = 0; j0 < a.J; j0 += kJC) {
    const int jn = min(kJC, a.J - j0);
    __syncthreads();
    for (int t = tid; t < jn * ncolT; t += blockDim.x) {
      const int jj = t / ncolT, c = t - jj * ncolT;
      const int cg = 3 * b0 + c;
      double2 v1 = make_double2(0, 0), v2 = v1;
      if (cg < ncol) {
        v1 = a.four[((int64_t)(j0 + jj) * M1 + m) * ncol + cg];
        v2 = a.four[((int64_t)(a.nlat - 1 - j0 - jj) * M1 + m) * ncol + cg];
      }
      xe[jj * ncolT + c] = make_double2(v1.x + v2.x, v1.y + v2.y);
      xo[jj * ncolT + c] = make_double2(v1.x - v2.x, v1.y - v2.y);
    }
    for (int t = tid; t < TN * jn; t += blockDim.x) {
      const int r = t / jn, jj = t - r * jn;
      const int row = r0 + r;
      double p = 0.0, h = 0.0;
      if (row < nrows) {
        p = a.tabP[(idx0 + row) * a.J + j0 + jj];
        h = a.tabH[(idx0 + row) * a.J + j0 + jj];
      }
      tp[r * kJC + jj] = p;
      th[r * kJC + jj] = h;
    }
    __syncthreads();
    if (live) {
      const double2 *xp = par ? xo : xe;   // data with the parity of Pbar_n
      const double2 *xh = par ? xe : xo;   // data with the parity of H_n
      for (int jj = 0; jj < jn; ++jj) {
        const double p = tp[rl * kJC + jj], h = th[rl * kJC + jj];
        const double2 *rp = xp + jj * ncolT + 3 * bl;
        const double2 *rh = xh + jj * ncolT + 3 * bl;
        aPhi = zmad(aPhi, p, rp[0]);
        aPU = zmad(aPU, p, rp[1]);
        aPV = zmad(aPV, p, rp[2]);
        aHU = zmad(aHU, h, rh[1]);
        aHV = zmad(aHV, h, rh[2]);
      }
    }
  }
  if (!live) return;
  const int64_t ix = idx0 + (n - m);
  const double s = a.zd[ix];
  const double fm = (double)m;
  // zeta = i m (P V) + H U,  delta = i m (P U) - H V
  const double2 zeta = make_double2(s * (-fm * aPV.y + aHU.x), s * (fm * aPV.x + aHU.y));
  const double2 delta = make_double2(s * (-fm * aPU.y - aHV.x), s * (fm * aPU.x - aHV.y));
  const int b = b0 + bl;
  a.sint[ix * a.B + b] = aPhi;
  a.sint[(a.nspec + ix) * a.B + b] = zeta;
  a.sint[(2 * a.nspec + ix) * a.B + b] = delta;
}

// grid: (latitude tiles of TN northern rows, m, b tiles); block = TN * TB threads
__global__ void __launch_bounds__(256) leg_syn_kernel(LegArgs a) {
  extern __shared__ double smem[];
  const int m = blockIdx.y;
  const int nrows = a.N - m + 1;
  const int j0 = blockIdx.x * a.TN;
  const int b0 = blockIdx.z * a.TB;
  const int TB = a.TB, TN = a.TN;
  double2 *sv = reinterpret_cast<double2 *>(smem);          // [kNC][3 TB]: Phi, psi', chi'
  double *tp = reinterpret_cast<double *>(sv + kNC * 3 * TB);  // [kNC][TN]
  double *th = tp + kNC * TN;
  const int tid = threadIdx.x;
  const int jl = tid / TB, bl = tid - jl * TB;
  const int j = j0 + jl;
  const bool live = j < a.J && (b0 + bl) < a.B;
  const int64_t idx0 = (int64_t)m * (2 * a.N + 3 - m) / 2;
  // accumulators per symmetry class (0: even in mu, 1: odd)
  double2 aPhi[2], aPpsi[2], aPchi[2], aHpsi[2], aHchi[2];
  for (int c = 0; c < 2; ++c) aPhi[c] = aPpsi[c] = aPchi[c] = aHpsi[c] = aHchi[c] = make_double2(0, 0);
  for (int r0 = 0; r0 < nrows; r0 += kNC) {
    const int rn = min(kNC, nrows - r0);
    __syncthreads();
    for (int t = tid; t < rn * 3 * TB; t += blockDim.x) {
      const int rr = t / (3 * TB), c = t - rr * 3 * TB;
      const int f = c / TB, bb = c - f * TB;
      const int64_t ix = idx0 + r0 + rr;
      double2 v = make_double2(0, 0);
      if (b0 + bb < a.B) {
        v = a.sint[((int64_t)f * a.nspec + ix) * a.B + b0 + bb];
        if (f > 0) {
          const double s = a.zd[ix];
          v = make_double2(s * v.x, s * v.y);
        }
      }
      sv[rr * 3 * TB + c] = v;
    }
    for (int t = tid; t < rn * TN; t += blockDim.x) {
      const int rr = t / TN, jj = t - rr * TN;
      double p = 0.0, h = 0.0;
      if (j0 + jj < a.J) {
        p = a.tabP[(idx0 + r0 + rr) * a.J + j0 + jj];
        h = a.tabH[(idx0 + r0 + rr) * a.J + j0 + jj];
      }
      tp[rr * TN + jj] = p;
      th[rr * TN + jj] = h;
    }
    __syncthreads();
    if (live) {
      for (int rr = 0; rr < rn; ++rr) {
        const int par = (r0 + rr) & 1;
        const double p = tp[rr * TN + jl], h = th[rr * TN + jl];
        const double2 *v = sv + rr * 3 * TB;
        const double2 phi = v[bl], psi = v[TB + bl], chi = v[2 * TB + bl];
        aPhi[par] = zmad(aPhi[par], p, phi);
        aPpsi[par] = zmad(aPpsi[par], p, psi);
        aPchi[par] = zmad(aPchi[par], p, chi);
        aHpsi[par ^ 1] = zmad(aHpsi[par ^ 1], h, psi);
        aHchi[par ^ 1] = zmad(aHchi[par ^ 1], h, chi);
      }
    }
  }
  if (!live) return;
  const double fm = (double)m;
  double2 F[2][3];
  for (int c = 0; c < 2; ++c) {
    F[c][0] = aPhi[c];
    // U = -H psi' + i m P chi',  V = i m P psi' + H chi'
    F[c][1] = make_double2(-aHpsi[c].x - fm * aPchi[c].y, -aHpsi[c].y + fm * aPchi[c].x);
    F[c][2] = make_double2(-fm * aPpsi[c].y + aHchi[c].x, fm * aPpsi[c].x + aHchi[c].y);
  }
  const int M1 = a.N + 1, ncol = 3 * a.B, b = b0 + bl;
  double2 *north = a.four + ((int64_t)j * M1 + m) * ncol + 3 * b;
  double2 *south = a.four + ((int64_t)(a.nlat - 1 - j) * M1 + m) * ncol + 3 * b;
  for (int f = 0; f < 3; ++f) {
    north[f] = make_double2(F[0][f].x + F[1][f].x, F[0][f].y + F[1][f].y);
    south[f] = make_double2(F[0][f].x - F[1][f].x, F[0][f].y - F[1][f].y);
  }
}

void tiles(int B, int *TB, int *TN) {
  int tb = 1;
  while (tb < B && tb < 16) tb *= 2;
  *TB = tb;
  *TN = std::min(64, 256 / tb);
}

}  // namespace

cudaError_t launch_leg_ana(Plan &pl, const double2 *four, double2 *sint, int B, const double *zd,
                           cudaStream_t st) {
  LegArgs a{pl.tabP, pl.tabH, const_cast<double2 *>(four), sint, zd, pl.N, pl.nlat, pl.J, B, 0, 0, pl.nspec};
  tiles(B, &a.TB, &a.TN);
  dim3 g((unsigned)((pl.N + 1 + a.TN - 1) / a.TN), (unsigned)(pl.N + 1), (unsigned)((B + a.TB - 1) / a.TB));
  size_t sm = (size_t)2 * kJC * 3 * a.TB * sizeof(double2) + (size_t)2 * a.TN * kJC * sizeof(double);
  leg_ana_kernel<<<g, a.TN * a.TB, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_leg_syn(Plan &pl, const double2 *sint, double2 *four, int B, const double *zd,
                           cudaStream_t st) {
  LegArgs a{pl.tabP, pl.tabH, four, const_cast<double2 *>(sint), zd, pl.N, pl.nlat, pl.J, B, 0, 0, pl.nspec};
  tiles(B, &a.TB, &a.TN);
  dim3 g((unsigned)((pl.J + a.TN - 1) / a.TN), (unsigned)(pl.N + 1), (unsigned)((B + a.TB - 1) / a.TB));
  size_t sm = (size_t)kNC * 3 * a.TB * sizeof(double2) + (size_t)2 * kNC * a.TN * sizeof(double);
  leg_syn_kernel<<<g, a.TN * a.TB, sm, st>>>(a);
  return cudaGetLastError();
}

cudaError_t legendre_configure() {
  cudaError_t e = cudaFuncSetAttribute(leg_ana_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(leg_syn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
}

}  // namespace rexi
