// Internal declarations of librexi (not part of the C-ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <map>
#include <string>
#include <vector>

#include "../../include/rexi.h"

namespace rexi {

#ifdef __CUDACC__
// IEEE-754 binary64 <-> binary32 conversions on the integer pipe.  On GB300 the FP64
// unit, which also executes the hardware conversions, issues 1/64 of the FP32 rate; the
// mixed-form transform kernels convert every element once, so they do it with integer
// operations instead.  Round to nearest even; results below 2^-126 in magnitude are
// flushed to signed zero (the transform data are many orders of magnitude larger);
// infinities and NaNs are preserved.
__device__ __forceinline__ float f64_to_f32(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int e11 = (int)((b >> 52) & 0x7ffu);
  const unsigned long long mant = b & 0xfffffffffffffull;
  if (e11 == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (mant ? 0x400000u : 0u));
  const int e = e11 - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned m = (unsigned)(mant >> 29);
  const unsigned rem = (unsigned)(mant & 0x1fffffffull);
  unsigned r = ((unsigned)e << 23) | m;
  if (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) r += 1u;  // a carry bumps the exponent
  return __uint_as_float(sign | r);
}
__device__ __forceinline__ double f32_to_f64(float x) {
  const unsigned u = __float_as_uint(x);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  const unsigned e = (u >> 23) & 0xffu;
  const unsigned long long m = u & 0x7fffffu;
  if (e == 0) return __longlong_as_double((long long)sign);
  if (e == 255) return __longlong_as_double((long long)(sign | 0x7ff0000000000000ull | (m << 29)));
  return __longlong_as_double((long long)(sign | ((unsigned long long)(e - 127 + 1023) << 52) | (m << 29)));
}
#endif

using cplx = std::complex<double>;

constexpr int kGaussTerms = 11;  // K of the Gaussian rational approximation (Sec. 4.1)

// ---- host math (coeffs.cpp) -------------------------------------------------
// Refitted Gaussian rational approximation psi(y) ~ Re sum_l a_l/(i y + mu + i l).
struct GaussFit {
  double mu;
  cplx a[2 * kGaussTerms + 1];  // l = -K..K
  double sup_err;
};
const GaussFit &gauss_fit();
void rexi_coeffs_host(int M, double h, bool normalize, std::vector<cplx> &alpha,
                      std::vector<cplx> &beta, double *eps);
void gauss_legendre_host(int nlat, std::vector<double> &mu, std::vector<double> &w);

// ---- spectral indexing ---------------------------------------------------------
inline int64_t spec_idx(int N, int m, int n) { return (int64_t)m * (2 * N + 3 - m) / 2 + (n - m); }
inline int64_t nspec_of(int N) { return (int64_t)(N + 1) * (N + 2) / 2; }

// One row of a banded system: zonal order m, parity p (of n - m), position i.
// Rows of a (m, p) system are n = n0(m, p) + 2 i, i = 0..len-1; zeta_0^0 and
// delta_0^0 are excluded (so m = 0 starts at n = 2 / n = 1).
struct SysInfo {
  int m, p, n0, len;
  int64_t row0;  // first global row id
};

// Solve-kernel work item: (m, pole-slot group, first state) for one warp.
struct WorkItem {
  int32_t m, g, b0, len;
};

// Lane layout of the solve kernel for a given batch: lane = (b_local, p, kk)
// with bw * 2 * kk_per_warp = 32.
struct SolveLayout {
  int batch, bw, kk, groups, slots;  // slots = groups * kk: the partial buffer's slot stride
  int shape = 0;                     // 0: same groups for every order; 1: in proportion to length
  int nitems;
  WorkItem *items_dev = nullptr;     // nitems items, followed by slots_m (one allocation)
  // per zonal order: pole groups proportional to the system length, so that items carry
  // similar work; order m uses slots_m[m] = groups_m[m] * kk <= slots partial sums
  std::vector<int> groups_m;
  int32_t *slots_m_dev = nullptr;
};

// CTA shape and work list of the fused solve (solve_fused.cu) for one batch size: ST
// states per CTA tile over WS warps of SB states; WP warps split the poles when the tile
// has fewer than four states; NG CTAs split the poles of one (system, tile) in groups of
// gsz poles, the last of them to finish adding the groups' partial sums.  items: (system
// 2 m + p, first state, pole group, (system, tile) index), longest first.
struct FusedLayout {
  int sb = 0, ws = 0, wp = 0, st = 0;
  int nw = 8;       // warps per CTA: 8 (one CTA per SM), 4 (two per SM, or the lean form) or 2 (lean)
  int per_sm = 1;   // CTAs per SM (lean form: 3 or 4 of four warps, 7 or 8 of two)
  int ng = 1, gsz = 0;  // pole groups per (system, tile) and poles per group
  int ntiles = 0;       // (system, tile) pairs
  int nitems = 0;
  int4 *items_dev = nullptr;
  double2 *part_dev = nullptr;   // NG > 1: [B / st][ng][st][nrows][4] partial sums
  unsigned *sync_dev = nullptr;  // [1 + ntiles]: the work counter, then per (system, tile) arrivals
  size_t smem = 0;  // dynamic shared memory per CTA (running sums and the exchange buffer)
};
void free_fused_layout(FusedLayout &F);

// The fused solve over the states of several plans in one launch (ragged batches).
struct FusedRagged {
  void *views_dev = nullptr;  // per plan (solve_fused.cu's FusedView)
  int4 *items_dev = nullptr;
  unsigned *counter = nullptr;
  int nitems = 0, nviews = 0, lmax = 0, per_sm = 0, ws = 0, wp = 0, nw = 4;
  size_t smem = 0;
};

struct FftPlan {
  int n;
  int nstages;
  int radix[24];
  int nsplit;     // rows per CTA (pairs of real rows packed as one complex row)
  void *tw_dev;   // n twiddles e^{-2 pi i k/n}, double2
  void *tw32_dev; // the same as float2 (mixed form)
};

enum FacComp { F_L = 0, F_G, F_E, F_F, F_C, F_BD, F_BAD, F_ZP, F_ZM, F_NCOMP };

// factor c in the compact float-float set (F_G and F_BAD are formed in the sweep: -1)
__host__ __device__ constexpr int compact_comp(int c) {
  return c == F_G || c == F_BAD ? -1 : (c < F_G ? c : (c < F_BAD ? c - 1 : c - 2));
}
constexpr int F_NCOMPACT = F_NCOMP - 2;

// bits of a plan's device error word (rexi_check_device)
enum DevErr {
  DEV_ERR_TIMEOUT = 1,  // a bounded wait (tensor-core completion barrier) expired
  DEV_ERR_RANGE = 2     // a finite binary64 value outside binary32's range met a float-float split
};

// Poles a lane sweeps at once in the solve kernel; the forward-sweep buffer holds lmax
// rows of that many values per lane.
inline int sweep_width(bool) { return 2; }

struct Plan {
  rexi_params prm{};
  int N = 0, nlat = 0, nlon = 0, J = 0, P = 0;
  int64_t nspec = 0, nrows = 0;
  std::vector<cplx> alpha, beta;
  double eps0 = 0;
  int device = 0, num_sms = 0;
  size_t bytes = 0;

  // systems and rows
  std::vector<SysInfo> sys;  // index 2 m + p
  // per-coefficient coupling data on the device: {sigma, ct, dt, G} per idx(m, n)
  double *coef_dev = nullptr;
  // per system (index 2 m + p): {m, n0, len, row0}; per idx: zonal order m
  int4 *sys_dev = nullptr;
  int32_t *m_of_dev = nullptr;

  // solve factors (forward and adjoint): [F_NCOMP][nrows][P] double2; float-float plans
  // hold the compact set as float-float values (float4 in the double2 slots):
  // [F_NCOMPACT][nrows][P], or [nrows][P][F_NCOMPACT] when ffil
  double2 *fac_fwd = nullptr, *fac_adj = nullptr;
  double2 *alpha_dev = nullptr, *beta_dev = nullptr;
  // pole-independent parts: W[idx] = sum_k beta_k/s_{k,n} (zeta), scalar S_Phi
  double2 *w_fwd = nullptr, *w_adj = nullptr;
  double2 sphi_fwd{}, sphi_adj{};
  // reduce flags per (field, idx): bit0 has partials, bit1 forced zero
  uint8_t *rflags_dev = nullptr;

  // grid / Legendre
  double *mu_dev = nullptr;
  double *tabP = nullptr, *tabH = nullptr;       // [nspec][J] FP64
  float *tabP_hi = nullptr, *tabP_lo = nullptr;  // mixed: TF32 hi/lo splits
  float *tabH_hi = nullptr, *tabH_lo = nullptr;
  double *scale_ana_in = nullptr;   // [3][nlat]: analysis pre-scale (g w, cos w/(a(1-mu^2)))
  double *scale_syn_out = nullptr;  // [3][nlat]: synthesis post-scale (1/g, 1/cos)
  double *mscale_fwd = nullptr;     // [N+1]: 1/nlon
  double *mscale_c = nullptr;       // [N+1]: c_m = 1, 2, 2, ...
  double *mscale_adj = nullptr;     // [N+1]: 1/nlon, 1/(2 nlon), ...
  double *mscale_one = nullptr;     // [N+1]: 1
  // the same six scales rounded to binary32 (the mixed form's FFTs scale in FP32)
  float *scale_ana_in32 = nullptr, *scale_syn_out32 = nullptr, *mscale_fwd32 = nullptr, *mscale_c32 = nullptr,
        *mscale_adj32 = nullptr, *mscale_one32 = nullptr;
  double *zd_syn = nullptr;         // [nspec]: -a/(n(n+1)) (0 at n = 0)
  double *zd_ana_adj = nullptr;     // [nspec]: +a/(n(n+1))
  double *zd_one = nullptr;         // [nspec]: 1
  double *zd_mone = nullptr;        // [nspec]: -1
  FftPlan fft{};
  // mixed precision: packed TF32 hi/lo tables and per-CTA work lists of the tensor-core kernels
  uint32_t *tc_tab_ana = nullptr, *tc_tab_syn = nullptr;
  int4 *tc_work_ana = nullptr, *tc_work_syn = nullptr;
  int tc_nwork_ana = 0, tc_nwork_syn = 0;
  int *dev_err = nullptr;  // device error word: DEV_ERR_* bits

  // geopotential-only solver (REXI_SOLVER_PHI): Z coefficients [nspec][12] (Z2, Z3, Z6
  // entries by degree offset), right-hand-side coefficients Q_p [5][nspec][max_batch],
  // sum of the beta_k; its factors [7][nrows][P] live in fac_fwd
  double *phi_zc = nullptr;
  double2 *phi_q = nullptr;
  double2 *phi_abf = nullptr;  // float-float plans: alpha, beta, beta alpha per pole ([3][P] float4)
  double2 sumb{};

  // float-float solves (REXI_SOLVE_FP32X2): the factors hold float-float values in place
  // of binary64 ones, and s_ff [3][nspec][B] the step's input states split the same way
  bool ff = false;
  double2 *s_ff = nullptr;
  // float-float factor layout: interleaved ([nrows][P][comp], the factors of a (row, pole)
  // adjacent) when a warp's lanes share their poles (max_batch >= 8: 8 or 16 states per
  // warp); otherwise the pole-fastest layout of the binary64 factors, where a warp's lanes
  // hold consecutive poles and its loads coalesce
  bool ffil = false;
  // float-float plans keep 7 of the 9 factors (compact_comp): g = tau G_n / alpha and the
  // Phi weight beta/d' tau Phibar / alpha (adjoint: -tau Phibar / conj(alpha) and
  // -beta/d' tau G_n / conj(alpha)) are formed in the sweep from these
  float2 *ffc_rows = nullptr;  // [nspec] tau G_n as float-float values
  float4 *ffc_ia = nullptr;    // [P] 1/alpha as float-float values

  // workspaces (max_batch)
  double2 *four = nullptr;     // [nlat][N+1][3 B] complex (FP64 or FP32 pairs in mixed mode)
  double2 *s_in = nullptr;     // [3][nspec][B]
  double2 *s_out = nullptr;    // [3][nspec][B]
  double2 *partial = nullptr;  // [3][nspec][slots][B]
  double2 *yscratch = nullptr; // [resident warps][Lmax][32]
  int resident_warps = 0, lmax = 0;
  unsigned *counter = nullptr;
  size_t partial_cap = 0;

  std::map<int, SolveLayout> layouts;  // per batch size
  // bumped whenever a slot layout is replaced (its device work list freed): objects that
  // cached views of the old one (ragged batches) rebuild them
  uint64_t layout_gen = 0;
  int slots_override = 0;
  // fused solve (binary64 delta solver): per batch size its layout, and whether the slot
  // layout above was chosen instead (rexi_tune, rexi_set_pole_slots, pole_slots)
  std::map<int, FusedLayout> fused;
  std::map<int, bool> use_slots;
  std::map<int, int> fused_tile;  // requested states per CTA tile (0: the default)
  std::map<int, int> fused_form;  // 0: register form; lean form with CTAs of 1: four warps, 2: two warps
  std::map<int, int> fused_groups; // requested CTAs per system's poles (0: the default)

  // optional per-stage timing with CUDA events on the launching stream
  bool prof = false;
  std::vector<cudaEvent_t> prof_ev;  // [calls][kStages + 1], in recording order
  std::vector<int> prof_sid;         // stage id of each recorded mark (kStages = end)
  std::vector<int> prof_n;           // marks recorded per call
  int prof_calls = 0, prof_cap = 0;
};

// components stored per (row, pole) for the delta solver's factors of this plan (the
// compact set for float-float plans)
inline int fac_ncomp(const Plan &pl) { return pl.ff ? F_NCOMPACT : F_NCOMP; }

enum Stage { ST_FFT_FWD = 0, ST_LEG_ANA, ST_SOLVE, ST_REDUCE, ST_LEG_SYN, ST_FFT_INV, ST_TRANS_IN,
             ST_TRANS_OUT, kStages };

// ---- kernels (launchers) ------------------------------------------------------------
cudaError_t launch_factor_setup(Plan &pl, bool adjoint, cudaStream_t st);
// geopotential-only solver (REXI_SOLVER_PHI): plan-time factors; per step the right-hand
// sides and the pentadiagonal solves into the slot partials, then the ordered reduction
cudaError_t launch_phi_factor(Plan &pl, cudaStream_t st);
cudaError_t launch_phi_solve(Plan &pl, const SolveLayout &lay, const double2 *sin, int B, cudaStream_t st);
cudaError_t launch_phi_reduce(Plan &pl, const SolveLayout &lay, const double2 *sin, double2 *sout, int B,
                              cudaStream_t st);
// f-sphere plans: closed-form per-degree solves and the pole sum, sin -> sout ([3][nspec][B])
cudaError_t launch_fsphere(Plan &pl, bool adjoint, const double2 *sin, double2 *sout, int B, bool single,
                           int pole, cudaStream_t st);
cudaError_t launch_solve(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin,
                         int B, int pole_begin, int pole_end, bool use_beta, cudaStream_t st);
// One plan's view for the solve kernels: factors, internal states, partial sums,
// systems and the lane layout of its batch.
struct SolveView {
  const double2 *fac;   // [F_NCOMP][nrows][P] (float-float: the compact set, interleaved when ffil)
  const double2 *sin;   // [3][nspec][B]
  double2 *part;        // [3][nspec][slots][B]
  const int4 *sys;      // per (m, p): {m, n0, len, row0}
  int P, N, B, bw, kk, slots, pole_begin, pole_end;
  int64_t nspec, nrows;
  const int32_t *slots_m;  // per zonal order slot count (<= slots), or null for slots everywhere
  int ffil;                // float-float factors interleaved (Plan::ffil)
  int adj;                 // adjoint factors (the compact float-float set forms g and the Phi weight per direction)
  const float2 *ffc_rows;  // compact float-float factors: tau G_n per idx
  const float4 *ffc_ia;    // compact float-float factors: 1/alpha per pole
  float2 ffc_tpb;          // tau Phibar as a float-float value
};
SolveView make_view(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin, double2 *part, int B,
                    int pole_begin, int pole_end);
// fused solve: eligible plans (binary64 delta solver on the rotating sphere) whose running
// sums fit in shared memory; sin -> sout ([3][nspec][B]) with no partial sums and no reduction
bool build_fused_layout(Plan &pl, int B, int tile, int form, int groups, FusedLayout &F);
bool build_fused_ragged(const std::vector<Plan *> &plans, const std::vector<int> &counts, FusedRagged &R);
void free_fused_ragged(FusedRagged &R);
cudaError_t launch_fused_ragged(const FusedRagged &R, double2 *ybuf, int num_sms, cudaStream_t st);
cudaError_t launch_solve_fused(Plan &pl, const FusedLayout &F, bool adjoint, const double2 *sin, double2 *sout,
                               int B, cudaStream_t st);
cudaError_t launch_solve_ragged(const SolveView *views_dev, const WorkItem *items, int nitems, double2 *ybuf,
                                int lmax, unsigned *counter, int resident_warps, bool ff, cudaStream_t st);
// float-float solves: convert n complex values in place (factors), or split n binary64
// states into out (float-float values in double2 slots)
cudaError_t launch_to_ff(Plan &pl, double2 *v, int64_t n, cudaStream_t st);
cudaError_t launch_split_state(Plan &pl, const double2 *in, double2 *out, int64_t n, cudaStream_t st);
// reads and clears DEV_ERR_RANGE after a synchronisation: REXI_ERANGE when set
rexi_status take_range_error(Plan &pl, const char *what);
cudaError_t launch_reduce(Plan &pl, const SolveLayout &lay, bool adjoint, const double2 *sin,
                          double2 *sout, int B, bool single_pole, int pole, cudaStream_t st);
cudaError_t launch_transpose_in(const double2 *user, double2 *sint, int64_t nspec, int B,
                                cudaStream_t st);
cudaError_t launch_transpose_out(const double2 *sint, double2 *user, int64_t nspec, int B, int N,
                                 cudaStream_t st);
// scales: binary64 arrays in the FP64 form, their binary32 copies in the mixed form
cudaError_t launch_fft_fwd(Plan &pl, const double *grid, double2 *four, int B,
                           const void *in_scale, const void *m_scale, cudaStream_t st);
cudaError_t launch_fft_inv(Plan &pl, const double2 *four, double *grid, int B,
                           const void *m_scale, const void *out_scale, cudaStream_t st);
cudaError_t launch_leg_ana(Plan &pl, const double2 *four, double2 *sint, int B,
                           const double *zdscale, cudaStream_t st);
cudaError_t launch_leg_syn(Plan &pl, const double2 *sint, double2 *four, int B,
                           const double *zdscale, cudaStream_t st);
cudaError_t launch_leg_ana_tc(Plan &pl, const double2 *four, double2 *sint, int B,
                              const double *zdscale, cudaStream_t st);
cudaError_t launch_leg_syn_tc(Plan &pl, const double2 *sint, double2 *four, int B,
                              const double *zdscale, cudaStream_t st);

void set_error(const std::string &msg);

}  // namespace rexi
