// C-ABI entry points of librexi (declared in include/rexi.h).
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <utility>
#include <string>

#include "rexi_internal.h"

struct rexi_plan {
  rexi::Plan *pl;
};

namespace rexi {

static thread_local std::string g_last_error;
void set_error(const std::string &msg) { g_last_error = msg; }

rexi_status build_plan(const rexi_params &prm, Plan *pl);
rexi_status get_layout(Plan &pl, int B, bool single, SolveLayout **out);
void free_plan(Plan *pl);
rexi_status step_static(Plan &pl, const void *in, void *out, int B, cudaStream_t st);
rexi_status tune_layout(Plan &pl, int B, int *slots_out, int *shape_out);
rexi_status set_layout(Plan &pl, int B, int slots, int shape, int *used);
const FusedLayout *fused_layout(Plan &pl, int B);

namespace {

rexi_status cuda_fail(const char *what, cudaError_t e) {
  set_error(std::string(what) + ": " + cudaGetErrorString(e));
  return REXI_ECUDA;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Event marks: a timed call records one event at the start of each stage it
// runs and one at its end; each interval is attributed to the stage that
// opened it.
// Stage boundaries of one call: NVTX ranges (a host-side timeline for profilers; no cost
// without one attached) and, when rexi_profile_enable is on, CUDA events on the stream.
const char *const kStageNames[kStages] = {"fft_fwd", "leg_ana", "solve", "reduce",
                                          "leg_syn", "fft_inv", "transpose_in", "transpose_out"};

struct Marks {
  Plan &pl;
  cudaStream_t st;
  int call = -1;
  bool open = false;
  Marks(Plan &p, cudaStream_t s, bool timed = true) : pl(p), st(s) {
    nvtxRangePushA("rexi");
    if (timed && pl.prof && pl.prof_calls < pl.prof_cap) {
      call = pl.prof_calls++;
      pl.prof_n[call] = 0;
    }
  }
  ~Marks() {
    if (open) nvtxRangePop();
    nvtxRangePop();
  }
  void mark(int stage) {
    if (open) nvtxRangePop();
    open = stage < kStages;
    if (open) nvtxRangePushA(kStageNames[stage]);
    if (call < 0) return;
    int &k = pl.prof_n[call];
    if (k > kStages) return;
    const size_t at = (size_t)call * (kStages + 1) + k;
    cudaEventRecord(pl.prof_ev[at], st);
    pl.prof_sid[at] = stage;
    ++k;
  }
};

rexi_status check_io2(const Plan &pl, const void *in, const void *out, int B, bool grid_in, bool grid_out);
rexi_status check_io(const Plan &pl, const void *in, const void *out, int B, bool grid) {
  return check_io2(pl, in, out, B, grid, grid);
}

rexi_status check_io2(const Plan &pl, const void *in, const void *out, int B, bool grid_in, bool grid_out) {
  if (!in || !out) {
    set_error("null device pointer");
    return REXI_EINVAL;
  }
  if (B < 1 || B > pl.prm.max_batch) {
    set_error("batch must be in [1, max_batch]");
    return REXI_EINVAL;
  }
  if (!aligned16(in) || !aligned16(out)) {
    set_error("device pointers must be 16-byte aligned");
    return REXI_EINVAL;
  }
  const size_t gbytes = (size_t)B * 3 * pl.nlat * pl.nlon * sizeof(double);
  const size_t sbytes = (size_t)B * 3 * pl.nspec * 2 * sizeof(double);
  const size_t ibytes = grid_in ? gbytes : sbytes, obytes = grid_out ? gbytes : sbytes;
  const char *a = static_cast<const char *>(in), *b = static_cast<const char *>(out);
  if (a < b + obytes && b < a + ibytes) {
    set_error("in and out overlap");
    return REXI_EINVAL;
  }
  return REXI_OK;
}

rexi_status ensure_adjoint_factors(Plan &pl) {
  if (pl.fac_adj || pl.prm.fsphere) return REXI_OK;
  const size_t n = (size_t)fac_ncomp(pl) * pl.nrows * pl.P;
  cudaError_t e = cudaMalloc(&pl.fac_adj, n * sizeof(double2));
  if (e != cudaSuccess) {
    pl.fac_adj = nullptr;
    set_error(std::string("adjoint factors: ") + cudaGetErrorString(e));
    return REXI_ENOMEM;
  }
  pl.bytes += n * sizeof(double2);
  e = launch_factor_setup(pl, true, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail("adjoint factor setup", e);
  if (pl.ff) {
    const rexi_status r = take_range_error(pl, "adjoint float-float factors");
    if (r != REXI_OK) {  // not kept: every adjoint call on this plan fails the same way
      cudaFree(pl.fac_adj);
      pl.fac_adj = nullptr;
      pl.bytes -= n * sizeof(double2);
      return r;
    }
  }
  return REXI_OK;
}

// Spectral REXI core on the plan's internal layout: s_in -> s_out.
rexi_status core(Plan &pl, int B, bool adjoint, cudaStream_t st, Marks &mk) {
  if (pl.prm.fsphere) {
    mk.mark(ST_SOLVE);
    cudaError_t e = launch_fsphere(pl, adjoint, pl.s_in, pl.s_out, B, false, 0, st);
    return e == cudaSuccess ? REXI_OK : cuda_fail("f-sphere solve", e);
  }
  SolveLayout *lay = nullptr;
  rexi_status r = get_layout(pl, B, false, &lay);
  if (r != REXI_OK) return r;
  if (pl.prm.solver == REXI_SOLVER_PHI) {
    mk.mark(ST_SOLVE);
    cudaError_t e = launch_phi_solve(pl, *lay, pl.s_in, B, st);
    if (e != cudaSuccess) return cuda_fail("phi solve", e);
    mk.mark(ST_REDUCE);
    e = launch_phi_reduce(pl, *lay, pl.s_in, pl.s_out, B, st);
    return e == cudaSuccess ? REXI_OK : cuda_fail("phi reduce", e);
  }
  const FusedLayout *fl = fused_layout(pl, B);
  if (fl) {  // the pole sum stays on chip: one kernel, outputs written once
    mk.mark(ST_SOLVE);
    cudaError_t e = launch_solve_fused(pl, *fl, adjoint, pl.s_in, pl.s_out, B, st);
    return e == cudaSuccess ? REXI_OK : cuda_fail("solve", e);
  }
  mk.mark(ST_SOLVE);
  cudaError_t e = launch_solve(pl, *lay, adjoint, pl.s_in, B, 0, pl.P, true, st);
  if (e != cudaSuccess) return cuda_fail("solve", e);
  mk.mark(ST_REDUCE);
  e = launch_reduce(pl, *lay, adjoint, pl.s_in, pl.s_out, B, false, 0, st);
  if (e != cudaSuccess) return cuda_fail("reduce", e);
  return REXI_OK;
}

rexi_status analyze(Plan &pl, const double *grid, int B, bool adjoint, cudaStream_t st, Marks &mk) {
  const bool f32 = pl.prm.precision == REXI_MIXED;  // the mixed form's FFTs scale in binary32
  const void *isc = adjoint ? (f32 ? (const void *)pl.scale_syn_out32 : pl.scale_syn_out)
                            : (f32 ? (const void *)pl.scale_ana_in32 : pl.scale_ana_in);
  const void *msc = adjoint ? (f32 ? (const void *)pl.mscale_c32 : pl.mscale_c)
                            : (f32 ? (const void *)pl.mscale_fwd32 : pl.mscale_fwd);
  const double *zd = adjoint ? pl.zd_ana_adj : pl.zd_one;
  mk.mark(ST_FFT_FWD);
  cudaError_t e = launch_fft_fwd(pl, grid, pl.four, B, isc, msc, st);
  if (e != cudaSuccess) return cuda_fail("fft forward", e);
  mk.mark(ST_LEG_ANA);
  e = pl.prm.precision == REXI_MIXED ? launch_leg_ana_tc(pl, pl.four, pl.s_in, B, zd, st)
                                     : launch_leg_ana(pl, pl.four, pl.s_in, B, zd, st);
  if (e != cudaSuccess) return cuda_fail("legendre analysis", e);
  return REXI_OK;
}

rexi_status synthesize(Plan &pl, const double2 *spec, double *grid, int B, bool adjoint,
                       cudaStream_t st, Marks &mk) {
  const double *zd = adjoint ? pl.zd_mone : pl.zd_syn;
  const bool f32 = pl.prm.precision == REXI_MIXED;
  const void *msc = adjoint ? (f32 ? (const void *)pl.mscale_adj32 : pl.mscale_adj)
                            : (f32 ? (const void *)pl.mscale_one32 : pl.mscale_one);
  const void *osc = adjoint ? (f32 ? (const void *)pl.scale_ana_in32 : pl.scale_ana_in)
                            : (f32 ? (const void *)pl.scale_syn_out32 : pl.scale_syn_out);
  mk.mark(ST_LEG_SYN);
  cudaError_t e = pl.prm.precision == REXI_MIXED ? launch_leg_syn_tc(pl, spec, pl.four, B, zd, st)
                                                 : launch_leg_syn(pl, spec, pl.four, B, zd, st);
  if (e != cudaSuccess) return cuda_fail("legendre synthesis", e);
  mk.mark(ST_FFT_INV);
  e = launch_fft_inv(pl, pl.four, grid, B, msc, osc, st);
  if (e != cudaSuccess) return cuda_fail("fft inverse", e);
  mk.mark(kStages);
  return REXI_OK;
}

rexi_status step_impl(rexi_plan *plan, const void *in, void *out, int32_t B, void *stream, bool adjoint) {
  if (!plan || !plan->pl) {
    set_error("null plan");
    return REXI_EINVAL;
  }
  Plan &pl = *plan->pl;
  const bool grid = pl.prm.layout == REXI_GRID;
  rexi_status r = check_io(pl, in, out, B, grid);
  if (r != REXI_OK) return r;
  if (adjoint && pl.prm.solver == REXI_SOLVER_PHI) {
    set_error("rexi_step_adjoint: not available for REXI_SOLVER_PHI plans");
    return REXI_EINVAL;
  }
  if (adjoint && (r = ensure_adjoint_factors(pl)) != REXI_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Marks mk(pl, st);
  if (grid) {
    if ((r = analyze(pl, static_cast<const double *>(in), B, adjoint, st, mk)) != REXI_OK) return r;
  } else {
    mk.mark(ST_TRANS_IN);
    cudaError_t e = launch_transpose_in(static_cast<const double2 *>(in), pl.s_in, pl.nspec, B, st);
    if (e != cudaSuccess) return cuda_fail("transpose", e);
  }
  if ((r = core(pl, B, adjoint, st, mk)) != REXI_OK) return r;
  if (grid) return synthesize(pl, pl.s_out, static_cast<double *>(out), B, adjoint, st, mk);
  mk.mark(ST_TRANS_OUT);
  cudaError_t e = launch_transpose_out(pl.s_out, static_cast<double2 *>(out), pl.nspec, B, pl.N, st);
  if (e != cudaSuccess) return cuda_fail("transpose", e);
  mk.mark(kStages);
  return REXI_OK;
}

}  // namespace
}  // namespace rexi

using namespace rexi;

extern "C" {

size_t rexi_params_size(void) { return sizeof(rexi_params); }

void rexi_params_default(rexi_params *p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->ntrunc = 63;
  p->nlat = 96;
  p->nlon = 192;
  p->M = 128;
  p->h = 0.2;
  p->tau = 3600.0;
  p->radius = 6.37122e6;
  p->omega = 7.292e-5;
  p->gravity = 9.80616;
  p->mean_depth = 1.0e4;
  p->normalize = 1;
  p->precision = REXI_FP64;
  p->layout = REXI_GRID;
  p->max_batch = 1;
}

rexi_status rexi_coefficients(int32_t M, double h, int32_t normalize, double *alpha, double *beta,
                              int32_t *P, double *eps) {
  if (M < 1 || !(h > 0.0) || !alpha || !beta) {
    set_error("rexi_coefficients: need M >= 1, h > 0 and output arrays");
    return REXI_EINVAL;
  }
  std::vector<cplx> al, be;
  double e0 = 0;
  rexi_coeffs_host(M, h, normalize != 0, al, be, &e0);
  for (size_t k = 0; k < al.size(); ++k) {
    alpha[2 * k] = al[k].real();
    alpha[2 * k + 1] = al[k].imag();
    beta[2 * k] = be[k].real();
    beta[2 * k + 1] = be[k].imag();
  }
  if (P) *P = (int32_t)al.size();
  if (eps) *eps = e0;
  return REXI_OK;
}

rexi_status rexi_plan_create(const rexi_params *prm, rexi_plan **out) {
  if (!out) {
    set_error("null output pointer");
    return REXI_EINVAL;
  }
  *out = nullptr;
  if (!prm) {
    set_error("null params");
    return REXI_EINVAL;
  }
  const rexi_params &p = *prm;
  if (p.ntrunc < 1 || p.max_batch < 1 || !(p.tau > 0) || !(p.radius > 0) || !(p.gravity > 0) ||
      !(p.mean_depth > 0) || (p.precision != REXI_FP64 && p.precision != REXI_MIXED) ||
      (p.layout != REXI_GRID && p.layout != REXI_SPECTRAL)) {
    set_error("rexi_plan_create: invalid truncation, batch, constants, precision or layout");
    return REXI_EINVAL;
  }
  if ((p.alpha == nullptr) != (p.beta == nullptr) || (p.alpha && p.npoles < 1) ||
      (!p.alpha && (p.M < 1 || !(p.h > 0)))) {
    set_error("rexi_plan_create: give both alpha and beta with npoles >= 1, or M >= 1 and h > 0");
    return REXI_EINVAL;
  }
  if (p.nlat % 2 != 0 || p.nlon % 2 != 0 || p.nlat < p.ntrunc + 1 || p.nlon < 2 * p.ntrunc + 2) {
    set_error("rexi_plan_create: need even nlat >= N + 1 and even nlon >= 2N + 2");
    return REXI_EINVAL;
  }
  {
    int m = p.nlon;
    for (int q : {2, 3, 5})
      while (m % q == 0) m /= q;
    if (m != 1) {
      set_error("rexi_plan_create: nlon must be a product of 2, 3 and 5");
      return REXI_EINVAL;
    }
  }
  if (p.precision == REXI_MIXED && p.layout != REXI_GRID) {
    set_error("rexi_plan_create: REXI_MIXED applies to the grid layout (the spectral step is all FP64)");
    return REXI_EINVAL;
  }
  if ((p.solver != REXI_SOLVER_DELTA && p.solver != REXI_SOLVER_PHI) || (p.solver == REXI_SOLVER_PHI && p.fsphere)) {
    set_error("rexi_plan_create: solver must be REXI_SOLVER_DELTA or REXI_SOLVER_PHI (the latter on the rotating sphere)");
    return REXI_EINVAL;
  }
  {
    const int64_t Pfull = p.alpha ? p.npoles : 2 * ((int64_t)p.M + kGaussTerms) + 1;
    if ((p.pole_begin != 0 || p.pole_end != 0) &&
        (p.pole_begin < 0 || p.pole_end <= p.pole_begin || p.pole_end > Pfull)) {
      set_error("rexi_plan_create: need 0 <= pole_begin < pole_end <= P (P = " + std::to_string(Pfull) + ")");
      return REXI_EINVAL;
    }
  }
  if ((p.solve_arith != REXI_SOLVE_FP64 && p.solve_arith != REXI_SOLVE_FP32X2) ||
      (p.solve_arith == REXI_SOLVE_FP32X2 && p.fsphere)) {
    set_error("rexi_plan_create: solve_arith must be REXI_SOLVE_FP64 or REXI_SOLVE_FP32X2 (the latter on the "
              "rotating sphere)");
    return REXI_EINVAL;
  }
  Plan *pl = new Plan();
  rexi_status r = build_plan(p, pl);
  if (r != REXI_OK) {
    free_plan(pl);
    return r;
  }
  *out = new rexi_plan{pl};
  return REXI_OK;
}

rexi_status rexi_step(rexi_plan *plan, const void *in_dev, void *out_dev, int32_t batch, void *stream) {
  return step_impl(plan, in_dev, out_dev, batch, stream, false);
}

rexi_status rexi_step_adjoint(rexi_plan *plan, const void *gout_dev, void *gin_dev, int32_t batch,
                              void *stream) {
  return step_impl(plan, gout_dev, gin_dev, batch, stream, true);
}

rexi_status rexi_analyze(rexi_plan *plan, const void *grid_dev, void *spec_dev, int32_t B, void *stream) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  rexi_status r = check_io2(pl, grid_dev, spec_dev, B, true, false);
  if (r != REXI_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Marks mk(pl, st);
  mk.call = -1;
  if ((r = analyze(pl, static_cast<const double *>(grid_dev), B, false, st, mk)) != REXI_OK) return r;
  cudaError_t e = launch_transpose_out(pl.s_in, static_cast<double2 *>(spec_dev), pl.nspec, B, pl.N, st);
  return e == cudaSuccess ? REXI_OK : cuda_fail("transpose", e);
}

rexi_status rexi_synthesize(rexi_plan *plan, const void *spec_dev, void *grid_dev, int32_t B, void *stream) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  rexi_status r = check_io2(pl, spec_dev, grid_dev, B, false, true);
  if (r != REXI_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = launch_transpose_in(static_cast<const double2 *>(spec_dev), pl.s_out, pl.nspec, B, st);
  if (e != cudaSuccess) return cuda_fail("transpose", e);
  Marks mk(pl, st);
  mk.call = -1;
  return synthesize(pl, pl.s_out, static_cast<double *>(grid_dev), B, false, st, mk);
}

rexi_status rexi_solve_pole(rexi_plan *plan, int32_t k, const void *in_dev, void *out_dev, int32_t B,
                            void *stream) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  if (k < 0 || k >= pl.P) { set_error("pole index out of range"); return REXI_EINVAL; }
  if (pl.prm.solver == REXI_SOLVER_PHI) { set_error("rexi_solve_pole: not available for REXI_SOLVER_PHI plans"); return REXI_EINVAL; }
  rexi_status r = check_io(pl, in_dev, out_dev, B, false);
  if (r != REXI_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  SolveLayout *lay = nullptr;
  if (!pl.prm.fsphere && (r = get_layout(pl, B, true, &lay)) != REXI_OK) return r;
  cudaError_t e = launch_transpose_in(static_cast<const double2 *>(in_dev), pl.s_in, pl.nspec, B, st);
  if (pl.prm.fsphere) {
    if (e == cudaSuccess) e = launch_fsphere(pl, false, pl.s_in, pl.s_out, B, true, k, st);
  } else {
    if (e == cudaSuccess) e = launch_solve(pl, *lay, false, pl.s_in, B, k, k + 1, true, st);
    if (e == cudaSuccess) e = launch_reduce(pl, *lay, false, pl.s_in, pl.s_out, B, true, k, st);
  }
  if (e == cudaSuccess) e = launch_transpose_out(pl.s_out, static_cast<double2 *>(out_dev), pl.nspec, B, pl.N, st);
  return e == cudaSuccess ? REXI_OK : cuda_fail("solve_pole", e);
}

rexi_status rexi_integrate(rexi_plan *plan, const void *in_dev, void *out_dev, int32_t batch, int32_t nsteps,
                           void *stream) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  if (nsteps < 1) { set_error("rexi_integrate: nsteps must be >= 1"); return REXI_EINVAL; }
  const bool grid = pl.prm.layout == REXI_GRID;
  rexi_status r = check_io(pl, in_dev, out_dev, batch, grid);
  if (r != REXI_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Marks mk(pl, st, false);
  if (grid) {
    if ((r = analyze(pl, static_cast<const double *>(in_dev), batch, false, st, mk)) != REXI_OK) return r;
  } else {
    mk.mark(ST_TRANS_IN);
    cudaError_t e = launch_transpose_in(static_cast<const double2 *>(in_dev), pl.s_in, pl.nspec, batch, st);
    if (e != cudaSuccess) return cuda_fail("transpose", e);
  }
  // the spectral state ping-pongs between the plan's two internal buffers: each step
  // reads s_in and writes s_out, and the pointers swap (kernels take them at launch)
  double2 *const s_in0 = pl.s_in, *const s_out0 = pl.s_out;
  for (int k = 0; k < nsteps && r == REXI_OK; ++k) {
    r = core(pl, batch, false, st, mk);
    std::swap(pl.s_in, pl.s_out);
  }
  double2 *const result = pl.s_in;
  pl.s_in = s_in0;
  pl.s_out = s_out0;
  if (r != REXI_OK) return r;
  if (grid) return synthesize(pl, result, static_cast<double *>(out_dev), batch, false, st, mk);
  mk.mark(ST_TRANS_OUT);
  cudaError_t e = launch_transpose_out(result, static_cast<double2 *>(out_dev), pl.nspec, batch, pl.N, st);
  return e == cudaSuccess ? REXI_OK : cuda_fail("transpose", e);
}

rexi_status rexi_step_static(rexi_plan *plan, const void *in_dev, void *out_dev, int32_t batch, void *stream) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  if (pl.prm.layout != REXI_SPECTRAL || pl.prm.solver == REXI_SOLVER_PHI) {
    set_error("rexi_step_static: needs a REXI_SPECTRAL plan with REXI_SOLVER_DELTA");
    return REXI_EINVAL;
  }
  rexi_status r = check_io(pl, in_dev, out_dev, batch, false);
  if (r != REXI_OK) return r;
  return step_static(pl, in_dev, out_dev, batch, static_cast<cudaStream_t>(stream));
}

rexi_status rexi_get_coefficients(const rexi_plan *plan, double *alpha, double *beta, int32_t *P) {
  if (!plan || !plan->pl || !alpha || !beta) { set_error("null argument"); return REXI_EINVAL; }
  const Plan &pl = *plan->pl;
  for (int k = 0; k < pl.P; ++k) {
    alpha[2 * k] = pl.alpha[k].real();
    alpha[2 * k + 1] = pl.alpha[k].imag();
    beta[2 * k] = pl.beta[k].real();
    beta[2 * k + 1] = pl.beta[k].imag();
  }
  if (P) *P = pl.P;
  return REXI_OK;
}

rexi_status rexi_tune(rexi_plan *plan, int32_t batch, int32_t *slots, int32_t *shape) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  if (batch < 1 || batch > pl.prm.max_batch) { set_error("rexi_tune: batch must be in [1, max_batch]"); return REXI_EINVAL; }
  int s = 0, sh = 0;
  if (pl.prm.fsphere) {  // no banded solves, nothing to tune
    if (slots) *slots = 0;
    if (shape) *shape = 0;
    return REXI_OK;
  }
  rexi_status r = tune_layout(pl, batch, &s, &sh);
  if (r == REXI_OK && slots) *slots = s;
  if (r == REXI_OK && shape) *shape = sh;
  return r;
}

rexi_status rexi_set_pole_slots(rexi_plan *plan, int32_t batch, int32_t slots, int32_t shape, int32_t *used) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  if (batch < 1 || batch > pl.prm.max_batch || (shape < 2 && slots < 1) || slots < 0 || shape < 0 || shape > 4) {
    set_error("rexi_set_pole_slots: batch must be in [1, max_batch], shape 0 to 4, slots >= 1 for "
              "shapes 0 and 1 and >= 0 for shapes 2 to 4");
    return REXI_EINVAL;
  }
  if (pl.prm.fsphere) {  // no banded solves, no layout
    if (shape >= 2) {
      set_error("rexi_set_pole_slots: the fused solve (shapes 2 to 4) does not apply to f-sphere plans");
      return REXI_EINVAL;
    }
    if (used) *used = 0;
    return REXI_OK;
  }
  int u = 0;
  rexi_status r = set_layout(pl, batch, slots, shape, &u);
  if (r == REXI_OK && used) *used = u;
  return r;
}

rexi_status rexi_plan_info(const rexi_plan *plan, int64_t *info, int32_t n) {
  if (!plan || !plan->pl || !info) { set_error("null argument"); return REXI_EINVAL; }
  const Plan &pl = *plan->pl;
  int slots = 0;  // 0 when steps of max_batch states use the fused solve (no slot partials)
  auto it = pl.layouts.find(pl.prm.max_batch);
  auto us = pl.use_slots.find(pl.prm.max_batch);
  if (it != pl.layouts.end() && us != pl.use_slots.end() && us->second) slots = it->second.slots;
  const int64_t v[8] = {pl.N, pl.nspec, pl.P, pl.nlat, pl.nlon, pl.prm.max_batch, slots, (int64_t)pl.bytes};
  for (int i = 0; i < n && i < 8; ++i) info[i] = v[i];
  return REXI_OK;
}

void rexi_destroy(rexi_plan *plan) {
  if (!plan) return;
  free_plan(plan->pl);
  delete plan;
}

rexi_status rexi_profile_enable(rexi_plan *plan, int32_t max_calls) {
  if (!plan || !plan->pl || max_calls < 0) { set_error("bad argument"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  for (cudaEvent_t ev : pl.prof_ev) cudaEventDestroy(ev);
  pl.prof_ev.clear();
  pl.prof_calls = 0;
  pl.prof_cap = max_calls;
  pl.prof = max_calls > 0;
  pl.prof_ev.resize((size_t)max_calls * (kStages + 1));
  pl.prof_sid.assign((size_t)max_calls * (kStages + 1), kStages);
  pl.prof_n.assign((size_t)max_calls, 0);
  for (auto &ev : pl.prof_ev) {
    cudaError_t e = cudaEventCreate(&ev);
    if (e != cudaSuccess) return cuda_fail("event create", e);
  }
  return REXI_OK;
}

rexi_status rexi_profile_read(rexi_plan *plan, double *stage_ms, int32_t n, int32_t *calls) {
  if (!plan || !plan->pl || !stage_ms) { set_error("bad argument"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  std::vector<double> acc(kStages, 0.0);
  for (int c = 0; c < pl.prof_calls; ++c) {
    const size_t base = (size_t)c * (kStages + 1);
    const int k = pl.prof_n[c];
    if (k < 2) continue;
    cudaError_t e = cudaEventSynchronize(pl.prof_ev[base + k - 1]);
    if (e != cudaSuccess) return cuda_fail("event sync", e);
    for (int i = 0; i + 1 < k; ++i) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, pl.prof_ev[base + i], pl.prof_ev[base + i + 1]);
      if (e != cudaSuccess) return cuda_fail("event time", e);
      const int sid = pl.prof_sid[base + i];
      if (sid >= 0 && sid < kStages) acc[sid] += ms;
    }
  }
  for (int s = 0; s < n && s < kStages; ++s) stage_ms[s] = acc[s];
  if (calls) *calls = pl.prof_calls;
  pl.prof_calls = 0;
  return REXI_OK;
}

rexi_status rexi_check_device(rexi_plan *plan) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  Plan &pl = *plan->pl;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail("rexi_check_device", e);
  int flag = 0;
  e = cudaMemcpy(&flag, pl.dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail("rexi_check_device", e);
  if (flag) cudaMemset(pl.dev_err, 0, sizeof(int));
  if (flag & DEV_ERR_TIMEOUT) {
    set_error("a bounded device-side wait expired; the affected outputs were not written");
    return REXI_ETIMEOUT;
  }
  if (flag & DEV_ERR_RANGE) {
    set_error("a float-float solve met a value beyond binary32's range (|x| > 3.4e38); its outputs are "
              "not finite; use REXI_SOLVE_FP64 for such states");
    return REXI_ERANGE;
  }
  return REXI_OK;
}

rexi_status rexi_inject_device_error(rexi_plan *plan, int32_t bits) {
  if (!plan || !plan->pl) { set_error("null plan"); return REXI_EINVAL; }
  if (bits <= 0 || (bits & ~(DEV_ERR_TIMEOUT | DEV_ERR_RANGE))) {
    set_error("rexi_inject_device_error: bits must be a non-empty set of 1 (timeout) and 2 (range)");
    return REXI_EINVAL;
  }
  Plan &pl = *plan->pl;
  cudaError_t e = cudaDeviceSynchronize();
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, pl.dev_err, sizeof(int), cudaMemcpyDeviceToHost);
  flag |= bits;
  if (e == cudaSuccess) e = cudaMemcpy(pl.dev_err, &flag, sizeof(int), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? REXI_OK : cuda_fail("rexi_inject_device_error", e);
}

const char *rexi_last_error(void) { return g_last_error.c_str(); }

}  // extern "C"
