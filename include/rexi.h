/*
 * rexi.h -- C-ABI of librexi: one T-REXI time step of the linearised
 * shallow-water equations (SWE) on the rotating sphere, on one GB300 GPU.
 *
 * Method (Schreiber & Loft, "A parallel time-integrator for solving the
 * linearized shallow water equations on the rotating sphere", Sec. 4-5,
 * Algorithm 1):
 *
 *     U(t + tau)  ~  Re  sum_{k=1}^{P}  beta_k (alpha_k + tau L)^{-1} U(t)
 *
 * with L the linear SWE operator of Eq. (1) in vorticity-divergence form and
 * (alpha_k, beta_k) the T-REXI poles of Sec. 4.1.  This is the paper's form
 * (alpha + L); the equivalent form sum beta'(alpha' - tau L)^{-1} has
 * alpha' = -alpha, beta' = -beta.  L is block-diagonal in the zonal
 * wavenumber m, so every (pole, m) pair is an independent banded solve in the
 * spherical-harmonic degree n (Sec. 5).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Spectral state: complex128 (interleaved re, im doubles), layout
 *   [batch][3][nspec], fields (Phi, zeta, delta) = (geopotential perturbation
 *   g h' in m^2/s^2, relative vorticity in 1/s, divergence in 1/s); within a
 *   field the coefficients xi_n^m, 0 <= m <= n <= N, are m-major:
 *   idx(m, n) = m (2N + 3 - m) / 2 + (n - m),  nspec = (N + 1)(N + 2) / 2.
 *   Orthonormal associated Legendre functions, int_{-1}^{1} Pbar^2 dmu = 1,
 *   no Condon-Shortley phase; a real field is sum over m = -N..N with
 *   xi^{-m} = conj(xi^m).  zeta_0^0 and delta_0^0 are not state variables:
 *   ignored on input, zero on output.  m = 0 outputs are real.
 * Grid state: float64, layout [batch][3][nlat][nlon], fields (h', u, v) in
 *   (m, m/s, m/s) on the Gaussian grid: latitude j = 0..nlat-1 from north to
 *   south (mu_j = sin(lat_j) are the Gauss-Legendre nodes, descending),
 *   longitude lambda_i = 2 pi i / nlon.  Robert's cos(lat) scaling (Sec. 3) is
 *   applied inside.
 * Device pointers: every in/out pointer below named *_dev is a device pointer
 *   to caller-owned, contiguous, 16-byte aligned memory; in and out must not
 *   overlap (REXI_EINVAL).  The plan owns every other allocation.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream).  Calls
 *   enqueue work and return without synchronising the host; no device memory
 *   is allocated inside rexi_step / rexi_step_adjoint once a batch size has
 *   been seen by the plan (its work list is cached), so those calls can be
 *   captured in a CUDA graph after a first eager call with the same batch.
 *   Such a graph holds that batch's solve layout: rexi_tune or
 *   rexi_set_pole_slots for the batch afterwards frees it, and the graph must be
 *   captured again.
 *   A plan's workspaces (transposed states, Fourier data, slot partials) serve
 *   one call at a time: calls on one plan must be ordered on the GPU (one
 *   stream, or events between streams); independent plans may run
 *   concurrently.
 * Errors: negative rexi_status; rexi_last_error() gives a thread-local
 *   message.  A CUDA launch error is reported by the call that launched.
 */
#ifndef REXI_H
#define REXI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  REXI_OK = 0,
  REXI_EINVAL = -1,   /* bad argument, size or alignment */
  REXI_ENOMEM = -2,   /* device or host allocation failed */
  REXI_ECUDA = -3,    /* a CUDA runtime call or kernel launch failed */
  REXI_ERANGE = -4,   /* tau * max|omega| outside the poles' valid range (strict plans only);
                         for REXI_SOLVE_FP32X2: a value beyond binary32's range */
  REXI_ETIMEOUT = -5  /* a bounded device-side wait expired */
} rexi_status;

enum { REXI_FP64 = 0,      /* every transform in FP64 */
       REXI_MIXED = 1 };   /* Legendre contractions as 3xTF32 tensor-core products with FP32
                              accumulation and FP32 longitude FFTs.  The banded solves and the
                              beta-weighted pole sum follow `solve_arith` in both forms
                              (binary64 by default). */
enum { REXI_GRID = 0,      /* rexi_step in/out are grid states */
       REXI_SPECTRAL = 1 }; /* rexi_step in/out are spectral states */
enum { REXI_SOLVER_DELTA = 0, /* per (pole, m, parity): Phi and zeta eliminated, a tridiagonal
                                 system in delta (default) */
       REXI_SOLVER_PHI = 1 };  /* the paper's geopotential-only system (Sec. 4.3 and 5): the Phi
                                 equation multiplied through by D^2, D = alpha^2 + tau^2 f^2, so
                                 that its coefficients are polynomials in mu; Galerkin-truncated
                                 it couples degrees n, n +- 2, n +- 4 (a pentadiagonal system
                                 per parity).  delta and zeta follow from the Phi and zeta rows
                                 of the system in spectral space.  Truncating the multiplied
                                 equation is a different discretisation from truncating L, so
                                 the result differs from REXI_SOLVER_DELTA at the highest
                                 degrees (it agrees in the interior of a band-limited state). */

enum { REXI_SOLVE_FP64 = 0,    /* banded solves and pole sum in binary64 (default) */
       REXI_SOLVE_FP32X2 = 1 }; /* the same solves and pole sum in float-float arithmetic: every
                                  value is an unevaluated pair hi + lo of binary32 numbers
                                  (48-bit significand, unit roundoff ~3.6e-15; Dekker's
                                  double-length arithmetic with error-free sums and FMA
                                  products), run on the FP32 pipes.  The factors are built in
                                  binary64 and stored as pairs; inputs and outputs stay
                                  binary64.  Values must lie in binary32's range: magnitudes
                                  above ~3e38 overflow and below ~1e-31 lose relative precision
                                  (the SWE states and factors of Sec. 6 are within 1e-20 .. 1e6).
                                  Either solver, on the rotating sphere only. */

typedef struct rexi_plan rexi_plan;
typedef struct rexi_ragged rexi_ragged;

/* Plan parameters.  Defaults (rexi_params_default): earth constants of
 * Sec. 6 (a = 6.37122e6 m, Omega = 7.292e-5 1/s, g = 9.80616 m/s^2,
 * Hbar = 1e4 m), h = 0.2, normalize = 1, FP64, grid layout, max_batch = 1. */
typedef struct {
  int32_t ntrunc;       /* N: triangular truncation, 1 <= N */
  int32_t nlat, nlon;   /* Gaussian grid; nlat even, nlat >= N + 1, nlon even, nlon >= 2N + 2,
                           nlon = 2^a 3^b 5^c (the Legendre tables are built for every layout) */
  int32_t M;            /* Gaussian basis functions per side (Sec. 4.1); P = 2 (M + 11) + 1 */
  double h;             /* width parameter of the Gaussian basis (Sec. 4.1) */
  double tau;           /* time-step size (s) */
  double radius, omega, gravity, mean_depth; /* a, Omega, g, Hbar */
  int32_t normalize;    /* 1: beta <- beta / sum(beta/alpha) (Sec. 6.1) */
  int32_t precision;    /* REXI_FP64 | REXI_MIXED */
  int32_t layout;       /* REXI_GRID | REXI_SPECTRAL */
  int32_t max_batch;    /* largest batch passed to rexi_step (sizes workspaces) */
  int32_t strict_range; /* 1: plan creation fails with REXI_ERANGE when tau * max|omega|
                           exceeds h (M - 10), the range where Re of the REXI symbol
                           matches cos to the fit level */
  int32_t pole_slots;   /* 0: the default solve -- for batches of up to four states with
                           binary64 solves of the delta solver on the rotating sphere, the
                           fused solve that keeps the pole sum on chip (one kernel, every
                           output written once), else the pole-slot solve (rexi_tune picks
                           per batch); > 0: the pole-slot solve with this many pole groups
                           summed separately, then reduced in slot order (a deterministic
                           tuning knob, any >= 1) */
  const double *alpha;  /* optional: P complex poles (re, im interleaved); NULL -> computed */
  const double *beta;   /* optional: P complex weights, used as given (no renormalisation) */
  int32_t npoles;       /* P when alpha/beta are given */
  int32_t fsphere;      /* 1: constant Coriolis parameter f = 2 Omega (the f-sphere of Sec. 4,
                           used for the eigenvalue analysis of Sec. 6.3): every degree n is a
                           closed 3x3 system solved in closed form, no banded solves; 0: the
                           rotating sphere, f = 2 Omega mu (default).  rexi_ragged_create
                           rejects f-sphere plans. */
  int32_t solver;       /* REXI_SOLVER_DELTA | REXI_SOLVER_PHI.  REXI_SOLVER_PHI needs the
                           rotating sphere (fsphere = 0) and serves rexi_step,
                           rexi_analyze / rexi_synthesize and rexi_tune only:
                           rexi_step_adjoint, rexi_step_static, rexi_solve_pole and
                           rexi_ragged_create return REXI_EINVAL for such plans. */
  int32_t solve_arith;  /* REXI_SOLVE_FP64 | REXI_SOLVE_FP32X2: arithmetic of the banded solves
                           and the beta-weighted pole sum (the transforms follow `precision`).
                           rexi_ragged_create needs the same value on every plan. */
  int32_t pole_begin, pole_end; /* 0, 0: every pole.  Otherwise the plan keeps only the poles
                           k in [pole_begin, pole_end) of the full ascending set (computed,
                           and renormalised over the full set, or given by alpha/beta), and
                           rexi_step returns the partial sum
                             Re sum_{pole_begin <= k < pole_end} beta_k (alpha_k + tau L)^{-1} U,
                           transforms included: the plans of a partition of the poles return
                           outputs that add up to the full step (the paper's even split of
                           the REXI terms over ranks and one reduction, Sec. 6.4; the sum is
                           the caller's, e.g. an allreduce).  Such a plan's P and
                           rexi_get_coefficients are those of its own poles; every call works
                           on them.  Needs 0 <= pole_begin < pole_end <= P. */
} rexi_params;

/* Fill *p with the defaults above (ntrunc = 63, nlat = 96, nlon = 192, M = 128,
 * tau = 3600).  Host only. */
void rexi_params_default(rexi_params *p);

/* sizeof(rexi_params) as compiled into the library, so that a binding can check that
 * its copy of the struct matches before passing one (no counterpart in the paper).  Host
 * only. */
size_t rexi_params_size(void);

/* T-REXI coefficients on the host, no GPU needed (Sec. 4.1; Sec. 6.1 for the
 * renormalisation).  alpha_n = h (mu + i n), n = -(M+11)..(M+11) ascending,
 * beta_n = h sum_{l+m=n} Re(b_m) a_l with the refitted Gaussian rational
 * approximation (mu, a_l) and b_m = e^{h^2} e^{-i m h}.  alpha and beta must
 * hold 2P doubles each (P = 2(M+11)+1, re/im interleaved); *P receives P and
 * *eps the x = 0 residual 1 - sum beta/alpha before renormalisation (may be
 * NULL).  Returns REXI_EINVAL for M < 1 or h <= 0. */
rexi_status rexi_coefficients(int32_t M, double h, int32_t normalize,
                              double *alpha, double *beta, int32_t *P, double *eps);

/* Create a plan on the current CUDA device: Gaussian grid, Legendre tables,
 * REXI poles, the per-(pole, m, n) factors of the banded solves for the step
 * (those of the adjoint are built on the first rexi_step_adjoint call), and
 * workspaces for max_batch states.  Allocates device memory; synchronises the
 * device once.  *out is NULL on failure (REXI_ENOMEM when the device memory does
 * not suffice; REXI_ERANGE when a REXI_SOLVE_FP32X2 plan's factors exceed
 * binary32's range, as do those of rexi_step_adjoint's first call). */
rexi_status rexi_plan_create(const rexi_params *params, rexi_plan **out);

/* One T-REXI step (Algorithm 1): out = Re sum_k beta_k (alpha_k + tau L)^{-1} in,
 * with the spherical-harmonic transforms of Sec. 3 around it in the grid layout.
 * in_dev/out_dev: [batch][3][nspec] complex128 (REXI_SPECTRAL) or
 * [batch][3][nlat][nlon] float64 (REXI_GRID).  1 <= batch <= max_batch. */
rexi_status rexi_step(rexi_plan *plan, const void *in_dev, void *out_dev,
                      int32_t batch, void *stream);

/* Transpose of rexi_step for the Euclidean inner products (sum x y on the grid,
 * Re sum conj(x) y on coefficients): sum_k conj(beta_k) (conj(alpha_k) + tau L^H)^{-1}
 * framed by the transposed transforms.  Gives dJ/dU0 from dJ/dU1 (no paper
 * counterpart; the adjoint of the paper's operator).  Same layouts as rexi_step. */
rexi_status rexi_step_adjoint(rexi_plan *plan, const void *gout_dev, void *gin_dev,
                              int32_t batch, void *stream);

/* nsteps >= 1 consecutive T-REXI steps from in_dev, the result in out_dev (same layouts
 * as rexi_step): the state stays in spectral space between steps (the grid layout
 * analyses once at the start and synthesises once at the end), ping-ponging between
 * the plan's two internal buffers, so a long time integration (Sec. 6.2) costs one
 * launch sequence per step and no transforms in between.  For spectral plans the
 * result equals nsteps rexi_step calls bit for bit; for grid plans it differs from
 * them only by the rounding of the skipped intermediate transforms.  No device memory
 * is allocated once the batch size has been seen. */
rexi_status rexi_integrate(rexi_plan *plan, const void *in_dev, void *out_dev, int32_t batch, int32_t nsteps,
                           void *stream);

/* Allocation-free spectral step (no counterpart in the paper).  Some callers
 * cannot allocate device memory while they step -- for example a time loop
 * inside an application that hands all device memory out at start-up, or code
 * that must not re-enter an allocator.  This entry point computes the same
 * result as rexi_step on a REXI_SPECTRAL plan (up to the summation order of the
 * poles) and allocates nothing: every per-call scratch buffer lives in one
 * file-scope device array of 64 MiB that each device loading the library holds
 * until exit.  The plan's read-only tables and the caller's in/out buffers are
 * used as usual.
 *   - Sizes whose scratch would exceed 64 MiB (3 nspec batch x 32 B for the two
 *     state copies, plus the pole-slot partial sums, the sweep buffers of four
 *     warps per SM and the work list) return REXI_EINVAL with the needed size.
 *     The sweep buffers grow with the GPU's number of SMs and with N but not with
 *     the batch, so the largest truncation served at all depends on the GPU (on a
 *     152-SM GB300, N up to about 170 for one state); the message says when no
 *     batch fits.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current and caches it for the life
 *     of the device context; make that first call before any stream capture.
 *     First calls from several host threads are serialised by a lock.
 *   - All calls share the one array and it keeps the last call's contents; the
 *     work counter is cleared on the stream at the start of every call.  Calls
 *     that overlap on the GPU (other streams, other threads) race on it.
 * Plan layout must be REXI_SPECTRAL; in/out as for rexi_step. */
rexi_status rexi_step_static(rexi_plan *plan, const void *in_dev, void *out_dev,
                             int32_t batch, void *stream);

/* Spectral <-> grid transforms of the plan's grid (Sec. 3): analysis maps
 * grid (h', u, v) to spectral (Phi, zeta, delta); synthesis the reverse. */
rexi_status rexi_analyze(rexi_plan *plan, const void *grid_dev, void *spec_dev,
                         int32_t batch, void *stream);
rexi_status rexi_synthesize(rexi_plan *plan, const void *spec_dev, void *grid_dev,
                            int32_t batch, void *stream);

/* One shifted system (alpha_k + tau L) X = U for pole index k (0 <= k < P, the
 * ascending order of rexi_get_coefficients), spectral layout, no beta weight.
 * For tests of a single (pole, m) family of banded solves (Sec. 5). */
rexi_status rexi_solve_pole(rexi_plan *plan, int32_t k, const void *in_dev, void *out_dev,
                            int32_t batch, void *stream);

/* Copy the plan's poles (Sec. 4.1's alpha_k, beta_k, ascending k; a plan over a share of
 * the poles gives its own) to host arrays of 2P doubles each; *P receives P.  For tests of
 * bit-exact pole indexing. */
rexi_status rexi_get_coefficients(const rexi_plan *plan, double *alpha, double *beta, int32_t *P);

/* Autotuner (no paper counterpart; a tuning knob of this implementation): times
 * the banded solve and the slot reduction at this batch size for 1, 2, 4, ... pole
 * groups (the number of partial sums per coefficient, which trades load balance
 * against reduction work) in two shapes -- 0: the same number of groups for every
 * zonal order; 1: groups in proportion to the order's system length -- and, where it
 * applies (binary64 delta solver on the rotating sphere), shape 2: the fused solve
 * with the pole sum on chip and no slots, in CTA tiles of 32 down to 2 states (down to
 * 1 for batches of 1 and 2) and, for batches up to 8, with each tile's poles split over
 * 1, 2, 3, 4, 6 or 8 CTAs, and shapes 3 and 4: its lean forms (see rexi_set_pole_slots).
 * Keeps the fastest for later steps with this batch (the fused solve unless a slot layout
 * is more than 0.5 % faster: it needs no reduction) and writes its slot count (for shapes
 * 2 to 4: tile + 256 x pole groups, as rexi_set_pole_slots takes it) to *slots and its
 * shape to *shape (either may be NULL).  Synchronous; uses the plan's workspaces, so no
 * step of this plan may be in flight. */
rexi_status rexi_tune(rexi_plan *plan, int32_t batch, int32_t *slots, int32_t *shape);

/* Sets the pole-slot layout for steps with this batch size without timing (for instance
 * from a cache of earlier rexi_tune results): slots >= 1 (rounded down to a multiple of
 * the lanes a warp gives each state and capped by the partial-sum buffer) and shape 0
 * or 1 as for rexi_tune, or shape 2 for the fused solve with slots = tile + 256 x groups
 * >= 0: `tile` states per CTA tile (0: the default tile, the smallest power of two >=
 * batch up to 32; a request is rounded down to a power of two) and each tile's poles
 * split over `groups` CTAs in whole passes of the CTA's pole lanes (0: the default, more
 * than one only when a batch is too small to fill the GPU; a request is capped at the
 * passes), the last CTA of a tile to finish adding the groups' partial sums in group
 * order, or shape 3 for its lean form (three or four CTAs of four warps per SM, fewer
 * registers, the next rows prefetched into the caches; tiles of up to 8 states), or shape
 * 4 for the lean form on CTAs of two warps (seven or eight per SM; tiles of up to 4
 * states; a tile of 2 states puts each state on a warp of its own, so no CTA splits its
 * poles over warps), REXI_EINVAL where that does not apply; the slot count used (for
 * shapes 2 to 4: the tile + 256 x the groups) is
 * written to *used (may be NULL).  Results are deterministic for any layout; only the
 * order of the final pole sum changes.  Synchronous, like rexi_tune. */
rexi_status rexi_set_pole_slots(rexi_plan *plan, int32_t batch, int32_t slots, int32_t shape, int32_t *used);

/* Host-side description of a plan (no counterpart in the paper): writes up to 8 int64 values
 * {N, nspec, P, nlat, nlon, max_batch, pole_slots, device bytes held}; pole_slots is
 * that of steps with max_batch states, 0 when they use the fused solve. */
rexi_status rexi_plan_info(const rexi_plan *plan, int64_t *info, int32_t n);

/* Ragged batches (mixed truncations and pole counts): the banded solves of
 * every state of several plans run as ONE persistent launch over the merged
 * work list of every plan's items sorted longest first (Sec. 5: every (pole, m)
 * system is independent).  With binary64 solves that launch is the fused solve:
 * items are (system, tile of 2 states, plan), the pole sum stays on chip and no
 * reduction follows, provided the largest plan's running sums leave seven CTAs of two
 * warps, or three of four warps, per SM.  Otherwise (and with float-float solves) it is the pole-slot solve over
 * (m, pole group, state group, plan) items, then each plan's reduction.  Plans must use
 * REXI_SPECTRAL, the rotating sphere and REXI_SOLVER_DELTA; the ragged object
 * keeps pointers to them (destroy it first).
 * rexi_ragged_step: in_dev[s], out_dev[s] are state s's [3][nspec_p] complex128
 * device arrays (p = state_plan[s]); at most max_batch of plan p's states per
 * call, nstates <= max_states.  A call with a new per-plan state count
 * allocates its work list once; after that the call allocates nothing and can
 * be captured in a CUDA graph.  rexi_tune or rexi_set_pole_slots on one of the
 * plans replaces the slot layout the work lists were built from: the next call
 * rebuilds them (allocating once more), and a graph captured before must be
 * captured again.  Results equal each plan's rexi_step up to the summation order
 * of the poles. */
rexi_status rexi_ragged_create(rexi_plan *const *plans, int32_t nplans, int32_t max_states,
                               rexi_ragged **out);
rexi_status rexi_ragged_step(rexi_ragged *rg, const void *const *in_dev, void *const *out_dev,
                             const int32_t *state_plan, int32_t nstates, void *stream);
void rexi_ragged_destroy(rexi_ragged *rg);

/* Optional per-stage timing (no counterpart in the paper): with max_calls > 0 the next max_calls calls of
 * rexi_step / rexi_step_adjoint record CUDA events on their stream around each
 * stage (0 FFT forward, 1 Legendre analysis, 2 banded solve + pole sum,
 * 3 slot reduction (zero with the fused solve, which has none), 4 Legendre
 * synthesis, 5 FFT inverse, 6/7 layout transposes).  max_calls = 0 turns it off.  rexi_profile_read waits for the
 * recorded events, writes the summed milliseconds per stage to stage_ms[0..n)
 * and the number of timed calls to *calls, and restarts the count. */
rexi_status rexi_profile_enable(rexi_plan *plan, int32_t max_calls);
rexi_status rexi_profile_read(rexi_plan *plan, double *stage_ms, int32_t n, int32_t *calls);

/* No counterpart in the paper.  Synchronise the device and report whether any kernel of this plan gave up a
 * bounded device-side wait (tensor-core completion barriers) since the last
 * check: REXI_ETIMEOUT (and the flag is cleared) or REXI_OK.  Kernels that give
 * up skip their outputs, free their tensor memory and return.  For
 * REXI_SOLVE_FP32X2 plans it also reports REXI_ERANGE when a step's input (or a
 * Phi-only right-hand side) held a finite value beyond binary32's range since the
 * last check: such values become infinite in float-float, and the outputs of that
 * step are not finite. */
rexi_status rexi_check_device(rexi_plan *plan);

/* Test hook (no counterpart in the paper): ORs `bits` (1: a bounded device-side wait
 * expired, 2: a float-float range error; other bits are rejected) into the plan's
 * device error word from the host, as a kernel that gave up would, so that the
 * reporting path of rexi_check_device can be tested without making a kernel wait
 * out its limit.  Synchronises the device.  REXI_EINVAL for a NULL plan or unknown
 * bits. */
rexi_status rexi_inject_device_error(rexi_plan *plan, int32_t bits);

/* Free everything the plan holds (no counterpart in the paper); NULL-safe.  The caller synchronises streams
 * that still use the plan first. */
void rexi_destroy(rexi_plan *plan);

/* Message of the last failed call on this host thread ("" if none); no counterpart in the
 * paper. */
const char *rexi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* REXI_H */
