// Banded shifted solves with the beta-weighted pole sum kept on chip (paper Sec. 4.2,
// Sec. 5, Algorithm 1), binary64.
//
// The systems and factors are those of solve.cu: per (pole k, zonal order m, parity p)
// a complex tridiagonal system in delta over the degrees n = n0 + 2 i, pre-factored per
// plan, swept forward
//   y_i = delta0_n - g Phi0_n - e zeta0_{n-1} - f zeta0_{n+1} - l y_{i-1}
// and backward  w_i = y_i - Chat w_{i+1}, after which the step needs, per row i,
//   Sum_k bd_{k,i} w_{k,i}   (delta),      Sum_k bad_{k,i} w_{k,i}   (Phi),
//   Sum_k zp_{k,i} w_{k,i}   (zeta at n_i + 1),  Sum_k zm_{k,i} w_{k,i}   (zeta at n_i - 1),
// with the factors bd, bad, zp, zm carrying beta_k (Algorithm 1's accumulation).
//
// Here one CTA owns a whole (m, p, tile of states) system for every pole, so that each
// of those sums is complete inside the CTA and its result is written once:
//   - lanes of a warp are (state in the warp, pole): a pass of the warp sweeps PL poles of
//     SB states at once, lane by lane, and the warps of the CTA cover further states (WS
//     groups) or further poles (WP groups);
//   - after every R rows of the backward sweep the lanes trade roles through shared
//     memory: lane (row r, state s, stream t) takes the w of all PL poles of that row and
//     state and adds them to its stream's running sum with complex FMAs, in ascending
//     pole order -- so the pole sum costs no additions beyond the FMAs that apply the
//     weights, and its order is fixed (results are bit-reproducible);
//   - the running sums of every (state, row, stream) stay in shared memory across the
//     passes; at the end of the item the CTA adds the pole-independent terms
//     (Sum beta/alpha Phi0, Sum beta/(alpha + i tau sigma_n) zeta0), takes the real part
//     at m = 0 and writes each output coefficient once.
// The forward-sweep values y go through a per-warp global buffer of 32 lanes x lmax rows
// (in L2 while the resident warps' buffers fit: 8 warps per SM at T341, 16 at T170).  No
// partial sums leave the SM and no reduction kernel
// follows -- except when a batch is too small to fill the GPU (one state has 2 (N + 1)
// systems for 608 schedulers, and the longest one alone would set the time): then NG
// CTAs split a tile's poles in whole passes, each writes its group's sums to global
// memory, and the last of them to arrive (an atomic count; nothing waits) adds the NG
// partials in group order and writes the outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <string>
#include <vector>

#include "rexi_internal.h"

namespace rexi {
namespace {

__device__ __forceinline__ double2 cfms_(double2 acc, double2 a, double2 b) {  // acc - a b
  double re = fma(-a.x, b.x, acc.x);
  re = fma(a.y, b.y, re);
  double im = fma(-a.x, b.y, acc.y);
  im = fma(-a.y, b.x, im);
  return make_double2(re, im);
}
__device__ __forceinline__ double2 cfma_(double2 acc, double2 a, double2 b) {  // acc + a b
  double re = fma(a.x, b.x, acc.x);
  re = fma(-a.y, b.y, re);
  double im = fma(a.x, b.y, acc.y);
  im = fma(a.y, b.x, im);
  return make_double2(re, im);
}
__device__ __forceinline__ double2 ldg2(const double2 *p) { return __ldg(p); }
__device__ __forceinline__ void pf_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" : : "l"(p)); }
__device__ __forceinline__ void pf_l1(const void *p) { asm volatile("prefetch.global.L1 [%0];" : : "l"(p)); }

constexpr int kWarpsPerSM = 8;         // two warps per SM sub-partition: one CTA of 8 or two of 4
constexpr int kStreams = 4;            // delta, Phi, zeta at n + 1, zeta at n - 1

// per-plan arguments of the fused solve (a ragged launch holds one per plan)
struct FusedView {
  const double2 *fac;   // [F_NCOMP][nrows][P]
  const double2 *sin;   // [3][nspec][B]
  double2 *sout;        // [3][nspec][B]
  const int4 *sys;      // per (m, p): {m, n0, len, row0}
  const double2 *wz;    // [nspec] Sum beta_k / (alpha_k + i tau sigma_n) (adjoint: its counterpart)
  double2 sphi;         // Sum beta_k / alpha_k over the plan's poles
  unsigned *arrivals;   // NG > 1: per (system, tile), pole groups finished
  double2 *part;        // NG > 1: [B / ST][NG][ST][nrows][4] the groups' partial sums
  int P, N, B, pole_begin, pole_end, realm0, NG, gsz;
  int64_t nspec, nrows;
};

struct FusedArgs {
  FusedView v;              // the plan of a single-plan launch
  const FusedView *views;   // a ragged launch: one per plan, the item's plan selects it
  double2 *ybuf;            // [gridDim.x * NW][lmax][32]
  const int4 *items;        // (system 2 m + p, first state of the tile, pole group (+ 256 x plan
                            // in a ragged launch), tile index), longest first
  unsigned *counter;        // work counter
  int nitems, WS, WP, lmax;  // lmax: the largest over the launch's plans
};

template <bool RG>
__device__ __forceinline__ const FusedView &pick_view(const FusedView &param, const FusedView &shared) {
  if constexpr (RG) return shared;
  else return param;
}

// one forward-sweep row of one lane: its factors and the states it reads
struct FwdRow {
  double2 l, g, e, f, d0, p0, zn;
};

// SB states per warp, PL = 32 / SB poles per warp pass, R = 8 / SB rows per task round
// (lanes = R rows x SB states x 4 streams).  Shared memory: the running sums
// [WP * ST][lmax * 4 + 1] (an odd plane stride spreads the states over the banks), then
// per warp two exchange buffers of R rows x (32 + SB) values (a pad after every state's
// PL lanes and a row stride of SB mod 8 put the R x SB (row, state) groups that a task
// instruction reads on distinct banks).
//
// MINB CTAs per SM.  MINB = kWarpsPerSM / NW: the running sums and two exchange buffers per
// warp, and the next rows' factors, states and sweep values prefetched into registers
// (up to 222 registers).  MINB x NW > kWarpsPerSM (three or four CTAs of four warps, or
// seven or eight of two, per SM): the lean form for 12 to 16 warps per SM -- registers
// capped at 170, 146 or 128, one exchange buffer per warp, and the next rows brought into
// the caches instead of registers.
template <int SB, int NW, int MINB = kWarpsPerSM / NW, bool RAGGED = false>
__global__ void __launch_bounds__(32 * NW, MINB) solve_fused_kernel(FusedArgs a) {
  constexpr int PL = 32 / SB, R = 8 / SB, RS = 32 + SB, kThreads = 32 * NW;
  constexpr bool kLean = MINB * NW > kWarpsPerSM;
  constexpr int kBufs = kLean ? 1 : 2;  // exchange buffers per warp
  extern __shared__ double2 smem[];
  __shared__ int s_item, s_last;
  __shared__ FusedView s_view;  // a ragged launch: the current item's plan
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ws = warp / a.WP, wp = warp - ws * a.WP;  // state group, pole group of this warp
  const int ST = a.WS * SB;                           // states per CTA tile
  const int lmax = a.lmax;
  const int ACS = lmax * kStreams + 1;                // running-sum plane stride
  double2 *acc = smem;                                                           // [WP * ST][ACS]
  double2 *wbase = smem + (size_t)a.WP * ST * ACS + (size_t)warp * kBufs * R * RS;  // [kBufs][R][RS]
  double2 *ybuf = a.ybuf + ((size_t)blockIdx.x * NW + warp) * (size_t)lmax * 32 + lane;
  // sweep role: lane = (state s_sw, pole pl); task role: lane = (row r, state t_s, stream t)
  const int s_sw = lane / PL, pl = lane - s_sw * PL;
  const int wslot = lane + s_sw;  // this lane's place in an exchange row
  const int t_r = lane / (4 * SB), t_s = (lane >> 2) % SB, t_t = lane & 3;
  const int t_comp = t_t == 0 ? F_BD : (t_t == 1 ? F_BAD : (t_t == 2 ? F_ZP : F_ZM));

  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(a.counter, 1u);
    __syncthreads();
    const int it = s_item;
    __syncthreads();
    if (it >= a.nitems) break;
    const int4 item = a.items[it];
    if constexpr (RAGGED) {
      if (threadIdx.x == 0) s_view = a.views[item.z >> 8];
      __syncthreads();
    }
    const FusedView &V = pick_view<RAGGED>(a.v, s_view);
    const int gi = RAGGED ? (item.z & 255) : item.z;  // the item's pole group
    const int N = V.N, B = V.B;
    const int64_t NS = V.nspec, NR = V.nrows, P = V.P;
    const int4 sy = V.sys[item.x];
    const int m = sy.x, n0 = sy.y, len = sy.z;
    const int64_t row0 = sy.w;
    const int p = item.x & 1, b0 = item.y;
    const int kg0 = V.pole_begin + gi * V.gsz;  // this CTA's poles [kg0, kg1)
    const int kg1 = min(V.pole_end, kg0 + V.gsz);
    const int64_t base_idx = (int64_t)m * (2 * N + 3 - m) / 2 - m;  // idx(m, n) = base_idx + n
    const int nmin = m > 1 ? m : 1;

    // running sums of this item start at zero
    for (int q = threadIdx.x; q < a.WP * ST * len * kStreams; q += kThreads) {
      const int t = q % kStreams, rest = q / kStreams, i = rest % len, g = rest / len;  // g = wp * ST + st
      acc[(size_t)g * ACS + i * kStreams + t] = make_double2(0.0, 0.0);
    }
    __syncthreads();

    // a warp group whose states all lie past the batch (the last tile of an odd batch)
    // skips the sweeps: its running sums stay zero and no output of it is written
    if (len > 0 && b0 + ws * SB < B) {
      const int bsw = b0 + ws * SB + s_sw;  // the sweep lane's state (clamped for loads)
      const int bq = bsw < B ? bsw : b0;
      const double2 *sPhi = V.sin + bq, *sZeta = V.sin + NS * B + bq, *sDel = V.sin + 2 * NS * B + bq;
      const int npp = a.WP * PL;  // poles per CTA pass
      const int nr = (len + R - 1) / R;  // task rounds of the backward sweep
      for (int kb = kg0; kb < kg1; kb += npp) {
        const int kw = kb + wp * PL;         // this warp's first pole
        const int npa = min(PL, kg1 - kw);   // its active poles (warp-uniform)
        if (npa <= 0) continue;
        const bool active = pl < npa;              // inactive lanes repeat a valid pole, add zero
        const int k = kw + min(pl, npa - 1);
        const double2 *fL = V.fac + ((int64_t)F_L * NR + row0) * P + k;
        const double2 *fG = V.fac + ((int64_t)F_G * NR + row0) * P + k;
        const double2 *fE = V.fac + ((int64_t)F_E * NR + row0) * P + k;
        const double2 *fF = V.fac + ((int64_t)F_F * NR + row0) * P + k;
        const double2 *fC = V.fac + ((int64_t)F_C * NR + row0) * P + k;

        // ---- forward sweep, two rows per iteration: the next row's factors and states
        // are loaded while the current row computes (two register sets, no copies)
        auto load_fwd = [&](int i, FwdRow &r) {
          const int64_t o = (int64_t)i * P;
          const int n = n0 + 2 * i;
          const int64_t ix = base_idx + n;
          if (i + 4 < len) {
            const int64_t o4 = o + 4 * P;
            pf_l2(fL + o4);
            pf_l2(fG + o4);
            pf_l2(fE + o4);
            pf_l2(fF + o4);
          }
          r.l = ldg2(fL + o);
          r.g = ldg2(fG + o);
          r.e = ldg2(fE + o);
          r.f = ldg2(fF + o);
          r.d0 = ldg2(sDel + ix * B);
          r.p0 = ldg2(sPhi + ix * B);
          r.zn = (n + 1 <= N) ? ldg2(sZeta + (ix + 1) * B) : make_double2(0.0, 0.0);
        };
        double2 yprev = make_double2(0.0, 0.0);
        double2 zprev = (n0 - 1 >= nmin) ? ldg2(sZeta + (base_idx + n0 - 1) * B) : make_double2(0.0, 0.0);
        auto fwd = [&](int i, const FwdRow &r) {
          double2 y = cfms_(r.d0, r.g, r.p0);
          y = cfms_(y, r.e, zprev);
          y = cfms_(y, r.f, r.zn);
          y = cfms_(y, r.l, yprev);
          ybuf[(size_t)i * 32] = y;
          yprev = y;
          zprev = r.zn;
        };
        if constexpr (kLean) {
          // each row's values two rows ahead into L1 (no registers held), then loaded
          auto pf_row = [&](int i) {
            const int64_t o = (int64_t)i * P;
            const int64_t ix = base_idx + n0 + 2 * i;
            pf_l1(fL + o);
            pf_l1(fG + o);
            pf_l1(fE + o);
            pf_l1(fF + o);
            pf_l1(sDel + ix * B);
            pf_l1(sPhi + ix * B);
            pf_l1(sZeta + (ix + 1) * B);  // the state array's next field follows: in bounds
          };
          if (len > 1) pf_row(1);
          for (int i = 0; i < len; ++i) {
            if (i + 2 < len) pf_row(i + 2);
            FwdRow r;
            load_fwd(i, r);
            fwd(i, r);
          }
        } else {
          FwdRow A, Bn;
          load_fwd(0, A);
          int i = 0;
          for (; i + 1 < len; i += 2) {
            load_fwd(i + 1, Bn);
            fwd(i, A);
            if (i + 2 < len) load_fwd(i + 2, A);
            fwd(i + 1, Bn);
          }
          if (i < len) fwd(i, A);
        }

        // ---- backward sweep in rounds of R rows from the top, software-pipelined: the
        // recurrence of round rr + 1 and the pole sum of round rr are independent work in
        // one block, and the sweep values of round rr + 2 are loaded meanwhile
        double2 wnext = make_double2(0.0, 0.0);
        double2 yv[R], cv[R];
        auto load_round = [&](int rr) {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            const int i = max(len - 1 - rr * R - j, 0);
            yv[j] = ybuf[(size_t)i * 32];
            cv[j] = ldg2(fC + (int64_t)i * P);
          }
        };
        auto rec_round = [&](int rr, double2 *wbuf) {
#pragma unroll
          for (int j = 0; j < R; ++j) {
            if (len - 1 - rr * R - j >= 0) {
              const double2 w = cfms_(yv[j], cv[j], wnext);
              wbuf[j * RS + wslot] = active ? w : make_double2(0.0, 0.0);
              wnext = w;
            }
          }
        };
        auto task_round = [&](int rr, const double2 *wbuf) {
          const int iv = len - 1 - rr * R - t_r;  // the row this lane sums (< 0: none)
          const int ii = max(iv, 0);
          double2 *ap = acc + ((size_t)wp * ST + ws * SB + t_s) * ACS + ii * kStreams + t_t;
          const double2 *W = V.fac + ((int64_t)t_comp * NR + row0 + ii) * P + kw;
          const double2 *wv = wbuf + t_r * RS + t_s * (PL + 1);
          double2 s = *ap;
#pragma unroll
          for (int q = 0; q < PL; ++q) s = cfma_(s, ldg2(W + min(q, npa - 1)), wv[q]);  // w = 0 past npa
          if (iv >= 0) *ap = s;
          if (iv - R >= 0) {  // the next round's weights (R rows further down) into L1
            const double2 *Wn = W - (int64_t)R * P;
#pragma unroll
            for (int q = 0; q < PL; q += 8)
              if (q < npa) pf_l1(Wn + q);  // poles of this pass only: every address inside the factors
          }
        };
        // The last round of a pass holds rv = len - rr R rows (1 ... R).  With rv <= R / H the
        // lanes of the missing rows would sum nothing useful, so the round is laid out as
        // R / H rows x SB states x 4 streams x H pole slices: each lane sums PL / H poles of
        // its row and the H slices are added by shuffles (lanes 4 SB apart).  Slice 0 starts
        // from the running sum; the order of every addition is fixed.
        auto task_split = [&](auto Hc, int rr, const double2 *wbuf) {
          constexpr int H = decltype(Hc)::value, QH = PL / H;
          const int h = (lane / (4 * SB)) % H, tr = lane / (4 * SB * H);
          const int iv = len - 1 - rr * R - tr;
          const int ii = max(iv, 0);
          double2 *ap = acc + ((size_t)wp * ST + ws * SB + t_s) * ACS + ii * kStreams + t_t;
          const double2 *W = V.fac + ((int64_t)t_comp * NR + row0 + ii) * P + kw;
          const double2 *wv = wbuf + tr * RS + t_s * (PL + 1) + h * QH;
          double2 s = h == 0 ? *ap : make_double2(0.0, 0.0);
#pragma unroll
          for (int q = 0; q < QH; ++q) s = cfma_(s, ldg2(W + min(h * QH + q, npa - 1)), wv[q]);
#pragma unroll
          for (int o = 4 * SB; o < 4 * SB * H; o *= 2) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
          }
          if (h == 0 && iv >= 0) *ap = s;
        };
        auto task_last = [&](int rr, const double2 *wbuf) {
          const int rv = len - rr * R;
          if constexpr (R >= 8) {
            if (rv <= R / 8) { task_split(std::integral_constant<int, 8>{}, rr, wbuf); return; }
          }
          if constexpr (R >= 4) {
            if (rv <= R / 4) { task_split(std::integral_constant<int, 4>{}, rr, wbuf); return; }
          }
          if constexpr (R >= 2) {
            if (rv <= R / 2) { task_split(std::integral_constant<int, 2>{}, rr, wbuf); return; }
          }
          task_round(rr, wbuf);
        };
        if constexpr (kLean) {
          // one exchange buffer: each round's recurrence, then its sums; the next round's
          // sweep values and factors two rounds ahead into L1
          auto pf_round = [&](int rr) {
#pragma unroll
            for (int j = 0; j < R; ++j) {
              const int i = max(len - 1 - rr * R - j, 0);
              pf_l1(ybuf + (size_t)i * 32);
              pf_l1(fC + (int64_t)i * P);
            }
          };
          pf_round(0);
          if (nr > 1) pf_round(1);
          for (int rr = 0; rr < nr; ++rr) {
            if (rr + 2 < nr) pf_round(rr + 2);
            load_round(rr);
            rec_round(rr, wbase);
            __syncwarp();
            if (rr + 1 < nr) task_round(rr, wbase);
            else task_last(rr, wbase);
            __syncwarp();
          }
        } else {
          load_round(0);
          rec_round(0, wbase);
          if (nr > 1) load_round(1);
          __syncwarp();
          for (int rr = 0; rr < nr; ++rr) {
            double2 *wcur = wbase + (rr & 1) * R * RS, *wnxt = wbase + ((rr + 1) & 1) * R * RS;
            if (rr + 1 < nr) rec_round(rr + 1, wnxt);
            if (rr + 2 < nr) load_round(rr + 2);
            if (rr + 1 < nr) task_round(rr, wcur);
            else task_last(rr, wcur);
            __syncwarp();
          }
        }
      }
    }
    __syncthreads();

    // ---- NG > 1: the NG CTAs of one (system, tile) each hold the sums over their own
    // pole group.  Each writes them (added over its WP warp groups) to the tile's partial
    // slots and counts its arrival; the last to arrive adds the NG partials in group order
    // and writes the outputs.  No CTA waits for another, and the order of the sum does not
    // depend on which CTA comes last.
    const int64_t PS = NR * kStreams;  // one state's partial sums of one group
    const double2 *pg = nullptr;       // the tile's partials at this system (NG > 1, last CTA)
    if (V.NG > 1) {
      double2 *mine = V.part + ((size_t)(b0 / ST) * V.NG + gi) * ST * PS + row0 * kStreams;
      for (int q = threadIdx.x; q < ST * len * kStreams; q += kThreads) {
        const int st = q / (len * kStreams), r = q - st * (len * kStreams);
        double2 v = make_double2(0.0, 0.0);
        for (int g = 0; g < a.WP; ++g) {
          const double2 u = acc[((size_t)g * ST + st) * ACS + r];
          v.x += u.x;
          v.y += u.y;
        }
        mine[(size_t)st * PS + r] = v;
      }
      __threadfence();  // the partials are visible device-wide before the arrival counts
      __syncthreads();
      if (threadIdx.x == 0) s_last = atomicAdd(V.arrivals + item.w, 1u) == (unsigned)(V.NG - 1);
      __syncthreads();
      if (!s_last) continue;  // block-uniform
      __threadfence();
      pg = V.part + (size_t)(b0 / ST) * V.NG * ST * PS + row0 * kStreams;
    }

    // ---- outputs of this item: delta and Phi at the degrees of parity p, zeta at the
    // other parity; every coefficient of the item written once
    {
      const int nown = (N - (m + p)) >= 0 ? (N - (m + p)) / 2 + 1 : 0;          // n = m + p + 2 j
      const int noth = (N - (m + 1 - p)) >= 0 ? (N - (m + 1 - p)) / 2 + 1 : 0;  // n = m + 1 - p + 2 j
      const int tot = (nown + noth) * ST;
      for (int q = threadIdx.x; q < tot; q += kThreads) {
        const int st = q % ST, jj = q / ST;
        const int b = b0 + st;
        if (b >= B) continue;
        auto sumacc = [&](int i, int t) {
          double2 v = make_double2(0.0, 0.0);
          if (pg) {  // the groups' partials, from L2 (written by other SMs)
            for (int g = 0; g < V.NG; ++g) {
              const double2 u = __ldcg(pg + ((size_t)g * ST + st) * PS + i * kStreams + t);
              v.x += u.x;
              v.y += u.y;
            }
            return v;
          }
          for (int g = 0; g < a.WP; ++g) {
            const double2 u = acc[((size_t)g * ST + st) * ACS + i * kStreams + t];
            v.x += u.x;
            v.y += u.y;
          }
          return v;
        };
        if (jj < nown) {
          const int n = m + p + 2 * jj;
          const int64_t ix = base_idx + n;
          const int i = (n - n0) / 2;
          const bool row = n >= n0 && i < len;
          double2 dl = row ? sumacc(i, 0) : make_double2(0.0, 0.0);
          double2 ph = row ? sumacc(i, 1) : make_double2(0.0, 0.0);
          ph = cfma_(ph, V.sphi, V.sin[ix * B + b]);
          if (V.realm0 && m == 0) {
            dl.y = 0.0;
            ph.y = 0.0;
          }
          V.sout[ix * B + b] = ph;
          V.sout[(2 * NS + ix) * B + b] = dl;
        } else {
          const int n = m + 1 - p + 2 * (jj - nown);
          const int64_t ix = base_idx + n;
          double2 ze = make_double2(0.0, 0.0);
          if (n > 0) {  // zeta_0^0 is not state
            const int ia = (n - 1 - n0) / 2, ib = (n + 1 - n0) / 2;  // delta rows n - 1 and n + 1
            if (n - 1 >= n0 && ia < len) ze = sumacc(ia, 2);
            if (n + 1 >= n0 && ib < len) {
              const double2 u = sumacc(ib, 3);
              ze.x += u.x;
              ze.y += u.y;
            }
            ze = cfma_(ze, V.wz[ix], V.sin[(NS + ix) * B + b]);
            if (V.realm0 && m == 0) ze.y = 0.0;
          }
          V.sout[(NS + ix) * B + b] = ze;
        }
      }
    }
    __syncthreads();
  }
}

}  // namespace

void free_fused_layout(FusedLayout &F) {
  if (F.items_dev) cudaFree(F.items_dev);
  if (F.part_dev) cudaFree(F.part_dev);
  if (F.sync_dev) cudaFree(F.sync_dev);
  F = FusedLayout{};
}

// Work items and CTA shape of the fused solve for a batch of B states: ST states per
// CTA tile (the smallest power of two >= B, at most 32, or a smaller requested tile),
// split over the eight warps as WS state groups of SB states; when the tile has fewer
// than eight states the remaining warps split the poles (WP groups).  Smaller tiles give
// more, shorter work items (better balance over the SMs) at the cost of reading each
// factor once per tile.  `groups` CTAs (0: the default below) split each (system, tile)'s
// poles in whole passes.  Returns false when the running sums of a tile do not fit in
// shared memory (the slot-partial path then serves the plan).
bool build_fused_layout(Plan &pl, int B, int tile, int form, int groups, FusedLayout &F) {
  F = FusedLayout{};
  int st = 1;
  while (st < B && st < 32) st *= 2;
  if (tile > 0)  // a requested tile: the largest power of two <= tile (and <= the default)
    while (st > 1 && st > tile) st /= 2;
  const int dev = pl.device;
  int smem_max = 0, smem_sm = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  auto smem_of = [&](int nw, int sb, int wp, int t, int bufs) {
    return ((size_t)wp * t * (pl.lmax * kStreams + 1) + (size_t)nw * bufs * (8 / sb) * (32 + sb)) * sizeof(double2);
  };
  for (; st >= 1; st /= 2) {
    if (form != 0) {
      // lean: CTAs of four warps (form 1; 4 or 3 per SM) or two warps (form 2; 8 or 7 per
      // SM), one exchange buffer per warp, as many CTAs per SM as fit
      const int nwl = form == 2 ? 2 : 4;
      int sb, ws, wp;
      if (st >= nwl) { sb = st / nwl; ws = nwl; wp = 1; }
      else { sb = 1; ws = st; wp = nwl / st; }
      if (sb > 2) continue;
      const size_t smem = smem_of(nwl, sb, wp, st, 1);
      if (smem + 1024 > (size_t)smem_max) continue;
      const int per_sm = std::min<int>(2 * kWarpsPerSM / nwl, (int)(smem_sm / (smem + 1024)));
      if (per_sm < (nwl == 2 ? 7 : 3)) continue;
      F.sb = sb;
      F.ws = ws;
      F.wp = wp;
      F.st = st;
      F.nw = nwl;
      F.per_sm = per_sm;
      F.smem = smem;
      break;
    }
    // two CTAs of four warps when both fit on an SM (a tile's poles then need no split over
    // warps down to four states), else one CTA of eight warps; at most two states per warp
    // unless nothing else fits (four states per warp, in tiles of 16 states at T170, left
    // the FP64 pipe 50 % idle)
    for (int nw : {4, 8, 4 + 0x100, 8 + 0x100}) {
      const bool wide = nw & 0x100;
      nw &= 0xff;
      int sb, ws, wp;
      if (st >= nw) { sb = st / nw; ws = nw; wp = 1; }
      else { sb = 1; ws = st; wp = nw / st; }
      if (sb > 4 || (sb > 2 && !wide)) continue;
      const int per_sm = kWarpsPerSM / nw;
      const size_t smem = smem_of(nw, sb, wp, st, 2);
      if (smem + 1024 > (size_t)smem_max || per_sm * (smem + 1024) > (size_t)smem_sm) continue;
      F.sb = sb;
      F.ws = ws;
      F.wp = wp;
      F.st = st;
      F.nw = nw;
      F.per_sm = per_sm;
      F.smem = smem;
      break;
    }
    if (F.st) break;
  }
  if (F.st == 0) return false;
  // the kernel's shared-memory limit, set here once (not per launch, so that steps can be
  // captured in a CUDA graph): the device's opt-in maximum less the 1 KiB every layout
  // leaves for the static shared memory, which covers every layout
  const int smem_opt = smem_max - 1024;
  auto allow = [&](auto kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opt);
  };
  cudaError_t ea;
  if (F.nw == 2 && F.per_sm == 8) ea = F.sb == 2 ? allow(solve_fused_kernel<2, 2, 8>) : allow(solve_fused_kernel<1, 2, 8>);
  else if (F.nw == 2) ea = F.sb == 2 ? allow(solve_fused_kernel<2, 2, 7>) : allow(solve_fused_kernel<1, 2, 7>);
  else if (F.per_sm == 4) ea = F.sb == 2 ? allow(solve_fused_kernel<2, 4, 4>) : allow(solve_fused_kernel<1, 4, 4>);
  else if (F.per_sm == 3) ea = F.sb == 2 ? allow(solve_fused_kernel<2, 4, 3>) : allow(solve_fused_kernel<1, 4, 3>);
  else if (F.nw == 4)
    ea = F.sb == 4 ? allow(solve_fused_kernel<4, 4>) : F.sb == 2 ? allow(solve_fused_kernel<2, 4>)
                                                      : allow(solve_fused_kernel<1, 4>);
  else
    ea = F.sb == 4 ? allow(solve_fused_kernel<4, 8>) : F.sb == 2 ? allow(solve_fused_kernel<2, 8>)
                                                      : allow(solve_fused_kernel<1, 8>);
  if (ea != cudaSuccess) {
    F = FusedLayout{};
    return false;
  }

  // pole groups: NG CTAs share a (system, tile), each taking whole passes of WP x PL poles.
  // Default: the fewest groups for which the longest system's CTA (its warps sharing their
  // schedulers with the SM's other resident warps) needs at most half the FP64 work the
  // average scheduler has in all -- so that the longest items, taken first, leave room to
  // balance the rest; with a large batch, or many orders, that is one group.
  const int npp = F.wp * (32 / F.sb), passes = (pl.P + npp - 1) / npp;
  const int ntile_b = (B + F.st - 1) / F.st;
  int ng = 1;
  if (groups > 0) {
    ng = std::min(groups, passes);
  } else {
    double work = 0;  // warp passes x rows over every (system, tile)
    int lmax_sys = 0;
    const double wpasses = (double)F.ws * ((pl.P + 32 / F.sb - 1) / (32 / F.sb));  // per tile, per row
    for (int sy = 0; sy < 2 * (pl.N + 1); ++sy) {
      work += wpasses * pl.sys[sy].len * ntile_b;
      lmax_sys = std::max(lmax_sys, pl.sys[sy].len);
    }
    const double avg = work / (4.0 * pl.num_sms);        // per scheduler (four per SM)
    const double share = std::max(1.0, F.per_sm * F.nw / 4.0);  // warps per scheduler, SM full
    for (ng = 1; ng < passes; ++ng)
      if (share * lmax_sys * ((passes + ng - 1) / ng) <= 0.5 * avg) break;
  }
  // the groups' partial sums take B x NG x rows x 64 bytes: at most 1 GiB
  while (ng > 1 && (double)ntile_b * F.st * ng * pl.nrows * kStreams * sizeof(double2) > 1073741824.0) --ng;
  F.gsz = ((passes + ng - 1) / ng) * npp;
  F.ng = (pl.P + F.gsz - 1) / F.gsz;

  // items (system, first state, group, tile index), longest system first; m ascending
  // breaks ties and a tile's groups stay together
  struct Keyed { int4 it; int len; };
  std::vector<Keyed> keyed;
  int ti = 0;
  for (int m = 0; m <= pl.N; ++m)
    for (int p = 0; p < 2; ++p)
      for (int b0 = 0; b0 < B; b0 += F.st, ++ti)
        for (int g = 0; g < F.ng; ++g) keyed.push_back(Keyed{make_int4(2 * m + p, b0, g, ti), pl.sys[2 * m + p].len});
  std::stable_sort(keyed.begin(), keyed.end(), [](const Keyed &x, const Keyed &y) { return x.len > y.len; });
  std::vector<int4> items;
  for (const Keyed &k : keyed) items.push_back(k.it);
  F.ntiles = ti;
  F.nitems = (int)items.size();
  cudaError_t e = cudaMalloc(&F.items_dev, items.size() * sizeof(int4));
  if (e == cudaSuccess) e = cudaMemcpy(F.items_dev, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&F.sync_dev, (size_t)(1 + (F.ng > 1 ? F.ntiles : 0)) * sizeof(unsigned));
  if (e == cudaSuccess && F.ng > 1)
    e = cudaMalloc(&F.part_dev, (size_t)ntile_b * F.ng * F.st * pl.nrows * kStreams * sizeof(double2));
  if (e != cudaSuccess) {
    free_fused_layout(F);
    return false;
  }
  return true;
}

// the per-plan arguments of a fused solve of B states of plan pl with layout F
FusedView fused_view(Plan &pl, const FusedLayout &F, bool adjoint, const double2 *sin, double2 *sout, int B,
                     unsigned *arrivals, double2 *part) {
  FusedView v;
  v.fac = adjoint ? pl.fac_adj : pl.fac_fwd;
  v.sin = sin;
  v.sout = sout;
  v.sys = pl.sys_dev;
  v.wz = adjoint ? pl.w_adj : pl.w_fwd;
  v.sphi = adjoint ? pl.sphi_adj : pl.sphi_fwd;
  v.arrivals = arrivals;
  v.part = part;
  v.P = pl.P;
  v.N = pl.N;
  v.B = B;
  v.pole_begin = 0;
  v.pole_end = pl.P;
  v.realm0 = 1;
  v.NG = F.ng;
  v.gsz = F.gsz;
  v.nspec = pl.nspec;
  v.nrows = pl.nrows;
  return v;
}

cudaError_t launch_solve_fused(Plan &pl, const FusedLayout &F, bool adjoint, const double2 *sin, double2 *sout,
                               int B, cudaStream_t st) {
  FusedArgs a;
  a.v = fused_view(pl, F, adjoint, sin, sout, B, F.sync_dev + 1, F.part_dev);
  a.views = nullptr;
  a.ybuf = pl.yscratch;  // sized for 16 warps x 2 poles per SM: eight warps of one pole here
  a.items = F.items_dev;
  a.counter = F.sync_dev;
  a.nitems = F.nitems;
  a.WS = F.ws;
  a.WP = F.wp;
  a.lmax = pl.lmax;
  cudaError_t e = cudaMemsetAsync(F.sync_dev, 0, (size_t)(1 + (F.ng > 1 ? F.ntiles : 0)) * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int grid = pl.num_sms * F.per_sm;
  const int smem = (int)F.smem;
  auto go = [&](auto kernel) {  // the shared-memory limit was raised when the layout was built
    kernel<<<grid, 32 * F.nw, smem, st>>>(a);
    return cudaSuccess;
  };
  if (F.nw == 2 && F.per_sm == 8) {
    e = F.sb == 2 ? go(solve_fused_kernel<2, 2, 8>) : go(solve_fused_kernel<1, 2, 8>);
  } else if (F.nw == 2) {
    e = F.sb == 2 ? go(solve_fused_kernel<2, 2, 7>) : go(solve_fused_kernel<1, 2, 7>);
  } else if (F.per_sm == 4) {
    e = F.sb == 2 ? go(solve_fused_kernel<2, 4, 4>) : go(solve_fused_kernel<1, 4, 4>);
  } else if (F.per_sm == 3) {
    e = F.sb == 2 ? go(solve_fused_kernel<2, 4, 3>) : go(solve_fused_kernel<1, 4, 3>);
  } else if (F.nw == 4) {
    e = F.sb == 4 ? go(solve_fused_kernel<4, 4>) : F.sb == 2 ? go(solve_fused_kernel<2, 4>) : go(solve_fused_kernel<1, 4>);
  } else {
    e = F.sb == 4 ? go(solve_fused_kernel<4, 8>) : F.sb == 2 ? go(solve_fused_kernel<2, 8>) : go(solve_fused_kernel<1, 8>);
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}


// ---- ragged launches: the fused solve over the states of several plans -----------------
// One persistent launch of the lean form (tiles of 2 states; CTAs of two warps, else four)
// over the merged work list of every plan's (system, tile) items, longest (rows x poles)
// first; each item names its plan, whose arguments the CTA reads from a per-plan view.  One
// pole group per tile: the merged list is long enough to balance the SMs.  Needs the
// largest plan's running sums to leave seven two-warp or three four-warp CTAs per SM;
// returns false otherwise (the slot path serves).
bool build_fused_ragged(const std::vector<Plan *> &plans, const std::vector<int> &counts, FusedRagged &R) {
  R = FusedRagged{};
  int lmax = 1;
  for (size_t p = 0; p < plans.size(); ++p)
    if (counts[p] > 0) {
      if (plans[p]->ff) return false;
      lmax = std::max(lmax, plans[p]->lmax);
    }
  const int dev = plans[0]->device;
  int smem_max = 0, smem_sm = 0;
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  // CTAs of two warps (one state each, seven or eight per SM) where they fit, else of four
  // warps (two per state, splitting its poles; three or four per SM)
  int nw = 0, per_sm = 0, wp = 0;
  size_t smem = 0;
  const int st = 2, sb = 1, ws = 2;
  for (int nwc : {2, 4}) {
    const int wpc = nwc / st;
    const size_t sm = ((size_t)wpc * st * (lmax * kStreams + 1) + (size_t)nwc * 1 * (8 / sb) * (32 + sb)) * sizeof(double2);
    if (sm + 1024 > (size_t)smem_max) continue;
    const int ps = std::min<int>(2 * kWarpsPerSM / nwc, (int)(smem_sm / (sm + 1024)));
    if (ps < (nwc == 2 ? 7 : 3)) continue;
    nw = nwc;
    per_sm = ps;
    wp = wpc;
    smem = sm;
    break;
  }
  if (nw == 0) return false;
  const int smem_opt = smem_max - 1024;
  cudaError_t e;
  if (nw == 2)
    e = per_sm == 8 ? cudaFuncSetAttribute(solve_fused_kernel<1, 2, 8, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opt)
                    : cudaFuncSetAttribute(solve_fused_kernel<1, 2, 7, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opt);
  else
    e = per_sm == 4 ? cudaFuncSetAttribute(solve_fused_kernel<1, 4, 4, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opt)
                    : cudaFuncSetAttribute(solve_fused_kernel<1, 4, 3, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_opt);
  if (e != cudaSuccess) return false;
  // one pole group per tile: gsz covers every pole
  FusedLayout F1;
  F1.ng = 1;
  std::vector<FusedView> views(plans.size());
  struct Keyed { int4 it; double work; };
  std::vector<Keyed> keyed;
  for (size_t p = 0; p < plans.size(); ++p) {
    if (counts[p] == 0) continue;
    Plan &pl = *plans[p];
    F1.gsz = pl.P;
    views[p] = fused_view(pl, F1, false, pl.s_in, pl.s_out, counts[p], nullptr, nullptr);
    int ti = 0;
    for (int m = 0; m <= pl.N; ++m)
      for (int par = 0; par < 2; ++par)
        for (int b0 = 0; b0 < counts[p]; b0 += st, ++ti)
          keyed.push_back(Keyed{make_int4(2 * m + par, b0, (int)(p << 8), ti), (double)pl.sys[2 * m + par].len * pl.P});
  }
  std::stable_sort(keyed.begin(), keyed.end(), [](const Keyed &x, const Keyed &y) { return x.work > y.work; });
  std::vector<int4> items;
  for (const Keyed &k : keyed) items.push_back(k.it);
  R.nitems = (int)items.size();
  R.nviews = (int)views.size();
  R.lmax = lmax;
  R.per_sm = per_sm;
  R.smem = smem;
  R.ws = ws;
  R.wp = wp;
  R.nw = nw;
  e = cudaMalloc(&R.views_dev, views.size() * sizeof(FusedView));
  if (e == cudaSuccess) e = cudaMemcpy(R.views_dev, views.data(), views.size() * sizeof(FusedView), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&R.items_dev, std::max<size_t>(1, items.size()) * sizeof(int4));
  if (e == cudaSuccess) e = cudaMemcpy(R.items_dev, items.data(), items.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&R.counter, sizeof(unsigned));
  if (e != cudaSuccess) {
    free_fused_ragged(R);
    return false;
  }
  return true;
}

void free_fused_ragged(FusedRagged &R) {
  if (R.views_dev) cudaFree(R.views_dev);
  if (R.items_dev) cudaFree(R.items_dev);
  if (R.counter) cudaFree(R.counter);
  R = FusedRagged{};
}

cudaError_t launch_fused_ragged(const FusedRagged &R, double2 *ybuf, int num_sms, cudaStream_t st) {
  FusedArgs a{};
  a.views = static_cast<const FusedView *>(R.views_dev);
  a.ybuf = ybuf;
  a.items = R.items_dev;
  a.counter = R.counter;
  a.nitems = R.nitems;
  a.WS = R.ws;
  a.WP = R.wp;
  a.lmax = R.lmax;
  cudaError_t e = cudaMemsetAsync(R.counter, 0, sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  const int grid = num_sms * R.per_sm;
  if (R.nw == 2 && R.per_sm == 8) solve_fused_kernel<1, 2, 8, true><<<grid, 64, R.smem, st>>>(a);
  else if (R.nw == 2) solve_fused_kernel<1, 2, 7, true><<<grid, 64, R.smem, st>>>(a);
  else if (R.per_sm == 4) solve_fused_kernel<1, 4, 4, true><<<grid, 128, R.smem, st>>>(a);
  else solve_fused_kernel<1, 4, 3, true><<<grid, 128, R.smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace rexi
