// Legendre transforms per zonal order m (paper Sec. 3) on the 5th-generation
// tensor cores: tcgen05.mma kind::tf32 with 3xTF32 split products
// (a b ~ a_hi b_hi + a_hi b_lo + a_lo b_hi) accumulated in FP32 in tensor memory.
//
// Analysis, per (m, parity p of n - m, tile of 128 degrees, group of G states):
//   D1[n][8b + 2f + c] = sum_j Pbar_n(mu_j) X^{p}_f(j)      f in (Phi, U, V), c = re/im
//   D2[n][4b + 2f + c] = sum_j H_n(mu_j)    X^{1-p}_f(j)    f in (U, V)
//   with X^0 = F(mu_j) + F(-mu_j), X^1 = F(mu_j) - F(-mu_j) over the J northern
//   latitudes (the FFT has already applied g w_j and cos w_j / (a (1 - mu^2))), and
//   Phi = D1[Phi], zeta = i m D1[V] + D2[U], delta = i m D1[U] - D2[V].
// Synthesis, per (m, tile of 128 northern latitudes, group of G states), for both
// symmetry classes s:
//   D1_s[j][8b + ...] = sum_{n: (n-m)%2 = s}   Pbar_n(mu_j) (Phi, psi', chi')_n
//   D2_s[j][4b + ...] = sum_{n: (n-m)%2 = 1-s} H_n(mu_j)    (psi', chi')_n
//   F_s(Phi) = D1_s[Phi], F_s(U) = -D2_s[psi'] + i m D1_s[chi'],
//   F_s(V) = i m D1_s[psi'] + D2_s[chi'];  F(mu) = F_0 + F_1, F(-mu) = F_0 - F_1.
//
// Operands are staged in shared memory in the no-swizzle K-major canonical layout:
// core matrices of 8 rows x 16 bytes (4 tf32), adjacent along K at LBO bytes and
// along M/N at SBO = 128 bytes.  The tables come pre-split into TF32 hi/lo and
// pre-packed in exactly that layout (plan time); the data are folded, split and
// packed while staging.  The Fourier data are FP32 (the mixed form's FFTs are FP32),
// so staging and epilogues run in FP32 and the FP64 spectral coefficients are
// converted on the integer pipe: the kernels issue no FP64 instruction, which on
// GB300 would otherwise bound them.  One thread issues the MMAs; completion is tracked with an
// mbarrier whose waits are bounded (on expiry the kernel records an error word,
// skips its output and still frees its tensor memory).
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "rexi_internal.h"

namespace rexi {

namespace {

constexpr int TM = 128;              // rows (analysis: degrees; synthesis: latitudes) per tile
constexpr int KB = 32;               // K per staged block (latitudes or degrees)
constexpr int SUB = TM * KB * 4;     // bytes of one packed 128 x 32 tf32 sub-tile (16 KiB)
constexpr unsigned kSpinLimit = 1u << 26;
constexpr int THREADS = 256;         // 8 warps: all stage; warp 0 allocates TMEM, thread 0 issues MMAs

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// tcgen05 shared-memory matrix descriptor, SWIZZLE_NONE, K-major canonical layout.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;  // descriptor version of sm_100-family tensor cores
  return d;                // base offset 0, absolute LBO mode 0, layout type 0 (no swizzle)
}

// Instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, M x N.
__device__ __forceinline__ uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
      smem_u32(mbar)));
}

__device__ __forceinline__ void mbar_init(uint64_t *mbar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count));
}

// Bounded wait for the mbarrier phase with parity `par`; false on expiry.
__device__ __forceinline__ bool mbar_wait(uint64_t *mbar, uint32_t par) {
  const uint32_t a = smem_u32(mbar);
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(a), "r"(par));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
               "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}

// 4 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float *v) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}

// 16-byte asynchronous global -> shared copy (completion: cp_async_wait_all)
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x ~ hi + lo with hi, lo TF32 (plan-time table packing, from FP64)
__device__ __forceinline__ void split_tf32(double x, uint32_t &hi, uint32_t &lo) {
  hi = to_tf32((float)x);
  lo = to_tf32((float)(x - (double)__uint_as_float(hi)));
}
// the same from FP32 data: x - hi is exact in FP32 (hi keeps the top 11 bits of x)
__device__ __forceinline__ void split_tf32f(float x, uint32_t &hi, uint32_t &lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// byte offset of element (row r, k) in a packed K-major tile with `groups` 8-row groups
__device__ __forceinline__ uint32_t core_off(int r, int k, int groups) {
  return (uint32_t)(((k >> 2) * groups + (r >> 3)) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Packs FP64 tables into TF32 hi/lo core-matrix sub-tiles.
//   analysis:  for each (m, p, tile, kb): [P_hi, P_lo, H_hi, H_lo], rows = degrees
//              n = m + p + 2 (tile*128 + r), K = latitudes j = kb*32 + k
//   synthesis: for each (m, jt, kb): [P0_hi, P0_lo, P1_hi, P1_lo, H0_hi, H0_lo, H1_hi, H1_lo],
//              rows = latitudes j = jt*128 + r, K = degree index i of parity q:
//              n = m + q + 2 (kb*32 + k)
struct PackArgs {
  const double *tabP, *tabH;
  uint32_t *dst;
  const int64_t *blk_off;  // per (m, p or jt, tile) first block (in sub-tile-set units), analysis
  int N, J, synth;
  int64_t nblocks;         // total (m, ., tile, kb) blocks
  const int4 *blk;         // per block: {m, p or jt, tile (ana) / 0, kb}
};

__global__ void pack_tables_kernel(PackArgs a) {
  const int64_t b = blockIdx.x;
  if (b >= a.nblocks) return;
  const int4 info = a.blk[b];
  const int m = info.x, pq = info.y, tile = info.z, kb = info.w;
  const int N = a.N, J = a.J;
  const int64_t idx0 = (int64_t)m * (2 * N + 3 - m) / 2;
  const int nsub = a.synth ? 8 : 4;
  uint32_t *out = a.dst + b * (int64_t)nsub * (SUB / 4);
  for (int t = threadIdx.x; t < TM * KB; t += blockDim.x) {
    const int r = t / KB, k = t - r * KB;
    const uint32_t off = core_off(r, k, TM / 8) / 4;
    if (!a.synth) {
      const int n = m + pq + 2 * (tile * TM + r);
      const int j = kb * KB + k;
      double p = 0.0, h = 0.0;
      if (n <= N && j < J) {
        p = a.tabP[(idx0 + n - m) * J + j];
        h = a.tabH[(idx0 + n - m) * J + j];
      }
      uint32_t hi, lo;
      split_tf32(p, hi, lo);
      out[0 * (SUB / 4) + off] = hi;
      out[1 * (SUB / 4) + off] = lo;
      split_tf32(h, hi, lo);
      out[2 * (SUB / 4) + off] = hi;
      out[3 * (SUB / 4) + off] = lo;
    } else {
      const int j = pq * TM + r;
      for (int q = 0; q < 2; ++q) {
        const int n = m + q + 2 * (kb * KB + k);
        double p = 0.0, h = 0.0;
        if (n <= N && j < J) {
          p = a.tabP[(idx0 + n - m) * J + j];
          h = a.tabH[(idx0 + n - m) * J + j];
        }
        uint32_t hi, lo;
        split_tf32(p, hi, lo);
        out[(2 * q + 0) * (SUB / 4) + off] = hi;
        out[(2 * q + 1) * (SUB / 4) + off] = lo;
        split_tf32(h, hi, lo);
        out[(4 + 2 * q + 0) * (SUB / 4) + off] = hi;
        out[(4 + 2 * q + 1) * (SUB / 4) + off] = lo;
      }
    }
  }
}

struct TcArgs {
  const uint32_t *tab;   // packed tables
  const int4 *work;      // per CTA: {m, p (analysis) or jt (synthesis), tile, first packed block}
  float2 *four;          // [nlat][N+1][3B], FP32 in the mixed form
  double2 *sint;         // [3][nspec][B]
  const double *zd;      // [nspec]
  int *err;              // device error word
  int N, nlat, J, B, G, nkb_fixed;
  int64_t nspec;
};

// ---- analysis -------------------------------------------------------------------------
// dynamic smem: [A: 4 x 16 KiB][B1 hi, B1 lo: 8G x 32 tf32 each][B2 hi, B2 lo: 4G x 32 each]
__global__ void __launch_bounds__(THREADS) leg_ana_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int4 w = a.work[blockIdx.x];
  const int m = w.x, p = w.y, tile = w.z;
  const int64_t blk0 = w.w;
  const int b0 = blockIdx.y * a.G;
  const int G = a.G, N1 = 8 * G, N2 = 4 * G;
  const int nkb = (a.J + KB - 1) / KB;
  unsigned char *sA = sm;
  unsigned char *sB1 = sm + 4 * SUB;
  unsigned char *sB2 = sB1 + 2 * N1 * KB * 4;
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(N1 + N2)) ncols <<= 1;
  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const int M1 = a.N + 1, ncol = 3 * a.B;
  bool ok = true;
  for (int kb = 0; kb < nkb; ++kb) {
    // tables: the packed 64 KiB block, copied asynchronously while the data are staged
    const uint4 *src = reinterpret_cast<const uint4 *>(a.tab + (blk0 + kb) * (int64_t)(4 * SUB / 4));
    uint4 *dstA = reinterpret_cast<uint4 *>(sA);
    for (int t = tid; t < 4 * SUB / 16; t += THREADS) cp_async16(dstA + t, src + t);
    // data: unit = (4 latitudes kq, state bl, field f in Phi, U, V, pad); every load of
    // the thread is issued before any use (one memory latency per block).  A unit
    // writes B1 columns 8 bl + 2 f + {re, im} (class of Pbar_n) and, for U and V,
    // B2 columns 4 bl + 2 (f - 1) + {re, im} (class of H_n), as 16-byte rows.
    {
      constexpr int RMAX = 512 / THREADS;  // units per thread: 8 kq x 4 G <= 512
      const int nun = (KB / 4) * 4 * G;
      float2 xn[RMAX][4], xs[RMAX][4];
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        const int u = tid + r * THREADS;
        const int kq = u / (4 * G), rem = u - kq * (4 * G), bl = rem >> 2, f = rem & 3;
        const int b = b0 + bl;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int j = kb * KB + 4 * kq + q;
          xn[r][q] = xs[r][q] = make_float2(0.f, 0.f);
          if (u < nun && f < 3 && j < a.J && b < a.B) {
            xn[r][q] = a.four[((int64_t)j * M1 + m) * ncol + 3 * b + f];
            xs[r][q] = a.four[((int64_t)(a.nlat - 1 - j) * M1 + m) * ncol + 3 * b + f];
          }
        }
      }
#pragma unroll
      for (int r = 0; r < RMAX; ++r) {
        const int u = tid + r * THREADS;
        if (u >= nun) continue;
        const int kq = u / (4 * G), rem = u - kq * (4 * G), bl = rem >> 2, f = rem & 3;
        uint32_t eh[2][4], el[2][4], oh[2][4], ol[2][4];  // [re/im][latitude]
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          split_tf32f(xn[r][q].x + xs[r][q].x, eh[0][q], el[0][q]);
          split_tf32f(xn[r][q].y + xs[r][q].y, eh[1][q], el[1][q]);
          split_tf32f(xn[r][q].x - xs[r][q].x, oh[0][q], ol[0][q]);
          split_tf32f(xn[r][q].y - xs[r][q].y, oh[1][q], ol[1][q]);
        }
        // Pbar_n has the class of p (E for p = 0); H_n the other one
        uint32_t(*ph)[4] = p ? oh : eh, (*pl)[4] = p ? ol : el;
        uint32_t(*hh)[4] = p ? eh : oh, (*hl)[4] = p ? el : ol;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint32_t off = core_off(8 * bl + 2 * f + c, 4 * kq, N1 / 8);
          *reinterpret_cast<uint4 *>(sB1 + off) = make_uint4(ph[c][0], ph[c][1], ph[c][2], ph[c][3]);
          *reinterpret_cast<uint4 *>(sB1 + N1 * KB * 4 + off) = make_uint4(pl[c][0], pl[c][1], pl[c][2], pl[c][3]);
          if (f == 1 || f == 2) {
            const uint32_t off2 = core_off(4 * bl + 2 * (f - 1) + c, 4 * kq, N2 / 8);
            *reinterpret_cast<uint4 *>(sB2 + off2) = make_uint4(hh[c][0], hh[c][1], hh[c][2], hh[c][3]);
            *reinterpret_cast<uint4 *>(sB2 + N2 * KB * 4 + off2) =
                make_uint4(hl[c][0], hl[c][1], hl[c][2], hl[c][3]);
          }
        }
      }
    }
    cp_async_wait_all();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc1 = make_idesc(TM, N1), idesc2 = make_idesc(TM, N2);
      const uint32_t aP = smem_u32(sA), aPl = aP + SUB, aH = aP + 2 * SUB, aHl = aP + 3 * SUB;
      const uint32_t b1 = smem_u32(sB1), b1l = b1 + N1 * KB * 4;
      const uint32_t b2 = smem_u32(sB2), b2l = b2 + N2 * KB * 4;
      const uint32_t lboA = (TM / 8) * 128, lbo1 = (N1 / 8) * 128, lbo2 = (N2 / 8) * 128;
      for (int s = 0; s < KB / 8; ++s) {
        const uint32_t oA = 2 * s * lboA, o1 = 2 * s * lbo1, o2 = 2 * s * lbo2;
        const uint32_t first = (kb == 0 && s == 0) ? 0u : 1u;
        // small products first, then hi * hi
        mma_tf32(tbase, make_desc(aPl + oA, lboA, 128), make_desc(b1 + o1, lbo1, 128), idesc1, first);
        mma_tf32(tbase, make_desc(aP + oA, lboA, 128), make_desc(b1l + o1, lbo1, 128), idesc1, 1u);
        mma_tf32(tbase, make_desc(aP + oA, lboA, 128), make_desc(b1 + o1, lbo1, 128), idesc1, 1u);
        mma_tf32(tbase + N1, make_desc(aHl + oA, lboA, 128), make_desc(b2 + o2, lbo2, 128), idesc2, first);
        mma_tf32(tbase + N1, make_desc(aH + oA, lboA, 128), make_desc(b2l + o2, lbo2, 128), idesc2, 1u);
        mma_tf32(tbase + N1, make_desc(aH + oA, lboA, 128), make_desc(b2 + o2, lbo2, 128), idesc2, 1u);
      }
      mma_commit(&mbar);
    }
    if (!mbar_wait(&mbar, (uint32_t)(kb & 1))) ok = false;
    tc_fence_after();
    ok = __syncthreads_and(ok) != 0;  // block-uniform, so every thread leaves the loop together
    if (!ok) break;
  }
  if (!ok) {
    if (tid == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
  } else {
    // epilogue: TMEM lane = row of the tile (warp w owns lanes 32w .. 32w + 31)
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (rows of the tile) for half w / 4 of the states
    const int wq = warp & 3, half = warp >> 2;
    const int r = tile * TM + wq * 32 + (tid & 31);
    const int n = m + p + 2 * r;
    const uint32_t lane_addr = tbase + ((uint32_t)(wq * 32) << 16);
    for (int bl = half * (G / 2); bl < (half + 1) * (G / 2); ++bl) {
      float d1[8], d2[4];
      tmem_ld4(lane_addr + 8 * bl, d1);
      tmem_ld4(lane_addr + 8 * bl + 4, d1 + 4);
      tmem_ld4(lane_addr + N1 + 4 * bl, d2);
      const int b = b0 + bl;
      if (n <= a.N && b < a.B) {
        const int64_t ix = (int64_t)m * (2 * a.N + 3 - m) / 2 + (n - m);
        // FP32 arithmetic, FP64 stores (the solve's input) converted on the integer pipe
        const float s = f64_to_f32(a.zd[ix]), fm = (float)m;
        const float2 pu = make_float2(d1[2], d1[3]), pv = make_float2(d1[4], d1[5]);
        const float2 hu = make_float2(d2[0], d2[1]), hv = make_float2(d2[2], d2[3]);
        a.sint[ix * a.B + b] = make_double2(f32_to_f64(d1[0]), f32_to_f64(d1[1]));
        a.sint[(a.nspec + ix) * a.B + b] =
            make_double2(f32_to_f64(s * (-fm * pv.y + hu.x)), f32_to_f64(s * (fm * pv.x + hu.y)));
        a.sint[(2 * a.nspec + ix) * a.B + b] =
            make_double2(f32_to_f64(s * (-fm * pu.y - hv.x)), f32_to_f64(s * (fm * pu.x - hv.y)));
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, ncols);
}

// ---- synthesis ------------------------------------------------------------------------
// Two accumulator classes per tile: class c holds the Pbar rows of parity c against B1_c
// (Phi, psi', chi' of degrees n - m = c mod 2) and the H rows of parity 1 - c against B2_c
// (psi', chi' of the other parity); north and south are their sum and difference.
// SPLIT = false: each degree block stages both classes, dynamic smem [A: 8 x 16 KiB]
// [B1_0, B1_1: (hi, lo) 8G x 32][B2_0, B2_1: (hi, lo) 4G x 32], one CTA per SM.
// SPLIT = true (groups of up to 8 states): each block is staged one class at a time, smem
// [A: 4 x 16 KiB][B1: (hi, lo) 8G x 32][B2: (hi, lo) 4G x 32], so that two CTAs fit on
// an SM and one fetches tables while the other converts and multiplies.
template <bool SPLIT>
__global__ void __launch_bounds__(THREADS, SPLIT ? 2 : 1) leg_syn_tc_kernel(TcArgs a) {
  extern __shared__ __align__(1024) unsigned char sm[];
  __shared__ uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const int4 w = a.work[blockIdx.x];
  const int m = w.x, jt = w.y;
  const int64_t blk0 = w.w;
  const int b0 = blockIdx.y * a.G;
  const int G = a.G, N1 = 8 * G, N2 = 4 * G;
  const int L0 = (a.N - m) / 2 + 1;                    // degrees with n - m even
  const int L1 = (a.N - m - 1) >= 0 ? (a.N - m - 1) / 2 + 1 : 0;
  const int nkb = (max(L0, L1) + KB - 1) / KB;
  constexpr int kCls = SPLIT ? 1 : 2;                  // classes staged per iteration
  unsigned char *sA = sm;
  unsigned char *sB1 = sm + 4 * kCls * SUB;            // class slot s at sB1 + s * 2 * N1 * KB * 4
  unsigned char *sB2 = sB1 + kCls * (2 * N1 * KB * 4); // class slot s at sB2 + s * 2 * N2 * KB * 4
  const int tid = threadIdx.x, warp = tid >> 5;
  uint32_t ncols = 32;
  while (ncols < (uint32_t)(2 * (N1 + N2))) ncols <<= 1;
  if (warp == 0) tmem_alloc(&tmem_base, ncols);
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = tmem_base;
  const int64_t idx0 = (int64_t)m * (2 * a.N + 3 - m) / 2;
  bool ok = true;
  const int nit = SPLIT ? 2 * nkb : nkb;
  for (int it = 0; it < nit; ++it) {
    const int kb = SPLIT ? it >> 1 : it;
    const int c0 = SPLIT ? (it & 1) : 0;  // the (first) class of this iteration
    const uint4 *src = reinterpret_cast<const uint4 *>(a.tab + (blk0 + kb) * (int64_t)(8 * SUB / 4));
    uint4 *dstA = reinterpret_cast<uint4 *>(sA);
    if constexpr (SPLIT) {
      // class c0: sub-tiles Pbar parity c0 (2 c0, 2 c0 + 1) and H parity 1 - c0 (4 + 2 (1 - c0), +1)
      const uint4 *srcP = src + (2 * c0) * (SUB / 16), *srcH = src + (4 + 2 * (1 - c0)) * (SUB / 16);
      for (int t = tid; t < 2 * SUB / 16; t += THREADS) {
        cp_async16(dstA + t, srcP + t);
        cp_async16(dstA + 2 * SUB / 16 + t, srcH + t);
      }
    } else {
      for (int t = tid; t < 8 * SUB / 16; t += THREADS) cp_async16(dstA + t, src + t);
    }
    // spectral data: unit = (parity q, 4 degrees kq, state bl, field f in Phi, psi', chi',
    // pad); rows i = kb*32 + 4 kq + r have n = m + q + 2 i.  P-terms feed class q (B1_q),
    // H-terms (psi', chi') class 1 - q (B2_{1-q}); with SPLIT only those of class c0 are
    // loaded and staged.  All loads are issued first.
    {
      constexpr int RMAX = 1024 / THREADS;  // 2 q x 8 kq x 4 G <= 1024
      const int nun = 2 * (KB / 4) * 4 * G;
      // every load of the block first (an element outside the data reads element 0 and
      // is zeroed), then the conversions: converting inside the load loop puts one memory
      // latency per load on the critical path (measured: 11.6 of the block's 14 us at T341)
      double2 xr[RMAX][4];
      double zr[RMAX][4];
      bool vr[RMAX][4];
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr) {
        const int u = tid + rr * THREADS;
        const int q = u / ((KB / 4) * 4 * G), u2 = u - q * ((KB / 4) * 4 * G);
        const int kq = u2 / (4 * G), rem = u2 - kq * (4 * G), bl = rem >> 2, f = rem & 3;
        const int b = b0 + bl;
#pragma unroll
        const bool need = !SPLIT || q == c0 || f == 1 || f == 2;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const int n = m + q + 2 * (kb * KB + 4 * kq + r);
          const bool v = need && u < nun && f < 3 && n <= a.N && b < a.B;
          const int64_t ix = v ? idx0 + (n - m) : 0;
          xr[rr][r] = a.sint[((int64_t)(v ? f : 0) * a.nspec + ix) * a.B + (v ? b : 0)];
          zr[rr][r] = f > 0 ? a.zd[ix] : 1.0;
          vr[rr][r] = v;
        }
      }
      float2 xv[RMAX][4];
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float sc = f64_to_f32(zr[rr][r]);
          xv[rr][r] = vr[rr][r] ? make_float2(sc * f64_to_f32(xr[rr][r].x), sc * f64_to_f32(xr[rr][r].y))
                                : make_float2(0.f, 0.f);
        }
#pragma unroll
      for (int rr = 0; rr < RMAX; ++rr) {
        const int u = tid + rr * THREADS;
        if (u >= nun) continue;
        const int q = u / ((KB / 4) * 4 * G), u2 = u - q * ((KB / 4) * 4 * G);
        const int kq = u2 / (4 * G), rem = u2 - kq * (4 * G), bl = rem >> 2, f = rem & 3;
        uint32_t hi[2][4], lo[2][4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          split_tf32f(xv[rr][r].x, hi[0][r], lo[0][r]);
          split_tf32f(xv[rr][r].y, hi[1][r], lo[1][r]);
        }
        const bool w1 = !SPLIT || q == c0, w2 = !SPLIT || 1 - q == c0;  // B1 of class q, B2 of class 1 - q
        unsigned char *b1 = sB1 + (SPLIT ? 0 : q) * (2 * N1 * KB * 4);
        unsigned char *b2 = sB2 + (SPLIT ? 0 : 1 - q) * (2 * N2 * KB * 4);
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint32_t off = core_off(8 * bl + 2 * f + c, 4 * kq, N1 / 8);
          if (w1) {
            *reinterpret_cast<uint4 *>(b1 + off) = make_uint4(hi[c][0], hi[c][1], hi[c][2], hi[c][3]);
            *reinterpret_cast<uint4 *>(b1 + N1 * KB * 4 + off) = make_uint4(lo[c][0], lo[c][1], lo[c][2], lo[c][3]);
          }
          if (w2 && (f == 1 || f == 2)) {
            const uint32_t off2 = core_off(4 * bl + 2 * (f - 1) + c, 4 * kq, N2 / 8);
            *reinterpret_cast<uint4 *>(b2 + off2) = make_uint4(hi[c][0], hi[c][1], hi[c][2], hi[c][3]);
            *reinterpret_cast<uint4 *>(b2 + N2 * KB * 4 + off2) =
                make_uint4(lo[c][0], lo[c][1], lo[c][2], lo[c][3]);
          }
        }
      }
    }
    cp_async_wait_all();
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t idesc1 = make_idesc(TM, N1), idesc2 = make_idesc(TM, N2);
      const uint32_t lboA = (TM / 8) * 128, lbo1 = (N1 / 8) * 128, lbo2 = (N2 / 8) * 128;
      const uint32_t A0 = smem_u32(sA);
      for (int cs = 0; cs < kCls; ++cs) {
        // class cls: Pbar rows of parity cls with B1_cls; H rows of parity 1 - cls with B2_cls
        // (SPLIT: the staged class sits in slot 0, its Pbar tiles then its H tiles)
        const int cls = c0 + cs;
        const uint32_t aP = A0 + (SPLIT ? 0 : 2 * cls) * SUB, aPl = aP + SUB;
        const uint32_t aH = A0 + (SPLIT ? 2 : 4 + 2 * (1 - cls)) * SUB, aHl = aH + SUB;
        const uint32_t b1 = smem_u32(sB1 + cs * (2 * N1 * KB * 4)), b1l = b1 + N1 * KB * 4;
        const uint32_t b2 = smem_u32(sB2 + cs * (2 * N2 * KB * 4)), b2l = b2 + N2 * KB * 4;
        const uint32_t d1 = tbase + cls * (N1 + N2), d2 = d1 + N1;
        for (int s = 0; s < KB / 8; ++s) {
          const uint32_t oA = 2 * s * lboA, o1 = 2 * s * lbo1, o2 = 2 * s * lbo2;
          const uint32_t first = (kb == 0 && s == 0) ? 0u : 1u;
          mma_tf32(d1, make_desc(aPl + oA, lboA, 128), make_desc(b1 + o1, lbo1, 128), idesc1, first);
          mma_tf32(d1, make_desc(aP + oA, lboA, 128), make_desc(b1l + o1, lbo1, 128), idesc1, 1u);
          mma_tf32(d1, make_desc(aP + oA, lboA, 128), make_desc(b1 + o1, lbo1, 128), idesc1, 1u);
          mma_tf32(d2, make_desc(aHl + oA, lboA, 128), make_desc(b2 + o2, lbo2, 128), idesc2, first);
          mma_tf32(d2, make_desc(aH + oA, lboA, 128), make_desc(b2l + o2, lbo2, 128), idesc2, 1u);
          mma_tf32(d2, make_desc(aH + oA, lboA, 128), make_desc(b2 + o2, lbo2, 128), idesc2, 1u);
        }
      }
      mma_commit(&mbar);
    }
    if (!mbar_wait(&mbar, (uint32_t)(it & 1))) ok = false;
    tc_fence_after();
    ok = __syncthreads_and(ok) != 0;  // block-uniform, so every thread leaves the loop together
    if (!ok) break;
  }
  if (!ok) {
    if (tid == 0) atomicOr(a.err, DEV_ERR_TIMEOUT);
  } else {
    const int wq = warp & 3, half = warp >> 2;
    const int jl = wq * 32 + (tid & 31);  // this thread's latitude row of the tile
    const uint32_t lane_addr = tbase + ((uint32_t)(wq * 32) << 16);
    const int M1 = a.N + 1, ncol = 3 * a.B;
    const float fm = (float)m;
    // With 8 or more states a group, the tile's results go through shared memory (free
    // once the last MMA has completed), [north, south][TM latitudes][3G columns + 1], so
    // that each latitude's 3G columns reach the Fourier array as one contiguous row (the
    // odd row stride puts the 32 latitudes a warp writes on distinct banks): -14 % at 16
    // states.  Smaller groups store directly, a few columns per latitude.
    const bool via_smem = G >= 8;
    const int CW = 3 * G, RSW = 3 * G + 1;
    float2 *tr = reinterpret_cast<float2 *>(sm);
    for (int bl = half * (G / 2); bl < (half + 1) * (G / 2); ++bl) {
      float2 F[2][3];
      for (int cls = 0; cls < 2; ++cls) {
        float d1[8], d2[4];
        const uint32_t base = lane_addr + cls * (N1 + N2);
        tmem_ld4(base + 8 * bl, d1);
        tmem_ld4(base + 8 * bl + 4, d1 + 4);
        tmem_ld4(base + N1 + 4 * bl, d2);
        // d1: Phi re/im, psi' re/im, chi' re/im; d2: psi' re/im, chi' re/im (H-terms)
        F[cls][0] = make_float2(d1[0], d1[1]);
        F[cls][1] = make_float2(-d2[0] - fm * d1[5], -d2[1] + fm * d1[4]);
        F[cls][2] = make_float2(-fm * d1[3] + d2[2], fm * d1[2] + d2[3]);
      }
      if (via_smem) {
        for (int f = 0; f < 3; ++f) {
          tr[jl * RSW + 3 * bl + f] = make_float2(F[0][f].x + F[1][f].x, F[0][f].y + F[1][f].y);
          tr[(TM + jl) * RSW + 3 * bl + f] = make_float2(F[0][f].x - F[1][f].x, F[0][f].y - F[1][f].y);
        }
      } else {
        const int j = jt * TM + jl, b = b0 + bl;
        if (j < a.J && b < a.B) {
          float2 *north = a.four + ((int64_t)j * M1 + m) * ncol + 3 * b;
          float2 *south = a.four + ((int64_t)(a.nlat - 1 - j) * M1 + m) * ncol + 3 * b;
          for (int f = 0; f < 3; ++f) {
            north[f] = make_float2(F[0][f].x + F[1][f].x, F[0][f].y + F[1][f].y);
            south[f] = make_float2(F[0][f].x - F[1][f].x, F[0][f].y - F[1][f].y);
          }
        }
      }
    }
    if (via_smem) {  // block-uniform
      __syncthreads();
      // one warp per row: the valid columns (states < B) of latitude j, north then south
      const int ncw = min(CW, ncol - 3 * b0), lane = tid & 31;
      for (int row = warp; row < 2 * TM; row += THREADS / 32) {
        const int side = row / TM, jr = row - side * TM, j = jt * TM + jr;
        if (j >= a.J) continue;
        float2 *dst = a.four + ((int64_t)(side ? a.nlat - 1 - j : j) * M1 + m) * ncol + 3 * b0;
        const float2 *srow = tr + row * RSW;
        for (int c = lane; c < ncw; c += 32) dst[c] = srow[c];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tbase, ncols);
}

int group_size(int B) { return std::min(B, 16) + (4 - std::min(B, 16) % 4) % 4; }

size_t ana_smem(int G) { return 4 * (size_t)SUB + 2 * (8 * G) * KB * 4 + 2 * (4 * G) * KB * 4; }
// The synthesis stages one accumulator class per block iteration (two CTAs per SM) when
//  - two CTAs' tensor-memory accumulators (2 classes x 12 G columns each, rounded up to a
//    power of two) fit in the SM's 512 columns: groups of up to 8 states, and
//  - the grid has at least three CTAs per SM, so that CTAs do share SMs.  With fewer, the
//    split only doubles each CTA's chain of table fetches and MMA round trips (measured,
//    T170 one state, 171 CTAs: 0.0335 against 0.0242 ms; T255 one state, 512 CTAs: 0.0609
//    against 0.0669 ms; T1279 one state: 3.77 against 4.24 ms).
bool syn_split(int G, int64_t ncta, int num_sms) { return G <= 8 && ncta >= 3 * (int64_t)num_sms; }
size_t syn_smem(int G, bool split) {
  const int cls = split ? 1 : 2;
  return 4 * (size_t)cls * SUB + cls * (2 * (8 * G) * KB * 4) + cls * (2 * (4 * G) * KB * 4);
}

}  // namespace

// Plan-time: work lists and packed TF32 hi/lo tables for both directions.
cudaError_t tc_setup(Plan &pl) {
  const int N = pl.N, J = pl.J;
  const int nkb_ana = (J + KB - 1) / KB;
  std::vector<int4> work_a, blk_a, work_s, blk_s;
  int64_t nb = 0;
  for (int m = 0; m <= N; ++m)
    for (int p = 0; p < 2; ++p) {
      if (m + p > N) continue;
      const int L = (N - m - p) / 2 + 1;
      for (int t = 0; t * TM < L; ++t) {
        work_a.push_back(make_int4(m, p, t, (int)nb));
        for (int kb = 0; kb < nkb_ana; ++kb) blk_a.push_back(make_int4(m, p, t, kb));
        nb += nkb_ana;
      }
    }
  int64_t ns = 0;
  const int njt = (J + TM - 1) / TM;
  for (int m = 0; m <= N; ++m) {
    const int L0 = (N - m) / 2 + 1, L1 = (N - m - 1) >= 0 ? (N - m - 1) / 2 + 1 : 0;
    const int nkb = (std::max(L0, L1) + KB - 1) / KB;
    for (int jt = 0; jt < njt; ++jt) {
      work_s.push_back(make_int4(m, jt, 0, (int)ns));
      for (int kb = 0; kb < nkb; ++kb) blk_s.push_back(make_int4(m, jt, 0, kb));
      ns += nkb;
    }
  }
  auto up = [&](const std::vector<int4> &v, int4 **d) -> cudaError_t {
    cudaError_t e = cudaMalloc(d, std::max<size_t>(1, v.size()) * sizeof(int4));
    if (e != cudaSuccess) return e;
    pl.bytes += v.size() * sizeof(int4);
    return cudaMemcpy(*d, v.data(), v.size() * sizeof(int4), cudaMemcpyHostToDevice);
  };
  cudaError_t e;
  int4 *blk_a_dev = nullptr, *blk_s_dev = nullptr;
  if ((e = up(work_a, &pl.tc_work_ana))) return e;
  if ((e = up(work_s, &pl.tc_work_syn))) return e;
  if ((e = up(blk_a, &blk_a_dev))) return e;
  if ((e = up(blk_s, &blk_s_dev))) return e;
  pl.tc_nwork_ana = (int)work_a.size();
  pl.tc_nwork_syn = (int)work_s.size();
  const size_t bytes_a = (size_t)nb * 4 * SUB, bytes_s = (size_t)ns * 8 * SUB;
  if ((e = cudaMalloc(&pl.tc_tab_ana, bytes_a))) return e;
  if ((e = cudaMalloc(&pl.tc_tab_syn, bytes_s))) return e;
  pl.bytes += bytes_a + bytes_s;
  PackArgs pa{pl.tabP, pl.tabH, pl.tc_tab_ana, nullptr, N, J, 0, nb, blk_a_dev};
  pack_tables_kernel<<<(unsigned)nb, 256>>>(pa);
  if ((e = cudaGetLastError())) return e;
  PackArgs ps{pl.tabP, pl.tabH, pl.tc_tab_syn, nullptr, N, J, 1, ns, blk_s_dev};
  pack_tables_kernel<<<(unsigned)ns, 256>>>(ps);
  if ((e = cudaGetLastError())) return e;
  e = cudaDeviceSynchronize();
  cudaFree(blk_a_dev);
  cudaFree(blk_s_dev);
  if (e != cudaSuccess) return e;
  const int Gmax = group_size(pl.prm.max_batch);
  if ((e = cudaFuncSetAttribute(leg_ana_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)ana_smem(Gmax))))
    return e;
  if ((e = cudaFuncSetAttribute(leg_syn_tc_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)syn_smem(std::min(Gmax, 8), true))))
    return e;
  return cudaFuncSetAttribute(leg_syn_tc_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)syn_smem(Gmax, false));
}

cudaError_t launch_leg_ana_tc(Plan &pl, const double2 *four, double2 *sint, int B, const double *zd,
                              cudaStream_t st) {
  const int G = group_size(B);
  // the mixed form's Fourier array holds FP32 pairs
  TcArgs a{pl.tc_tab_ana, pl.tc_work_ana, reinterpret_cast<float2 *>(const_cast<double2 *>(four)), sint, zd,
           pl.dev_err, pl.N, pl.nlat, pl.J, B, G, 0, pl.nspec};
  dim3 grid((unsigned)pl.tc_nwork_ana, (unsigned)((B + G - 1) / G));
  leg_ana_tc_kernel<<<grid, THREADS, ana_smem(G), st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_leg_syn_tc(Plan &pl, const double2 *sint, double2 *four, int B, const double *zd,
                              cudaStream_t st) {
  const int G = group_size(B);
  TcArgs a{pl.tc_tab_syn, pl.tc_work_syn, reinterpret_cast<float2 *>(four), const_cast<double2 *>(sint), zd,
           pl.dev_err, pl.N, pl.nlat, pl.J, B, G, 0, pl.nspec};
  dim3 grid((unsigned)pl.tc_nwork_syn, (unsigned)((B + G - 1) / G));
  if (syn_split(G, (int64_t)grid.x * grid.y, pl.num_sms))
    leg_syn_tc_kernel<true><<<grid, THREADS, syn_smem(G, true), st>>>(a);
  else
    leg_syn_tc_kernel<false><<<grid, THREADS, syn_smem(G, false), st>>>(a);
  return cudaGetLastError();
}

}  // namespace rexi
