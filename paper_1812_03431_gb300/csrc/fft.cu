// Longitude transforms (paper Sec. 3): for every latitude row of every field,
//   forward  F_m = s_m sum_i x_i e^{-i m lambda_i},   m = 0..N,
//   inverse  x_i = sum_{m=-N}^{N} X_m e^{i m lambda_i},  X_{-m} = conj(X_m),  X_m = s_m F_m,
// with per-(field, latitude) input/output scales that carry Robert's cos(lat)
// factor, g, the Gaussian weights and the transposes' scalings.
//
// Each real row of even length n is transformed on its own: its even and odd
// samples form one complex sequence z_k = x_{2k} + i x_{2k+1} of length n/2,
// transformed by a mixed-radix (2, 3, 4, 5, 8) Stockham autosort FFT in shared
// memory; X_m = E_m + e^{-2 pi i m/n} O_m with E_m = (Z_m + conj Z_{n/2-m})/2,
// O_m = (Z_m - conj Z_{n/2-m})/(2i).  (Packing two different rows instead would
// let the rounding of a large row leak into a small one.)  The inverse builds
// Z'_m = E'_m + i O'_m from the Hermitian spectrum and evaluates
// conj(FFT(conj Z')).
//
// Layouts: grid [B][3][nlat][nlon] float64; Fourier [nlat][N+1][3B] complex (FP64 in
// the FP64 form, FP32 in the mixed form, where the transform itself is FP32), column
// c = 3 b + field, so that for each latitude the Legendre kernels read contiguous
// columns.  The mixed form scales in FP32 (scales rounded to binary32 once, at plan time)
// and converts the data between FP64 and FP32 on the integer pipe (f64_to_f32 /
// f32_to_f64): no FP64 instruction is left in its kernels.
#include <cuda_runtime.h>

#include <cmath>
#include <type_traits>

#include "rexi_internal.h"

namespace rexi {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };
template <typename T> __device__ __forceinline__ typename V2<T>::t mk(T x, T y) { return {x, y}; }

struct FftArgs {
  const void *tw;  // n twiddles e^{-2 pi i k / n} (n = nlon), double2 or float2
  int n, h, nstages, N, nlat, ncol, np;  // h = n / 2 complex points per row; np rows per CTA
  int radix[24];
  // division by run-time sizes as a multiply-high: x / d = umulhi(x, mag) for x, d < 2^16
  uint32_t mag_nb[24], mag_ns[24], mag_h, mag_np;
  double c3, s3, c5a, s5a, c5b, s5b;  // cos/sin of 2pi/3, 2pi/5, 4pi/5
};

__host__ __device__ inline uint32_t div_magic(int d) { return d > 1 ? (uint32_t)((1ull << 32) / (unsigned)d + 1) : 0u; }
// exact for 0 <= x < 2^16 and 1 <= d < 2^16 (x d < 2^32)
__device__ __forceinline__ int fdiv(int x, uint32_t mag, int d) {
  return d == 1 ? x : (int)__umulhi((uint32_t)x, mag);
}

template <typename C> __device__ __forceinline__ C cmulz(C a, C b) { return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
template <typename C> __device__ __forceinline__ C addz(C a, C b) { return {a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C subz(C a, C b) { return {a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C mulmi(C a) { return {a.y, -a.x}; }  // -i a

// In-register DFT of R points (forward, e^{-2 pi i jk/R}); R is a compile-time constant
// so v[] stays in registers and the loops unroll.
template <typename T, int R>
__device__ __forceinline__ void dft_small(typename V2<T>::t *v, const FftArgs &a) {
  using C = typename V2<T>::t;
  if constexpr (R == 2) {
    C t = v[0];
    v[0] = addz(t, v[1]);
    v[1] = subz(t, v[1]);
  } else if constexpr (R == 4) {
    C t0 = addz(v[0], v[2]), t1 = subz(v[0], v[2]);
    C t2 = addz(v[1], v[3]), t3 = mulmi(subz(v[1], v[3]));
    v[0] = addz(t0, t2);
    v[2] = subz(t0, t2);
    v[1] = addz(t1, t3);
    v[3] = subz(t1, t3);
  } else if constexpr (R == 8) {
    // two 4-point DFTs (even and odd samples) and the w8^k butterflies
    C a0 = addz(v[0], v[4]), a1 = subz(v[0], v[4]), a2 = addz(v[2], v[6]), a3 = mulmi(subz(v[2], v[6]));
    C b0 = addz(v[1], v[5]), b1 = subz(v[1], v[5]), b2 = addz(v[3], v[7]), b3 = mulmi(subz(v[3], v[7]));
    C e0 = addz(a0, a2), e2 = subz(a0, a2), e1 = addz(a1, a3), e3 = subz(a1, a3);
    C o0 = addz(b0, b2), o2 = subz(b0, b2), o1 = addz(b1, b3), o3 = subz(b1, b3);
    const T r2 = (T)0.70710678118654752440;  // 1/sqrt(2)
    C w1 = {r2 * (o1.x + o1.y), r2 * (o1.y - o1.x)};   // o1 (1 - i)/sqrt(2)
    C w2 = mulmi(o2);                                  // o2 (-i)
    C w3 = {r2 * (o3.y - o3.x), -r2 * (o3.x + o3.y)};  // o3 (-1 - i)/sqrt(2)
    v[0] = addz(e0, o0);
    v[4] = subz(e0, o0);
    v[1] = addz(e1, w1);
    v[5] = subz(e1, w1);
    v[2] = addz(e2, w2);
    v[6] = subz(e2, w2);
    v[3] = addz(e3, w3);
    v[7] = subz(e3, w3);
  } else if constexpr (R == 3) {
    const T c3 = (T)a.c3, s3 = (T)a.s3;
    C s = addz(v[1], v[2]);
    C d = subz(v[1], v[2]);
    C y0 = addz(v[0], s);
    C t = {v[0].x + c3 * s.x, v[0].y + c3 * s.y};
    C u = mulmi(C{s3 * d.x, s3 * d.y});
    v[0] = y0;
    v[1] = addz(t, u);
    v[2] = subz(t, u);
  } else {  // R == 5
    const T c5a = (T)a.c5a, s5a = (T)a.s5a, c5b = (T)a.c5b, s5b = (T)a.s5b;
    C b1 = addz(v[1], v[4]), b2 = addz(v[2], v[3]);
    C d1 = subz(v[1], v[4]), d2 = subz(v[2], v[3]);
    C y0 = addz(v[0], addz(b1, b2));
    C t1 = {v[0].x + c5a * b1.x + c5b * b2.x, v[0].y + c5a * b1.y + c5b * b2.y};
    C t2 = {v[0].x + c5b * b1.x + c5a * b2.x, v[0].y + c5b * b1.y + c5a * b2.y};
    C u1 = mulmi(C{s5a * d1.x + s5b * d2.x, s5a * d1.y + s5b * d2.y});
    C u2 = mulmi(C{s5b * d1.x - s5a * d2.x, s5b * d1.y - s5a * d2.y});
    v[0] = y0;
    v[1] = addz(t1, u1);
    v[4] = subz(t1, u1);
    v[2] = addz(t2, u2);
    v[3] = subz(t2, u2);
  }
}

// One Stockham pass of radix R over np rows of n points: src -> dst.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const typename V2<T>::t *src, typename V2<T>::t *dst, int n, int Ns,
                                              uint32_t mnb, uint32_t mns, const FftArgs &a) {
  using C = typename V2<T>::t;
  const C *tw = static_cast<const C *>(a.tw);
  const int nb = n / R;
  const int tstep = 2 * (n / (Ns * R));  // twiddle e^{-2 pi i jm r / (Ns R)} = tw[r jm tstep]
  for (int t = threadIdx.x; t < a.np * nb; t += blockDim.x) {
    const int q = fdiv(t, mnb, nb), jb = t - q * nb;
    const C *in = src + q * n;
    C *out = dst + q * n;
    const int jd = fdiv(jb, mns, Ns), jm = jb - jd * Ns;
    C v[R];
    v[0] = in[jb];
#pragma unroll
    for (int r = 1; r < R; ++r) v[r] = cmulz(in[jb + r * nb], tw[r * jm * tstep]);  // tw[0] = 1 exactly
    dft_small<T, R>(v, a);
    const int od = jd * Ns * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out[od + r * Ns] = v[r];
  }
}

// In-shared-memory forward FFT of np rows of h points; returns the buffer holding
// the result (buf0 or buf1).
template <typename T>
__device__ typename V2<T>::t *fft_smem(typename V2<T>::t *buf0, typename V2<T>::t *buf1, const FftArgs &a) {
  using C = typename V2<T>::t;
  const int n = a.h;
  C *src = buf0, *dst = buf1;
  int Ns = 1;
  for (int s = 0; s < a.nstages; ++s) {
    const int R = a.radix[s];
    const uint32_t mnb = a.mag_nb[s], mns = a.mag_ns[s];
    switch (R) {  // uniform across the block
      case 8: stockham_pass<T, 8>(src, dst, n, Ns, mnb, mns, a); break;
      case 4: stockham_pass<T, 4>(src, dst, n, Ns, mnb, mns, a); break;
      case 2: stockham_pass<T, 2>(src, dst, n, Ns, mnb, mns, a); break;
      case 3: stockham_pass<T, 3>(src, dst, n, Ns, mnb, mns, a); break;
      default: stockham_pass<T, 5>(src, dst, n, Ns, mnb, mns, a); break;
    }
    __syncthreads();
    C *tmp = src;
    src = dst;
    dst = tmp;
    Ns *= R;
  }
  return src;
}

// T: arithmetic type inside the transform (double, or float in the mixed form, whose
// Fourier array is FP32); the grid stays FP64 either way, and the scales come in type T.
template <typename T>
__global__ void fft_fwd_kernel(FftArgs a, const double *grid, void *four_v, const T *in_scale, const T *m_scale) {
  using C = typename V2<T>::t;
  constexpr bool F32 = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  const C *tw = static_cast<const C *>(a.tw);
  C *four = static_cast<C *>(four_v);
  const int h = a.h;
  C *buf0 = sm, *buf1 = sm + a.np * h;
  const int j = blockIdx.y;
  const int c0 = blockIdx.x * a.np;
  const double2 *g2 = reinterpret_cast<const double2 *>(grid);
  // in chunks of kLd elements per thread: every load of a chunk first (an element outside
  // the data reads element 0 and is zeroed), then the conversions, so that the loads'
  // latencies overlap instead of one conversion waiting on each
  constexpr int kLd = 8;
  for (int t0 = 0; t0 < a.np * h; t0 += kLd * blockDim.x) {
    double2 x[kLd];
    T sv[kLd];
    bool ok[kLd];
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int t = t0 + i * blockDim.x + threadIdx.x;
      const int q = fdiv(t, a.mag_h, h), k = t - q * h;
      const int c = c0 + q;
      ok[i] = t < a.np * h && c < a.ncol;
      x[i] = g2[ok[i] ? ((int64_t)c * a.nlat + j) * h + k : 0];
      sv[i] = in_scale[ok[i] ? (c % 3) * a.nlat + j : 0];
    }
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int t = t0 + i * blockDim.x + threadIdx.x;
      if (t >= a.np * h) break;
      C v = {0, 0};
      if (ok[i]) {
        if constexpr (F32) {
          v = C{sv[i] * f64_to_f32(x[i].x), sv[i] * f64_to_f32(x[i].y)};
        } else {
          v = C{sv[i] * x[i].x, sv[i] * x[i].y};
        }
      }
      buf0[t] = v;
    }
  }
  __syncthreads();
  const C *Z = fft_smem<T>(buf0, buf1, a);
  const int M1 = a.N + 1;
  for (int t = threadIdx.x; t < a.np * M1; t += blockDim.x) {
    const int m = fdiv(t, a.mag_np, a.np), q = t - m * a.np;
    const int c = c0 + q;
    if (c >= a.ncol) continue;
    const C zm = Z[q * h + m];
    const C zr = Z[q * h + (m == 0 ? 0 : h - m)];
    // E = (Z_m + conj Z_{h-m}) / 2,  O = (Z_m - conj Z_{h-m}) / (2 i)
    const C E = {(T)0.5 * (zm.x + zr.x), (T)0.5 * (zm.y - zr.y)};
    const C O = {(T)0.5 * (zm.y + zr.y), (T)-0.5 * (zm.x - zr.x)};
    const C X = addz(E, cmulz(tw[m], O));
    const T s = m_scale[m];
    four[((int64_t)j * M1 + m) * a.ncol + c] = C{s * X.x, s * X.y};
  }
}

template <typename T>
__global__ void fft_inv_kernel(FftArgs a, const void *four_v, double *grid, const T *m_scale, const T *out_scale) {
  using C = typename V2<T>::t;
  constexpr bool F32 = std::is_same<T, float>::value;
  extern __shared__ __align__(16) unsigned char smraw[];
  C *sm = reinterpret_cast<C *>(smraw);
  const C *tw = static_cast<const C *>(a.tw);
  const C *four = static_cast<const C *>(four_v);
  const int h = a.h;
  C *buf0 = sm, *buf1 = sm + a.np * h;
  const int j = blockIdx.y;
  const int c0 = blockIdx.x * a.np;
  const int N = a.N, M1 = N + 1;
  // column index fastest, so that neighbouring threads read neighbouring Fourier columns;
  // in chunks of kLd elements per thread, every load of a chunk before any use (an element
  // outside the data reads element 0 and is zeroed)
  constexpr int kLd = 4;
  for (int t0 = 0; t0 < a.np * h; t0 += kLd * blockDim.x) {
    C va[kLd], vb[kLd];
    T sa[kLd], sb[kLd];
    bool oka[kLd], okb[kLd];
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int t = t0 + i * blockDim.x + threadIdx.x;
      const int m = fdiv(t, a.mag_np, a.np), q = t - m * a.np;
      const int c = c0 + q;
      const bool in = t < a.np * h && c < a.ncol;
      const int mr = h - m;  // partner X_{h-m}, present when h - m <= N
      oka[i] = in && m <= N;
      okb[i] = in && m > 0 && mr <= N;
      va[i] = four[oka[i] ? ((int64_t)j * M1 + m) * a.ncol + c : 0];
      vb[i] = four[okb[i] ? ((int64_t)j * M1 + mr) * a.ncol + c : 0];
      sa[i] = m_scale[oka[i] ? m : 0];
      sb[i] = m_scale[okb[i] ? mr : 0];
    }
#pragma unroll
    for (int i = 0; i < kLd; ++i) {
      const int t = t0 + i * blockDim.x + threadIdx.x;
      if (t >= a.np * h) break;
      const int m = fdiv(t, a.mag_np, a.np), q = t - m * a.np;
      const int mr = h - m;
      C A = {0, 0}, Bc = {0, 0};
      if (oka[i]) A = C{sa[i] * va[i].x, m == 0 ? (T)0 : sa[i] * va[i].y};
      if (okb[i]) Bc = C{sb[i] * vb[i].x, mr == 0 ? (T)0 : -sb[i] * vb[i].y};  // conj(X_{h-m})
      // E' = X_m + conj X_{h-m},  O' = (X_m - conj X_{h-m}) e^{+2 pi i m / n},  Z' = E' + i O'
      const C E = addz(A, Bc);
      const C w = tw[m];
      const C O = cmulz(subz(A, Bc), C{w.x, -w.y});
      const C Zp = {E.x - O.y, E.y + O.x};
      buf0[q * h + m] = C{Zp.x, -Zp.y};  // conj(Z') for the inverse by a forward FFT
    }
  }
  __syncthreads();
  const C *r = fft_smem<T>(buf0, buf1, a);
  double2 *g2 = reinterpret_cast<double2 *>(grid);
  for (int t = threadIdx.x; t < a.np * h; t += blockDim.x) {
    const int q = fdiv(t, a.mag_h, h), k = t - q * h;
    const int c = c0 + q;
    if (c >= a.ncol) continue;
    const T s = out_scale[(c % 3) * a.nlat + j];
    const C v = r[t];  // conj of z_k = x_{2k} + i x_{2k+1}
    if constexpr (F32) {
      g2[((int64_t)c * a.nlat + j) * h + k] = make_double2(f32_to_f64(s * v.x), f32_to_f64(-s * v.y));
    } else {
      g2[((int64_t)c * a.nlat + j) * h + k] = make_double2(s * v.x, -s * v.y);
    }
  }
}

FftArgs make_args(const Plan &pl, int B) {
  FftArgs a;
  a.tw = pl.prm.precision == REXI_MIXED ? pl.fft.tw32_dev : pl.fft.tw_dev;
  a.n = pl.fft.n;
  a.h = pl.fft.n / 2;
  a.nstages = pl.fft.nstages;
  for (int s = 0; s < 24; ++s) a.radix[s] = pl.fft.radix[s];
  a.N = pl.N;
  a.nlat = pl.nlat;
  a.ncol = 3 * B;
  // rows per CTA: the plan's nsplit (its shared memory holds that many), spread evenly
  // over the fewest CTAs a latitude needs, so that a small batch does not transform rows
  // of zeros (one state at T63: 3 rows, not 21)
  {
    const int nblk = (a.ncol + pl.fft.nsplit - 1) / pl.fft.nsplit;
    a.np = (a.ncol + nblk - 1) / nblk;
  }
  {
    int Ns = 1;
    for (int s = 0; s < a.nstages; ++s) {
      a.mag_nb[s] = div_magic(a.h / a.radix[s]);
      a.mag_ns[s] = div_magic(Ns);
      Ns *= a.radix[s];
    }
    a.mag_h = div_magic(a.h);
    a.mag_np = div_magic(a.np);
  }
  a.c3 = std::cos(2.0 * M_PI / 3.0);
  a.s3 = std::sin(2.0 * M_PI / 3.0);
  a.c5a = std::cos(2.0 * M_PI / 5.0);
  a.s5a = std::sin(2.0 * M_PI / 5.0);
  a.c5b = std::cos(4.0 * M_PI / 5.0);
  a.s5b = std::sin(4.0 * M_PI / 5.0);
  return a;
}

}  // namespace

// Factor n into radices 8, 4, 2, 3, 5 (largest powers of two first); false if another
// prime divides n.
bool fft_factor(int n, int *radix, int *nstages) {
  int k = 0, m = n;
  while (m % 8 == 0) { radix[k++] = 8; m /= 8; }
  while (m % 4 == 0) { radix[k++] = 4; m /= 4; }
  while (m % 2 == 0) { radix[k++] = 2; m /= 2; }
  while (m % 3 == 0) { radix[k++] = 3; m /= 3; }
  while (m % 5 == 0) { radix[k++] = 5; m /= 5; }
  *nstages = k;
  return m == 1 && k < 24;
}

bool fft32(const Plan &pl) { return pl.prm.precision == REXI_MIXED; }
size_t fft_smem_bytes(const Plan &pl) {
  return (size_t)pl.fft.nsplit * pl.fft.n * (fft32(pl) ? sizeof(float2) : sizeof(double2));
}

cudaError_t launch_fft_fwd(Plan &pl, const double *grid, double2 *four, int B, const void *in_scale,
                           const void *m_scale, cudaStream_t st) {
  FftArgs a = make_args(pl, B);
  dim3 g((unsigned)((a.ncol + a.np - 1) / a.np), (unsigned)pl.nlat);
  size_t sm = fft_smem_bytes(pl);
  if (fft32(pl))
    fft_fwd_kernel<float><<<g, 256, sm, st>>>(a, grid, four, static_cast<const float *>(in_scale),
                                              static_cast<const float *>(m_scale));
  else
    fft_fwd_kernel<double><<<g, 256, sm, st>>>(a, grid, four, static_cast<const double *>(in_scale),
                                               static_cast<const double *>(m_scale));
  return cudaGetLastError();
}

cudaError_t launch_fft_inv(Plan &pl, const double2 *four, double *grid, int B, const void *m_scale,
                           const void *out_scale, cudaStream_t st) {
  FftArgs a = make_args(pl, B);
  dim3 g((unsigned)((a.ncol + a.np - 1) / a.np), (unsigned)pl.nlat);
  size_t sm = fft_smem_bytes(pl);
  if (fft32(pl))
    fft_inv_kernel<float><<<g, 256, sm, st>>>(a, four, grid, static_cast<const float *>(m_scale),
                                              static_cast<const float *>(out_scale));
  else
    fft_inv_kernel<double><<<g, 256, sm, st>>>(a, four, grid, static_cast<const double *>(m_scale),
                                               static_cast<const double *>(out_scale));
  return cudaGetLastError();
}

cudaError_t fft_configure(Plan &pl) {
  const int bytes = (int)fft_smem_bytes(pl);
  cudaError_t e;
  if (fft32(pl)) {
    if ((e = cudaFuncSetAttribute(fft_fwd_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
    return cudaFuncSetAttribute(fft_inv_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  }
  if ((e = cudaFuncSetAttribute(fft_fwd_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes))) return e;
  return cudaFuncSetAttribute(fft_inv_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
}

}  // namespace rexi
