// Measured FP64 fused multiply-add rate of the current GPU: the denominator of the
// banded solve's roofline (the solve is bound by its FP64 FMAs; the device's FP64 rate
// is not among the vendor figures this library can read at run time).
//
// Every thread runs C independent FMA recurrences x <- x a + b for `iters` iterations,
// with a and b in registers (per-thread values, so that no operand comes from the
// constant bank).  A few shapes are timed -- chains per thread and warps per SM -- and
// the fastest counts: a shape with too few independent FMAs per scheduler is latency
// bound, one with too many may lose issue slots to register-bank conflicts, and which
// is which is measured rather than assumed.  The recurrence contracts towards
// b / (1 - a), so no value overflows, and the results are folded into one store that
// the compiler cannot drop.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "../../include/rexi_measure.h"
#include "rexi_internal.h"

namespace rexi {
namespace {

template <int C>
__global__ void __launch_bounds__(256) fp64_fma_kernel(double *sink, double a0, double b0, int iters) {
  const double a = a0 - 1e-12 * (threadIdx.x & 7), b = b0 + 1e-12 * (threadIdx.x & 3);
  double x[C];
#pragma unroll
  for (int c = 0; c < C; ++c) x[c] = 1e-3 * (threadIdx.x + 1) + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < C; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < C; ++c) s += x[c];
  if (s == -1.0) sink[blockIdx.x] = s;  // never true for these a, b; keeps the chains live
}

}  // namespace
}  // namespace rexi

extern "C" rexi_status rexi_measure_fp64_fma(int32_t reps, double *tflops, double *ms_best, void *stream) {
  using namespace rexi;
  if (reps < 1 || !tflops) {
    set_error("rexi_measure_fp64_fma: need reps >= 1 and an output pointer");
    return REXI_EINVAL;
  }
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    set_error(std::string("rexi_measure_fp64_fma: ") + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int threads = 256;
  // (chains per thread, CTAs of 8 warps per SM): 8-64 independent FMAs per scheduler
  const int shapes[][2] = {{4, 1}, {8, 1}, {4, 2}, {8, 2}, {16, 2}, {8, 4}};
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  double *sink = nullptr;
  e = cudaMalloc(&sink, (size_t)sms * 4 * sizeof(double));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double best_rate = 0.0, best_ms = 0.0;
  for (const auto &sh : shapes) {
    const int C = sh[0], blocks = sms * sh[1];
    const int iters = (int)(2.4e10 / ((double)blocks * threads * C));  // ~24 G FMA: ~40 ms per launch
    // one untimed launch (clocks ramp up), then the best of `reps`
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
      e = cudaEventRecord(e0, st);
      if (e == cudaSuccess) {
        if (C == 4) fp64_fma_kernel<4><<<blocks, threads, 0, st>>>(sink, 0.999999, 1e-6, iters);
        else if (C == 8) fp64_fma_kernel<8><<<blocks, threads, 0, st>>>(sink, 0.999999, 1e-6, iters);
        else fp64_fma_kernel<16><<<blocks, threads, 0, st>>>(sink, 0.999999, 1e-6, iters);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      const double rate = 2.0 * (double)blocks * threads * iters * C / (ms * 1e-3) / 1e12;
      if (e == cudaSuccess && r > 0 && rate > best_rate) {
        best_rate = rate;
        best_ms = ms;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    set_error(std::string("rexi_measure_fp64_fma: ") + cudaGetErrorString(e));
    return REXI_ECUDA;
  }
  *tflops = best_rate;
  if (ms_best) *ms_best = best_ms;
  return REXI_OK;
}
