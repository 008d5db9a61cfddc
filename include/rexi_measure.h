/*
 * rexi_measure.h -- measurement helpers of librexi (no counterpart in the paper).
 *
 * The banded solves of rexi_step (include/rexi.h) are bound by the GPU's binary64
 * fused multiply-add rate.  That rate is not among the figures a program can read
 * from the device, so the roofline of the solve divides by a measured one.
 */
#ifndef REXI_MEASURE_H
#define REXI_MEASURE_H

#include <stdint.h>

#include "rexi.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Measured binary64 FMA rate of the current device, in TFLOP/s (2 flops per FMA).
 * Times kernels of independent FMA chains (operands in registers) in six shapes --
 * 4 to 16 chains per thread, 8 to 32 warps per SM, ~24 G FMAs per launch, about
 * 40 ms each on GB300 -- each once untimed and then `reps` times on `stream` (a
 * cudaStream_t, NULL = legacy default stream) with CUDA events; writes the rate of
 * the fastest launch to *tflops and its milliseconds to *ms_best (may be NULL).  Allocates and frees a few KB of device
 * memory and synchronises the stream.  REXI_EINVAL for reps < 1 or a NULL
 * tflops, REXI_ECUDA if a CUDA call fails. */
rexi_status rexi_measure_fp64_fma(int32_t reps, double *tflops, double *ms_best, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* REXI_MEASURE_H */
