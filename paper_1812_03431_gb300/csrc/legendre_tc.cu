// Mixed-precision Legendre transforms on the tcgen05 tensor cores (3xTF32 split
// products, FP32 accumulation).  Until these kernels are built, plans with
// REXI_MIXED are rejected at creation.
#include <cuda_runtime.h>

#include "rexi_internal.h"

namespace rexi {

cudaError_t launch_leg_ana_tc(Plan &, const double2 *, double2 *, int, const double *, cudaStream_t) {
  return cudaErrorNotSupported;
}
cudaError_t launch_leg_syn_tc(Plan &, const double2 *, double2 *, int, const double *, cudaStream_t) {
  return cudaErrorNotSupported;
}

}  // namespace rexi
