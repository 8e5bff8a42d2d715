// FP64 adjoint of Eq. (3): placeholder until the adjoint kernels land.
#include "sse_internal.h"

namespace sse {
size_t fp64_bwd_workspace(const sse_dims&) { return 0; }
cudaError_t fp64_bwd(const Problem&, const double2*, const double2*, double2*, double2*, double2*, unsigned*, void*,
                     size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace sse
