// Mixed-precision forward of Eq. (3): placeholder until the tensor-core kernels land.
#include "sse_internal.h"

namespace sse {
size_t mixed_fwd_workspace(const sse_dims&, int) { return 0; }
cudaError_t mixed_fwd(const Problem&, int, double2*, double2*, unsigned*, void*, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace sse
