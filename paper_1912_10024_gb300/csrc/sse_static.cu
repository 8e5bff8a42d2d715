// sse_sigma_bwd_static: the FP64 adjoint without a caller-provided workspace.
//
// Some callers cannot call cudaMalloc: code that runs inside a host
// application whose device memory is owned by its own allocator or pool (the
// caller may only hand out buffers it already has), code that must not
// allocate on its hot path (an allocation can synchronise the device or fail
// under memory pressure), and foreign-language hosts that only pass through
// pointers they were given. For them this entry point takes the same inputs
// and outputs as sse_sigma_bwd but keeps its scratch -- the device status
// word and the per-(atom, slot, kz, type) partial gradients of dH -- in one
// file-scope static device array of SSE_STATIC_SCRATCH_BYTES. Every GPU that
// loads the library holds that array until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse.h"
#include "sse_internal.h"

namespace {

static __device__ __align__(256) unsigned char g_scratch[SSE_STATIC_SCRATCH_BYTES];

// Device address of g_scratch on the current device. In host code `g_scratch` names a host-side stand-in,
// never the device memory, so the address must come from cudaGetSymbolAddress with the device current. It is
// looked up on every call (a host-side query that allocates nothing): an address cached across calls would go
// stale if the process reset the device or re-created its primary context, which reloads the library's device
// code at another address.
cudaError_t scratch_on_current_device(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" int sse_sigma_bwd_static(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                                    const double* D_greater, const double* G_less, const double* G_greater,
                                    double scale, int mode, uint32_t flags, const double* gS_less,
                                    const double* gS_greater, double* g_dH, double* g_D_less, double* g_D_greater,
                                    void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    // The checks of sse_sigma_bwd and the same status codes, all before anything touches the device: invalid
    // arguments give SSE_ERR_INVALID_ARG; valid modes other than FP64 and valid sizes the kernels are not built for
    // give SSE_ERR_UNSUPPORTED; problems whose scratch exceeds the static array give SSE_ERR_WORKSPACE.
    const int rc = sse::abi_common_checks(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, mode, flags);
    if (rc != SSE_OK) return rc;
    if (!gS_less || !gS_greater || !g_dH || !g_D_less || !g_D_greater) return SSE_ERR_INVALID_ARG;
    if (!aligned(gS_less, 16) || !aligned(gS_greater, 16) || !aligned(g_dH, 16) || !aligned(g_D_less, 16) ||
        !aligned(g_D_greater, 16))
        return SSE_ERR_INVALID_ARG;
    if (mode != SSE_MODE_FP64) return SSE_ERR_UNSUPPORTED;
    const size_t need = sse_workspace_bytes(d, SSE_MODE_FP64, flags);  // nonzero: the checks above passed
    if (need == 0) return SSE_ERR_UNSUPPORTED;
    if (need > SSE_STATIC_SCRATCH_BYTES) return SSE_ERR_WORKSPACE;  // problem too large for the array
    if (d->a_begin == d->a_end) return SSE_OK;

    void* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return SSE_ERR_CUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(scratch);
    // the status word must start at zero; the partial gradients are fully overwritten
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    sse::Problem p;
    p.d = *d;
    p.nbr = nbr;
    p.dH = reinterpret_cast<const double2*>(dH);
    p.D[0] = reinterpret_cast<const double2*>(D_less);
    p.D[1] = reinterpret_cast<const double2*>(D_greater);
    p.G[0] = reinterpret_cast<const double2*>(G_less);
    p.G[1] = reinterpret_cast<const double2*>(G_greater);
    p.scale = scale;
    p.flags = flags;
    void* ws = static_cast<char*>(scratch) + sse::kStatusBytes;
    const cudaError_t e = sse::fp64_bwd(p, reinterpret_cast<const double2*>(gS_less),
                                        reinterpret_cast<const double2*>(gS_greater), reinterpret_cast<double2*>(g_dH),
                                        reinterpret_cast<double2*>(g_D_less), reinterpret_cast<double2*>(g_D_greater),
                                        status, ws, SSE_STATIC_SCRATCH_BYTES - sse::kStatusBytes, st);
    if (e == cudaErrorNotSupported) return SSE_ERR_UNSUPPORTED;
    if (e != cudaSuccess) return SSE_ERR_CUDA;
    if (!(flags & SSE_FLAG_CHECK)) return SSE_OK;
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SSE_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SSE_ERR_CUDA;
    if (h & sse::DEV_TIMEOUT) return SSE_ERR_TIMEOUT;
    if (h & sse::DEV_BAD_NEIGHBOUR) return SSE_ERR_DEVICE_CHECK;
    return SSE_OK;
}
