// Internal declarations shared by the translation units of libsse (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sse.h"

namespace sse {

// Bits of the device status word (first word of the workspace).
enum : unsigned {
    DEV_BAD_NEIGHBOUR = 1u,  // nbr[a][s] outside [0, NA): that bond contributed zero
    DEV_TIMEOUT = 2u,        // a bounded mbarrier / flag wait gave up
    DEV_NOT_ANTIHERMITIAN = 4u,  // SSE_FLAG_ANTIHERMITIAN with CHECK: an input block is not anti-Hermitian
};

// Device views of the inputs of Eq. (3). Complex tensors are double2 (re, im).
struct Problem {
    sse_dims d;
    const int32_t* nbr;
    const double2* dH;
    const double2* D[2];  // [0] = D^<, [1] = D^>
    const double2* G[2];  // [0] = G^<, [1] = G^>
    double scale;
    uint32_t flags;
};

// Kernel timing (SSE_FLAG_PROFILE, sse_profile.cu): while a ProfScope(true) is alive on this
// thread, prof_begin/prof_end record a CUDA event pair on the launching stream around a kernel.
class ProfScope {
  public:
    explicit ProfScope(bool on);
    ~ProfScope();

  private:
    bool prev_;
};
void prof_begin(const char* name, cudaStream_t st);
void prof_end(cudaStream_t st);
#define SSE_TIMED(name, st, ...)     \
    do {                              \
        ::sse::prof_begin(name, st);  \
        __VA_ARGS__;                  \
        ::sse::prof_end(st);          \
    } while (0)

// Argument checks shared by sse_sigma_fwd, sse_sigma_bwd and sse_sigma_bwd_static (sse_abi.cu): sizes, mode,
// flags, scale and the input pointers. SSE_ERR_INVALID_ARG for invalid values, SSE_ERR_UNSUPPORTED for valid sizes
// the kernels are not built for, SSE_OK otherwise. Host only.
int abi_common_checks(const sse_dims* d, const int32_t* nbr, const double* dH, const double* Dl, const double* Dg,
                      const double* Gl, const double* Gg, double scale, int mode, uint32_t flags);

// Workspace layout: [0, 256) status word + padding; the rest per mode.
constexpr size_t kStatusBytes = 256;

// FP64 forward (sse_fp64.cu).
size_t fp64_fwd_workspace(const sse_dims& d);
cudaError_t fp64_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                     size_t ws_bytes, cudaStream_t st);

// FP64 adjoint (sse_fp64_bwd.cu).
size_t fp64_bwd_workspace(const sse_dims& d);
cudaError_t fp64_bwd(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                     double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                     cudaStream_t st);

// Mixed-precision forward (sse_mixed.cu).
size_t mixed_fwd_workspace(const sse_dims& d, int mode);
bool mixed_supported(const sse_dims& d, int mode);  // host-only limits: Norb, shared memory, grid
cudaError_t mixed_fwd(const Problem& p, int mode, double2* S_less, double2* S_greater, unsigned* status,
                      void* ws, size_t ws_bytes, cudaStream_t st);

// Transform-based forward (sse_spectral_fwd.cu): FFT length along E, size limits, workspace.
int spectral_length(const sse_dims& d);
bool spectral_supported(const sse_dims& d);
// The forward's limits for FP64 (fp32 = false) or FP32 (true) transforms and block products; like every
// *_supported predicate below, a host-only function of the sizes that the entry points test before any device work.
bool spectral_fwd_supported(const sse_dims& d, bool fp32);
size_t spectral_fwd_workspace(const sse_dims& d);
cudaError_t spectral_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                         size_t ws_bytes, cudaStream_t st);
// Stream-ordered hand-offs between the copies of the host-buffer entry point and the transform forward, per kz
// slice: the forward waits for `inputs` (nbr, dH, D^<, D^>) before the lag-kernel transforms and for g[t][k]
// before transforming slice k of G^t, and records s[t][k] once slice k of Sigma^t is written.
struct FwdPipe {
    cudaEvent_t inputs;
    const cudaEvent_t* g[2];  // [Nkz] each
    const cudaEvent_t* s[2];  // [Nkz] each
};
cudaError_t spectral_fwd_pipelined(const Problem& p, int mode, double2* S_less, double2* S_greater, unsigned* status,
                                   void* ws, size_t ws_bytes, cudaStream_t st, const FwdPipe& pipe);
// FP32 transforms and block products (mode FP32_FFT), FP64 inputs and outputs.
size_t spectral_fwd32_workspace(const sse_dims& d);
cudaError_t spectral_fwd32(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                           size_t ws_bytes, cudaStream_t st);

// FP32 transforms with the block products on the tcgen05 tensor cores (mode F16X3_FFT, sse_spectral_tc.cu); the
// workspace is FP32_FFT's.
bool spectral_fwd_tc_supported(const sse_dims& d);
cudaError_t spectral_fwd_tc(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                            size_t ws_bytes, cudaStream_t st);

// Transform-based adjoint of Eq. (3), FP64 and FP32 (sse_spectral_adj.cu).
size_t spectral_bwd_workspace(const sse_dims& d);
bool spectral_bwd_supported(const sse_dims& d);
cudaError_t spectral_bwd(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                         double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                         cudaStream_t st);

// The same adjoint with FP32 transforms and products (mode FP32_FFT), FP64 final sums and outputs.
size_t spectral_bwd32_workspace(const sse_dims& d);
cudaError_t spectral_bwd32(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                           double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                           cudaStream_t st);

// Gradient with respect to G, transform-based: FP64 (spectral_bwd_g) or FP32 transforms and products with FP64
// inputs and outputs (spectral_bwd_g32) (sse_spectral_adj.cu).
size_t spectral_bwd_g_workspace(const sse_dims& d);
bool spectral_bwd_g_supported(const sse_dims& d, bool fp32);
cudaError_t spectral_bwd_g(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_G_less,
                           double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st);
size_t spectral_bwd_g32_workspace(const sse_dims& d);
cudaError_t spectral_bwd_g32(const Problem& p, const double2* gS_less, const double2* gS_greater,
                             double2* g_G_less, double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes,
                             cudaStream_t st);

// Phonon self-energy of Eq. (4), transform-based: FP64 (spectral_pi) or FP32 transforms and products with FP64
// inputs and outputs (spectral_pi32) (sse_spectral_pi.cu).
size_t spectral_pi_workspace(const sse_dims& d);
bool spectral_pi_supported(const sse_dims& d);
cudaError_t spectral_pi(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                        const double2* G_greater, double scale, uint32_t flags, double2* P_less, double2* P_greater,
                        unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st);
size_t spectral_pi32_workspace(const sse_dims& d);
cudaError_t spectral_pi32(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                          const double2* G_greater, double scale, uint32_t flags, double2* P_less,
                          double2* P_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st);

// Bond weights D_ba - D_bb - D_aa + D_ab from raw phonon Green's functions (sse_dcomb.cu).
cudaError_t dcomb_fwd(const sse_dims& d, const int32_t* nbr, const double2* raw_l, const double2* raw_g,
                      double2* Dl, double2* Dg, unsigned* status, cudaStream_t st);
cudaError_t dcomb_bwd(const sse_dims& d, const int32_t* nbr, const double2* g_l, const double2* g_g, double2* r_l,
                      double2* r_g, unsigned* status, cudaStream_t st);

}  // namespace sse
