// C ABI entry points of libsse: host-side validation, workspace bookkeeping,
// dispatch to the kernels and status reporting. Declarations and contracts
// are in include/sse.h.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <vector>

#include "sse.h"
#include "sse_internal.h"

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

bool valid_dims(const sse_dims* d) {
    if (!d) return false;
    if (d->NA < 1 || d->NB < 1 || d->Norb < 1 || d->NE < 1 || d->Nkz < 1 || d->Nqz < 1 || d->Nw < 1) return false;
    if (d->Nqz > d->Nkz || d->Nw >= d->NE) return false;
    if (d->a_begin < 0 || d->a_end > d->NA || d->a_begin > d->a_end) return false;
    return true;
}

// Sizes that are valid but outside what the kernels are built for.
bool supported_dims(const sse_dims* d) {
    if (d->Norb > 16 || d->NA > 32767 || d->Nkz > 65535) return false;
    // element counts of the largest tensors must fit comfortably in 63 bits
    const double g = (double)d->Nkz * d->NE * d->NA * d->Norb * d->Norb;
    const double dd = (double)d->Nqz * d->Nw * d->NA * d->NB * 9.0;
    return g < 4e18 && dd < 4e18;
}

bool valid_mode(int mode) {
    return mode == SSE_MODE_FP64 || mode == SSE_MODE_TF32 || mode == SSE_MODE_BF16X3 || mode == SSE_MODE_FP64_FFT ||
           mode == SSE_MODE_FP32_FFT || mode == SSE_MODE_F16X3_FFT;
}
bool fp64_mode(int mode) { return mode == SSE_MODE_FP64 || mode == SSE_MODE_FP64_FFT; }

// The kernels' own limits for these sizes in this mode (transform length, kz DFT size, shared memory of the
// configurations, Norb of the tensor-core epilogue): host-only functions of the sizes, tested before any device
// work. The direct FP64 kernels choose configurations that fit; their drivers keep their own checks.
enum class Op { Fwd, Bwd, BwdG, Pi };
bool op_supported(const sse_dims& d, int mode, Op op) {
    const bool fp32 = mode == SSE_MODE_FP32_FFT;
    switch (op) {
        case Op::Fwd:
            if (mode == SSE_MODE_TF32 || mode == SSE_MODE_BF16X3) return sse::mixed_supported(d, mode);
            if (mode == SSE_MODE_F16X3_FFT) return sse::spectral_fwd_tc_supported(d);
            return mode == SSE_MODE_FP64 || sse::spectral_fwd_supported(d, fp32);
        case Op::Bwd: return mode == SSE_MODE_FP64 || sse::spectral_bwd_supported(d);
        case Op::BwdG: return sse::spectral_bwd_g_supported(d, fp32);  // transforms in every mode it takes
        case Op::Pi: return sse::spectral_pi_supported(d);              // limits of the FP64 and FP32 kernels
    }
    return false;
}
bool valid_flags(uint32_t f) {
    return (f & ~(uint32_t)(SSE_FLAG_SYMMETRIZE | SSE_FLAG_CHECK | SSE_FLAG_PROFILE | SSE_FLAG_ANTIHERMITIAN)) == 0;
}

size_t fwd_ws(const sse_dims& d, int mode) {
    if (mode == SSE_MODE_FP64) return sse::fp64_fwd_workspace(d);
    if (mode == SSE_MODE_FP64_FFT) return sse::spectral_fwd_workspace(d);
    if (mode == SSE_MODE_FP32_FFT || mode == SSE_MODE_F16X3_FFT) return sse::spectral_fwd32_workspace(d);
    return sse::mixed_fwd_workspace(d, mode);
}

int finish(cudaError_t launch, unsigned* status, uint32_t flags, cudaStream_t st) {
    if (launch != cudaSuccess) return SSE_ERR_CUDA;
    if (!(flags & SSE_FLAG_CHECK)) return SSE_OK;
    unsigned h = 0;
    if (cudaMemcpyAsync(&h, status, sizeof h, cudaMemcpyDeviceToHost, st) != cudaSuccess) return SSE_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return SSE_ERR_CUDA;
    if (h & sse::DEV_TIMEOUT) return SSE_ERR_TIMEOUT;
    if (h & (sse::DEV_BAD_NEIGHBOUR | sse::DEV_NOT_ANTIHERMITIAN)) return SSE_ERR_DEVICE_CHECK;
    return SSE_OK;
}

}  // namespace

namespace sse {
int abi_common_checks(const sse_dims* d, const int32_t* nbr, const double* dH, const double* Dl, const double* Dg,
                      const double* Gl, const double* Gg, double scale, int mode, uint32_t flags) {
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags)) return SSE_ERR_INVALID_ARG;
    if (!isfinite(scale)) return SSE_ERR_INVALID_ARG;
    if (!nbr || !dH || !Dl || !Dg || !Gl || !Gg) return SSE_ERR_INVALID_ARG;
    if (!aligned(nbr, 4) || !aligned(dH, 16) || !aligned(Dl, 16) || !aligned(Dg, 16) || !aligned(Gl, 16) ||
        !aligned(Gg, 16))
        return SSE_ERR_INVALID_ARG;
    if (!supported_dims(d)) return SSE_ERR_UNSUPPORTED;
    return SSE_OK;
}
}  // namespace sse

namespace {
using sse::abi_common_checks;

sse::Problem make_problem(const sse_dims* d, const int32_t* nbr, const double* dH, const double* Dl,
                          const double* Dg, const double* Gl, const double* Gg, double scale, uint32_t flags) {
    sse::Problem p;
    p.d = *d;
    p.nbr = nbr;
    p.dH = reinterpret_cast<const double2*>(dH);
    p.D[0] = reinterpret_cast<const double2*>(Dl);
    p.D[1] = reinterpret_cast<const double2*>(Dg);
    p.G[0] = reinterpret_cast<const double2*>(Gl);
    p.G[1] = reinterpret_cast<const double2*>(Gg);
    p.scale = scale;
    p.flags = flags;
    return p;
}

}  // namespace

extern "C" const char* sse_strerror(int status) {
    switch (status) {
        case SSE_OK: return "success";
        case SSE_ERR_INVALID_ARG: return "invalid argument (null or misaligned pointer, bad size or range)";
        case SSE_ERR_UNSUPPORTED: return "unsupported mode, flag or problem size";
        case SSE_ERR_CUDA: return "a CUDA runtime call or kernel launch failed";
        case SSE_ERR_TIMEOUT: return "a bounded device-side wait gave up";
        case SSE_ERR_DEVICE_CHECK: return "device-side input check failed (neighbour index out of range)";
        case SSE_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        default: return "unknown status";
    }
}

extern "C" size_t sse_workspace_bytes(const sse_dims* d, int mode, uint32_t flags) {
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !supported_dims(d)) return 0;
    size_t f = fwd_ws(*d, mode);
    size_t b = mode == SSE_MODE_FP64       ? sse::fp64_bwd_workspace(*d)
               : mode == SSE_MODE_FP64_FFT ? sse::spectral_bwd_workspace(*d)
               : mode == SSE_MODE_FP32_FFT ? sse::spectral_bwd32_workspace(*d)
                                           : 0;
    return sse::kStatusBytes + (f > b ? f : b);
}

extern "C" int sse_sigma_fwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                             const double* D_greater, const double* G_less, const double* G_greater, double scale,
                             int mode, uint32_t flags, double* S_less, double* S_greater, void* workspace,
                             size_t ws_bytes, void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    int rc = abi_common_checks(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, mode, flags);
    if (rc != SSE_OK) return rc;
    if (!S_less || !S_greater || !aligned(S_less, 16) || !aligned(S_greater, 16)) return SSE_ERR_INVALID_ARG;
    if (!op_supported(*d, mode, Op::Fwd)) return SSE_ERR_UNSUPPORTED;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < sse::kStatusBytes + fwd_ws(*d, mode))
        return SSE_ERR_WORKSPACE;
    if (d->a_begin == d->a_end) return SSE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    void* ws = static_cast<char*>(workspace) + sse::kStatusBytes;
    const size_t wsb = ws_bytes - sse::kStatusBytes;
    const sse::Problem p = make_problem(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, flags);
    double2* Sl = reinterpret_cast<double2*>(S_less);
    double2* Sg = reinterpret_cast<double2*>(S_greater);
    cudaError_t e = mode == SSE_MODE_FP64       ? sse::fp64_fwd(p, Sl, Sg, status, ws, wsb, st)
                    : mode == SSE_MODE_FP64_FFT ? sse::spectral_fwd(p, Sl, Sg, status, ws, wsb, st)
                    : mode == SSE_MODE_FP32_FFT ? sse::spectral_fwd32(p, Sl, Sg, status, ws, wsb, st)
                    : mode == SSE_MODE_F16X3_FFT ? sse::spectral_fwd_tc(p, Sl, Sg, status, ws, wsb, st)
                                                : sse::mixed_fwd(p, mode, Sl, Sg, status, ws, wsb, st);
    if (e == cudaErrorNotSupported) return SSE_ERR_UNSUPPORTED;
    return finish(e, status, flags, st);
}

extern "C" int sse_sigma_bwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                             const double* D_greater, const double* G_less, const double* G_greater, double scale,
                             int mode, uint32_t flags, const double* gS_less, const double* gS_greater,
                             double* g_dH, double* g_D_less, double* g_D_greater, void* workspace, size_t ws_bytes,
                             void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    int rc = abi_common_checks(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, mode, flags);
    if (rc != SSE_OK) return rc;
    if (!gS_less || !gS_greater || !g_dH || !g_D_less || !g_D_greater) return SSE_ERR_INVALID_ARG;
    if (!aligned(gS_less, 16) || !aligned(gS_greater, 16) || !aligned(g_dH, 16) || !aligned(g_D_less, 16) ||
        !aligned(g_D_greater, 16))
        return SSE_ERR_INVALID_ARG;
    if (!fp64_mode(mode) && mode != SSE_MODE_FP32_FFT) return SSE_ERR_UNSUPPORTED;
    if (!op_supported(*d, mode, Op::Bwd)) return SSE_ERR_UNSUPPORTED;
    const size_t need = mode == SSE_MODE_FP64       ? sse::fp64_bwd_workspace(*d)
                        : mode == SSE_MODE_FP64_FFT ? sse::spectral_bwd_workspace(*d)
                                                    : sse::spectral_bwd32_workspace(*d);
    if (!workspace || !aligned(workspace, 256) || ws_bytes < sse::kStatusBytes + need) return SSE_ERR_WORKSPACE;
    if (d->a_begin == d->a_end) return SSE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    void* ws = static_cast<char*>(workspace) + sse::kStatusBytes;
    const size_t wsb = ws_bytes - sse::kStatusBytes;
    const sse::Problem p = make_problem(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, flags);
    const double2* gl = reinterpret_cast<const double2*>(gS_less);
    const double2* gg = reinterpret_cast<const double2*>(gS_greater);
    double2* gh = reinterpret_cast<double2*>(g_dH);
    double2* gdl = reinterpret_cast<double2*>(g_D_less);
    double2* gdg = reinterpret_cast<double2*>(g_D_greater);
    cudaError_t e = mode == SSE_MODE_FP64       ? sse::fp64_bwd(p, gl, gg, gh, gdl, gdg, status, ws, wsb, st)
                    : mode == SSE_MODE_FP64_FFT ? sse::spectral_bwd(p, gl, gg, gh, gdl, gdg, status, ws, wsb, st)
                                                : sse::spectral_bwd32(p, gl, gg, gh, gdl, gdg, status, ws, wsb, st);
    if (e == cudaErrorNotSupported) return SSE_ERR_UNSUPPORTED;
    return finish(e, status, flags, st);
}

namespace {
int dcomb_common(const sse_dims* d, const int32_t* nbr, const double* in_l, const double* in_g, double* out_l,
                 double* out_g, uint32_t flags, void* workspace, size_t ws_bytes) {
    if (!valid_dims(d) || !valid_flags(flags)) return SSE_ERR_INVALID_ARG;
    if (!nbr || !in_l || !in_g || !out_l || !out_g) return SSE_ERR_INVALID_ARG;
    if (!aligned(nbr, 4) || !aligned(in_l, 16) || !aligned(in_g, 16) || !aligned(out_l, 16) || !aligned(out_g, 16))
        return SSE_ERR_INVALID_ARG;
    if (!supported_dims(d)) return SSE_ERR_UNSUPPORTED;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < sse::kStatusBytes) return SSE_ERR_WORKSPACE;
    return SSE_OK;
}
}  // namespace

extern "C" int sse_dcomb_fwd(const sse_dims* d, const int32_t* nbr, const double* Draw_less,
                             const double* Draw_greater, double* D_less, double* D_greater, uint32_t flags,
                             void* workspace, size_t ws_bytes, void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    int rc = dcomb_common(d, nbr, Draw_less, Draw_greater, D_less, D_greater, flags, workspace, ws_bytes);
    if (rc != SSE_OK || d->a_begin == d->a_end) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    cudaError_t e = sse::dcomb_fwd(*d, nbr, reinterpret_cast<const double2*>(Draw_less),
                                   reinterpret_cast<const double2*>(Draw_greater), reinterpret_cast<double2*>(D_less),
                                   reinterpret_cast<double2*>(D_greater), status, st);
    return finish(e, status, flags, st);
}

extern "C" int sse_dcomb_bwd(const sse_dims* d, const int32_t* nbr, const double* gD_less, const double* gD_greater,
                             double* gDraw_less, double* gDraw_greater, uint32_t flags, void* workspace,
                             size_t ws_bytes, void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    int rc = dcomb_common(d, nbr, gD_less, gD_greater, gDraw_less, gDraw_greater, flags, workspace, ws_bytes);
    if (rc != SSE_OK || d->a_begin == d->a_end) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    cudaError_t e = sse::dcomb_bwd(*d, nbr, reinterpret_cast<const double2*>(gD_less),
                                   reinterpret_cast<const double2*>(gD_greater), reinterpret_cast<double2*>(gDraw_less),
                                   reinterpret_cast<double2*>(gDraw_greater), status, st);
    return finish(e, status, flags, st);
}

namespace {
// FP64 and FP64_FFT: FP64 transforms; FP32_FFT: FP32 transforms and products.
size_t pi_workspace(const sse_dims& d, int mode) {
    return mode == SSE_MODE_FP32_FFT ? sse::spectral_pi32_workspace(d) : sse::spectral_pi_workspace(d);
}
}  // namespace

extern "C" size_t sse_pi_workspace_bytes(const sse_dims* d, int mode, uint32_t flags) {
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !supported_dims(d)) return 0;
    return sse::kStatusBytes + pi_workspace(*d, mode);
}

extern "C" int sse_pi_fwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* G_less,
                          const double* G_greater, double scale, int mode, uint32_t flags, double* P_less,
                          double* P_greater, void* workspace, size_t ws_bytes, void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !isfinite(scale)) return SSE_ERR_INVALID_ARG;
    if (!nbr || !dH || !G_less || !G_greater || !P_less || !P_greater) return SSE_ERR_INVALID_ARG;
    if (!aligned(nbr, 4) || !aligned(dH, 16) || !aligned(G_less, 16) || !aligned(G_greater, 16) ||
        !aligned(P_less, 16) || !aligned(P_greater, 16))
        return SSE_ERR_INVALID_ARG;
    if (!supported_dims(d) || !(fp64_mode(mode) || mode == SSE_MODE_FP32_FFT)) return SSE_ERR_UNSUPPORTED;
    if (!op_supported(*d, mode, Op::Pi)) return SSE_ERR_UNSUPPORTED;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < sse::kStatusBytes + pi_workspace(*d, mode))
        return SSE_ERR_WORKSPACE;
    if (d->a_begin == d->a_end) return SSE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    auto* run = mode == SSE_MODE_FP32_FFT ? sse::spectral_pi32 : sse::spectral_pi;
    cudaError_t e = run(*d, nbr, reinterpret_cast<const double2*>(dH), reinterpret_cast<const double2*>(G_less),
                        reinterpret_cast<const double2*>(G_greater), scale, flags, reinterpret_cast<double2*>(P_less),
                        reinterpret_cast<double2*>(P_greater), status,
                        static_cast<char*>(workspace) + sse::kStatusBytes, ws_bytes - sse::kStatusBytes, st);
    if (e == cudaErrorNotSupported) return SSE_ERR_UNSUPPORTED;
    return finish(e, status, flags, st);
}

namespace {
// FP64 and FP64_FFT: FP64 transforms; FP32_FFT: FP32 transforms and products.
size_t gradg_workspace(const sse_dims& d, int mode) {
    return mode == SSE_MODE_FP32_FFT ? sse::spectral_bwd_g32_workspace(d) : sse::spectral_bwd_g_workspace(d);
}
}  // namespace

extern "C" size_t sse_sigma_bwd_g_workspace_bytes(const sse_dims* d, int mode, uint32_t flags) {
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !supported_dims(d)) return 0;
    return sse::kStatusBytes + gradg_workspace(*d, mode);
}

extern "C" int sse_sigma_bwd_g(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                               const double* D_greater, double scale, int mode, uint32_t flags, const double* gS_less,
                               const double* gS_greater, double* g_G_less, double* g_G_greater, void* workspace,
                               size_t ws_bytes, void* stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !isfinite(scale)) return SSE_ERR_INVALID_ARG;
    if (!nbr || !dH || !D_less || !D_greater || !gS_less || !gS_greater || !g_G_less || !g_G_greater)
        return SSE_ERR_INVALID_ARG;
    if (!aligned(nbr, 4) || !aligned(dH, 16) || !aligned(D_less, 16) || !aligned(D_greater, 16) ||
        !aligned(gS_less, 16) || !aligned(gS_greater, 16) || !aligned(g_G_less, 16) || !aligned(g_G_greater, 16))
        return SSE_ERR_INVALID_ARG;
    if (!supported_dims(d) || !(fp64_mode(mode) || mode == SSE_MODE_FP32_FFT)) return SSE_ERR_UNSUPPORTED;
    if (!op_supported(*d, mode, Op::BwdG)) return SSE_ERR_UNSUPPORTED;
    if (!workspace || !aligned(workspace, 256) || ws_bytes < sse::kStatusBytes + gradg_workspace(*d, mode))
        return SSE_ERR_WORKSPACE;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned* status = static_cast<unsigned*>(workspace);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return SSE_ERR_CUDA;
    // G does not enter the gradient (Sigma is linear in G); the Problem's G pointers stay null
    const sse::Problem p = make_problem(d, nbr, dH, D_less, D_greater, nullptr, nullptr, scale, flags);
    auto* run = mode == SSE_MODE_FP32_FFT ? sse::spectral_bwd_g32 : sse::spectral_bwd_g;
    cudaError_t e = run(p, reinterpret_cast<const double2*>(gS_less), reinterpret_cast<const double2*>(gS_greater),
                        reinterpret_cast<double2*>(g_G_less), reinterpret_cast<double2*>(g_G_greater), status,
                        static_cast<char*>(workspace) + sse::kStatusBytes, ws_bytes - sse::kStatusBytes, st);
    if (e == cudaErrorNotSupported) return SSE_ERR_UNSUPPORTED;
    return finish(e, status, flags, st);
}

// ---------------------------------------------------------------------------
// Host-buffer forward: copies in, computes, copies back, overlapping the copies with the compute.
// ---------------------------------------------------------------------------
namespace {

struct HostLayout {
    size_t nbr, dH, D[2], G[2], S[2], status, ws, total;
};

size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

HostLayout host_layout(const sse_dims& d, int mode) {
    HostLayout l{};
    const size_t nel = (size_t)d.Norb * d.Norb;
    const size_t g = (size_t)d.Nkz * d.NE * d.NA * nel * 16;
    const size_t dd = (size_t)d.Nqz * d.Nw * d.NA * d.NB * 9 * 16;
    size_t o = 0;
    l.nbr = o;
    o = a256(o + (size_t)d.NA * d.NB * 4);
    l.dH = o;
    o = a256(o + (size_t)d.NA * d.NB * 3 * nel * 16);
    for (int t = 0; t < 2; ++t) l.D[t] = o, o = a256(o + dd);
    for (int t = 0; t < 2; ++t) l.G[t] = o, o = a256(o + g);
    for (int t = 0; t < 2; ++t) l.S[t] = o, o = a256(o + g);
    l.status = o;
    l.ws = o + sse::kStatusBytes;
    l.total = a256(l.ws + fwd_ws(d, mode));
    return l;
}

}  // namespace

extern "C" size_t sse_sigma_fwd_host_bytes(const sse_dims* d, int mode, uint32_t flags) {
    if (!valid_dims(d) || !valid_mode(mode) || !valid_flags(flags) || !supported_dims(d)) return 0;
    return host_layout(*d, mode).total;
}

extern "C" int sse_sigma_fwd_host(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                                  const double* D_greater, const double* G_less, const double* G_greater,
                                  double scale, int mode, uint32_t flags, double* S_less, double* S_greater,
                                  void* device_buf, size_t buf_bytes, void* stream, void* copy_stream) {
    sse::ProfScope prof_scope((flags & SSE_FLAG_PROFILE) != 0);
    int rc = abi_common_checks(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, mode, flags);
    if (rc != SSE_OK) return rc;
    if (!S_less || !S_greater || !aligned(S_less, 16) || !aligned(S_greater, 16)) return SSE_ERR_INVALID_ARG;
    if (!op_supported(*d, mode, Op::Fwd)) return SSE_ERR_UNSUPPORTED;
    const HostLayout L = host_layout(*d, mode);
    if (!device_buf || !aligned(device_buf, 256) || buf_bytes < L.total) return SSE_ERR_WORKSPACE;
    if (d->a_begin == d->a_end) return SSE_OK;
    cudaStream_t st = static_cast<cudaStream_t>(stream), cp = static_cast<cudaStream_t>(copy_stream);
    if (cp == st) return SSE_ERR_INVALID_ARG;  // the overlap needs a second stream
    char* base = static_cast<char*>(device_buf);
    const sse_dims& dd = *d;
    const size_t nel = (size_t)dd.Norb * dd.Norb;
    const size_t slice = (size_t)dd.NE * dd.NA * nel * 16;  // one kz slice of G or Sigma
    const size_t db = (size_t)dd.Nqz * dd.Nw * dd.NA * dd.NB * 9 * 16;
    // events: inputs, then per type and kz slice "G slice on the device" and "Sigma slice written", then "out"
    const int nk = dd.Nkz;
    std::vector<cudaEvent_t> ev((size_t)2 + 4 * nk, nullptr);
    auto cleanup = [&](int code) {
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);  // released once the recorded work completes
        return code;
    };
    for (auto& e : ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return cleanup(SSE_ERR_CUDA);
    cudaEvent_t ev_in = ev[0], ev_out = ev[1];
    cudaEvent_t* ev_g[2] = {ev.data() + 2, ev.data() + 2 + nk};
    cudaEvent_t* ev_s[2] = {ev.data() + 2 + 2 * nk, ev.data() + 2 + 3 * nk};
    unsigned* status = reinterpret_cast<unsigned*>(base + L.status);
    if (cudaMemsetAsync(status, 0, sizeof(unsigned), st) != cudaSuccess) return cleanup(SSE_ERR_CUDA);
    // inputs on the copy stream: the small tensors, then G^< and G^> one kz slice at a time
    if (cudaEventRecord(ev_out, st) != cudaSuccess || cudaStreamWaitEvent(cp, ev_out, 0) != cudaSuccess)
        return cleanup(SSE_ERR_CUDA);  // the device buffer is free once earlier work on `stream` is done
    bool ok_in = cudaMemcpyAsync(base + L.nbr, nbr, (size_t)dd.NA * dd.NB * 4, cudaMemcpyHostToDevice, cp) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(base + L.dH, dH, (size_t)dd.NA * dd.NB * 3 * nel * 16, cudaMemcpyHostToDevice, cp) ==
                     cudaSuccess &&
                 cudaMemcpyAsync(base + L.D[0], D_less, db, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                 cudaMemcpyAsync(base + L.D[1], D_greater, db, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                 cudaEventRecord(ev_in, cp) == cudaSuccess;
    const double* Gh[2] = {G_less, G_greater};
    for (int t = 0; t < 2 && ok_in; ++t)
        for (int k = 0; k < nk && ok_in; ++k)
            ok_in = cudaMemcpyAsync(base + L.G[t] + (size_t)k * slice, reinterpret_cast<const char*>(Gh[t]) + k * slice,
                                    slice, cudaMemcpyHostToDevice, cp) == cudaSuccess &&
                    cudaEventRecord(ev_g[t][k], cp) == cudaSuccess;
    if (!ok_in) return cleanup(SSE_ERR_CUDA);
    const sse::Problem p = make_problem(d, reinterpret_cast<const int32_t*>(base + L.nbr),
                                        reinterpret_cast<const double*>(base + L.dH),
                                        reinterpret_cast<const double*>(base + L.D[0]),
                                        reinterpret_cast<const double*>(base + L.D[1]),
                                        reinterpret_cast<const double*>(base + L.G[0]),
                                        reinterpret_cast<const double*>(base + L.G[1]), scale, flags);
    double2* Sd[2] = {reinterpret_cast<double2*>(base + L.S[0]), reinterpret_cast<double2*>(base + L.S[1])};
    void* ws = base + L.ws;
    const size_t wsb = L.total - L.ws;
    cudaError_t e;
    if (mode == SSE_MODE_FP64_FFT || mode == SSE_MODE_FP32_FFT || mode == SSE_MODE_F16X3_FFT) {
        const sse::FwdPipe pipe{ev_in, {ev_g[0], ev_g[1]}, {ev_s[0], ev_s[1]}};
        e = sse::spectral_fwd_pipelined(p, mode, Sd[0], Sd[1], status, ws, wsb, st, pipe);
    } else {  // one kernel sequence for both types: wait for every input, hand every slice over at the end
        if (cudaStreamWaitEvent(st, ev_g[1][nk - 1], 0) != cudaSuccess) return cleanup(SSE_ERR_CUDA);
        e = mode == SSE_MODE_FP64 ? sse::fp64_fwd(p, Sd[0], Sd[1], status, ws, wsb, st)
                                  : sse::mixed_fwd(p, mode, Sd[0], Sd[1], status, ws, wsb, st);
        for (int t = 0; t < 2 && e == cudaSuccess; ++t)
            for (int k = 0; k < nk && e == cudaSuccess; ++k) e = cudaEventRecord(ev_s[t][k], st);
    }
    if (e == cudaErrorNotSupported) return cleanup(SSE_ERR_UNSUPPORTED);
    if (e != cudaSuccess) return cleanup(SSE_ERR_CUDA);
    // results back on the copy stream, slice by slice as written, rows of the atom range only (pitched copies)
    const size_t pitch = (size_t)dd.NA * nel * 16, off = (size_t)dd.a_begin * nel * 16;
    const size_t width = (size_t)(dd.a_end - dd.a_begin) * nel * 16;
    double* Sh[2] = {S_less, S_greater};
    for (int t = 0; t < 2; ++t)
        for (int k = 0; k < nk; ++k)
            if (cudaStreamWaitEvent(cp, ev_s[t][k], 0) != cudaSuccess ||
                cudaMemcpy2DAsync(reinterpret_cast<char*>(Sh[t]) + k * slice + off, pitch,
                                  base + L.S[t] + k * slice + off, pitch, width, (size_t)dd.NE,
                                  cudaMemcpyDeviceToHost, cp) != cudaSuccess)
                return cleanup(SSE_ERR_CUDA);
    // `stream` observes the completion of the copies
    if (cudaEventRecord(ev_out, cp) != cudaSuccess || cudaStreamWaitEvent(st, ev_out, 0) != cudaSuccess)
        return cleanup(SSE_ERR_CUDA);
    return cleanup(finish(cudaSuccess, status, flags, st));
}
