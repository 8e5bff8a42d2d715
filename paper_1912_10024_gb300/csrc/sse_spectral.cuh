// Shared machinery of the transform-based (convolution-theorem) evaluation of Eqs. (3) and (4) and of the
// adjoint of Eq. (3): the E-direction FFT kernel with its loaders and stores, the frequency maps of the half
// spectrum, complex helpers, the frequency-per-CTA picker and the FP64 product configuration; sse_fft32.cuh, included
// at the end, adds the kz DFT and the FP32 E-transforms with register codelets. Included by
// sse_spectral_fwd.cu (Sigma), sse_spectral_pi.cu (Pi) and sse_spectral_adj.cu (adjoint, gradient in G); each
// translation unit gets its own copy of the internal-linkage kernels and helpers.
//
// For one bond (a, s), b = nbr[a][s], Eq. (3) is a 2-D convolution of G^t_b
// with a lag kernel K:
//
//   Sigma^t_a(E,k) = i*scale * sum_s sum_ij sum_{q,l} K^{t,(a,s)}_ij(q,l) dH_i G^t_b(E-l, k-q) dH_j^H,
//   K(q, l = +(w+1)) = D^t(q,w,a,s),  K(q, l = -(w+1)) = D^{t'}(q,w,a,s)   (t' = other type),
//
// cyclic in kz (period Nkz) and linear in E (G is zero outside [0, NE)). With
// G zero-padded to a length L >= NE + Nw the linear convolution equals the
// cyclic one of period L on [0, NE), so with DFTs over (kz, E) -> (kappa, eps)
//
//   Sigma^^t_a(kappa,eps) = i*scale * sum_s sum_i dH_i G^^t_b(kappa,eps) W_i(kappa,eps),
//   W_i = sum_j K^^_ij(kappa,eps) dH_j^H,
//
// i.e. per frequency and bond 6 products of Norb x Norb blocks instead of the
// 2*Nqz*Nw*3 of the direct form. Steps, per type t:
//   1. G^t -> E-FFT (length L, zero-padded) -> kz-DFT (length Nkz)   -> G^^   [Nkz][L][NA][Norb^2]
//   2. D^t, D^t' placed at lags +-(w+1) -> E-FFT -> qz->kappa DFT      -> K^^   [Nkz][L][nA][NB][9]
//   3. per (a, frequency): the block products above                   -> S^^   [Nkz][L][nA][Norb^2]
//   4. inverse kz-DFT, inverse E-FFT, scale 1/(Nkz L), keep E < NE     -> Sigma^t
// Eq. (4) and the adjoint are correlations of the same kind and use the same transforms. Every transform and
// spectrum is templated on the real type: double (modes FP64, FP64_FFT) or float (FP32_FFT; FP64 inputs and
// outputs). The E-FFT is a Stockham radix-4/2/3 transform of CC columns at once in shared memory
// (L = smallest 2^a 3^b >= NE + Nw); twiddles come from one table of exp(-2 pi i m / L) built with sincospi. In
// FP64 the results equal the direct sums up to the rounding of the transforms (normwise ~1e-15).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {
namespace {

// Transform CTAs: 512 threads and at most 100 KB of shared memory, two CTAs (32 warps) per SM; each thread keeps
// 8 global loads in flight (the shape was chosen by timing 256/512/1024 threads and 8/12/16 loads). The FP64
// transforms are bound by the FP64 pipe; the FP32 ones (lengths without a register-codelet kernel) by instruction
// issue and the waits on their loads.
constexpr int kFftThreads = 512;
constexpr int kFftSmemBudget = 100 * 1024;
constexpr int kFftLoadBatch = 8;
constexpr int kMaxStages = 24;
constexpr int kMaxNk = 16;  // kz grid sizes handled by the kz DFT pass (one kernel instantiation each)

struct FftPlan {
    int L, C, nst;
    int radix[kMaxStages];
    int ns[kMaxStages];           // product of the earlier stages' radices
    int ns_shift[kMaxStages];     // log2(ns) if ns is a power of two, else -1
    unsigned ns_mul[kMaxStages];  // floor(2^32 / ns) + 1: j / ns = umulhi(j, ns_mul), exact for j, ns < 2^16
    int smem;                     // two L x C buffers + the twiddle table
};

constexpr int kFftMaxLength = 1 << 16;  // bound of the umulhi quotient

inline FftPlan make_plan(int L, int esz = 16) {
    FftPlan p{};
    p.L = L;
    int m = L;
    while (m % 4 == 0) p.radix[p.nst++] = 4, m /= 4;
    while (m % 2 == 0) p.radix[p.nst++] = 2, m /= 2;
    while (m % 3 == 0) p.radix[p.nst++] = 3, m /= 3;
    int ns = 1;
    for (int s = 0; s < p.nst; ++s) {
        p.ns[s] = ns;
        p.ns_shift[s] = -1;
        for (int b = 0; b < 31; ++b)
            if ((1 << b) == ns) p.ns_shift[s] = b;
        p.ns_mul[s] = (unsigned)((1ull << 32) / (unsigned long long)ns + 1ull);
        ns *= p.radix[s];
    }
    p.C = 16;
    while (p.C > 1 && (2 * (size_t)L * p.C + L) * esz > (size_t)kFftSmemBudget) p.C /= 2;
    p.smem = (int)((2 * (size_t)L * p.C + L) * esz);
    return p;
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cconj(float2 a) { return make_float2(a.x, -a.y); }
// 8-byte shared-memory access of two consecutive floats
__device__ __forceinline__ float2 ld2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void st2(float* p, float a, float b) { *reinterpret_cast<float2*>(p) = make_float2(a, b); }

// acc[dm][dn] (re/im in ar/ai, index dm * 2 + dn) += x[dm] * y[dn], x or y conjugated on request: 16 FMAs
template <bool CONJX, bool CONJY>
__device__ __forceinline__ void cmac2x2(float* ar, float* ai, float2 xr, float2 xi, float2 yr, float2 yi) {
    const float sx = CONJX ? -1.f : 1.f, sy = CONJY ? -1.f : 1.f;
    const float xrv[2] = {xr.x, xr.y}, xiv[2] = {sx * xi.x, sx * xi.y};
    const float yrv[2] = {yr.x, yr.y}, yiv[2] = {sy * yi.x, sy * yi.y};
#pragma unroll
    for (int dm = 0; dm < 2; ++dm)
#pragma unroll
        for (int dn = 0; dn < 2; ++dn) {
            const int q = dm * 2 + dn;
            ar[q] = fmaf(xrv[dm], yrv[dn], ar[q]);
            ar[q] = fmaf(-xiv[dm], yiv[dn], ar[q]);
            ai[q] = fmaf(xrv[dm], yiv[dn], ai[q]);
            ai[q] = fmaf(xiv[dm], yrv[dn], ai[q]);
        }
}


// complex element type of the transforms: double2 (FP64 modes) or float2 (FP32_FFT)
template <class C>
struct CT;
template <>
struct CT<double2> {
    using R = double;
    static __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }
};
template <>
struct CT<float2> {
    using R = float;
    static __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
};
template <class T>
struct CX;
template <>
struct CX<double> {
    using C = double2;
};
template <>
struct CX<float> {
    using C = float2;
};

// tw[m] = exp(-2 pi i m / L)
__global__ void twiddle_kernel(int L, double2* __restrict__ tw) {
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x) {
        double s, c;
        sincospi(2.0 * (double)m / (double)L, &s, &c);
        tw[m] = make_double2(c, -s);
    }
}

// In-place forward DFT of R values (R in {2, 3, 4}); w3 = exp(-2 pi i / 3) from the twiddle table.
template <int R, class C>
__device__ __forceinline__ void dft_small(C* v, C w3) {
    if constexpr (R == 2) {
        const C a = v[0], b = v[1];
        v[0] = cadd(a, b);
        v[1] = csub(a, b);
    } else if constexpr (R == 4) {
        const C s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        const C s13 = cadd(v[1], v[3]), d13 = csub(v[1], v[3]);
        const C md13 = CT<C>::mk(d13.y, -d13.x);  // -i * d13
        v[0] = cadd(s02, s13);
        v[2] = csub(s02, s13);
        v[1] = cadd(d02, md13);
        v[3] = csub(d02, md13);
    } else {
        static_assert(R == 3, "radix 2, 3 or 4");
        const C t = cadd(v[1], v[2]), d = csub(v[1], v[2]);
        const C m = CT<C>::mk(v[0].x + w3.x * t.x, v[0].y + w3.x * t.y);
        const C r = CT<C>::mk(-w3.y * d.y, w3.y * d.x);  // i * Im(w3) * d
        v[0] = cadd(v[0], t);
        v[1] = cadd(m, r);
        v[2] = csub(m, r);
    }
}

// One Stockham stage of radix R on CC columns stored [L][CC]: butterfly j = q * Ns + k reads rows j + r * L/R,
// multiplies by the twiddles exp(-2 pi i r k / (Ns R)) and writes rows q * Ns * R + k + r * Ns.
template <int R, int CC, class C>
__device__ __forceinline__ void fft_stage(const C* __restrict__ src, C* __restrict__ dst, const C* __restrict__ tw,
                                          int L, int Ns, int ns_shift, unsigned ns_mul) {
    constexpr int lgC = CC == 1 ? 0 : CC == 2 ? 1 : CC == 4 ? 2 : CC == 8 ? 3 : 4;
    static_assert((1 << lgC) == CC, "CC in {1, 2, 4, 8, 16}");
    const int nb = L / R;
    const int span = nb / Ns;  // L / (Ns R)
    const C w3 = tw[L / 3 * (R == 3)];
    for (int it = threadIdx.x; it < nb * CC; it += blockDim.x) {
        const int c = it & (CC - 1), j = it >> lgC;
        const int q = ns_shift >= 0 ? (j >> ns_shift) : (int)__umulhi((unsigned)j, ns_mul);
        const int k = j - q * Ns;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * CC + c];
        if (k > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw[r * k * span]);
        }
        dft_small<R>(v, w3);
        const int d0 = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) dst[(d0 + r * Ns) * CC + c] = v[r];
    }
}

// The same stage for FP32 tiles of at least two columns: each thread takes the adjacent columns (c, c+1) of a
// butterfly with one 16-byte shared access per row, sharing the index arithmetic and the twiddles.
template <int R, int CC>
__device__ __forceinline__ void fft_stage_pairs(const float2* __restrict__ src, float2* __restrict__ dst,
                                                const float2* __restrict__ tw, int L, int Ns, int ns_shift,
                                                unsigned ns_mul) {
    constexpr int CP = CC / 2;  // column pairs per row
    constexpr int lgP = CP == 1 ? 0 : CP == 2 ? 1 : CP == 4 ? 2 : 3;
    static_assert(CC >= 2 && (1 << lgP) == CP, "CC in {2, 4, 8, 16}");
    const int nb = L / R;
    const int span = nb / Ns;
    const float2 w3 = tw[L / 3 * (R == 3)];
    for (int it = threadIdx.x; it < nb * CP; it += blockDim.x) {
        const int c = (it & (CP - 1)) * 2, j = it >> lgP;
        const int q = ns_shift >= 0 ? (j >> ns_shift) : (int)__umulhi((unsigned)j, ns_mul);
        const int k = j - q * Ns;
        float2 a[R], b[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float4 v = *reinterpret_cast<const float4*>(src + (j + r * nb) * CC + c);
            a[r] = make_float2(v.x, v.y);
            b[r] = make_float2(v.z, v.w);
        }
        if (k > 0) {
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const float2 w = tw[r * k * span];
                a[r] = cmul(a[r], w);
                b[r] = cmul(b[r], w);
            }
        }
        dft_small<R>(a, w3);
        dft_small<R>(b, w3);
        const int d0 = q * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r)
            *reinterpret_cast<float4*>(dst + (d0 + r * Ns) * CC + c) = make_float4(a[r].x, a[r].y, b[r].x, b[r].y);
    }
}

template <int R, int CC, class C>
__device__ __forceinline__ void fft_stage_any(const C* src, C* dst, const C* tw, int L, int Ns, int ns_shift,
                                              unsigned ns_mul) {
    if constexpr (sizeof(C) == 8 && CC >= 2)
        fft_stage_pairs<R, CC>(src, dst, tw, L, Ns, ns_shift, ns_mul);
    else
        fft_stage<R, CC>(src, dst, tw, L, Ns, ns_shift, ns_mul);
}

// Stockham autosort FFT of CC columns stored [L][CC] in `src`; returns the buffer holding the result.
template <int CC, class C>
__device__ C* fft_columns(const FftPlan& p, C* src, C* dst, const C* tw) {
    for (int st = 0; st < p.nst; ++st) {
        const int R = p.radix[st];
        if (R == 4) fft_stage_any<4, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
        else if (R == 2) fft_stage_any<2, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
        else fft_stage_any<3, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
    }
    return src;
}

// ---------------------------------------------------------------------------
// E-direction transforms. Each CTA transforms C consecutive columns of one
// batch (kz slice or qz slice); the loader yields row r (r < L) of column col.
// ---------------------------------------------------------------------------

// G^t[k][E][col] (col over NA*Norb^2), rows E >= NE are zero  ->  out[k][eps][col]
template <class CC>
struct LoadGT {
    using C = CC;
    const double2* G;
    int NE;
    size_t ncols;
    __device__ C operator()(int k, int r, size_t col) const {
        if (r >= NE) return CT<C>::mk(0, 0);
        const double2 v = G[((size_t)k * NE + r) * ncols + col];
        return CT<C>::mk(v.x, v.y);
    }
    // the same element for an asynchronous copy: rows below src_rows() are read raw from src() and converted
    using Raw = double2;
    __host__ __device__ int src_rows() const { return NE; }
    __device__ const Raw* src(int k, int r, size_t col) const { return G + ((size_t)k * NE + r) * ncols + col; }
    static __device__ C cvt(Raw v) { return CT<C>::mk(v.x, v.y); }
};
using LoadG = LoadGT<double2>;
// lag kernel of one qz slice: row w+1 <- D^t(q,w), row L-(w+1) <- D^t'(q,w), else zero.
// col over (a - a_begin, s, ij); D rows have NA*NB*9 entries, the range starts at a_begin*NB*9.
template <class CC>
struct LoadLagT {
    using C = CC;
    const double2* Dt;
    const double2* Dtb;
    int Nw, L;
    size_t rowlen, col0;
    __device__ C operator()(int q, int r, size_t col) const {
        double2 v = make_double2(0.0, 0.0);
        if (r >= 1 && r <= Nw) v = Dt[((size_t)q * Nw + (r - 1)) * rowlen + col0 + col];
        else if (r >= L - Nw) v = Dtb[((size_t)q * Nw + (L - 1 - r)) * rowlen + col0 + col];
        return CT<C>::mk(v.x, v.y);
    }
};
using LoadLag = LoadLagT<double2>;
// spectrum [k][eps][col], conjugated (inverse transform = conj(FFT(conj(x))))
template <class CC>
struct LoadSpecConjT {
    using C = CC;
    const C* X;
    int L;
    size_t ncols;
    __device__ C operator()(int k, int r, size_t col) const { return cconj(X[((size_t)k * L + r) * ncols + col]); }
    using Raw = C;
    __host__ __device__ int src_rows() const { return L; }
    __device__ const Raw* src(int k, int r, size_t col) const { return X + ((size_t)k * L + r) * ncols + col; }
    static __device__ C cvt(Raw v) { return cconj(v); }
};
using LoadSpecConj = LoadSpecConjT<double2>;

template <class C>
struct StoreSpecT {  // out[batch][r][col]
    C* X;
    int L;
    size_t ncols;
    int rows;
    __device__ void operator()(int b, int r, size_t col, C v) const { X[((size_t)b * L + r) * ncols + col] = v; }
};
using StoreSpec = StoreSpecT<double2>;
template <class C>
struct StoreSigmaT {  // S[k][E][a_begin*nel + col] = conj(v) * inv in FP64, E < NE
    double2* S;
    int NE;
    size_t rowlen, col0;
    double inv;
    int rows;
    __device__ void operator()(int k, int r, size_t col, C v) const {
        using R = typename CT<C>::R;
        const R s = (R)inv;  // scaled in the transform's precision, then widened
        S[((size_t)k * NE + r) * rowlen + col0 + col] = make_double2((double)(v.x * s), (double)(-v.y * s));
    }
};
using StoreSigma = StoreSigmaT<double2>;

template <class Load, class Store, int CC>
__global__ void __launch_bounds__(kFftThreads) fft_e_kernel(FftPlan p, const double2* __restrict__ tw_g, Load ld,
                                                            Store sv, size_t ncols) {
    using C = typename Load::C;
    constexpr int lgC = CC == 1 ? 0 : CC == 2 ? 1 : CC == 4 ? 2 : CC == 8 ? 3 : 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* b0 = reinterpret_cast<C*>(smem_raw);
    C* b1 = b0 + p.L * CC;
    C* tw = b1 + p.L * CC;
    const size_t col0 = (size_t)blockIdx.x * CC;
    const int batch = blockIdx.y;
    for (int m = threadIdx.x; m < p.L; m += blockDim.x) tw[m] = CT<C>::mk(tw_g[m].x, tw_g[m].y);
    const int n = p.L * CC;
    for (int base = threadIdx.x; base < n; base += kFftLoadBatch * blockDim.x) {
        C v[kFftLoadBatch];
#pragma unroll
        for (int u = 0; u < kFftLoadBatch; ++u) {
            const int it = base + u * blockDim.x;
            const int r = it >> lgC, c = it & (CC - 1);
            v[u] = (it < n && col0 + c < ncols) ? ld(batch, r, col0 + c) : CT<C>::mk(0, 0);
        }
#pragma unroll
        for (int u = 0; u < kFftLoadBatch; ++u) {
            const int it = base + u * blockDim.x;
            if (it < n) b0[it] = v[u];
        }
    }
    __syncthreads();
    const C* res = fft_columns<CC>(p, b0, b1, tw);
    for (int it = threadIdx.x; it < sv.rows * CC; it += blockDim.x) {
        const int r = it >> lgC, c = it & (CC - 1);
        if (col0 + c < ncols) sv(batch, r, col0 + c, res[it]);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// frequency index maps. With anti-Hermitian inputs (SSE_FLAG_ANTIHERMITIAN) the spectra obey
// S^(-f) = -S^(f)^H (Sigma) and C^(-f) = C^(f)^H (Pi), so only one frequency of each pair (f, -f)
// is computed: eps in [1, (L-1)/2] for every kappa, and on the rows eps = 0 and eps = L/2 (L even)
// kappa in [0, Nk/2]; a mirror kernel fills the partners. (Outside the file-local namespace: the
// tensor-core product kernel in sse_spectral_tc.cu takes the same map.)
// ---------------------------------------------------------------------------
struct FreqMap {
    int Nk, L, half, Lh, nK0;
    size_t count;
};

inline FreqMap make_freq_map(int Nk, int L, bool half) {
    FreqMap m{};
    m.Nk = Nk;
    m.L = L;
    m.half = half ? 1 : 0;
    m.Lh = (L - 1) / 2;
    m.nK0 = Nk / 2 + 1;
    m.count = half ? (size_t)Nk * m.Lh + (size_t)m.nK0 * ((L % 2 == 0) ? 2 : 1) : (size_t)Nk * L;
    return m;
}

__device__ __forceinline__ size_t freq_of(const FreqMap& m, size_t i) {
    if (!m.half) return i;
    const size_t body = (size_t)m.Nk * m.Lh;
    if (i < body) return (i / m.Lh) * (size_t)m.L + 1 + (i % m.Lh);
    const size_t r = i - body;
    const size_t row = r / m.nK0, kap = r - row * m.nK0;
    return kap * (size_t)m.L + (row == 0 ? 0 : (size_t)(m.L / 2));
}

__device__ __forceinline__ size_t freq_neg(const FreqMap& m, size_t f) {
    const int kap = (int)(f / m.L), eps = (int)(f - (size_t)kap * m.L);
    return (size_t)((m.Nk - kap) % m.Nk) * m.L + (size_t)((m.L - eps) % m.L);
}

// Block products of the F16X3_FFT forward on the tcgen05 tensor cores (sse_spectral_tc.cu): S^ of one type from the
// FP32 spectra G^ [Nkz*L][NA][Norb^2] and K^ [Nkz*L][nA][NB][9] into S^ [Nkz*L][nA][Norb^2] (frequencies of `fm`).
// Limits (host-only): Norb <= 10, NB <= 4.
bool spectral_prod_tc_supported(const sse_dims& d);
cudaError_t spectral_prod_tc(const sse_dims& d, const FreqMap& fm, const int32_t* nbr, const double2* dH,
                             const float2* Gh, const float2* Kh, float2* Sh, double scale, unsigned* status,
                             cudaStream_t st);

namespace {

// Sigma^(-f) = -Sigma^(f)^H per atom block, for the computed half
template <class C>
__global__ void mirror_sigma_kernel(FreqMap fm, size_t nA, int Norb, C* __restrict__ Sh) {
    const int nel = Norb * Norb;
    const size_t total = fm.count * nA * nel;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % nel);
        const size_t r = i / nel;
        const size_t la = r % nA, ix = r / nA;
        const size_t f = freq_of(fm, ix), fn = freq_neg(fm, f);
        if (fn == f) continue;
        const int m = e / Norb, n = e - m * Norb;
        const C v = Sh[(f * nA + la) * nel + e];
        Sh[(fn * nA + la) * nel + n * Norb + m] = CT<C>::mk(-v.x, v.y);
    }
}

// C^(-f) = C^(f)^H per 3x3 block (Pi), for the computed half
template <class C>
__global__ void mirror_pi_kernel(FreqMap fm, size_t nblk, C* __restrict__ Ch) {
    const size_t total = fm.count * nblk * 9;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int ij = (int)(i % 9);
        const size_t r = i / 9;
        const size_t blk = r % nblk, ix = r / nblk;
        const size_t f = freq_of(fm, ix), fn = freq_neg(fm, f);
        if (fn == f) continue;
        const int ii = ij / 3, jj = ij - 3 * ii;
        const C v = Ch[(f * nblk + blk) * 9 + ij];
        Ch[(fn * nblk + blk) * 9 + jj * 3 + ii] = CT<C>::mk(v.x, -v.y);
    }
}

// With CHECK: every n x n block must be exactly anti-Hermitian, B[r][c] = -conj(B[c][r]).
__global__ void check_antiherm_kernel(const double2* __restrict__ X, size_t nblk, int n,
                                      unsigned* __restrict__ status) {
    const size_t total = nblk * n * n;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % (n * n));
        const size_t b = i / (n * n);
        const int r = e / n, c2 = e - r * n;
        const double2 x = X[b * n * n + e], y = X[b * n * n + c2 * n + r];
        if (x.x != -y.x || x.y != y.y) atomicOr(status, DEV_NOT_ANTIHERMITIAN);
    }
}

// ---------------------------------------------------------------------------
// per-frequency block products
// ---------------------------------------------------------------------------
constexpr int kProdMaxThreads = 512;

// Frequencies per CTA for the product kernels: the F that keeps the most lanes (F * nel of them, nel threads per
// frequency) busy per SM (whole warps issue, so lanes past F * nel are lost), given the shared memory per CTA,
// 64 warps per SM, `regs` registers per thread and at most `max_threads` threads per CTA.
template <class SmemOf>
int pick_frequencies(int nel, SmemOf smem_of, int regs = 64, int max_threads = kProdMaxThreads) {
    int best = 1;
    long best_useful = -1, best_smem = 0;
    for (int F = 1; F * nel <= max_threads; ++F) {
        const int threads = ((F * nel + 31) / 32) * 32;
        const long sm = smem_of(F);
        if (sm > 227 * 1024) break;
        long ctas = (228L * 1024) / (sm + 1024);
        ctas = ctas < 2048 / threads ? ctas : 2048 / threads;
        ctas = ctas < 65536 / (threads * regs) ? ctas : 65536 / (threads * regs);
        const long useful = ctas * F * nel;
        if (useful > best_useful || (useful == best_useful && sm < best_smem)) {
            best = F;
            best_useful = useful;
            best_smem = sm;
        }
    }
    return best;
}

struct ProdCfg {
    int nel, F, threads, fchunk;
    int off_A, off_G, off_K, off_W, off_U, smem;
};

inline ProdCfg make_prod_cfg(const sse_dims& d, size_t nfreq, int tsz = 8) {
    ProdCfg c{};
    c.nel = d.Norb * d.Norb;
    const int pl = c.nel * 3 * tsz;  // one (re, im, re+im) plane triple
    auto a16 = [](int x) { return (x + 15) & ~15; };  // every region starts on a 16-byte boundary
    c.F = pick_frequencies(c.nel, [&](int F) {
        return (long)a16(a16(a16(a16(d.NB * 3 * pl) + F * pl) + F * 9 * 2 * tsz) + F * 3 * pl) + F * 3 * pl;
    });
    c.threads = ((c.F * c.nel + 31) / 32) * 32;
    c.off_A = 0;                                   // [NB][3][planes]
    c.off_G = a16(c.off_A + d.NB * 3 * pl);        // [F][planes]
    c.off_K = a16(c.off_G + c.F * pl);             // [F][9] complex
    c.off_W = a16(c.off_K + c.F * 9 * 2 * tsz);    // [F][3][planes]
    c.off_U = a16(c.off_W + c.F * 3 * pl);         // [F][3][planes]
    c.smem = a16(c.off_U + c.F * 3 * pl);
    // frequencies per CTA: enough CTAs for ~8 waves of 2 CTAs per SM over all atoms
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

// Planes of a complex block: re, im, re+im (Gauss 3-multiply MACs).
template <class T, class C>
__device__ __forceinline__ void put3(T* P, int nel, int e, C v) {
    P[e] = v.x;
    P[nel + e] = v.y;
    P[2 * nel + e] = v.x + v.y;
}

// The FP32 tile kernels place the tile threads of two adjacent frequencies in one warp; per-frequency strides of
// 16 mod 32 floats put their rows of a plane on disjoint shared-memory banks.
inline int bank_pad16(int floats) { return floats + ((16 - floats % 32) + 32) % 32; }

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

inline unsigned grid_for(size_t work, int threads) {
    size_t g = (work + threads - 1) / threads;
    const size_t cap = (size_t)152 * 16;
    return (unsigned)(g < 1 ? 1 : (g > cap ? cap : g));
}

template <int CC, class Load, class Store>
cudaError_t launch_fft_c(const char* name, const FftPlan& p, const double2* tw, Load ld, Store sv, size_t ncols,
                         int batches, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(fft_e_kernel<Load, Store, CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
    if (e != cudaSuccess) return e;
    const size_t gx = (ncols + CC - 1) / CC;
    if (gx > 0x7fffffffu || batches > 65535) return cudaErrorInvalidValue;
    SSE_TIMED(name, st,
              fft_e_kernel<Load, Store, CC><<<dim3((unsigned)gx, (unsigned)batches), kFftThreads, p.smem, st>>>(
                  p, tw, ld, sv, ncols));
    return cudaGetLastError();
}

template <class Load, class Store>
cudaError_t launch_fft(const char* name, const FftPlan& p, const double2* tw, Load ld, Store sv, size_t ncols,
                       int batches, cudaStream_t st) {
    switch (p.C) {
        case 16: return launch_fft_c<16>(name, p, tw, ld, sv, ncols, batches, st);
        case 8: return launch_fft_c<8>(name, p, tw, ld, sv, ncols, batches, st);
        case 4: return launch_fft_c<4>(name, p, tw, ld, sv, ncols, batches, st);
        case 2: return launch_fft_c<2>(name, p, tw, ld, sv, ncols, batches, st);
        case 1: return launch_fft_c<1>(name, p, tw, ld, sv, ncols, batches, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace sse

#include "sse_fft32.cuh"
