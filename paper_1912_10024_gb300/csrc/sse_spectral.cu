// Transform-based FP64 forward of Eq. (3) (the convolution theorem along kz and E).
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
// 2*Nqz*Nw*3 of the direct form. Steps, per type t (FP64 throughout):
//   1. G^t -> E-FFT (length L, zero-padded) -> kz-DFT (length Nkz)   -> G^^   [Nkz][L][NA][Norb^2]
//   2. D^t, D^t' placed at lags +-(w+1) -> E-FFT -> qz->kappa DFT      -> K^^   [Nkz][L][nA][NB][9]
//   3. per (a, frequency): the block products above (Gauss 3-multiply
//      complex MACs on pre-formed (re, im, re+im) planes)             -> S^^   [Nkz][L][nA][Norb^2]
//   4. inverse kz-DFT, inverse E-FFT, scale 1/(Nkz L), keep E < NE     -> Sigma^t
// The E-FFT is a Stockham radix-4/2/3 transform of C columns at once in
// shared memory (L = smallest 2^a 3^b >= NE + Nw); twiddles come from one
// table of exp(-2 pi i m / L) built with sincospi. The results equal Eq. (3)
// up to the rounding of the transforms (normwise ~1e-15).
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {
namespace {

// Transform CTAs: 512 threads and at most 100 KB of shared memory, two CTAs (32 warps) per SM; each thread keeps
// 8 global loads in flight. The FP32 transforms are bound by the latency of those loads (the shape was chosen by
// timing 256/512/1024 threads and 8/12/16 loads), the FP64 ones by the FP64 pipe.
constexpr int kFftThreads = 512;
constexpr int kFftSmemBudget = 100 * 1024;
constexpr int kFftLoadBatch = 8;
constexpr int kMaxStages = 24;
constexpr int kMaxNk = 16;  // kz grid sizes handled by the small DFT pass

struct FftPlan {
    int L, C, nst;
    int radix[kMaxStages];
    int ns[kMaxStages];           // product of the earlier stages' radices
    int ns_shift[kMaxStages];     // log2(ns) if ns is a power of two, else -1
    unsigned ns_mul[kMaxStages];  // floor(2^32 / ns) + 1: j / ns = umulhi(j, ns_mul), exact for j, ns < 2^16
    int smem;                     // two L x C buffers + the twiddle table
};

constexpr int kFftMaxLength = 1 << 16;  // bound of the umulhi quotient

FftPlan make_plan(int L, int esz = 16) {
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

// Stockham autosort FFT of CC columns stored [L][CC] in `src`; returns the buffer holding the result.
template <int CC, class C>
__device__ C* fft_columns(const FftPlan& p, C* src, C* dst, const C* tw) {
    for (int st = 0; st < p.nst; ++st) {
        const int R = p.radix[st];
        if (R == 4) fft_stage<4, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
        else if (R == 2) fft_stage<2, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
        else fft_stage<3, CC>(src, dst, tw, p.L, p.ns[st], p.ns_shift[st], p.ns_mul[st]);
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

// ---------------------------------------------------------------------------
// kz-direction DFT, in place on X[Nk][M]: out[kappa] = sum_{k < n_in} in[k] exp(-+2 pi i k kappa / Nk).
// Inputs k and Nk-k are paired (p = x_k + x_{Nk-k}, m = x_k - x_{Nk-k}) and so are outputs kappa and
// Nk-kappa: out[kappa] = C -+ i S, out[Nk-kappa] = C +- i S with C = x_0 (+ (-1)^kappa x_{Nk/2}) +
// sum_k p_k cos(2 pi k kappa / Nk), S = sum_k m_k sin(2 pi k kappa / Nk).
// ---------------------------------------------------------------------------
template <class C>
__global__ void dft_k_kernel(C* __restrict__ X, int Nk, int n_in, size_t M, int inverse) {
    using R = typename CT<C>::R;
    __shared__ R cs[kMaxNk], sn[kMaxNk];
    if (threadIdx.x < Nk) {
        double s, c;
        sincospi(2.0 * (double)threadIdx.x / (double)Nk, &s, &c);
        cs[threadIdx.x] = (R)c;
        sn[threadIdx.x] = (R)s;
    }
    __syncthreads();
    const int half = (Nk - 1) / 2;  // number of (k, Nk-k) pairs
    const bool even = (Nk % 2) == 0;
    const R sgn = inverse ? (R)1 : (R)-1;  // out = C + sgn * i * S for kappa <= half
    for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < M; m += (size_t)gridDim.x * blockDim.x) {
        C x[kMaxNk];
        for (int k = 0; k < Nk; ++k) x[k] = k < n_in ? X[(size_t)k * M + m] : CT<C>::mk(0, 0);
        C p[kMaxNk / 2 + 1], q[kMaxNk / 2 + 1];
        C c0 = x[0];
        for (int k = 1; k <= half; ++k) {
            p[k] = cadd(x[k], x[Nk - k]);
            q[k] = csub(x[k], x[Nk - k]);
            c0 = cadd(c0, p[k]);
        }
        const C xh = even ? x[Nk / 2] : CT<C>::mk(0, 0);
        X[m] = cadd(c0, xh);  // kappa = 0
        for (int kap = 1; kap <= half; ++kap) {
            C Cs = x[0], S = CT<C>::mk(0, 0);
            for (int k = 1; k <= half; ++k) {
                const int r = (k * kap) % Nk;
                Cs.x = fma(p[k].x, cs[r], Cs.x);
                Cs.y = fma(p[k].y, cs[r], Cs.y);
                S.x = fma(q[k].x, sn[r], S.x);
                S.y = fma(q[k].y, sn[r], S.y);
            }
            if (even) {
                const R e = (kap & 1) ? (R)-1 : (R)1;
                Cs.x = fma(e, xh.x, Cs.x);
                Cs.y = fma(e, xh.y, Cs.y);
            }
            // i*S = (-S.y, S.x)
            X[(size_t)kap * M + m] = CT<C>::mk(Cs.x - sgn * S.y, Cs.y + sgn * S.x);
            X[(size_t)(Nk - kap) * M + m] = CT<C>::mk(Cs.x + sgn * S.y, Cs.y - sgn * S.x);
        }
        if (even && Nk > 1) {  // kappa = Nk/2: cos(pi k) = (-1)^k, sin = 0
            C Cs = x[0];
            for (int k = 1; k <= half; ++k) {
                const R e = (k & 1) ? (R)-1 : (R)1;
                Cs.x = fma(e, p[k].x, Cs.x);
                Cs.y = fma(e, p[k].y, Cs.y);
            }
            const R e = ((Nk / 2) & 1) ? (R)-1 : (R)1;
            X[(size_t)(Nk / 2) * M + m] = CT<C>::mk(fma(e, xh.x, Cs.x), fma(e, xh.y, Cs.y));
        }
    }
}

// ---------------------------------------------------------------------------
// frequency index maps. With anti-Hermitian inputs (SSE_FLAG_ANTIHERMITIAN) the spectra obey
// S^(-f) = -S^(f)^H (Sigma) and C^(-f) = C^(f)^H (Pi), so only one frequency of each pair (f, -f)
// is computed: eps in [1, (L-1)/2] for every kappa, and on the rows eps = 0 and eps = L/2 (L even)
// kappa in [0, Nk/2]; a mirror kernel fills the partners.
// ---------------------------------------------------------------------------
struct FreqMap {
    int Nk, L, half, Lh, nK0;
    size_t count;
};

FreqMap make_freq_map(int Nk, int L, bool half) {
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

ProdCfg make_prod_cfg(const sse_dims& d, size_t nfreq, int tsz = 8) {
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

template <class T>
__global__ void spec_prod_kernel(ProdCfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr,
                                 const double2* __restrict__ dH, const typename CX<T>::C* __restrict__ Ghat,
                                 const typename CX<T>::C* __restrict__ Khat, typename CX<T>::C* __restrict__ Shat,
                                 double scale, unsigned* __restrict__ status) {
    using C = typename CX<T>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;  // frequency indices of the map
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    T* sA = reinterpret_cast<T*>(smem + c.off_A);
    T* sG = reinterpret_cast<T*>(smem + c.off_G);
    C* sK = reinterpret_cast<C*>(smem + c.off_K);
    T* sW = reinterpret_cast<T*>(smem + c.off_W);
    T* sU = reinterpret_cast<T*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;

    for (int i = tid; i < d.NB * 3 * nel; i += blockDim.x) {
        const int si = i / nel, ee = i - si * nel;
        const double2 v = dH[((size_t)a * d.NB) * 3 * nel + i];
        put3(sA + (size_t)si * 3 * nel, nel, ee, CT<C>::mk((T)v.x, (T)v.y));
    }
    int bnb[16];
    for (int s = 0; s < d.NB && s < 16; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        bnb[s] = (b >= 0 && b < d.NA) ? b : -1;
        if (bnb[s] < 0 && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
    }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        T T1 = 0, T2 = 0, T3 = 0;
        for (int s = 0; s < d.NB; ++s) {
            const int b = s < 16 ? bnb[s] : -1;
            // stage G^_b(f) and K^_(a,s)(f)
            if (lane) {
                C g = CT<C>::mk(0, 0);
                if (act && b >= 0) g = Ghat[(f * d.NA + b) * nel + e];
                put3(sG + (size_t)fl * 3 * nel, nel, e, g);
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                C k = CT<C>::mk(0, 0);
                if (i0 + fk < i_end && b >= 0) k = Khat[((freq_of(fm, i0 + fk) * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            // W_i[m][n] = sum_j K_ij conj(dH_j[n][m])
            if (lane) {
                const T* A = sA + (size_t)s * 9 * nel;
                const int et = n * Norb + m;
                T ar[3], ai[3];  // conj(dH_j[n][m]) = (ar, -ai)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    ar[j] = A[(size_t)j * 3 * nel + et];
                    ai[j] = A[(size_t)j * 3 * nel + nel + et];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    C acc = CT<C>::mk(0, 0);  // plain FMA chains: no separate multiplies or adds
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const C k = sK[fl * 9 + i * 3 + j];
                        acc.x = fma(k.x, ar[j], acc.x);
                        acc.x = fma(k.y, ai[j], acc.x);
                        acc.y = fma(k.y, ar[j], acc.y);
                        acc.y = fma(-k.x, ai[j], acc.y);
                    }
                    put3(sW + ((size_t)fl * 3 + i) * 3 * nel, nel, e, acc);
                }
            }
            __syncthreads();
            // U_i = G^ W_i
            if (lane) {
                const T* Gp = sG + (size_t)fl * 3 * nel;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Wp = sW + ((size_t)fl * 3 + i) * 3 * nel;
                    T t1 = 0, t2 = 0, t3 = 0;
                    for (int l = 0; l < Norb; ++l) {
                        const int ga = m * Norb + l, wb = l * Norb + n;
                        t1 = fma(Gp[ga], Wp[wb], t1);
                        t2 = fma(Gp[nel + ga], Wp[nel + wb], t2);
                        t3 = fma(Gp[2 * nel + ga], Wp[2 * nel + wb], t3);
                    }
                    put3(sU + ((size_t)fl * 3 + i) * 3 * nel, nel, e, CT<C>::mk(t1 - t2, t3 - t1 - t2));
                }
            }
            __syncthreads();
            // acc += sum_i dH_i U_i
            if (lane) {
                const T* A = sA + (size_t)s * 9 * nel;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Ap = A + (size_t)i * 3 * nel;
                    const T* Up = sU + ((size_t)fl * 3 + i) * 3 * nel;
                    for (int l = 0; l < Norb; ++l) {
                        const int aa = m * Norb + l, ub = l * Norb + n;
                        T1 = fma(Ap[aa], Up[ub], T1);
                        T2 = fma(Ap[nel + aa], Up[nel + ub], T2);
                        T3 = fma(Ap[2 * nel + aa], Up[2 * nel + ub], T3);
                    }
                }
            }
        }
        if (act) {
            const T re = T1 - T2, im = T3 - T1 - T2;
            Shat[(f * nA + la) * nel + e] = CT<C>::mk((T)(-scale * (double)im), (T)(scale * (double)re));  // i*scale*(re+i im)
        }
    }
}

// ---------------------------------------------------------------------------
// phonon self-energy, Eq. (4): per (a, slot s, frequency)
//   C^_ij(kappa,eps) = tr( dH_i^H G^t_a(kappa,eps) dH_j G^t'_b(-kappa,-eps) ),
// the transform of the correlation sum_{k,E} tr(dH_i^H G^t_a(E+l, k+q) dH_j G^t'_b(E, k)) over the lags
// (q, l); slot NB (the diagonal block) is the sum over the bonds.
// ---------------------------------------------------------------------------
struct PiCfg {
    int nel, F, threads, fchunk;
    int off_A, off_X, off_Y, off_P, off_R, off_D, off_self, smem;
};

PiCfg make_pi_cfg(const sse_dims& d, size_t nfreq) {
    PiCfg c{};
    c.nel = d.Norb * d.Norb;
    const int pl = c.nel * 8;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    c.F = pick_frequencies(c.nel, [&](int F) {
        return (long)d.NB * 3 * 4 * pl + F * 3 * pl * 2 + F * 6 * pl * 2 + F * 9 * d.Norb * 16 + F * 9 * 16 + 96;
    });
    c.threads = ((c.F * c.nel + 31) / 32) * 32;
    c.off_A = 0;                                     // [NB][3][4 planes: re, im, re+im, re-im]
    c.off_X = a16(c.off_A + d.NB * 3 * 4 * pl);      // [F][3 planes]
    c.off_Y = a16(c.off_X + c.F * 3 * pl);           // [F][3 planes]
    c.off_P = a16(c.off_Y + c.F * 3 * pl);           // [F][3 i][2 planes]
    c.off_R = a16(c.off_P + c.F * 6 * pl);           // [F][3 j][2 planes]
    c.off_D = a16(c.off_R + c.F * 6 * pl);           // [F][9][Norb] complex: diagonal terms
    c.off_self = a16(c.off_D + c.F * 9 * d.Norb * 16);  // [F][9] complex: diagonal-block sums
    c.smem = a16(c.off_self + c.F * 9 * 16);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + 2 * nA - 1) / (2 * nA ? 2 * nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void __launch_bounds__(kProdMaxThreads, 2)
spec_pi_kernel(PiCfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
               const double2* __restrict__ Gl_hat, const double2* __restrict__ Gg_hat, double2* __restrict__ Cl_hat,
               double2* __restrict__ Cg_hat, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const int t = blockIdx.z;
    const double2* X_hat = t == 0 ? Gl_hat : Gg_hat;  // G^t of atom a
    const double2* Y_hat = t == 0 ? Gg_hat : Gl_hat;  // G^t' of the neighbour
    double2* C_hat = t == 0 ? Cl_hat : Cg_hat;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;  // frequency indices of the map
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    double* sA = reinterpret_cast<double*>(smem + c.off_A);
    double* sX = reinterpret_cast<double*>(smem + c.off_X);
    double* sY = reinterpret_cast<double*>(smem + c.off_Y);
    double* sP = reinterpret_cast<double*>(smem + c.off_P);
    double* sR = reinterpret_cast<double*>(smem + c.off_R);
    double2* sD = reinterpret_cast<double2*>(smem + c.off_D);
    double2* sSelf = reinterpret_cast<double2*>(smem + c.off_self);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;
    const int slots = d.NB + 1;
    const int ndiag = c.F * 9 * Norb;

    for (int i = tid; i < d.NB * 3 * nel; i += blockDim.x) {
        const int si = i / nel, ee = i - si * nel;
        const double2 v = dH[((size_t)a * d.NB) * 3 * nel + i];
        double* P = sA + (size_t)si * 4 * nel;
        P[ee] = v.x;
        P[nel + ee] = v.y;
        P[2 * nel + ee] = v.x + v.y;
        P[3 * nel + ee] = v.x - v.y;
    }
    if (tid == 0 && t == 0)
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            if (b < 0 || b >= d.NA) atomicOr(status, DEV_BAD_NEIGHBOUR);
        }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        const size_t fneg = act ? freq_neg(fm, f) : 0;
        if (lane) {
            double2 x = make_double2(0.0, 0.0);
            if (act) x = X_hat[(f * d.NA + a) * nel + e];
            put3(sX + (size_t)fl * 3 * nel, nel, e, x);
        }
        // diagonal-block sums: entry g = (frequency, ij) belongs to thread g mod blockDim for the whole batch
        for (int g = tid; g < c.F * 9; g += blockDim.x) sSelf[g] = make_double2(0.0, 0.0);
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            if (lane) {
                double2 y = make_double2(0.0, 0.0);
                if (act && bok) y = Y_hat[(fneg * d.NA + b) * nel + e];
                put3(sY + (size_t)fl * 3 * nel, nel, e, y);
            }
            __syncthreads();
            // half products P_i = dH_i^H X, R_j = dH_j Y (Gauss 3-multiply MACs)
            if (lane) {
                const double* A = sA + (size_t)s * 12 * nel;
                const double* Xp = sX + (size_t)fl * 3 * nel;
                const double* Yp = sY + (size_t)fl * 3 * nel;
#pragma unroll 1
                for (int i = 0; i < 3; ++i) {
                    const double* Ai = A + (size_t)i * 4 * nel;
                    double t1 = 0.0, u2 = 0.0, t3 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
                    for (int l = 0; l < Norb; ++l) {
                        const int lm = l * Norb + m, ml = m * Norb + l, ln = l * Norb + n;
                        t1 = fma(Ai[lm], Xp[ln], t1);                  // conj(A_i[l][m]) X[l][n]
                        u2 = fma(Ai[nel + lm], Xp[nel + ln], u2);
                        t3 = fma(Ai[3 * nel + lm], Xp[2 * nel + ln], t3);
                        r1 = fma(Ai[ml], Yp[ln], r1);                  // A_i[m][l] Y[l][n]
                        r2 = fma(Ai[nel + ml], Yp[nel + ln], r2);
                        r3 = fma(Ai[2 * nel + ml], Yp[2 * nel + ln], r3);
                    }
                    double* P = sP + ((size_t)fl * 3 + i) * 2 * nel;
                    P[e] = t1 + u2;
                    P[nel + e] = t3 - t1 + u2;
                    double* R = sR + ((size_t)fl * 3 + i) * 2 * nel;
                    R[e] = r1 - r2;
                    R[nel + e] = r3 - r1 - r2;
                }
            }
            __syncthreads();
            // diagonal terms D_ij[m] = sum_n P_i[m][n] R_j[n][m]
            for (int g = tid; g < ndiag; g += blockDim.x) {
                const int fi = g / (9 * Norb), rem = g - fi * 9 * Norb;
                const int ij = rem / Norb, mm = rem - ij * Norb;
                const int i = ij / 3, j = ij - 3 * i;
                const double* P = sP + ((size_t)fi * 3 + i) * 2 * nel;
                const double* R = sR + ((size_t)fi * 3 + j) * 2 * nel;
                double re = 0.0, im = 0.0;
                for (int nn = 0; nn < Norb; ++nn) {
                    const double pr = P[mm * Norb + nn], pi = P[nel + mm * Norb + nn];
                    const double rr = R[nn * Norb + mm], ri = R[nel + nn * Norb + mm];
                    re = fma(pr, rr, re);
                    re = fma(-pi, ri, re);
                    im = fma(pr, ri, im);
                    im = fma(pi, rr, im);
                }
                sD[g] = make_double2(re, im);
            }
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {  // fixed-order sums over the rows m
                const int rf = g / 9, ij = g - rf * 9;
                const double2* v = sD + (size_t)g * Norb;
                double2 sum = v[0];
                for (int mm = 1; mm < Norb; ++mm) sum = cadd(sum, v[mm]);
                const double2 self = cadd(sSelf[g], sum);
                sSelf[g] = self;
                if (i0 + rf < i_end) {
                    const size_t ff = freq_of(fm, i0 + rf);
                    C_hat[((ff * nA + la) * slots + s) * 9 + ij] = sum;
                    if (s == d.NB - 1) C_hat[((ff * nA + la) * slots + d.NB) * 9 + ij] = self;
                }
            }
            // the next bond rewrites sY before its first barrier; sP, sR and sD only after it
        }
        __syncthreads();  // sX of the next frequency batch
    }
}

// ---------------------------------------------------------------------------
// FP32 phonon self-energy (mode FP32_FFT): the half products P_i = dH_i^H X^ and R_j = dH_j Y^ three at a time
// on 2 x 2 register tiles (4-multiply MACs on (re, im) planes); R_j goes to shared memory transposed, so each
// thread forms its tile's part of tr(P_i R_j) from P_i in registers; the parts are summed over the tile threads
// in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kPi32MaxThreads = 256;  // <= 128 registers at two CTAs per SM

struct Pi32Cfg {
    int Np, TN, T, pl, F, threads, fchunk;
    int off_A, off_X, off_Y, off_R, off_self, smem;
};

Pi32Cfg make_pi32_cfg(const sse_dims& d, size_t nfreq) {
    Pi32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    // per CTA: every bond's dH row-major and transposed (12 planes per bond); per frequency X^, Y^ (4 planes),
    // R_j transposed (6 planes; the trace parts reuse them) and the diagonal-block sums (9 float2)
    c.F = pick_frequencies(
        c.T, [&](int F) { return (long)d.NB * 12 * pb + F * (10L * pb + 9 * 8) + 96; }, 128, kPi32MaxThreads);
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                               // [NB][3][4 planes: re, im row-major; re, im transposed]
    c.off_X = a16(c.off_A + d.NB * 12 * pb);   // [F][2 planes] X^ row-major
    c.off_Y = a16(c.off_X + c.F * 2 * pb);     // [F][2 planes] Y^ row-major
    c.off_R = a16(c.off_Y + c.F * 2 * pb);     // [F][3 j][2 planes] R_j transposed
    c.off_self = a16(c.off_R + c.F * 6 * pb);  // [F][9] float2
    c.smem = a16(c.off_self + c.F * 9 * 8);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + 2 * nA - 1) / (2 * nA ? 2 * nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void __launch_bounds__(kPi32MaxThreads, 2)
spec_pi32_kernel(Pi32Cfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
                 const float2* __restrict__ Gl_hat, const float2* __restrict__ Gg_hat, float2* __restrict__ Cl_hat,
                 float2* __restrict__ Cg_hat, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb, T = c.T;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const int t = blockIdx.z;
    const float2* X_hat = t == 0 ? Gl_hat : Gg_hat;  // G^t of atom a
    const float2* Y_hat = t == 0 ? Gg_hat : Gl_hat;  // G^t' of the neighbour
    float2* C_hat = t == 0 ? Cl_hat : Cg_hat;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sX = reinterpret_cast<float*>(smem + c.off_X);
    float* sY = reinterpret_cast<float*>(smem + c.off_Y);
    float* sR = reinterpret_cast<float*>(smem + c.off_R);
    float2* sSelf = reinterpret_cast<float2*>(smem + c.off_self);
    const int tid = threadIdx.x;
    const int fl = tid / T, tt = tid - fl * T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;
    const int slots = d.NB + 1;

    // dH planes of every bond, zero-padded: row-major A[l][n] and transposed AT[l][m] = A[m][l]
    for (int i = tid; i < d.NB * 3 * pl; i += blockDim.x) {
        const int si = i / pl, e = i - si * pl;
        const int r = e / Np, q = e - r * Np;
        double2 v = make_double2(0.0, 0.0), w = make_double2(0.0, 0.0);
        if (r < Norb && q < Norb) {
            v = dH[((size_t)a * d.NB * 3 + si) * nel + r * Norb + q];
            w = dH[((size_t)a * d.NB * 3 + si) * nel + q * Norb + r];
        }
        float* P = sA + (size_t)si * 4 * pl;
        P[e] = (float)v.x;
        P[pl + e] = (float)v.y;
        P[2 * pl + e] = (float)w.x;
        P[3 * pl + e] = (float)w.y;
    }
    if (tid == 0 && t == 0)
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            if (b < 0 || b >= d.NA) atomicOr(status, DEV_BAD_NEIGHBOUR);
        }

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        const size_t fneg = act ? freq_neg(fm, f) : 0;
        __syncthreads();  // the previous batch is done with sX and sSelf
        if (lane) {
            float* Xp = sX + (size_t)fl * 2 * pl;
#pragma unroll
            for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                for (int dn = 0; dn < 2; ++dn) {
                    const int m = m0 + dm, n = n0 + dn;
                    float2 x = make_float2(0.f, 0.f);
                    if (act && m < Norb && n < Norb) x = X_hat[(f * d.NA + a) * nel + m * Norb + n];
                    Xp[m * Np + n] = x.x;
                    Xp[pl + m * Np + n] = x.y;
                }
        }
        for (int g = tid; g < c.F * 9; g += blockDim.x) sSelf[g] = make_float2(0.f, 0.f);
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            if (lane) {
                float* Yp = sY + (size_t)fl * 2 * pl;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 y = make_float2(0.f, 0.f);
                        if (act && bok && m < Norb && n < Norb) y = Y_hat[(fneg * d.NA + b) * nel + m * Norb + n];
                        Yp[m * Np + n] = y.x;
                        Yp[pl + m * Np + n] = y.y;
                    }
            }
            __syncthreads();
            const float* A = sA + (size_t)s * 12 * pl;
            // P_i[m][n] = sum_l conj(A_i[l][m]) X[l][n];  R_j[m][n] = sum_l A_j[m][l] Y[l][n] (= AT_j[l][m])
            float pr[3][4] = {}, pim[3][4] = {};
            if (lane) {
                const float* Xp = sX + (size_t)fl * 2 * pl;
                const float* Yp = sY + (size_t)fl * 2 * pl;
                float rr[3][4] = {}, ri[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 xr = ld2(Xp + l * Np + n0), xi = ld2(Xp + pl + l * Np + n0);
                    const float2 yr = ld2(Yp + l * Np + n0), yi = ld2(Yp + pl + l * Np + n0);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float* Ai = A + (size_t)i * 4 * pl;
                        cmac2x2<true, false>(pr[i], pim[i], ld2(Ai + l * Np + m0), ld2(Ai + pl + l * Np + m0), xr, xi);
                        cmac2x2<false, false>(rr[i], ri[i], ld2(Ai + 2 * pl + l * Np + m0),
                                              ld2(Ai + 3 * pl + l * Np + m0), yr, yi);
                    }
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float* Rp = sR + ((size_t)fl * 3 + j) * 2 * pl;
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {  // transposed: (R[m0][n], R[m0+1][n]) at row n
                        const int o = (n0 + dn) * Np + m0;
                        st2(Rp + o, rr[j][dn], rr[j][2 + dn]);
                        st2(Rp + pl + o, ri[j][dn], ri[j][2 + dn]);
                    }
                }
            }
            __syncthreads();
            // this tile's part of C_ij = sum_{m,n} P_i[m][n] R_j[n][m] = sum_{m,n} P_i[m][n] RT_j[m][n]
            float hp[9][2];
            if (lane) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float* Rp = sR + ((size_t)fl * 3 + j) * 2 * pl;
                    float tr[4], ti[4];
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        const float2 r2 = ld2(Rp + (m0 + dm) * Np + n0), i2 = ld2(Rp + pl + (m0 + dm) * Np + n0);
                        tr[dm * 2] = r2.x;
                        tr[dm * 2 + 1] = r2.y;
                        ti[dm * 2] = i2.x;
                        ti[dm * 2 + 1] = i2.y;
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float hr = 0.f, hi = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            hr = fmaf(pr[i][q], tr[q], hr);
                            hr = fmaf(-pim[i][q], ti[q], hr);
                            hi = fmaf(pr[i][q], ti[q], hi);
                            hi = fmaf(pim[i][q], tr[q], hi);
                        }
                        hp[i * 3 + j][0] = hr;
                        hp[i * 3 + j][1] = hi;
                    }
                }
            }
            __syncthreads();  // every read of sR and sY for this bond is done
            float2* sP = reinterpret_cast<float2*>(sR);  // [F][T][9] trace parts (fit in the R_j planes)
            if (lane)
#pragma unroll
                for (int ij = 0; ij < 9; ++ij) sP[((size_t)fl * T + tt) * 9 + ij] = make_float2(hp[ij][0], hp[ij][1]);
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {  // fixed-order sums over the tile threads
                const int rf = g / 9, ij = g - rf * 9;
                float2 sum = sP[(size_t)rf * T * 9 + ij];
                for (int u = 1; u < T; ++u) {
                    const float2 v = sP[((size_t)rf * T + u) * 9 + ij];
                    sum.x += v.x;
                    sum.y += v.y;
                }
                const float2 self = make_float2(sSelf[g].x + sum.x, sSelf[g].y + sum.y);
                sSelf[g] = self;
                if (i0 + rf < i_end) {
                    const size_t ff = freq_of(fm, i0 + rf);
                    C_hat[((ff * nA + la) * slots + s) * 9 + ij] = sum;
                    if (s == d.NB - 1) C_hat[((ff * nA + la) * slots + d.NB) * 9 + ij] = self;
                }
            }
            // the next bond writes sY before its first barrier and sR (sP) only after it
        }
    }
}

// Pi^t[q][w][a][slot][ij] = -i*scale * conj(v) * inv for rows l = w+1 in [1, Nw]
template <class C>
struct StorePiT {
    double2* P;
    int Nw, NA, slots;
    size_t col0;
    double inv_scale;  // scale / (Nkz L)
    int rows;
    __device__ void operator()(int q, int r, size_t col, C v) const {
        if (r < 1 || r > Nw) return;
        const size_t rowlen = (size_t)NA * slots * 9;
        // C = conj(v) * inv; Pi = -i * scale * C, in FP64
        P[((size_t)q * Nw + (r - 1)) * rowlen + col0 + col] =
            make_double2(-(double)v.y * inv_scale, -(double)v.x * inv_scale);
    }
};
using StorePi = StorePiT<double2>;

// (P - P^H)/2 on every 3x3 block of the atoms in range
__global__ void symmetrize3_kernel(sse_dims d, double2* __restrict__ P) {
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const int slots = d.NB + 1;
    const size_t nblk = (size_t)d.Nqz * d.Nw * nA * slots;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nblk; i += (size_t)gridDim.x * blockDim.x) {
        const size_t qw = i / (nA * slots), rem = i - qw * nA * slots;
        double2* B = P + ((qw * d.NA + d.a_begin) * slots + rem) * 9;
        for (int r = 0; r < 3; ++r)
            for (int c2 = r; c2 < 3; ++c2) {
                const double2 x = B[r * 3 + c2], y = B[c2 * 3 + r];
                B[r * 3 + c2] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
                if (r != c2) B[c2 * 3 + r] = make_double2(0.5 * (y.x - x.x), 0.5 * (y.y + x.y));
            }
    }
}

// ---------------------------------------------------------------------------
// adjoint of Eq. (3) through the transforms. With W = gS^t (upstream), Z = G^H blockwise and
// N = Nkz L, Parseval and the correlation theorem give, per bond (a, s) and frequency f,
//   Q_j = W^ dH_j G^_b^H,  R_i = W^^H dH_i G^_b,
//   grad D:  H^_ij(f) = tr(dH_i^H Q_j(f)) -> H_ij(q, l) = IDFT; grad D^tau(q,w) = conj(c) [H^tau(q, w+1) +
//            H^tau'(q, -(w+1))] (emission lags of the same type, absorption lags of the other),
//   grad dH_m = (1/N) sum_f [ sum_j conj(c) conj(K^_mj(f)) Q_j(f) + sum_i c K^_im(f) R_i(f) ],
// K^ the transformed lag kernel of the forward (c = i*scale).
// ---------------------------------------------------------------------------
struct AdjCfg {
    int nel, F, threads, fchunk, nchunks;
    int off_A, off_W, off_G, off_K, off_T, off_V, off_Q, off_D, smem;
};

constexpr int kAdjMaxThreads = 320;

AdjCfg make_adj_cfg(const sse_dims& d, size_t nfreq, int tsz = 8) {
    AdjCfg c{};
    c.nel = d.Norb * d.Norb;
    const int pl = c.nel * tsz;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    // per CTA: the current bond's dH planes, then per frequency 27 plane-sized buffers and the traces
    auto smem_of = [&](int F) {
        return (long)3 * 4 * pl + F * (8 * pl + 9 * 2 * tsz + 9 * pl * 2 + 6 * pl + 9 * d.Norb * 2 * tsz) + 128;
    };
    c.F = 1;
    long best = -1;
    for (int F = 1; F * c.nel <= kAdjMaxThreads; ++F) {  // most busy lanes per SM (see pick_frequencies)
        const int threads = ((F * c.nel + 31) / 32) * 32;
        const long sm = smem_of(F);
        if (sm > 227 * 1024) break;
        long ctas = (228L * 1024) / (sm + 1024);
        ctas = ctas < 2 ? ctas : 2;  // registers: up to ~100 per thread at 2 x 320 threads
        const long useful = ctas * F * c.nel;
        if (useful > best) best = useful, c.F = F;
        (void)threads;
    }
    c.threads = ((c.F * c.nel + 31) / 32) * 32;
    c.off_A = 0;                                   // [3][4 planes: re, im, re+im, re-im] of the current bond
    c.off_W = a16(c.off_A + 3 * 4 * pl);           // [F][4 planes]
    c.off_G = a16(c.off_W + c.F * 4 * pl);         // [F][4 planes]
    c.off_K = a16(c.off_G + c.F * 4 * pl);         // [F][9] complex
    c.off_T = a16(c.off_K + c.F * 9 * 2 * tsz);    // [F][3 j][3 planes]  W^ dH_j
    c.off_V = a16(c.off_T + c.F * 9 * pl);         // [F][3 i][3 planes]  W^^H dH_i
    c.off_Q = a16(c.off_V + c.F * 9 * pl);         // [F][3 j][2 planes]
    c.off_D = a16(c.off_Q + c.F * 6 * pl);         // [F][9][Norb] complex
    c.smem = a16(c.off_D + c.F * 9 * d.Norb * 2 * tsz);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    c.nchunks = (int)((nfreq + c.fchunk - 1) / c.fchunk);
    return c;
}

template <class T, class C>
__device__ __forceinline__ void put4(T* P, int nel, int e, C v) {
    P[e] = v.x;
    P[nel + e] = v.y;
    P[2 * nel + e] = v.x + v.y;
    P[3 * nel + e] = v.x - v.y;
}

template <class T>
__global__ void __launch_bounds__(kAdjMaxThreads, 2)
spec_adj_kernel(AdjCfg c, sse_dims d, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
                const typename CX<T>::C* __restrict__ What, const typename CX<T>::C* __restrict__ Ghat,
                const typename CX<T>::C* __restrict__ Khat, typename CX<T>::C* __restrict__ Hhat,
                double2* __restrict__ gdh_part, int L, double scale, unsigned* __restrict__ status) {
    using C = typename CX<T>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nfreq = (size_t)d.Nkz * L;
    const size_t f_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t f_end = min(nfreq, f_begin + c.fchunk);
    T* sA = reinterpret_cast<T*>(smem + c.off_A);
    T* sW = reinterpret_cast<T*>(smem + c.off_W);
    T* sG = reinterpret_cast<T*>(smem + c.off_G);
    C* sK = reinterpret_cast<C*>(smem + c.off_K);
    T* sT = reinterpret_cast<T*>(smem + c.off_T);
    T* sV = reinterpret_cast<T*>(smem + c.off_V);
    T* sQ = reinterpret_cast<T*>(smem + c.off_Q);
    C* sD = reinterpret_cast<C*>(smem + c.off_D);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;
    const int ndiag = c.F * 9 * Norb;

    for (int s = 0; s < d.NB; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        const bool bok = b >= 0 && b < d.NA;
        if (!bok && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        // this bond's dH planes (the previous bond's last barrier has passed)
        for (int i = tid; i < 3 * nel; i += blockDim.x) {
            const int di = i / nel, ee = i - di * nel;
            const double2 v = dH[((size_t)a * d.NB + s) * 3 * nel + i];
            put4(sA + (size_t)di * 4 * nel, nel, ee, CT<C>::mk((T)v.x, (T)v.y));
        }
        __syncthreads();
        const T* A = sA;
        C acc[3] = {CT<C>::mk(0, 0), CT<C>::mk(0, 0), CT<C>::mk(0, 0)};
        for (size_t f0 = f_begin; f0 < f_end; f0 += c.F) {
            const size_t f = f0 + fl;
            const bool act = lane && f < f_end && bok;
            if (lane) {
                C w = CT<C>::mk(0, 0), g = CT<C>::mk(0, 0);
                if (act) {
                    w = What[(f * nA + la) * nel + e];
                    g = Ghat[(f * d.NA + b) * nel + e];
                }
                put4(sW + (size_t)fl * 4 * nel, nel, e, w);
                put4(sG + (size_t)fl * 4 * nel, nel, e, g);
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                const size_t ff = f0 + fk;
                C k = CT<C>::mk(0, 0);
                if (ff < f_end && bok) k = Khat[((ff * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            // T_j = W^ dH_j,  V_i = W^^H dH_i
            if (lane) {
                const T* Wp = sW + (size_t)fl * 4 * nel;
#pragma unroll 1
                for (int j = 0; j < 3; ++j) {
                    const T* Aj = A + (size_t)j * 4 * nel;
                    T t1 = 0, t2 = 0, t3 = 0, v1 = 0, u2 = 0, v3 = 0;
                    for (int l = 0; l < Norb; ++l) {
                        const int ml = m * Norb + l, lm = l * Norb + m, ln = l * Norb + n;
                        t1 = fma(Wp[ml], Aj[ln], t1);                  // W[m][l] A_j[l][n]
                        t2 = fma(Wp[nel + ml], Aj[nel + ln], t2);
                        t3 = fma(Wp[2 * nel + ml], Aj[2 * nel + ln], t3);
                        v1 = fma(Wp[lm], Aj[ln], v1);                  // conj(W[l][m]) A_j[l][n]
                        u2 = fma(Wp[nel + lm], Aj[nel + ln], u2);
                        v3 = fma(Wp[3 * nel + lm], Aj[2 * nel + ln], v3);
                    }
                    put3(sT + ((size_t)fl * 3 + j) * 3 * nel, nel, e, CT<C>::mk(t1 - t2, t3 - t1 - t2));
                    put3(sV + ((size_t)fl * 3 + j) * 3 * nel, nel, e, CT<C>::mk(v1 + u2, v3 - v1 + u2));
                }
            }
            __syncthreads();
            // Q_j = T_j G^^H (stored for the traces), R_i = V_i G^; grad dH accumulation
            if (lane) {
                const T* Gp = sG + (size_t)fl * 4 * nel;
                const C* K = sK + fl * 9;
#pragma unroll 1
                for (int j = 0; j < 3; ++j) {
                    const T* Tp = sT + ((size_t)fl * 3 + j) * 3 * nel;
                    const T* Vp = sV + ((size_t)fl * 3 + j) * 3 * nel;
                    T q1 = 0, q2 = 0, q3 = 0, r1 = 0, r2 = 0, r3 = 0;
                    for (int l = 0; l < Norb; ++l) {
                        const int ml = m * Norb + l, nl = n * Norb + l, ln = l * Norb + n;
                        q1 = fma(Tp[ml], Gp[nl], q1);                  // T[m][l] conj(G[n][l])
                        q2 = fma(Tp[nel + ml], Gp[nel + nl], q2);
                        q3 = fma(Tp[2 * nel + ml], Gp[3 * nel + nl], q3);
                        r1 = fma(Vp[ml], Gp[ln], r1);                  // V[m][l] G[l][n]
                        r2 = fma(Vp[nel + ml], Gp[nel + ln], r2);
                        r3 = fma(Vp[2 * nel + ml], Gp[2 * nel + ln], r3);
                    }
                    // (T conj(G^T)): re = q1 + q2, im = q3 - q1 + q2  (Gauss with (re - im) of G)
                    const C Q = CT<C>::mk(q1 + q2, q3 - q1 + q2);
                    const C R = CT<C>::mk(r1 - r2, r3 - r1 - r2);
                    T* Qs = sQ + ((size_t)fl * 3 + j) * 2 * nel;
                    Qs[e] = Q.x;
                    Qs[nel + e] = Q.y;
#pragma unroll
                    for (int mu = 0; mu < 3; ++mu) {
                        // conj(c) conj(K_mu,j) Q = -i*scale*conj(K) Q ;  c K_j,mu R = i*scale*K R
                        const C k1 = K[mu * 3 + j], k2 = K[j * 3 + mu];
                        // alpha = -i conj(k1) = (-k1.y, -k1.x);  beta = i k2 = (-k2.y, k2.x)
                        acc[mu].x = fma(-k1.y, Q.x, acc[mu].x);
                        acc[mu].x = fma(k1.x, Q.y, acc[mu].x);
                        acc[mu].y = fma(-k1.y, Q.y, acc[mu].y);
                        acc[mu].y = fma(-k1.x, Q.x, acc[mu].y);
                        acc[mu].x = fma(-k2.y, R.x, acc[mu].x);
                        acc[mu].x = fma(-k2.x, R.y, acc[mu].x);
                        acc[mu].y = fma(-k2.y, R.y, acc[mu].y);
                        acc[mu].y = fma(k2.x, R.x, acc[mu].y);
                    }
                }
            }
            __syncthreads();
            // diagonal terms sum_n conj(A_i[mm][n]) Q_j[mm][n]
            for (int g = tid; g < ndiag; g += blockDim.x) {
                const int fi = g / (9 * Norb), rem = g - fi * 9 * Norb;
                const int ij = rem / Norb, mm = rem - ij * Norb;
                const int i = ij / 3, j = ij - 3 * i;
                const T* Ai = A + (size_t)i * 4 * nel;
                const T* Qs = sQ + ((size_t)fi * 3 + j) * 2 * nel;
                T re = 0, im = 0;
                for (int nn = 0; nn < Norb; ++nn) {
                    const int o = mm * Norb + nn;
                    const T ar = Ai[o], ai = Ai[nel + o], qr = Qs[o], qi = Qs[nel + o];
                    re = fma(ar, qr, re);
                    re = fma(ai, qi, re);
                    im = fma(ar, qi, im);
                    im = fma(-ai, qr, im);
                }
                sD[g] = CT<C>::mk(re, im);
            }
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {
                const int rf = g / 9, ij = g - rf * 9;
                const size_t ff = f0 + rf;
                const C* v = sD + (size_t)g * Norb;
                C sum = v[0];
                for (int mm = 1; mm < Norb; ++mm) sum = cadd(sum, v[mm]);
                if (ff < f_end) Hhat[((ff * nA + la) * d.NB + s) * 9 + ij] = sum;
            }
            // the next batch rewrites sW, sG, sK before its first barrier (last read before the second),
            // sT, sV, sQ, sD only after it
        }
        // sum the frequency lanes' accumulators (fixed order) and write this chunk's partial
        __syncthreads();
        C* sAcc = reinterpret_cast<C*>(sT);  // [F][3][nel] complex fits in the T planes
        if (lane)
#pragma unroll
            for (int mu = 0; mu < 3; ++mu) sAcc[((size_t)fl * 3 + mu) * nel + e] = acc[mu];
        __syncthreads();
        const double inv = scale / (double)nfreq;
        for (int i = tid; i < 3 * nel; i += blockDim.x) {
            double2 sum = make_double2((double)sAcc[i].x, (double)sAcc[i].y);  // FP64 sums from here on
            for (int f2 = 1; f2 < c.F; ++f2) {
                const C v = sAcc[(size_t)f2 * 3 * nel + i];
                sum.x += (double)v.x;
                sum.y += (double)v.y;
            }
            gdh_part[(((size_t)blockIdx.y * nA + la) * d.NB + s) * 3 * nel + i] = make_double2(sum.x * inv, sum.y * inv);
        }
        __syncthreads();  // sT is rewritten by the next bond's first batch
    }
}

// ---------------------------------------------------------------------------
// FP32 gradient with respect to G (mode FP32_FFT): per target atom b and frequency, over the bonds (a, s)
// into b, P_j = W^_a A_j for the three j at once on 2 x 2 register tiles (4-multiply MACs on (re, im)
// planes), U_i = sum_j conj(K^_ij) P_j in registers, then acc += sum_i A_i^H U_i; the result is
// conj(c) acc = -i scale acc, as in spec_gradg_kernel.
// ---------------------------------------------------------------------------
struct GradG32Cfg {
    int Np, TN, T, pl, F, threads, fchunk;
    int off_A, off_W, off_K, off_U, smem;
};

GradG32Cfg make_gradg32_cfg(const sse_dims& d, size_t nfreq) {
    GradG32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    c.F = pick_frequencies(c.T, [&](int F) { return (long)6 * pb + F * (8L * pb + 9 * 8) + 64; });
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                            // [3 j][2 planes] the current bond's A_j row-major
    c.off_W = a16(c.off_A + 6 * pb);        // [F][2 planes] W^_a transposed: WT[l][m] = W^[m][l]
    c.off_K = a16(c.off_W + c.F * 2 * pb);  // [F][9] float2
    c.off_U = a16(c.off_K + c.F * 9 * 8);   // [F][3 i][2 planes] U_i row-major
    c.smem = a16(c.off_U + c.F * 6 * pb);
    // every target atom gets a CTA column: enough frequency chunks for ~8 waves of 2 CTAs per SM
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + (size_t)d.NA - 1) / (size_t)(d.NA ? d.NA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void spec_gradg32_kernel(GradG32Cfg c, sse_dims d, const int* __restrict__ off,
                                    const int* __restrict__ list, const double2* __restrict__ dH,
                                    const float2* __restrict__ What, const float2* __restrict__ Khat,
                                    float2* __restrict__ Rhat, int L, double scale) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb;
    const int b = blockIdx.x;  // target atom
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nfreq = (size_t)d.Nkz * L;
    const size_t f_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t f_end = min(nfreq, f_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sW = reinterpret_cast<float*>(smem + c.off_W);
    float2* sK = reinterpret_cast<float2*>(smem + c.off_K);
    float* sU = reinterpret_cast<float*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / c.T, tt = tid - fl * c.T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;
    const int i0 = off[b], i1 = off[b + 1];

    for (size_t f0 = f_begin; f0 < f_end; f0 += c.F) {
        const size_t f = f0 + fl;
        const bool act = lane && f < f_end;
        float accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};
        for (int ib = i0; ib < i1; ++ib) {
            const int bond = list[ib];  // (a - a_begin) * NB + s
            const int la = bond / d.NB;
            // this bond's A_j (zero-padded), W^_a(f) transposed, K^(f) of the bond
            for (int i = tid; i < 3 * pl; i += blockDim.x) {
                const int j = i / pl, e = i - j * pl;
                const int l = e / Np, n = e - l * Np;
                double2 v = make_double2(0.0, 0.0);
                if (l < Norb && n < Norb) v = dH[(((size_t)d.a_begin * d.NB + bond) * 3 + j) * nel + l * Norb + n];
                sA[(size_t)j * 2 * pl + e] = (float)v.x;
                sA[(size_t)j * 2 * pl + pl + e] = (float)v.y;
            }
            if (lane) {
                float* Wp = sW + (size_t)fl * 2 * pl;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 w = make_float2(0.f, 0.f);
                        if (act && m < Norb && n < Norb) w = What[(f * nA + la) * nel + m * Norb + n];
                        Wp[n * Np + m] = w.x;
                        Wp[pl + n * Np + m] = w.y;
                    }
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                const size_t ff = f0 + fk;
                sK[i] = ff < f_end ? Khat[(ff * nA * d.NB + bond) * 9 + ij] : make_float2(0.f, 0.f);
            }
            __syncthreads();
            // P_j = W^ A_j (three at once), U_i = sum_j conj(K_ij) P_j
            if (lane) {
                const float* Wp = sW + (size_t)fl * 2 * pl;
                float pr[3][4] = {}, pi[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 xr = ld2(Wp + l * Np + m0), xi = ld2(Wp + pl + l * Np + m0);
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        cmac2x2<false, false>(pr[j], pi[j], xr, xi, ld2(sA + (size_t)j * 2 * pl + l * Np + n0),
                                              ld2(sA + (size_t)j * 2 * pl + pl + l * Np + n0));
                }
                const float2* K = sK + fl * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float ur[4] = {0, 0, 0, 0}, ui[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 k = K[i * 3 + j];  // conj(k) P = (kx pr + ky pi, kx pi - ky pr)
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            ur[q] = fmaf(k.x, pr[j][q], ur[q]);
                            ur[q] = fmaf(k.y, pi[j][q], ur[q]);
                            ui[q] = fmaf(k.x, pi[j][q], ui[q]);
                            ui[q] = fmaf(-k.y, pr[j][q], ui[q]);
                        }
                    }
                    float* Up = sU + ((size_t)fl * 3 + i) * 2 * pl;
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        st2(Up + (m0 + dm) * Np + n0, ur[dm * 2], ur[dm * 2 + 1]);
                        st2(Up + pl + (m0 + dm) * Np + n0, ui[dm * 2], ui[dm * 2 + 1]);
                    }
                }
            }
            __syncthreads();
            // acc += sum_i A_i^H U_i: acc[m][n] += sum_l conj(A_i[l][m]) U_i[l][n]
            if (lane) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float* Ap = sA + (size_t)i * 2 * pl;
                    const float* Up = sU + ((size_t)fl * 3 + i) * 2 * pl;
                    for (int l = 0; l < Norb; ++l)
                        cmac2x2<true, false>(accr, acci, ld2(Ap + l * Np + m0), ld2(Ap + pl + l * Np + m0),
                                             ld2(Up + l * Np + n0), ld2(Up + pl + l * Np + n0));
                }
            }
            __syncthreads();  // sA, sW, sK, sU are rewritten for the next bond
        }
        if (act) {
            const float sc = (float)scale;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + q / 2, n = n0 + (q & 1);
                if (m < Norb && n < Norb)  // -i*scale*(re + i im)
                    Rhat[(f * d.NA + b) * nel + m * Norb + n] = make_float2(sc * acci[q], -sc * accr[q]);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 adjoint (mode FP32_FFT): the steps of spec_adj_kernel on 2 x 2 register tiles with 4-multiply complex
// MACs on (re, im) planes; the three T_j = W^ A_j and V_j = W^^H A_j share the W^ loads, the three
// Q_j = T_j G^^H and R_j = V_j G^ the G^ loads. Trace partials come from the Q_j tiles in registers and are
// summed over the tile threads in a fixed order; the coupling-gradient partial sums go to FP64 as in the FP64
// kernel.
// ---------------------------------------------------------------------------
struct Adj32Cfg {
    int Np, TN, T, pl, F, threads, fchunk, nchunks;
    int off_A, off_W, off_G, off_K, off_T, off_V, smem;
};

constexpr int kAdj32MaxThreads = 256;

Adj32Cfg make_adj32_cfg(const sse_dims& d, size_t nfreq) {
    Adj32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    // per CTA: the bond's 3 dH (2 planes); per frequency W^ and G^ in both layouts (8 planes), K (9 float2),
    // T_j and V_j transposed (12 planes; the trace partials reuse the T_j planes)
    auto smem_of = [&](int F) { return (long)6 * pb + F * (20L * pb + 9 * 8) + 96; };
    c.F = 1;
    long best = -1, best_sm = 0;
    for (int F = 1; F * c.T <= kAdj32MaxThreads; ++F) {
        const int threads = ((F * c.T + 31) / 32) * 32;
        const long sm = smem_of(F);
        if (sm > 227 * 1024) break;
        long ctas = (228L * 1024) / (sm + 1024);
        ctas = ctas < 2048 / threads ? ctas : 2048 / threads;
        ctas = ctas < 65536 / (threads * 128) ? ctas : 65536 / (threads * 128);  // <= 128 registers
        const long useful = ctas * F * c.T;
        if (useful > best || (useful == best && sm < best_sm)) best = useful, best_sm = sm, c.F = F;
    }
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                                  // [3 j][2 planes] A_j row-major
    c.off_W = a16(c.off_A + 6 * pb);              // [F][4 planes] W^ row-major (re, im), transposed (re, im)
    c.off_G = a16(c.off_W + c.F * 4 * pb);        // [F][4 planes] G^ likewise
    c.off_K = a16(c.off_G + c.F * 4 * pb);        // [F][9] float2
    c.off_T = a16(c.off_K + c.F * 9 * 8);         // [F][3 j][2 planes] T_j transposed
    c.off_V = a16(c.off_T + c.F * 6 * pb);        // [F][3 j][2 planes] V_j transposed
    c.smem = a16(c.off_V + c.F * 6 * pb);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    c.nchunks = (int)((nfreq + c.fchunk - 1) / c.fchunk);
    return c;
}

__global__ void __launch_bounds__(kAdj32MaxThreads, 2)
spec_adj32_kernel(Adj32Cfg c, sse_dims d, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
                  const float2* __restrict__ What, const float2* __restrict__ Ghat, const float2* __restrict__ Khat,
                  float2* __restrict__ Hhat, double2* __restrict__ gdh_part, int L, double scale,
                  unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb, T = c.T;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nfreq = (size_t)d.Nkz * L;
    const size_t f_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t f_end = min(nfreq, f_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sW = reinterpret_cast<float*>(smem + c.off_W);
    float* sG = reinterpret_cast<float*>(smem + c.off_G);
    float2* sK = reinterpret_cast<float2*>(smem + c.off_K);
    float* sT = reinterpret_cast<float*>(smem + c.off_T);
    float* sV = reinterpret_cast<float*>(smem + c.off_V);
    const int tid = threadIdx.x;
    const int fl = tid / T, tt = tid - fl * T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;

    for (int s = 0; s < d.NB; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        const bool bok = b >= 0 && b < d.NA;
        if (!bok && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        // this bond's dH planes, zero-padded to Np x Np (the previous bond's last barrier has passed)
        for (int i = tid; i < 3 * pl; i += blockDim.x) {
            const int j = i / pl, e = i - j * pl;
            const int l = e / Np, n = e - l * Np;
            double2 v = make_double2(0.0, 0.0);
            if (l < Norb && n < Norb) v = dH[(((size_t)a * d.NB + s) * 3 + j) * nel + l * Norb + n];
            sA[(size_t)j * 2 * pl + e] = (float)v.x;
            sA[(size_t)j * 2 * pl + pl + e] = (float)v.y;
        }
        float accr[3][4] = {}, acci[3][4] = {};  // grad dH_mu on the tile, this bond
        for (size_t f0 = f_begin; f0 < f_end; f0 += c.F) {
            const size_t f = f0 + fl;
            const bool act = lane && f < f_end && bok;
            // W^_a(f) and G^_b(f), both layouts, zero-padded
            if (lane) {
                float* Wp = sW + (size_t)fl * 4 * pl;
                float* Gp = sG + (size_t)fl * 4 * pl;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 w = make_float2(0.f, 0.f), g = make_float2(0.f, 0.f);
                        if (act && m < Norb && n < Norb) {
                            w = What[(f * nA + la) * nel + m * Norb + n];
                            g = Ghat[(f * d.NA + b) * nel + m * Norb + n];
                        }
                        const int o = m * Np + n, ot = n * Np + m;
                        Wp[o] = w.x;
                        Wp[pl + o] = w.y;
                        Wp[2 * pl + ot] = w.x;
                        Wp[3 * pl + ot] = w.y;
                        Gp[o] = g.x;
                        Gp[pl + o] = g.y;
                        Gp[2 * pl + ot] = g.x;
                        Gp[3 * pl + ot] = g.y;
                    }
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                const size_t ff = f0 + fk;
                float2 k = make_float2(0.f, 0.f);
                if (ff < f_end && bok) k = Khat[((ff * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            // T_j[m][n] = sum_l W^[m][l] A_j[l][n],  V_j[m][n] = sum_l conj(W^[l][m]) A_j[l][n]
            if (lane) {
                const float* Wp = sW + (size_t)fl * 4 * pl;
                float tr[3][4] = {}, ti[3][4] = {}, vr[3][4] = {}, vi[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 xr = ld2(Wp + 2 * pl + l * Np + m0), xi = ld2(Wp + 3 * pl + l * Np + m0);
                    const float2 zr = ld2(Wp + l * Np + m0), zi = ld2(Wp + pl + l * Np + m0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 ar = ld2(sA + (size_t)j * 2 * pl + l * Np + n0);
                        const float2 ai = ld2(sA + (size_t)j * 2 * pl + pl + l * Np + n0);
                        cmac2x2<false, false>(tr[j], ti[j], xr, xi, ar, ai);
                        cmac2x2<true, false>(vr[j], vi[j], zr, zi, ar, ai);
                    }
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float* Tp = sT + ((size_t)fl * 3 + j) * 2 * pl;
                    float* Vp = sV + ((size_t)fl * 3 + j) * 2 * pl;
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {  // transposed: (T[m0][n], T[m0+1][n]) at row n
                        const int o = (n0 + dn) * Np + m0;
                        st2(Tp + o, tr[j][dn], tr[j][2 + dn]);
                        st2(Tp + pl + o, ti[j][dn], ti[j][2 + dn]);
                        st2(Vp + o, vr[j][dn], vr[j][2 + dn]);
                        st2(Vp + pl + o, vi[j][dn], vi[j][2 + dn]);
                    }
                }
            }
            __syncthreads();
            // Q_j[m][n] = sum_l T_j[m][l] conj(G^[n][l]),  R_j[m][n] = sum_l V_j[m][l] G^[l][n]
            float hp[9][2];  // this tile's part of tr(A_i^H Q_j)
            if (lane) {
                const float* Gp = sG + (size_t)fl * 4 * pl;
                float qr[3][4] = {}, qi[3][4] = {}, rr[3][4] = {}, ri[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 yr = ld2(Gp + 2 * pl + l * Np + n0), yi = ld2(Gp + 3 * pl + l * Np + n0);
                    const float2 gr = ld2(Gp + l * Np + n0), gi = ld2(Gp + pl + l * Np + n0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float* Tp = sT + ((size_t)fl * 3 + j) * 2 * pl;
                        const float* Vp = sV + ((size_t)fl * 3 + j) * 2 * pl;
                        cmac2x2<false, true>(qr[j], qi[j], ld2(Tp + l * Np + m0), ld2(Tp + pl + l * Np + m0), yr, yi);
                        cmac2x2<false, false>(rr[j], ri[j], ld2(Vp + l * Np + m0), ld2(Vp + pl + l * Np + m0), gr,
                                              gi);
                    }
                }
                // grad dH_mu += sum_j -i conj(K_mu,j) Q_j + i K_j,mu R_j
                const float2* K = sK + fl * 9;
#pragma unroll
                for (int mu = 0; mu < 3; ++mu)
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 k1 = K[mu * 3 + j], k2 = K[j * 3 + mu];
                        const float alr = -k1.y, ali = -k1.x, ber = -k2.y, bei = k2.x;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            accr[mu][q] = fmaf(alr, qr[j][q], accr[mu][q]);
                            accr[mu][q] = fmaf(-ali, qi[j][q], accr[mu][q]);
                            acci[mu][q] = fmaf(alr, qi[j][q], acci[mu][q]);
                            acci[mu][q] = fmaf(ali, qr[j][q], acci[mu][q]);
                            accr[mu][q] = fmaf(ber, rr[j][q], accr[mu][q]);
                            accr[mu][q] = fmaf(-bei, ri[j][q], accr[mu][q]);
                            acci[mu][q] = fmaf(ber, ri[j][q], acci[mu][q]);
                            acci[mu][q] = fmaf(bei, rr[j][q], acci[mu][q]);
                        }
                    }
                // trace parts: sum over the tile of conj(A_i[m][n]) Q_j[m][n]
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float ar[4], ai[4];
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        const float2 r2 = ld2(sA + (size_t)i * 2 * pl + (m0 + dm) * Np + n0);
                        const float2 i2 = ld2(sA + (size_t)i * 2 * pl + pl + (m0 + dm) * Np + n0);
                        ar[dm * 2] = r2.x;
                        ar[dm * 2 + 1] = r2.y;
                        ai[dm * 2] = i2.x;
                        ai[dm * 2 + 1] = i2.y;
                    }
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        float hr = 0.f, hi = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            hr = fmaf(ar[q], qr[j][q], hr);
                            hr = fmaf(ai[q], qi[j][q], hr);
                            hi = fmaf(ar[q], qi[j][q], hi);
                            hi = fmaf(-ai[q], qr[j][q], hi);
                        }
                        hp[i * 3 + j][0] = hr;
                        hp[i * 3 + j][1] = hi;
                    }
                }
            }
            __syncthreads();  // every read of sT, sV, sG, sK, sW for this batch is done
            float2* sP = reinterpret_cast<float2*>(sT);  // [F][T][9] trace parts (fit in the T_j planes)
            if (lane)
#pragma unroll
                for (int ij = 0; ij < 9; ++ij) sP[((size_t)fl * T + tt) * 9 + ij] = make_float2(hp[ij][0], hp[ij][1]);
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {
                const int fk = g / 9, ij = g - fk * 9;
                const size_t ff = f0 + fk;
                float2 sum = sP[(size_t)fk * T * 9 + ij];
                for (int u = 1; u < T; ++u) {
                    const float2 v = sP[((size_t)fk * T + u) * 9 + ij];
                    sum.x += v.x;
                    sum.y += v.y;
                }
                if (ff < f_end) Hhat[((ff * nA + la) * d.NB + s) * 9 + ij] = sum;
            }
            // the next batch writes sW, sG, sK before its first barrier and sT (sP) only after it
        }
        // sum the frequency lanes' accumulators (fixed order, FP64) and write this chunk's partial
        __syncthreads();
        float2* sAcc = reinterpret_cast<float2*>(sT);  // [F][3][nel]
        if (lane)
#pragma unroll
            for (int mu = 0; mu < 3; ++mu)
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int m = m0 + q / 2, n = n0 + (q & 1);
                    if (m < Norb && n < Norb)
                        sAcc[((size_t)fl * 3 + mu) * nel + m * Norb + n] = make_float2(accr[mu][q], acci[mu][q]);
                }
        __syncthreads();
        const double inv = scale / (double)nfreq;
        for (int i = tid; i < 3 * nel; i += blockDim.x) {
            double2 sum = make_double2(0.0, 0.0);
            for (int f2 = 0; f2 < c.F; ++f2) {
                const float2 v = sAcc[(size_t)f2 * 3 * nel + i];
                sum.x += (double)v.x;
                sum.y += (double)v.y;
            }
            gdh_part[(((size_t)blockIdx.y * nA + la) * d.NB + s) * 3 * nel + i] = make_double2(sum.x * inv, sum.y * inv);
        }
        __syncthreads();  // sA and sT are rewritten by the next bond
    }
}

// grad dH = sum over types and frequency chunks (fixed order) of the partials
__global__ void spec_gdh_reduce_kernel(sse_dims d, int nchunks, const double2* __restrict__ part0,
                                       const double2* __restrict__ part1, double2* __restrict__ g_dH) {
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t per = (size_t)d.NB * 3 * d.Norb * d.Norb;
    const size_t total = nA * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        double2 acc = make_double2(0.0, 0.0);
        for (int t = 0; t < 2; ++t) {
            const double2* P = t == 0 ? part0 : part1;
            for (int ch = 0; ch < nchunks; ++ch) acc = cadd(acc, P[(size_t)ch * total + i]);
        }
        g_dH[(size_t)d.a_begin * per + i] = acc;
    }
}

// upstream gradient gS^t[k][E][a][mn] of atoms in range, optionally projected to (W - W^H)/2
template <class CC>
struct LoadWT {
    using C = CC;
    const double2* W;
    int NE, Norb;
    size_t rowlen, col0;
    int sym;
    __device__ C operator()(int k, int r, size_t col) const {
        if (r >= NE) return CT<C>::mk(0, 0);
        const double2* row = W + ((size_t)k * NE + r) * rowlen + col0;
        const double2 x = row[col];
        if (!sym) return CT<C>::mk(x.x, x.y);
        const int nel = Norb * Norb;
        const size_t blk = col / nel;
        const int mn = (int)(col - blk * nel), mm = mn / Norb, nn = mn - mm * Norb;
        const double2 y = row[blk * nel + nn * Norb + mm];
        return CT<C>::mk(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
    }
};
using LoadW = LoadWT<double2>;

// grad D^t (rows l = w+1) and grad D^t' (rows L-(w+1)) from the inverse transform of H^t:
// value conj(c) * conj(v) / N = (-v.y, -v.x) * scale / N
template <class C>
struct StoreGDT {
    double2* gD_same;   // D of the same type as H: emission lags
    double2* gD_other;  // the other type: absorption lags
    int Nw, L;
    size_t rowlen, col0;
    double inv_scale;
    int add;
    int rows;
    __device__ void operator()(int q, int r, size_t col, C v) const {
        double2* out;
        int w;
        if (r >= 1 && r <= Nw) {
            out = gD_same;
            w = r - 1;
        } else if (r >= L - Nw) {
            out = gD_other;
            w = L - 1 - r;
        } else {
            return;
        }
        double2* o = out + ((size_t)q * Nw + w) * rowlen + col0 + col;
        const double2 x = make_double2(-(double)v.y * inv_scale, -(double)v.x * inv_scale);
        if (add) {
            const double2 cur = *o;
            *o = make_double2(cur.x + x.x, cur.y + x.y);
        } else {
            *o = x;
        }
    }
};

// ---------------------------------------------------------------------------
// gradient with respect to G: per atom b and frequency f,
//   grad^G_b(f) = conj(c) sum over bonds (a, s) into b  sum_i dH_i^H W^_a(f) B_i,  B_i = sum_j conj(K^_ij(f)) dH_j
// (the correlation of the upstream gradient with the lag kernel), then the inverse transforms.
// Incoming bonds come from a list built on the device in (a, s) order: deterministic sums.
// ---------------------------------------------------------------------------
__global__ void inbond_count_kernel(sse_dims d, const int32_t* __restrict__ nbr, int* __restrict__ cnt,
                                    unsigned* __restrict__ status) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.NA; b += gridDim.x * blockDim.x) {
        int c = 0;
        for (int a = d.a_begin; a < d.a_end; ++a)
            for (int s = 0; s < d.NB; ++s) c += nbr[(size_t)a * d.NB + s] == b;
        cnt[b] = c;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0)
        for (size_t e = (size_t)d.a_begin * d.NB; e < (size_t)d.a_end * d.NB; ++e)
            if (nbr[e] < 0 || nbr[e] >= d.NA) atomicOr(status, DEV_BAD_NEIGHBOUR);
}

__global__ void inbond_scan_kernel(int NA, const int* __restrict__ cnt, int* __restrict__ off) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        int acc = 0;
        for (int b = 0; b < NA; ++b) {
            off[b] = acc;
            acc += cnt[b];
        }
        off[NA] = acc;
    }
}

__global__ void inbond_fill_kernel(sse_dims d, const int32_t* __restrict__ nbr, const int* __restrict__ off,
                                   int* __restrict__ list) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < d.NA; b += gridDim.x * blockDim.x) {
        int o = off[b];
        for (int a = d.a_begin; a < d.a_end; ++a)
            for (int s = 0; s < d.NB; ++s)
                if (nbr[(size_t)a * d.NB + s] == b) list[o++] = (a - d.a_begin) * d.NB + s;
    }
}

template <class T>
__global__ void spec_gradg_kernel(ProdCfg c, sse_dims d, const int* __restrict__ off, const int* __restrict__ list,
                                  const double2* __restrict__ dH, const typename CX<T>::C* __restrict__ What,
                                  const typename CX<T>::C* __restrict__ Khat, typename CX<T>::C* __restrict__ Rhat,
                                  int L, double scale) {
    using C = typename CX<T>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int b = blockIdx.x;  // target atom
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nfreq = (size_t)d.Nkz * L;
    const size_t f_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t f_end = min(nfreq, f_begin + c.fchunk);
    // region reuse of the forward's layout: A = one bond's 3 x 4 planes, G = W^ planes, W = B_i planes, U = U_i
    T* sA = reinterpret_cast<T*>(smem + c.off_A);
    T* sWa = reinterpret_cast<T*>(smem + c.off_G);
    C* sK = reinterpret_cast<C*>(smem + c.off_K);
    T* sB = reinterpret_cast<T*>(smem + c.off_W);
    T* sU = reinterpret_cast<T*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;
    const int i0 = off[b], i1 = off[b + 1];

    for (size_t f0 = f_begin; f0 < f_end; f0 += c.F) {
        const size_t f = f0 + fl;
        const bool act = lane && f < f_end;
        T T1 = 0, T2 = 0, T3 = 0;
        for (int ib = i0; ib < i1; ++ib) {
            const int bond = list[ib];  // (a - a_begin) * NB + s
            const int la = bond / d.NB;
            __syncthreads();  // previous bond done with sA, sWa, sK, sB, sU
            for (int i = tid; i < 3 * nel; i += blockDim.x) {
                const double2 v = dH[((size_t)d.a_begin * d.NB + bond) * 3 * nel + i];
                T* P = sA + (size_t)(i / nel) * 4 * nel;
                const int ee = i % nel;
                const T vr = (T)v.x, vi = (T)v.y;
                P[ee] = vr;
                P[nel + ee] = vi;
                P[2 * nel + ee] = vr + vi;
                P[3 * nel + ee] = vr - vi;
            }
            if (lane) {
                C w = CT<C>::mk(0, 0);
                if (act) w = What[(f * nA + la) * nel + e];
                put3(sWa + (size_t)fl * 3 * nel, nel, e, w);
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                const size_t ff = f0 + fk;
                sK[i] = ff < f_end ? Khat[(ff * nA * d.NB + bond) * 9 + ij] : CT<C>::mk(0, 0);
            }
            __syncthreads();
            // B_i[m][n] = sum_j conj(K_ij) A_j[m][n]
            if (lane) {
                T ar[3], ai[3];
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    ar[j] = sA[(size_t)j * 4 * nel + e];
                    ai[j] = sA[(size_t)j * 4 * nel + nel + e];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    C acc = CT<C>::mk(0, 0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const C k = sK[fl * 9 + i * 3 + j];  // conj(k) A = (kx ar + ky ai, kx ai - ky ar)
                        acc.x = fma(k.x, ar[j], acc.x);
                        acc.x = fma(k.y, ai[j], acc.x);
                        acc.y = fma(k.x, ai[j], acc.y);
                        acc.y = fma(-k.y, ar[j], acc.y);
                    }
                    put3(sB + ((size_t)fl * 3 + i) * 3 * nel, nel, e, acc);
                }
            }
            __syncthreads();
            // U_i = W^ B_i
            if (lane) {
                const T* Wp = sWa + (size_t)fl * 3 * nel;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Bp = sB + ((size_t)fl * 3 + i) * 3 * nel;
                    T t1 = 0, t2 = 0, t3 = 0;
                    for (int l = 0; l < Norb; ++l) {
                        const int ml = m * Norb + l, ln = l * Norb + n;
                        t1 = fma(Wp[ml], Bp[ln], t1);
                        t2 = fma(Wp[nel + ml], Bp[nel + ln], t2);
                        t3 = fma(Wp[2 * nel + ml], Bp[2 * nel + ln], t3);
                    }
                    put3(sU + ((size_t)fl * 3 + i) * 3 * nel, nel, e, CT<C>::mk(t1 - t2, t3 - t1 - t2));
                }
            }
            __syncthreads();
            // acc += sum_i A_i^H U_i:  A_i^H[m][l] = conj(A_i[l][m])  (Gauss with planes re, im, re - im)
            if (lane) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Ap = sA + (size_t)i * 4 * nel;
                    const T* Up = sU + ((size_t)fl * 3 + i) * 3 * nel;
                    for (int l = 0; l < Norb; ++l) {
                        const int lm = l * Norb + m, ln = l * Norb + n;
                        T1 = fma(Ap[lm], Up[ln], T1);
                        T2 = fma(Ap[nel + lm], Up[nel + ln], T2);  // enters with + (conj)
                        T3 = fma(Ap[3 * nel + lm], Up[2 * nel + ln], T3);
                    }
                }
            }
        }
        if (act) {
            // sum conj(A) U: re = T1 + T2, im = T3 - T1 + T2; times conj(c) = -i*scale
            const T re = T1 + T2, im = T3 - T1 + T2;
            Rhat[(f * d.NA + b) * nel + e] = CT<C>::mk((T)(scale * im), (T)(-scale * re));
        }
    }
}

// ---------------------------------------------------------------------------
// FP32 block products with register tiles. The FP32 pipe issues 64x the FP64 rate, so the scalar
// kernel above becomes bound by shared-memory bandwidth (two scalar loads per FMA). Here each
// thread computes a 2 x 2 tile of the (zero-padded, Np = Norb rounded up to even) block for one
// frequency, with G^ and dH stored transposed so that every operand pair is one 8-byte load:
// per reduction step 12 FMA for 6 loads. Same arithmetic as spec_prod_kernel (Gauss MACs).
// ---------------------------------------------------------------------------
struct Prod32Cfg {
    int Np, TN, T, F, threads, fchunk;
    int pl;      // floats per Np x Np plane
    int gs, us;  // floats per frequency of the G^ and U regions, padded to 16 mod 32 (see below)
    int off_A, off_G, off_K, off_U, smem;
};

// A warp holds the tile threads of two adjacent frequencies; per-frequency strides of 16 mod 32 floats put their
// rows of a plane on disjoint shared-memory banks.
inline int bank_pad16(int floats) { return floats + ((16 - floats % 32) + 32) % 32; }

// FP32 products use the 4-multiply complex MAC on (re, im) planes: with shared-memory bandwidth, not the FP32
// pipe, the limit, two planes per operand (4 loads per 16 FMAs of a 2 x 2 tile) beat the 3-multiply form's
// three planes (6 loads per 12 FMAs). U_i = G^ W_i is formed as sum_j K_ij P_j with P_j = G^ A_j^H, so the
// weight blocks W_i never pass through shared memory.
Prod32Cfg make_prod32_cfg(const sse_dims& d, size_t nfreq) {
    Prod32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;  // bytes per plane
    auto a16 = [](int x) { return (x + 15) & ~15; };
    c.gs = bank_pad16(2 * c.pl);
    c.us = bank_pad16(6 * c.pl);
    c.F = pick_frequencies(c.T, [&](int F) { return (long)d.NB * 6 * pb + F * (4L * (c.gs + c.us) + 9 * 8) + 64; });
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                                  // [NB][3 dir][2 planes] dH transposed: AT[l][m] = dH[m][l]
    c.off_G = a16(c.off_A + d.NB * 6 * pb);       // [F][gs] G^ transposed (2 planes): GT[l][m] = G^[m][l]
    c.off_K = a16(c.off_G + c.F * c.gs * 4);      // [F][9] float2
    c.off_U = a16(c.off_K + c.F * 9 * 8);         // [F][us] U_i row-major (3 i x 2 planes)
    c.smem = a16(c.off_U + c.F * c.us * 4);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void spec_prod32_kernel(Prod32Cfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr,
                                   const double2* __restrict__ dH, const float2* __restrict__ Ghat,
                                   const float2* __restrict__ Khat, float2* __restrict__ Shat, double scale,
                                   unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sG = reinterpret_cast<float*>(smem + c.off_G);
    float2* sK = reinterpret_cast<float2*>(smem + c.off_K);
    float* sU = reinterpret_cast<float*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / c.T, tt = tid - fl * c.T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;

    // dH planes, transposed and zero-padded: AT[s][dir][plane][l][m] = dH(a,s,dir)[m][l]
    for (int i = tid; i < d.NB * 3 * pl; i += blockDim.x) {
        const int sd = i / pl, e = i - sd * pl;
        const int l = e / Np, m = e - l * Np;
        double2 v = make_double2(0.0, 0.0);
        if (l < Norb && m < Norb) v = dH[((size_t)a * d.NB * 3 + sd) * nel + m * Norb + l];
        float* P = sA + (size_t)sd * 2 * pl;
        P[e] = (float)v.x;
        P[pl + e] = (float)v.y;
    }
    for (int s = 0; s < d.NB; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        if ((b < 0 || b >= d.NA) && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
    }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        float accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};  // the 2 x 2 tile of sum_s sum_i dH_i U_i
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            // G^_b(f) -> GT planes: element (m, n) goes to GT[n][m]
            if (lane) {
                float* Gp = sG + (size_t)fl * c.gs;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 g = make_float2(0.f, 0.f);
                        if (act && bok && m < Norb && n < Norb) g = Ghat[(f * d.NA + b) * nel + m * Norb + n];
                        const int o = n * Np + m;
                        Gp[o] = g.x;
                        Gp[pl + o] = g.y;
                    }
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                float2 k = make_float2(0.f, 0.f);
                if (i0 + fk < i_end && bok) k = Khat[((freq_of(fm, i0 + fk) * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            const float* A = sA + (size_t)s * 6 * pl;
            // P_j = G^ A_j^H for the three j at once: P_j[m][n] = sum_l GT[l][m] conj(AT_j[l][n]);
            // U_i = G^ W_i = sum_j K_ij P_j
            if (lane) {
                const float* Gp = sG + (size_t)fl * c.gs;
                float pr[3][4] = {}, pim[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 gr = ld2(Gp + l * Np + m0), gi = ld2(Gp + pl + l * Np + m0);
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        cmac2x2<false, true>(pr[j], pim[j], gr, gi, ld2(A + (size_t)j * 2 * pl + l * Np + n0),
                                             ld2(A + (size_t)j * 2 * pl + pl + l * Np + n0));
                }
                const float2* K = sK + fl * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float ur[4] = {0, 0, 0, 0}, ui[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 k = K[i * 3 + j];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            ur[q] = fmaf(k.x, pr[j][q], ur[q]);
                            ur[q] = fmaf(-k.y, pim[j][q], ur[q]);
                            ui[q] = fmaf(k.x, pim[j][q], ui[q]);
                            ui[q] = fmaf(k.y, pr[j][q], ui[q]);
                        }
                    }
                    float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        float* o = Up + (m0 + dm) * Np + n0;
                        st2(o, ur[dm * 2], ur[dm * 2 + 1]);
                        st2(o + pl, ui[dm * 2], ui[dm * 2 + 1]);
                    }
                }
            }
            __syncthreads();
            // acc += sum_i dH_i U_i: acc[m][n] += sum_l AT_i[l][m] U_i[l][n]
            if (lane) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float* Ap = A + (size_t)i * 2 * pl;
                    const float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
                    for (int l = 0; l < Norb; ++l) {
                        const float2 ar = ld2(Ap + l * Np + m0), ai = ld2(Ap + pl + l * Np + m0);
                        const float2 vr = ld2(Up + l * Np + n0), vi = ld2(Up + pl + l * Np + n0);
                        cmac2x2<false, false>(accr, acci, ar, ai, vr, vi);
                    }
                }
            }
            __syncthreads();  // sG, sK, sU are rewritten for the next bond
        }
        if (act) {
            const float sc = (float)scale;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + q / 2, n = n0 + (q & 1);
                if (m < Norb && n < Norb)  // i*scale*(re + i im)
                    Shat[(f * nA + la) * nel + m * Norb + n] = make_float2(-sc * acci[q], sc * accr[q]);
            }
        }
    }
}

// (S - S^H)/2 on the blocks of atoms in range
__global__ void symmetrize_kernel(sse_dims d, double2* __restrict__ S) {
    const int Norb = d.Norb, nel = Norb * Norb;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nblk = (size_t)d.Nkz * d.NE * nA;
    const size_t total = nblk * nel;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % nel);
        const size_t blk = i / nel;
        const int m = e / Norb, n = e - m * Norb;
        if (n < m) continue;
        const size_t ke = blk / nA, la = blk - ke * nA;
        double2* B = S + (ke * d.NA + d.a_begin + la) * nel;
        const double2 x = B[m * Norb + n], y = B[n * Norb + m];
        B[m * Norb + n] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
        if (m != n) B[n * Norb + m] = make_double2(0.5 * (y.x - x.x), 0.5 * (y.y + x.y));
    }
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct SpecLayout {
    int L;
    size_t off_tw, off_G, off_K, off_S, total;
};

SpecLayout spec_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    SpecLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    l.off_tw = 0;
    l.off_G = align256(l.off_tw + (size_t)l.L * 16);
    l.off_K = align256(l.off_G + spec * d.NA * nel * csz);
    l.off_S = align256(l.off_K + spec * nA * d.NB * 9 * csz);
    l.total = align256(l.off_S + spec * nA * nel * csz);
    return l;
}

unsigned grid_for(size_t work, int threads) {
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

int spectral_length(const sse_dims& d) {
    for (int L = d.NE + d.Nw;; ++L) {  // smallest 2^a 3^b: radix-4/2/3 stages only
        int m = L;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        if (m == 1) return L;
    }
}

bool spectral_supported(const sse_dims& d) {
    const int L = spectral_length(d);
    return d.Nkz <= kMaxNk && L < kFftMaxLength && make_plan(L).smem <= 227 * 1024 && d.NB <= 16 &&
           make_prod_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024;
}

size_t spectral_fwd_workspace(const sse_dims& d) { return spec_layout(d).total; }
size_t spectral_fwd32_workspace(const sse_dims& d) { return spec_layout(d, 8).total; }

namespace {
// The forward in the real type T: double (FP64_FFT) or float (FP32_FFT: FP32 transforms and block
// products on the FP32 pipe, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_fwd_t(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                           size_t ws_bytes, cudaStream_t st, const cudaEvent_t* g_ready = nullptr,
                           const cudaEvent_t* s_done = nullptr) {
    // g_ready[t]: G^t (and, for t = 0, every other input) is on the device; s_done[t]: Sigma^t is written.
    using C = typename CX<T>::C;
    const sse_dims& d = p.d;
    if (!spectral_supported(d)) return cudaErrorNotSupported;
    const SpecLayout lay = spec_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Gh = reinterpret_cast<C*>(base + lay.off_G);
    C* Kh = reinterpret_cast<C*>(base + lay.off_K);
    C* Sh = reinterpret_cast<C*>(base + lay.off_S);
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, kcols = nA * d.NB * 9, scols = nA * nel;
    cudaError_t e;
    if (nA == 0) return cudaSuccess;

    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool half = (p.flags & SSE_FLAG_ANTIHERMITIAN) != 0;
    const FreqMap fm = make_freq_map(d.Nkz, L, half);
    if (half && (p.flags & SSE_FLAG_CHECK)) {
        if (g_ready)
            for (int t = 0; t < 2; ++t)
                if ((e = cudaStreamWaitEvent(st, g_ready[t], 0)) != cudaSuccess) return e;
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nkz * d.NE * d.NA * nel, 256), 256, 0, st>>>(
                          p.G[t], (size_t)d.Nkz * d.NE * d.NA, d.Norb, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nqz * d.Nw * d.NA * d.NB * 9, 256), 256, 0, st>>>(
                          p.D[t], (size_t)d.Nqz * d.Nw * d.NA * d.NB, 3, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    const ProdCfg pc = make_prod_cfg(d, fm.count, (int)sizeof(T));
    const Prod32Cfg pc32 = make_prod32_cfg(d, fm.count);
    const bool tiled = sizeof(T) == 4;  // FP32: register-tiled kernel
    if ((e = tiled ? cudaFuncSetAttribute(spec_prod32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc32.smem)
                   : cudaFuncSetAttribute(spec_prod_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          pc.smem)) != cudaSuccess)
        return e;
    double2* S[2] = {S_less, S_greater};
    for (int t = 0; t < 2; ++t) {
        if (g_ready && (e = cudaStreamWaitEvent(st, g_ready[t], 0)) != cudaSuccess) return e;
        // 1. G^t -> G^
        e = launch_fft("fft_e_kernel(G)", plan, tw, LoadGT<C>{p.G[t], d.NE, gcols}, StoreSpecT<C>{Gh, L, gcols, L},
                       gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(G)", st,
                  dft_k_kernel<<<grid_for((size_t)L * gcols, 256), 256, 0, st>>>(Gh, d.Nkz, d.Nkz, (size_t)L * gcols, 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // 2. lag kernel -> K^
        LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
        e = launch_fft("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(K)", st,
                  dft_k_kernel<<<grid_for((size_t)L * kcols, 256), 256, 0, st>>>(Kh, d.Nkz, d.Nqz, (size_t)L * kcols, 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // 3. block products (one frequency of each (f, -f) pair with anti-Hermitian inputs, then the mirror)
        if (tiled) {
            const size_t gy = (fm.count + pc32.fchunk - 1) / pc32.fchunk;
            SSE_TIMED("spec_prod_kernel", st,
                      spec_prod32_kernel<<<dim3((unsigned)nA, (unsigned)gy), pc32.threads, pc32.smem, st>>>(
                          pc32, d, fm, p.nbr, p.dH, reinterpret_cast<const float2*>(Gh),
                          reinterpret_cast<const float2*>(Kh), reinterpret_cast<float2*>(Sh), p.scale, status));
        } else {
            const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
            SSE_TIMED("spec_prod_kernel", st,
                      spec_prod_kernel<T><<<dim3((unsigned)nA, (unsigned)gy), pc.threads, pc.smem, st>>>(
                          pc, d, fm, p.nbr, p.dH, Gh, Kh, Sh, p.scale, status));
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (half) {
            SSE_TIMED("mirror_sigma_kernel", st,
                      mirror_sigma_kernel<<<grid_for(fm.count * nA * nel, 256), 256, 0, st>>>(fm, nA, d.Norb, Sh));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // 4. inverse transforms into Sigma^t
        SSE_TIMED("dft_k_kernel(S)", st,
                  dft_k_kernel<<<grid_for((size_t)L * scols, 256), 256, 0, st>>>(Sh, d.Nkz, d.Nkz, (size_t)L * scols, 1));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const double inv = 1.0 / ((double)d.Nkz * (double)L);
        e = launch_fft("fft_e_kernel(S)", plan, tw, LoadSpecConjT<C>{Sh, L, scols},
                       StoreSigmaT<C>{S[t], d.NE, (size_t)d.NA * nel, (size_t)d.a_begin * nel, inv, d.NE}, scols,
                       d.Nkz, st);
        if (e != cudaSuccess) return e;
        if (p.flags & SSE_FLAG_SYMMETRIZE) {
            SSE_TIMED("symmetrize_kernel", st,
                      symmetrize_kernel<<<grid_for((size_t)d.Nkz * d.NE * nA * nel, 256), 256, 0, st>>>(d, S[t]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if (s_done && (e = cudaEventRecord(s_done[t], st)) != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t spectral_fwd_pipelined(const Problem& p, bool fp32, double2* S_less, double2* S_greater, unsigned* status,
                                   void* ws, size_t ws_bytes, cudaStream_t st, const cudaEvent_t g_ready[2],
                                   const cudaEvent_t s_done[2]) {
    return fp32 ? spectral_fwd_t<float>(p, S_less, S_greater, status, ws, ws_bytes, st, g_ready, s_done)
                : spectral_fwd_t<double>(p, S_less, S_greater, status, ws, ws_bytes, st, g_ready, s_done);
}

cudaError_t spectral_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                         size_t ws_bytes, cudaStream_t st) {
    return spectral_fwd_t<double>(p, S_less, S_greater, status, ws, ws_bytes, st);
}

cudaError_t spectral_fwd32(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                           size_t ws_bytes, cudaStream_t st) {
    return spectral_fwd_t<float>(p, S_less, S_greater, status, ws, ws_bytes, st);
}

struct PiLayout {
    int L;
    size_t off_tw, off_G[2], off_C[2], total;
};

PiLayout pi_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    PiLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    l.off_tw = 0;
    l.off_G[0] = align256((size_t)l.L * 16);
    l.off_G[1] = align256(l.off_G[0] + spec * d.NA * nel * csz);
    l.off_C[0] = align256(l.off_G[1] + spec * d.NA * nel * csz);
    l.off_C[1] = align256(l.off_C[0] + spec * nA * (d.NB + 1) * 9 * csz);
    l.total = align256(l.off_C[1] + spec * nA * (d.NB + 1) * 9 * csz);
    return l;
}

size_t spectral_pi_workspace(const sse_dims& d) { return pi_layout(d).total; }
size_t spectral_pi32_workspace(const sse_dims& d) { return pi_layout(d, 8).total; }

bool spectral_pi_supported(const sse_dims& d) {
    const int L = spectral_length(d);
    return d.Nkz <= kMaxNk && L < kFftMaxLength && make_plan(L).smem <= 227 * 1024 && d.NB <= 16 &&
           make_pi_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024 &&
           make_pi32_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024;
}

namespace {
// Pi in the real type T: double (FP64) or float (FP32_FFT: FP32 transforms and products, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_pi_t(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                          const double2* G_greater, double scale, uint32_t flags, double2* P_less,
                          double2* P_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    using C = typename CX<T>::C;
    constexpr bool fp32 = sizeof(T) == 4;
    if (!spectral_pi_supported(d)) return cudaErrorNotSupported;
    const PiLayout lay = pi_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Gh[2] = {reinterpret_cast<C*>(base + lay.off_G[0]), reinterpret_cast<C*>(base + lay.off_G[1])};
    C* Ch[2] = {reinterpret_cast<C*>(base + lay.off_C[0]), reinterpret_cast<C*>(base + lay.off_C[1])};
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, ccols = nA * (d.NB + 1) * 9;
    if (nA == 0) return cudaSuccess;
    cudaError_t e;
    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double2* G[2] = {G_less, G_greater};
    for (int t = 0; t < 2; ++t) {
        e = launch_fft("fft_e_kernel(G)", plan, tw, LoadGT<C>{G[t], d.NE, gcols}, StoreSpecT<C>{Gh[t], L, gcols, L},
                       gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(G)", st,
                  dft_k_kernel<<<grid_for((size_t)L * gcols, 256), 256, 0, st>>>(Gh[t], d.Nkz, d.Nkz,
                                                                                 (size_t)L * gcols, 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const bool half = (flags & SSE_FLAG_ANTIHERMITIAN) != 0;
    const FreqMap fm = make_freq_map(d.Nkz, L, half);
    if (half && (flags & SSE_FLAG_CHECK))
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nkz * d.NE * d.NA * nel, 256), 256, 0, st>>>(
                          G[t], (size_t)d.Nkz * d.NE * d.NA, d.Norb, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    if constexpr (fp32) {
        const Pi32Cfg pc = make_pi32_cfg(d, fm.count);
        if ((e = cudaFuncSetAttribute(spec_pi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc.smem)) !=
            cudaSuccess)
            return e;
        const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
        SSE_TIMED("spec_pi_kernel", st,
                  spec_pi32_kernel<<<dim3((unsigned)nA, (unsigned)gy, 2), pc.threads, pc.smem, st>>>(
                      pc, d, fm, nbr, dH, Gh[0], Gh[1], Ch[0], Ch[1], status));
    } else {
        const PiCfg pc = make_pi_cfg(d, fm.count);
        if ((e = cudaFuncSetAttribute(spec_pi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc.smem)) !=
            cudaSuccess)
            return e;
        const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
        SSE_TIMED("spec_pi_kernel", st,
                  spec_pi_kernel<<<dim3((unsigned)nA, (unsigned)gy, 2), pc.threads, pc.smem, st>>>(
                      pc, d, fm, nbr, dH, Gh[0], Gh[1], Ch[0], Ch[1], status));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (half)
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("mirror_pi_kernel", st,
                      mirror_pi_kernel<<<grid_for(fm.count * nA * (d.NB + 1) * 9, 256), 256, 0, st>>>(
                          fm, nA * (d.NB + 1), Ch[t]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    double2* P[2] = {P_less, P_greater};
    const double inv_scale = scale / ((double)d.Nkz * (double)L);
    for (int t = 0; t < 2; ++t) {
        SSE_TIMED("dft_k_kernel(C)", st,
                  dft_k_kernel<<<grid_for((size_t)L * ccols, 256), 256, 0, st>>>(Ch[t], d.Nkz, d.Nkz,
                                                                                 (size_t)L * ccols, 1));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = launch_fft("fft_e_kernel(C)", plan, tw, LoadSpecConjT<C>{Ch[t], L, ccols},
                       StorePiT<C>{P[t], d.Nw, d.NA, d.NB + 1, (size_t)d.a_begin * (d.NB + 1) * 9, inv_scale,
                                   d.Nw + 1},
                       ccols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        if (flags & SSE_FLAG_SYMMETRIZE) {
            SSE_TIMED("symmetrize3_kernel", st,
                      symmetrize3_kernel<<<grid_for((size_t)d.Nqz * d.Nw * nA * (d.NB + 1), 256), 256, 0, st>>>(
                          d, P[t]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t spectral_pi(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                        const double2* G_greater, double scale, uint32_t flags, double2* P_less, double2* P_greater,
                        unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    return spectral_pi_t<double>(d, nbr, dH, G_less, G_greater, scale, flags, P_less, P_greater, status, ws,
                                 ws_bytes, st);
}

cudaError_t spectral_pi32(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                          const double2* G_greater, double scale, uint32_t flags, double2* P_less,
                          double2* P_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    return spectral_pi_t<float>(d, nbr, dH, G_less, G_greater, scale, flags, P_less, P_greater, status, ws,
                                ws_bytes, st);
}

struct AdjLayout {
    int L;
    size_t off_tw, off_W, off_G, off_K, off_H, off_part, total;
};

AdjLayout adj_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    AdjLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    const int nchunks = csz == 8 ? make_adj32_cfg(d, spec).nchunks : make_adj_cfg(d, spec).nchunks;
    l.off_tw = 0;
    l.off_W = align256((size_t)l.L * 16);
    l.off_G = align256(l.off_W + spec * nA * nel * csz);
    l.off_K = align256(l.off_G + spec * d.NA * nel * csz);
    l.off_H = align256(l.off_K + spec * nA * d.NB * 9 * csz);
    l.off_part = align256(l.off_H + spec * nA * d.NB * 9 * csz);
    l.total = align256(l.off_part + (size_t)2 * nchunks * nA * d.NB * 3 * nel * 16);
    return l;
}

size_t spectral_bwd_workspace(const sse_dims& d) { return adj_layout(d).total; }
size_t spectral_bwd32_workspace(const sse_dims& d) { return adj_layout(d, 8).total; }

bool spectral_bwd_supported(const sse_dims& d) {
    const int L = spectral_length(d);
    return spectral_supported(d) && make_adj_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024 &&
           make_adj32_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024;
}

namespace {
// The adjoint in the real type T: double (FP64_FFT) or float (FP32_FFT: FP32 transforms and products, FP64
// partial sums of the coupling gradient and FP64 outputs).
template <class T>
cudaError_t spectral_bwd_t(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                           double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    using C = typename CX<T>::C;
    const sse_dims& d = p.d;
    if (!spectral_bwd_supported(d)) return cudaErrorNotSupported;
    const AdjLayout lay = adj_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Wh = reinterpret_cast<C*>(base + lay.off_W);
    C* Gh = reinterpret_cast<C*>(base + lay.off_G);
    C* Kh = reinterpret_cast<C*>(base + lay.off_K);
    C* Hh = reinterpret_cast<C*>(base + lay.off_H);
    double2* part = reinterpret_cast<double2*>(base + lay.off_part);
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, wcols = nA * nel, kcols = nA * d.NB * 9;
    const size_t nfreq = (size_t)d.Nkz * L;
    constexpr bool fp32 = sizeof(T) == 4;
    const AdjCfg ac = make_adj_cfg(d, nfreq, (int)sizeof(T));
    const Adj32Cfg ac32 = make_adj32_cfg(d, nfreq);
    const int nchunks = fp32 ? ac32.nchunks : ac.nchunks;
    const size_t part_one = (size_t)nchunks * nA * d.NB * 3 * nel;
    if (nA == 0) return cudaSuccess;
    cudaError_t e;
    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if constexpr (fp32)
        e = cudaFuncSetAttribute(spec_adj32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, ac32.smem);
    else
        e = cudaFuncSetAttribute(spec_adj_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, ac.smem);
    if (e != cudaSuccess) return e;
    const double2* W[2] = {gS_less, gS_greater};
    double2* gD[2] = {g_D_less, g_D_greater};
    const int sym = (p.flags & SSE_FLAG_SYMMETRIZE) ? 1 : 0;
    for (int t = 0; t < 2; ++t) {
        e = launch_fft("fft_e_kernel(W)", plan, tw,
                       LoadWT<C>{W[t], d.NE, d.Norb, (size_t)d.NA * nel, (size_t)d.a_begin * nel, sym},
                       StoreSpecT<C>{Wh, L, wcols, L}, wcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(W)", st,
                  dft_k_kernel<<<grid_for((size_t)L * wcols, 256), 256, 0, st>>>(Wh, d.Nkz, d.Nkz, (size_t)L * wcols,
                                                                                 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        e = launch_fft("fft_e_kernel(G)", plan, tw, LoadGT<C>{p.G[t], d.NE, gcols}, StoreSpecT<C>{Gh, L, gcols, L},
                       gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(G)", st,
                  dft_k_kernel<<<grid_for((size_t)L * gcols, 256), 256, 0, st>>>(Gh, d.Nkz, d.Nkz, (size_t)L * gcols,
                                                                                 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
        e = launch_fft("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(K)", st,
                  dft_k_kernel<<<grid_for((size_t)L * kcols, 256), 256, 0, st>>>(Kh, d.Nkz, d.Nqz, (size_t)L * kcols,
                                                                                 0));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if constexpr (fp32) {
            SSE_TIMED("spec_adj_kernel", st,
                      spec_adj32_kernel<<<dim3((unsigned)nA, (unsigned)ac32.nchunks), ac32.threads, ac32.smem, st>>>(
                          ac32, d, p.nbr, p.dH, Wh, Gh, Kh, Hh, part + (size_t)t * part_one, L, p.scale, status));
        } else {
            SSE_TIMED("spec_adj_kernel", st,
                      spec_adj_kernel<T><<<dim3((unsigned)nA, (unsigned)ac.nchunks), ac.threads, ac.smem, st>>>(
                          ac, d, p.nbr, p.dH, Wh, Gh, Kh, Hh, part + (size_t)t * part_one, L, p.scale, status));
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        // grad D from H^t: emission lags -> D^t, absorption lags -> D^t'
        SSE_TIMED("dft_k_kernel(H)", st,
                  dft_k_kernel<<<grid_for((size_t)L * kcols, 256), 256, 0, st>>>(Hh, d.Nkz, d.Nkz, (size_t)L * kcols,
                                                                                 1));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        StoreGDT<C> sg{gD[t], gD[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9,
                       p.scale / (double)nfreq, t, L};
        e = launch_fft("fft_e_kernel(H)", plan, tw, LoadSpecConjT<C>{Hh, L, kcols}, sg, kcols, d.Nqz, st);
        if (e != cudaSuccess) return e;
    }
    SSE_TIMED("spec_gdh_reduce_kernel", st,
              spec_gdh_reduce_kernel<<<grid_for(nA * d.NB * 3 * nel, 256), 256, 0, st>>>(d, nchunks, part,
                                                                                         part + part_one, g_dH));
    return cudaGetLastError();
}
}  // namespace

cudaError_t spectral_bwd(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                         double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                         cudaStream_t st) {
    return spectral_bwd_t<double>(p, gS_less, gS_greater, g_dH, g_D_less, g_D_greater, status, ws, ws_bytes, st);
}

cudaError_t spectral_bwd32(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                           double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                           cudaStream_t st) {
    return spectral_bwd_t<float>(p, gS_less, gS_greater, g_dH, g_D_less, g_D_greater, status, ws, ws_bytes, st);
}

struct GradGLayout {
    int L;
    size_t off_tw, off_W, off_K, off_R, off_cnt, off_off, off_list, total;
};

GradGLayout gradg_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    GradGLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    l.off_tw = 0;
    l.off_W = align256((size_t)l.L * 16);
    l.off_K = align256(l.off_W + spec * nA * nel * csz);
    l.off_R = align256(l.off_K + spec * nA * d.NB * 9 * csz);
    l.off_cnt = align256(l.off_R + spec * d.NA * nel * csz);
    l.off_off = align256(l.off_cnt + (size_t)d.NA * 4);
    l.off_list = align256(l.off_off + ((size_t)d.NA + 1) * 4);
    l.total = align256(l.off_list + nA * d.NB * 4 + 4);
    return l;
}

size_t spectral_bwd_g_workspace(const sse_dims& d) { return gradg_layout(d).total; }
size_t spectral_bwd_g32_workspace(const sse_dims& d) { return gradg_layout(d, 8).total; }

namespace {
// The gradient with respect to G in the real type T: double (FP64_FFT) or float (FP32_FFT: FP32 transforms and
// products, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_bwd_g_t(const Problem& p, const double2* gS_less, const double2* gS_greater,
                             double2* g_G_less, double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
    using C = typename CX<T>::C;
    const sse_dims& d = p.d;
    if (!spectral_supported(d)) return cudaErrorNotSupported;
    const GradGLayout lay = gradg_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Wh = reinterpret_cast<C*>(base + lay.off_W);
    C* Kh = reinterpret_cast<C*>(base + lay.off_K);
    C* Rh = reinterpret_cast<C*>(base + lay.off_R);
    int* cnt = reinterpret_cast<int*>(base + lay.off_cnt);
    int* offs = reinterpret_cast<int*>(base + lay.off_off);
    int* list = reinterpret_cast<int*>(base + lay.off_list);
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, wcols = nA * nel, kcols = nA * d.NB * 9;
    const size_t nfreq = (size_t)d.Nkz * L;
    cudaError_t e;
    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SSE_TIMED("inbond_count_kernel", st,
              inbond_count_kernel<<<grid_for(d.NA, 128), 128, 0, st>>>(d, p.nbr, cnt, status));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SSE_TIMED("inbond_scan_kernel", st, inbond_scan_kernel<<<1, 32, 0, st>>>(d.NA, cnt, offs));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SSE_TIMED("inbond_fill_kernel", st,
              inbond_fill_kernel<<<grid_for(d.NA, 128), 128, 0, st>>>(d, p.nbr, offs, list));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the product kernel's grid: every atom b (also those no bond reaches: they get zero)
    sse_dims dall = d;
    dall.a_begin = 0;
    dall.a_end = d.NA;
    dall.NB = d.NB < 2 ? 2 : d.NB;  // the A region holds one bond's 3 x 4 planes (>= 12 Norb^2 doubles)
    constexpr bool fp32 = sizeof(T) == 4;
    const ProdCfg pc = make_prod_cfg(dall, nfreq, (int)sizeof(T));
    const GradG32Cfg gc = make_gradg32_cfg(d, nfreq);
    if ((fp32 ? gc.smem : pc.smem) > 227 * 1024) return cudaErrorNotSupported;
    if constexpr (fp32)
        e = cudaFuncSetAttribute(spec_gradg32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, gc.smem);
    else
        e = cudaFuncSetAttribute(spec_gradg_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, pc.smem);
    if (e != cudaSuccess) return e;
    const double2* W[2] = {gS_less, gS_greater};
    double2* gG[2] = {g_G_less, g_G_greater};
    const int sym = (p.flags & SSE_FLAG_SYMMETRIZE) ? 1 : 0;
    for (int t = 0; t < 2; ++t) {
        if (nA > 0) {
            e = launch_fft("fft_e_kernel(W)", plan, tw,
                           LoadWT<C>{W[t], d.NE, d.Norb, (size_t)d.NA * nel, (size_t)d.a_begin * nel, sym},
                           StoreSpecT<C>{Wh, L, wcols, L}, wcols, d.Nkz, st);
            if (e != cudaSuccess) return e;
            SSE_TIMED("dft_k_kernel(W)", st,
                      dft_k_kernel<<<grid_for((size_t)L * wcols, 256), 256, 0, st>>>(Wh, d.Nkz, d.Nkz,
                                                                                     (size_t)L * wcols, 0));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
            e = launch_fft("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
            if (e != cudaSuccess) return e;
            SSE_TIMED("dft_k_kernel(K)", st,
                      dft_k_kernel<<<grid_for((size_t)L * kcols, 256), 256, 0, st>>>(Kh, d.Nkz, d.Nqz,
                                                                                     (size_t)L * kcols, 0));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        if constexpr (fp32) {
            const size_t gy = (nfreq + gc.fchunk - 1) / gc.fchunk;
            SSE_TIMED("spec_gradg_kernel", st,
                      spec_gradg32_kernel<<<dim3((unsigned)d.NA, (unsigned)gy), gc.threads, gc.smem, st>>>(
                          gc, d, offs, list, p.dH, Wh, Kh, Rh, L, p.scale));
        } else {
            const size_t gy = (nfreq + pc.fchunk - 1) / pc.fchunk;
            SSE_TIMED("spec_gradg_kernel", st,
                      spec_gradg_kernel<T><<<dim3((unsigned)d.NA, (unsigned)gy), pc.threads, pc.smem, st>>>(
                          pc, d, offs, list, p.dH, Wh, Kh, Rh, L, p.scale));
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        SSE_TIMED("dft_k_kernel(R)", st,
                  dft_k_kernel<<<grid_for((size_t)L * gcols, 256), 256, 0, st>>>(Rh, d.Nkz, d.Nkz, (size_t)L * gcols,
                                                                                 1));
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const double inv = 1.0 / ((double)d.Nkz * (double)L);
        e = launch_fft("fft_e_kernel(R)", plan, tw, LoadSpecConjT<C>{Rh, L, gcols},
                       StoreSigmaT<C>{gG[t], d.NE, gcols, 0, inv, d.NE}, gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t spectral_bwd_g(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_G_less,
                           double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    return spectral_bwd_g_t<double>(p, gS_less, gS_greater, g_G_less, g_G_greater, status, ws, ws_bytes, st);
}

cudaError_t spectral_bwd_g32(const Problem& p, const double2* gS_less, const double2* gS_greater,
                             double2* g_G_less, double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
    return spectral_bwd_g_t<float>(p, gS_less, gS_greater, g_G_less, g_G_greater, status, ws, ws_bytes, st);
}

}  // namespace sse
