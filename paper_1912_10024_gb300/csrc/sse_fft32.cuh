// Transform kernels with compile-time sizes. (1) FP32 E-direction transforms with the DFT codelets in registers,
// for the transform lengths of the stated workloads and of the small test shapes: each CTA transforms 8 adjacent
// columns of one batch, of length L = L1 * L2, as two passes over a tile in shared memory (the four-step
// factorisation of the DFT: L2 DFTs of length L1 down the stride-L2 rows, the twiddles exp(-2 pi i n2 k1 / L), then
// L1 DFTs of length L2 along contiguous rows, both in place), and stores the frequencies in natural order. Every index
// inside a codelet is a constant; the radix-4/2/3 Stockham kernel fft_e_kernel keeps every other length and the FP64
// transforms. Same loader and store interface. At the FinFET workload (L = 576) the transform of G takes 2.9 ms per
// type against 3.8 ms for fft_e_kernel (2.6 ms with the prefetching variant below), the inverse transform into
// Sigma 2.3 ms against 3.2. (2) The kz DFT of FP32 and FP64 spectra with the grid size as a template parameter.
//
// Included at the end of sse_spectral.cuh (it uses that file's loaders, stores, CT, launch_fft and SSE_TIMED).
#pragma once

#include <string.h>

#include <algorithm>
#include <type_traits>

namespace sse {
namespace {

// cos(2 pi k / n) and sin(2 pi k / n), evaluated at compile time: the angle is reduced exactly on the integers to a
// quadrant and phi in [0, pi/2), then Taylor series of 16 terms (truncation below 1e-20).
struct CxCis {
    double c, s;
};
__host__ __device__ constexpr double cx_series(double x, bool sine) {
    double term = sine ? x : 1.0, sum = term;
    for (int i = 1; i < 16; ++i) {
        const double a = sine ? 2.0 * i : 2.0 * i - 1.0;
        term *= -x * x / (a * (a + 1.0));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr CxCis cx_cis(long k, long n) {
    k %= n;
    if (k < 0) k += n;
    const long q = (4 * k) / n, r = 4 * k - q * n;  // 2 pi k / n = (pi / 2) (q + r / n)
    const double phi = 1.5707963267948966 * (double)r / (double)n;
    const double c = cx_series(phi, false), s = cx_series(phi, true);
    return q == 0 ? CxCis{c, s} : q == 1 ? CxCis{-s, c} : q == 2 ? CxCis{-c, -s} : CxCis{s, -c};
}

template <int I, int End, class F>
__device__ __forceinline__ void static_for(F&& f) {
    if constexpr (I < End) {
        f(std::integral_constant<int, I>{});
        static_for<I + 1, End>(f);
    }
}

// v * exp(-2 pi i E / N) with the angle known at compile time (multiples of pi/2 without multiplies)
template <int E, int N>
__device__ __forceinline__ float2 tw_const(float2 v) {
    constexpr int e = ((E % N) + N) % N;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (4 * e == N) {
        return make_float2(v.y, -v.x);
    } else if constexpr (2 * e == N) {
        return make_float2(-v.x, -v.y);
    } else if constexpr (4 * e == 3 * N) {
        return make_float2(-v.y, v.x);
    } else {
        constexpr CxCis w = cx_cis(e, N);
        constexpr float c = (float)w.c, s = (float)-w.s;  // exp(-2 pi i e / N) = c + i s
        return make_float2(fmaf(v.x, c, -v.y * s), fmaf(v.x, s, v.y * c));
    }
}

// In-place DFT of N values held in registers, X[k] = sum_n x[n] exp(-2 pi i n k / N), N = 2^a 3^b: direct forms for
// N <= 4, otherwise decimation in time N = R * M (R = 4, 2 or 3): the R DFTs of length M of the stride-R
// subsequences, the twiddles exp(-2 pi i r k' / N), and the M DFTs of length R that give X[k' + M q].
template <int N>
struct RegDft;
template <>
struct RegDft<1> {
    __device__ __forceinline__ static void run(float2 (&)[1]) {}
};
template <>
struct RegDft<2> {
    __device__ __forceinline__ static void run(float2 (&x)[2]) {
        const float2 a = x[0], b = x[1];
        x[0] = cadd(a, b);
        x[1] = csub(a, b);
    }
};
template <>
struct RegDft<3> {
    __device__ __forceinline__ static void run(float2 (&x)[3]) {
        constexpr float h = 0.86602540378443865f;  // sin(pi / 3)
        const float2 t = cadd(x[1], x[2]), d = csub(x[1], x[2]);
        const float2 m = make_float2(fmaf(-0.5f, t.x, x[0].x), fmaf(-0.5f, t.y, x[0].y));
        const float2 r = make_float2(h * d.y, -h * d.x);  // -i sin(pi/3) (x1 - x2)
        x[0] = cadd(x[0], t);
        x[1] = cadd(m, r);
        x[2] = csub(m, r);
    }
};
template <>
struct RegDft<4> {
    __device__ __forceinline__ static void run(float2 (&x)[4]) {
        const float2 s02 = cadd(x[0], x[2]), d02 = csub(x[0], x[2]);
        const float2 s13 = cadd(x[1], x[3]), d13 = csub(x[1], x[3]);
        const float2 md = make_float2(d13.y, -d13.x);  // -i (x1 - x3)
        x[0] = cadd(s02, s13);
        x[2] = csub(s02, s13);
        x[1] = cadd(d02, md);
        x[3] = csub(d02, md);
    }
};

template <int N>
struct RegDft {
    static constexpr int R = (N % 4 == 0) ? 4 : (N % 2 == 0) ? 2 : 3;
    static constexpr int M = N / R;
    static_assert(M * R == N && M > 1, "N = 2^a 3^b above 4");
    __device__ __forceinline__ static void run(float2 (&x)[N]) {
        float2 y[R][M];
#pragma unroll
        for (int r = 0; r < R; ++r) {
#pragma unroll
            for (int m = 0; m < M; ++m) y[r][m] = x[R * m + r];
            RegDft<M>::run(y[r]);
        }
        static_for<0, M>([&](auto kc) {
            constexpr int k = decltype(kc)::value;
            float2 z[R];
            static_for<0, R>([&](auto rc) {
                constexpr int r = decltype(rc)::value;
                z[r] = tw_const<r * k, N>(y[r][k]);
            });
            RegDft<R>::run(z);
#pragma unroll
            for (int q = 0; q < R; ++q) x[k + M * q] = z[q];
        });
    }
};

constexpr int kE4Cols = 8;        // columns per CTA: 128-byte rows of FP64 input, 64-byte rows of FP32
constexpr int kE4Threads = 256;
constexpr int kE4LoadBatch = 8;   // global loads in flight per thread while the tile is read

template <int L1, int L2>
struct E4Shape {
    static constexpr int L = L1 * L2;
    static constexpr int P = (L2 % 2 == 0) ? 1 : 0;  // a block of L2 rows padded to an odd count (banks)
    static constexpr int LP = L2 + P;
    static constexpr int SL = L1 * LP * kE4Cols;     // float2 of the tile
    static constexpr int SMEM = SL * 8 + L * 8;      // tile + twiddle table
    // CTAs per SM the register budget is sized for (occupancy, not loads per thread, sets the load throughput):
    // four (64 registers) up to L = 576, two for the 32 x 36 codelets
    static constexpr int MIN_CTAS = L <= 576 ? 4 : 2;
    // position of input row r = L2 n1 + n2, and of output frequency e = k1 + L1 k2 after the two passes
    __device__ __forceinline__ static int pos_in(int r) { return (r / L2) * LP + r % L2; }
    __device__ __forceinline__ static int pos_out(int e) { return (e % L1) * LP + e / L1; }
};

// CTA: kE4Cols adjacent columns of one batch (blockIdx.y). ld(batch, r, col) gives row r < L (zero where the loader
// pads), sv(batch, e, col, v) takes frequency rows e < sv.rows, as for fft_e_kernel.
template <int L1, int L2, class Load, class Store>
__global__ void __launch_bounds__(kE4Threads, E4Shape<L1, L2>::MIN_CTAS)
    fft_e4_kernel(const double2* __restrict__ tw_g, Load ld, Store sv, size_t ncols) {
    using S = E4Shape<L1, L2>;
    constexpr int CC = kE4Cols, L = S::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);  // [L1][LP][CC]
    float2* tw = X + S::SL;                          // [L] exp(-2 pi i m / L)
    const int tid = threadIdx.x, nt = blockDim.x, batch = blockIdx.y;
    const size_t col0 = (size_t)blockIdx.x * CC;
    for (int m = tid; m < L; m += nt) tw[m] = make_float2((float)tw_g[m].x, (float)tw_g[m].y);
    // 1. the tile, kE4LoadBatch loads in flight per thread
    constexpr int total = L * CC;
    for (int b0 = tid; b0 < total; b0 += kE4LoadBatch * nt) {
        float2 v[kE4LoadBatch];
#pragma unroll
        for (int u = 0; u < kE4LoadBatch; ++u) {
            const int i = b0 + u * nt, c = i % CC, r = i / CC;
            v[u] = (i < total && col0 + c < ncols) ? ld(batch, r, col0 + c) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < kE4LoadBatch; ++u) {
            const int i = b0 + u * nt;
            if (i < total) X[S::pos_in(i / CC) * CC + i % CC] = v[u];
        }
    }
    __syncthreads();
    // 2. L2 DFTs of length L1 per column (rows L2 n1 + n2, n1 = 0 .. L1-1), twiddled by w_L^(n2 k1), in place
    for (int t = tid; t < CC * L2; t += nt) {
        const int c = t % CC, n2 = t / CC;
        float2* p = X + n2 * CC + c;
        float2 x[L1];
#pragma unroll
        for (int n1 = 0; n1 < L1; ++n1) x[n1] = p[n1 * S::LP * CC];
        RegDft<L1>::run(x);
#pragma unroll
        for (int k1 = 1; k1 < L1; ++k1) x[k1] = cmul(x[k1], tw[n2 * k1]);
#pragma unroll
        for (int k1 = 0; k1 < L1; ++k1) p[k1 * S::LP * CC] = x[k1];
    }
    __syncthreads();
    // 3. L1 DFTs of length L2 along each block of contiguous rows, in place: position L2 k1 + k2 then holds the
    //    frequency k1 + L1 k2
    for (int t = tid; t < CC * L1; t += nt) {
        const int c = t % CC, k1 = t / CC;
        float2* p = X + k1 * S::LP * CC + c;
        float2 x[L2];
#pragma unroll
        for (int n2 = 0; n2 < L2; ++n2) x[n2] = p[n2 * CC];
        RegDft<L2>::run(x);
#pragma unroll
        for (int k2 = 0; k2 < L2; ++k2) p[k2 * CC] = x[k2];
    }
    __syncthreads();
    // 4. frequencies in natural order
    for (int t = tid; t < sv.rows * CC; t += nt) {
        const int c = t % CC, e = t / CC;
        if (col0 + c < ncols) sv(batch, e, col0 + c, X[S::pos_out(e) * CC + c]);
    }
}

template <int L1, int L2, class Load, class Store>
cudaError_t launch_e4_t(const char* name, const double2* tw, Load ld, Store sv, size_t ncols, int batches,
                        cudaStream_t st) {
    using S = E4Shape<L1, L2>;
    cudaError_t e =
        cudaFuncSetAttribute(fft_e4_kernel<L1, L2, Load, Store>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
    if (e != cudaSuccess) return e;
    const size_t gx = (ncols + kE4Cols - 1) / kE4Cols;
    if (gx == 0 || batches == 0) return cudaSuccess;
    if (gx > 0x7fffffffu || batches > 65535) return cudaErrorInvalidValue;
    SSE_TIMED(name, st,
              fft_e4_kernel<L1, L2, Load, Store><<<dim3((unsigned)gx, (unsigned)batches), kE4Threads, S::SMEM, st>>>(
                  tw, ld, sv, ncols));
    return cudaGetLastError();
}

// profile labels of the register-codelet kernels (plain, prefetching) for a transform the drivers name
// "fft_e_kernel(X)"
inline const char* e4_label(const char* name, bool prefetch) {
    static const char* const labels[][3] = {
        {"fft_e_kernel(G)", "fft_e4_kernel(G)", "fft_e4p_kernel(G)"},
        {"fft_e_kernel(K)", "fft_e4_kernel(K)", "fft_e4p_kernel(K)"},
        {"fft_e_kernel(S)", "fft_e4_kernel(S)", "fft_e4p_kernel(S)"},
        {"fft_e_kernel(W)", "fft_e4_kernel(W)", "fft_e4p_kernel(W)"},
        {"fft_e_kernel(H)", "fft_e4_kernel(H)", "fft_e4p_kernel(H)"},
        {"fft_e_kernel(R)", "fft_e4_kernel(R)", "fft_e4p_kernel(R)"},
        {"fft_e_kernel(C)", "fft_e4_kernel(C)", "fft_e4p_kernel(C)"}};
    for (const auto& l : labels)
        if (strcmp(l[0], name) == 0) return l[prefetch ? 2 : 1];
    return name;
}

// The same transform in a persistent CTA that copies the next tile into a raw staging buffer (cp.async, the
// loader's own element type) while it transforms the current one, for loaders that read one global element per
// (batch, row, column): the tile's loads are no longer a wait between the CTA's compute phases.
constexpr int kE4pSmemMax = 113 * 1024;

template <class T, class = void>
struct HasRawSrc : std::false_type {};
template <class T>
struct HasRawSrc<T, std::void_t<typename T::Raw>> : std::true_type {};
template <class T, bool = HasRawSrc<T>::value>
struct HasRawSrcType {
    using type = char;
};
template <class T>
struct HasRawSrcType<T, true> {
    using type = typename T::Raw;
};

// asynchronous copy of one 8- or 16-byte element global -> shared; with ok false the destination is zero-filled and
// nothing is read
template <int B>
__device__ __forceinline__ void cp_async_elem(uint32_t dst, const void* src, bool ok) {
    static_assert(B == 8 || B == 16, "8- or 16-byte elements");
    if constexpr (B == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(ok ? 8 : 0) : "memory");
}

template <int L1, int L2, class Load>
size_t e4p_smem(const Load& ld) {
    return (size_t)E4Shape<L1, L2>::SMEM + (size_t)ld.src_rows() * kE4Cols * sizeof(typename Load::Raw);
}

template <int L1, int L2, class Load, class Store>
__global__ void __launch_bounds__(kE4Threads, 2)
    fft_e4p_kernel(const double2* __restrict__ tw_g, Load ld, Store sv, size_t ncols, int gx, int ntiles) {
    using S = E4Shape<L1, L2>;
    using Raw = typename Load::Raw;
    constexpr int CC = kE4Cols, L = S::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float2* X = reinterpret_cast<float2*>(smem_raw);  // [L1][LP][CC]
    float2* tw = X + S::SL;                          // [L]
    Raw* raw = reinterpret_cast<Raw*>(tw + L);       // [rows][CC]: the next tile as stored (16-byte aligned: L even)
    const int tid = threadIdx.x, nt = blockDim.x;
    const int rows = ld.src_rows();
    const uint32_t raw_s = (uint32_t)__cvta_generic_to_shared(raw);
    auto issue = [&](int tile) {
        const int batch = tile / gx;
        const size_t col0 = (size_t)(tile % gx) * CC;
        for (int i = tid; i < rows * CC; i += nt) {
            const int c = i % CC, r = i / CC;
            const bool ok = col0 + c < ncols;
            cp_async_elem<(int)sizeof(Raw)>(raw_s + (uint32_t)(i * (int)sizeof(Raw)),
                                           ld.src(ok ? batch : 0, ok ? r : 0, ok ? col0 + c : 0), ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    for (int m = tid; m < L; m += nt) tw[m] = make_float2((float)tw_g[m].x, (float)tw_g[m].y);
    if ((int)blockIdx.x < ntiles) issue(blockIdx.x);
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int batch = tile / gx;
        const size_t col0 = (size_t)(tile % gx) * CC;
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();  // the raw tile has landed for every thread; the previous tile's store has read X
        for (int i = tid; i < L * CC; i += nt) {
            const int r = i / CC;
            X[S::pos_in(r) * CC + i % CC] = r < rows ? Load::cvt(raw[i]) : make_float2(0.f, 0.f);
        }
        __syncthreads();  // the raw buffer is free
        if (tile + (int)gridDim.x < ntiles) issue(tile + gridDim.x);
        for (int t = tid; t < CC * L2; t += nt) {
            const int c = t % CC, n2 = t / CC;
            float2* p = X + n2 * CC + c;
            float2 x[L1];
#pragma unroll
            for (int n1 = 0; n1 < L1; ++n1) x[n1] = p[n1 * S::LP * CC];
            RegDft<L1>::run(x);
#pragma unroll
            for (int k1 = 1; k1 < L1; ++k1) x[k1] = cmul(x[k1], tw[n2 * k1]);
#pragma unroll
            for (int k1 = 0; k1 < L1; ++k1) p[k1 * S::LP * CC] = x[k1];
        }
        __syncthreads();
        for (int t = tid; t < CC * L1; t += nt) {
            const int c = t % CC, k1 = t / CC;
            float2* p = X + k1 * S::LP * CC + c;
            float2 x[L2];
#pragma unroll
            for (int n2 = 0; n2 < L2; ++n2) x[n2] = p[n2 * CC];
            RegDft<L2>::run(x);
#pragma unroll
            for (int k2 = 0; k2 < L2; ++k2) p[k2 * CC] = x[k2];
        }
        __syncthreads();
        for (int t = tid; t < sv.rows * CC; t += nt) {
            const int c = t % CC, e = t / CC;
            if (col0 + c < ncols) sv(batch, e, col0 + c, X[S::pos_out(e) * CC + c]);
        }
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
}

template <int L1, int L2, class Load, class Store>
cudaError_t launch_e4p_t(const char* name, const double2* tw, Load ld, Store sv, size_t ncols, int batches,
                         cudaStream_t st) {
    const size_t smem = e4p_smem<L1, L2>(ld);
    auto kern = fft_e4p_kernel<L1, L2, Load, Store>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const size_t gx = (ncols + kE4Cols - 1) / kE4Cols;
    if (gx == 0 || batches == 0) return cudaSuccess;
    if (gx * (size_t)batches > 0x7fffffffu) return cudaErrorInvalidValue;
    const int ntiles = (int)(gx * (size_t)batches);
    int dev = 0, nsm = 0, per_sm = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kE4Threads, smem)) != cudaSuccess) return e;
    const int grid = std::min(ntiles, std::max(1, per_sm) * nsm);
    SSE_TIMED(name, st, kern<<<grid, kE4Threads, smem, st>>>(tw, ld, sv, ncols, (int)gx, ntiles));
    return cudaGetLastError();
}

// The prefetching kernel for FP64 input tiles (G: 16-byte elements, the larger share of the transform's traffic)
// where the staging buffer fits; fft_e4_kernel otherwise. Measured at FinFET (L = 576), per step of two types: the
// transform of G 5.81 -> 5.27 ms with the prefetch; the inverse transform into Sigma (FP32 spectrum in, 8-byte
// elements) 4.62 -> 5.05 ms with it (two CTAs per SM instead of four), so it keeps fft_e4_kernel.
template <int L1, int L2, class Load, class Store>
cudaError_t launch_e4_any(const char* name, const double2* tw, Load ld, Store sv, size_t ncols, int batches,
                          cudaStream_t st) {
    if constexpr (HasRawSrc<Load>::value && sizeof(typename HasRawSrcType<Load>::type) == 16) {
        if (e4p_smem<L1, L2>(ld) <= (size_t)kE4pSmemMax)
            return launch_e4p_t<L1, L2>(e4_label(name, true), tw, ld, sv, ncols, batches, st);
    }
    return launch_e4_t<L1, L2>(e4_label(name, false), tw, ld, sv, ncols, batches, st);
}


// FP32 E-transforms at the lengths with an instantiation (those of the stated workloads and of the small test
// shapes); every other length, and the FP64 transforms, take fft_e_kernel.
template <class Load, class Store>
cudaError_t launch_fft32(const char* name, const FftPlan& p, const double2* tw, Load ld, Store sv, size_t ncols,
                         int batches, cudaStream_t st) {
    if constexpr (std::is_same<typename Load::C, float2>::value) {
        switch (p.L) {
            case 36: return launch_e4_any<6, 6>(name, tw, ld, sv, ncols, batches, st);
            case 54: return launch_e4_any<6, 9>(name, tw, ld, sv, ncols, batches, st);
            case 288: return launch_e4_any<16, 18>(name, tw, ld, sv, ncols, batches, st);
            case 576: return launch_e4_any<24, 24>(name, tw, ld, sv, ncols, batches, st);
            case 1152: return launch_e4_any<32, 36>(name, tw, ld, sv, ncols, batches, st);
            default: break;
        }
    }
    return launch_fft(name, p, tw, ld, sv, ncols, batches, st);
}

// kz-direction DFT with the grid size Nk as a template parameter (FP32 and FP64 spectra), in place on X[Nk][M]:
// out[kappa] = sum_{k < n_in} x_k exp(-+2 pi i k kappa / Nk), one column m per thread, the column in registers and
// the cosines and sines compile-time constants. Inputs k and Nk - k are paired (p = x_k + x_{Nk-k},
// q = x_k - x_{Nk-k}) and so are outputs kappa and Nk - kappa: out[kappa] = C -+ i S, out[Nk - kappa] = C +- i S
// with C = x_0 (+ (-1)^kappa x_{Nk/2}) + sum_k p_k cos(2 pi k kappa / Nk), S = sum_k q_k sin(2 pi k kappa / Nk).
template <class C, int NK>
__global__ void __launch_bounds__(256) dft_kz_kernel(C* __restrict__ X, int n_in, size_t M, int inverse) {
    using R = typename CT<C>::R;
    constexpr int H = (NK - 1) / 2;  // (k, NK - k) pairs
    constexpr bool EVEN = NK % 2 == 0;
    const R sgn = inverse ? (R)1 : (R)-1;
    for (size_t m = blockIdx.x * (size_t)blockDim.x + threadIdx.x; m < M; m += (size_t)gridDim.x * blockDim.x) {
        C x[NK];
#pragma unroll
        for (int k = 0; k < NK; ++k) x[k] = k < n_in ? X[(size_t)k * M + m] : CT<C>::mk(0, 0);
        C p[H + 1], q[H + 1];
        C c0 = x[0];
#pragma unroll
        for (int k = 1; k <= H; ++k) {
            p[k] = cadd(x[k], x[NK - k]);
            q[k] = csub(x[k], x[NK - k]);
            c0 = cadd(c0, p[k]);
        }
        const C xh = EVEN ? x[NK / 2] : CT<C>::mk(0, 0);
        X[m] = cadd(c0, xh);
        static_for<1, H + 1>([&](auto kc) {
            constexpr int kap = decltype(kc)::value;
            C Cs = x[0], Sn = CT<C>::mk(0, 0);
            static_for<1, H + 1>([&](auto jc) {
                constexpr int k = decltype(jc)::value;
                constexpr CxCis w = cx_cis((long)k * kap, NK);
                Cs.x = fma(p[k].x, (R)w.c, Cs.x);
                Cs.y = fma(p[k].y, (R)w.c, Cs.y);
                Sn.x = fma(q[k].x, (R)w.s, Sn.x);
                Sn.y = fma(q[k].y, (R)w.s, Sn.y);
            });
            if constexpr (EVEN) {
                constexpr R e = (kap & 1) ? (R)-1 : (R)1;
                Cs.x = fma(e, xh.x, Cs.x);
                Cs.y = fma(e, xh.y, Cs.y);
            }
            X[(size_t)kap * M + m] = CT<C>::mk(Cs.x - sgn * Sn.y, Cs.y + sgn * Sn.x);
            X[(size_t)(NK - kap) * M + m] = CT<C>::mk(Cs.x + sgn * Sn.y, Cs.y - sgn * Sn.x);
        });
        if constexpr (EVEN && NK > 1) {  // kappa = NK/2: cos(pi k) = (-1)^k, sin = 0
            C Cs = x[0];
#pragma unroll
            for (int k = 1; k <= H; ++k) {
                const R e = (k & 1) ? (R)-1 : (R)1;
                Cs.x = fma(e, p[k].x, Cs.x);
                Cs.y = fma(e, p[k].y, Cs.y);
            }
            constexpr R e = ((NK / 2) & 1) ? (R)-1 : (R)1;
            X[(size_t)(NK / 2) * M + m] = CT<C>::mk(fma(e, xh.x, Cs.x), fma(e, xh.y, Cs.y));
        }
    }
}

template <class C, int NK>
cudaError_t launch_dft_kz_t(const char* name, C* X, int n_in, size_t M, int inverse, cudaStream_t st) {
    SSE_TIMED(name, st, dft_kz_kernel<C, NK><<<grid_for(M, 256), 256, 0, st>>>(X, n_in, M, inverse));
    return cudaGetLastError();
}

// the kz DFT of a spectrum: the compile-time kernel for Nk = 1 .. kMaxNk
template <class C>
cudaError_t launch_dft_k(const char* name, C* X, int Nk, int n_in, size_t M, int inverse, cudaStream_t st) {
    if (M == 0) return cudaSuccess;
    switch (Nk) {
        case 1: return launch_dft_kz_t<C, 1>(name, X, n_in, M, inverse, st);
        case 2: return launch_dft_kz_t<C, 2>(name, X, n_in, M, inverse, st);
        case 3: return launch_dft_kz_t<C, 3>(name, X, n_in, M, inverse, st);
        case 4: return launch_dft_kz_t<C, 4>(name, X, n_in, M, inverse, st);
        case 5: return launch_dft_kz_t<C, 5>(name, X, n_in, M, inverse, st);
        case 6: return launch_dft_kz_t<C, 6>(name, X, n_in, M, inverse, st);
        case 7: return launch_dft_kz_t<C, 7>(name, X, n_in, M, inverse, st);
        case 8: return launch_dft_kz_t<C, 8>(name, X, n_in, M, inverse, st);
        case 9: return launch_dft_kz_t<C, 9>(name, X, n_in, M, inverse, st);
        case 10: return launch_dft_kz_t<C, 10>(name, X, n_in, M, inverse, st);
        case 11: return launch_dft_kz_t<C, 11>(name, X, n_in, M, inverse, st);
        case 12: return launch_dft_kz_t<C, 12>(name, X, n_in, M, inverse, st);
        case 13: return launch_dft_kz_t<C, 13>(name, X, n_in, M, inverse, st);
        case 14: return launch_dft_kz_t<C, 14>(name, X, n_in, M, inverse, st);
        case 15: return launch_dft_kz_t<C, 15>(name, X, n_in, M, inverse, st);
        case 16: return launch_dft_kz_t<C, 16>(name, X, n_in, M, inverse, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace
}  // namespace sse
