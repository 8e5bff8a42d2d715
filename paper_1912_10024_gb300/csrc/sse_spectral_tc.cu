// Per-frequency block products of the transform-based forward of Eq. (3) on the tcgen05 tensor cores
// (mode F16X3_FFT): the paper's mixed precision (Sec. 4.4: FP16 tensor-core products of split-complex operands with
// normalisation factors, wider accumulation) applied to the convolution-theorem form of the sum.
//
// Per atom a, bond s (b = nbr[a][s]) and frequency f the forward needs (Sec. 2, Eq. 3 after the transforms)
//
//   P_j(f) = G^_b(f) dH_j^H                      j = 0..2      (right products: a GEMM over stacked f)
//   U_i(f) = sum_j K^_ij(a,s,f) P_j(f)           i = 0..2      (per-frequency weights: CUDA cores)
//   S^(f) += sum_i dH_i U_i(f)                                  (left products: a GEMM over stacked f, transposed)
//
// dH_j is shared by every frequency of the bond, so stacking frequencies into the M dimension turns both products
// into dense GEMMs with a shared B operand:
//   GEMM1: rows (f, m) of G^_b(f), K = (l, re/im), N = (j, n, re/im):          D1 = [G^] x [dH_j^H]  (real embedding)
//   GEMM2: rows (f, n) of U_i(f)^T, K = (m, i, re/im), N = (m', re/im):         D2 = [U^T] x [dH_i^T] = S^(f)^T
// A 128-row tile holds four 32-row groups of FG = 32 / Norb frequencies each (12 frequencies at Norb = 10), so that
// every frequency's rows lie in one warp's TMEM lane quarter.
//
// Precision: every operand x is scaled by a power of two (per 32-row group for the frequency-stacked operands, per
// bond for dH; exact, undone in the epilogue) and split into FP16 hi = fp16(x), lo = fp16(x - hi); each GEMM runs
// as hi x [B_hi | B_lo] (one MMA with N doubled) + lo x B_hi, so one FP32 accumulation holds hi*hi + lo*hi and
// another hi*lo (lo*lo, ~2^-22 relative, is dropped). The result carries about 22 significant bits, the level of
// the FP32 transforms around it.
//
// Roles (one persistent CTA per SM, 13 warps):
//   warps 0-7   epilogue: two warps per TMEM lane quarter, each half of the columns. Per bond: P from TMEM, the
//               K^ combination, the group scale, the split, and U^T into shared memory (GEMM2's A operand). Per
//               tile: S^ from the bonds' GEMM2 accumulators, unscaled, summed, times i*scale, to the spectrum.
//   warps 8-11  producers: G^ rows of one 32-row group each (load, scale, split, store GEMM1's A operand); per work
//               item the dH operands of all bonds of the atom (GEMM1's and GEMM2's B).
//   warp 12     TMEM allocation and the MMA issuer (one thread).
// Work item = (frequency-tile group, atom) with the atom fastest, so the CTAs running at one time read the spectra of
// neighbouring atoms for the same frequencies (L2 reuse). Every mbarrier wait is bounded as in the direct
// tensor-core kernel: a wait that gives up sets the timeout status bit, later waits return at once, and the MMA
// thread waits (bounded) for its own MMAs before TMEM is released.
#include <cuda_fp16.h>

#include "sse_spectral.cuh"
#include "sse_tcgen05.cuh"

namespace sse {
namespace {

constexpr int kTcEpiWarps = 8, kTcProdWarps = 4;
constexpr int kTcThreads = (kTcEpiWarps + kTcProdWarps + 1) * 32;
constexpr int kTcMmaWarp = kTcEpiWarps + kTcProdWarps;
constexpr int kTcProd0 = kTcEpiWarps * 32;  // first producer thread
constexpr int kTcMaxNB = 4;                 // GEMM2 accumulators: one TMEM slot per bond
constexpr int kTcTilesPerItem = 8;          // frequency tiles per work item (the dH operands are staged per item)
constexpr int kTcExpTarget = 13;            // scaled operands have max |x| in [2^13, 2^14): FP16 holds up to 65504

template <int NORB>
struct TcShape {
    static constexpr int FG = 32 / NORB;                    // frequencies per 32-row group
    static constexpr int FT = 4 * FG;                       // frequencies per 128-row tile
    static constexpr int R = FG * NORB;                     // used rows per group
    static constexpr int CD = (NORB + 3) / 4;               // 16-B chunks of one G^ row (4 complex each)
    static constexpr int K1 = (2 * NORB + 15) / 16 * 16;    // GEMM1 K (fp16 elements)
    static constexpr int C1 = K1 / 8;                       // 16-B K chunks of GEMM1's operands
    static constexpr int N1 = (6 * NORB + 15) / 16 * 16;    // GEMM1 N of one part (hi or lo of dH)
    static constexpr int C2 = (NORB + 1) / 2 * 2;           // GEMM2 K chunks: one per m (8 fp16), even
    static constexpr int K2 = 8 * C2;
    static constexpr int N2 = (2 * NORB + 15) / 16 * 16;    // GEMM2 N of one part
    static constexpr int NH = (NORB + 1) / 2;               // columns n (or m') per epilogue half
    static constexpr int LA1 = 128 * 16;                    // A1 K-chunk stride (rows contiguous, 16 B each)
    static constexpr int LA2 = 128 * 16 + 16;               // A2 K-chunk stride: +16 B spreads the chunk planes
                                                            // over the banks for the epilogue's transposed stores
    static constexpr int LB1 = 2 * N1 * 16, LB2 = 2 * N2 * 16;
    static constexpr int A1_PLANE = C1 * LA1, A1_STAGE = 2 * A1_PLANE;
    static constexpr int A2_PLANE = C2 * LA2, A2_STAGE = 2 * A2_PLANE;
    static constexpr int B1_BOND = C1 * LB1, B2_BOND = C2 * LB2;
    static constexpr int TM_P = 2 * N1;                     // TMEM columns per P buffer (two)
    static constexpr int TM_O = 2 * N2;                     // TMEM columns per bond accumulator
};

// Barriers (8 B each) after the operand buffers.
enum { BA1F = 0, BA1E = 2, BPF = 4, BPE = 6, BA2F = 8, BA2E = 10, BXE = 12, BOF = 14, BBF = 15, BBE = 16, BMD = 17,
       kTcBars = 18 };

struct TcCfg {
    int NB, nA, ntiles, ngroups, nitems;
    int off_A1, off_A2, off_B1, off_B2, off_bar, off_x, smem, tmem_cols;
};

template <int NORB>
TcCfg make_tc_cfg(const sse_dims& d, size_t nfreq) {
    using S = TcShape<NORB>;
    TcCfg c{};
    c.NB = d.NB;
    c.nA = d.a_end - d.a_begin;
    c.ntiles = (int)((nfreq + S::FT - 1) / S::FT);
    c.ngroups = (c.ntiles + kTcTilesPerItem - 1) / kTcTilesPerItem;
    c.nitems = c.ngroups * c.nA;
    c.off_A1 = 0;
    c.off_A2 = c.off_A1 + 2 * S::A1_STAGE;
    c.off_B1 = c.off_A2 + 2 * S::A2_STAGE;
    c.off_B2 = c.off_B1 + d.NB * S::B1_BOND;
    c.off_bar = c.off_B2 + d.NB * S::B2_BOND;
    c.off_x = c.off_bar + kTcBars * 8;
    // exchange area: exponent ring [2][8] int, bond exponents [16] int, producer maxima [4] float,
    // epilogue pair maxima [2][4][2] float, TMEM base, abort flag
    c.smem = c.off_x + (16 + 16 + 4 + 16 + 2) * 4;
    const int cols = 2 * S::TM_P + d.NB * S::TM_O;
    c.tmem_cols = cols <= 32 ? 32 : cols <= 64 ? 64 : cols <= 128 ? 128 : cols <= 256 ? 256 : 512;
    return c;
}

__device__ __forceinline__ uint32_t tc_idesc_f16(int n) {
    // kind::f16: F32 accumulator, F16 A and B, both K-major, M = 128
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void umma_f16(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                 ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

// tcgen05.ld of N consecutive 32-bit columns (N = 2, 4, 8) of this warp's lane quarter; no wait.
template <int N>
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, float* v) {
    uint32_t r[8];
    if (N == 8)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(taddr));
    else if (N == 4)
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                     : "r"(taddr));
    else
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0,%1}, [%2];" : "=r"(r[0]), "=r"(r[1]) : "r"(taddr));
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = __uint_as_float(r[i]);
}

// 2*NH consecutive columns (NH <= 5: 10 = 8 + 2, 8, 6 = 4 + 2, 4, 2).
template <int NH>
__device__ __forceinline__ void tmem_ld_half(uint32_t taddr, float* v) {
    constexpr int n = 2 * NH;
    if (n >= 8) {
        tmem_ld_cols<8>(taddr, v);
        if (n == 10) tmem_ld_cols<2>(taddr + 8, v + 8);
    } else if (n >= 4) {
        tmem_ld_cols<4>(taddr, v);
        if (n == 6) tmem_ld_cols<2>(taddr + 4, v + 4);
    } else {
        tmem_ld_cols<2>(taddr, v);
    }
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ float warp_max_abs(float m) {  // max over the warp of non-negative values
    return __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(m)));
}

// Exponent e that brings max |x| into [2^13, 2^14); 0 for an all-zero (or non-finite) group.
__device__ __forceinline__ int scale_exp(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    return kTcExpTarget - floor_log2(m);
}
// x * 2^e for |e| <= 252 (two exact power-of-two factors, each a normal float).
__device__ __forceinline__ float mul_pow2(float x, int e) {
    const int e1 = max(-126, min(127, e));
    const int e2 = max(-126, min(127, e - e1));
    return x * __int_as_float((e1 + 127) << 23) * __int_as_float((e2 + 127) << 23);
}

// (a, b) -> packed fp16 pairs hi = fp16(.), lo = fp16(. - hi); element a in the low half (the lower K index).
__device__ __forceinline__ void split2(float a, float b, uint32_t& hi, uint32_t& lo) {
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *reinterpret_cast<const uint32_t*>(&h);
    lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t x, uint32_t y, uint32_t z, uint32_t w) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(x), "r"(y), "r"(z), "r"(w) : "memory");
}
__device__ __forceinline__ void st_shared_b32(uint32_t addr, uint32_t x) {
    asm volatile("st.shared.b32 [%0], %1;" ::"r"(addr), "r"(x) : "memory");
}

template <int NORB>
__global__ void __launch_bounds__(kTcThreads, 1)
    spec_prod_tc_kernel(TcCfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr,
                        const double2* __restrict__ dH, const float2* __restrict__ Ghat,
                        const float2* __restrict__ Khat, float2* __restrict__ Shat, double scale,
                        unsigned* __restrict__ status) {
    using S = TcShape<NORB>;
    constexpr int nel = NORB * NORB;
    extern __shared__ __align__(1024) unsigned char smem[];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bars = sbase + (uint32_t)c.off_bar;
    auto B_ = [&](int i) { return bars + 8u * (uint32_t)i; };
    int* xr = reinterpret_cast<int*>(smem + c.off_x);           // [2][8]: e1 of the four groups, eH of the bond
    int* ehs = xr + 16;                                          // [16] bond exponents of the current item
    float* pmax = reinterpret_cast<float*>(ehs + 16);            // [4] producer warp maxima
    float* xmax = pmax + 4;                                      // [2][4][2] epilogue pair maxima
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(xmax + 16);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
    const int NB = c.NB, nA = c.nA;

    // every operand byte that no role writes (K and N padding, padding rows) must be zero
    for (int i = tid; i < c.off_bar / 16; i += kTcThreads) reinterpret_cast<uint4*>(smem)[i] = make_uint4(0, 0, 0, 0);
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(B_(BA1F + i), kTcProdWarps * 32);
            mbar_init(B_(BA1E + i), 1);
            mbar_init(B_(BPF + i), 1);
            mbar_init(B_(BPE + i), kTcEpiWarps * 32);
            mbar_init(B_(BA2F + i), kTcEpiWarps * 32);
            mbar_init(B_(BA2E + i), 1);
            mbar_init(B_(BXE + i), kTcEpiWarps * 32);
        }
        mbar_init(B_(BOF), 1);
        mbar_init(B_(BBF), kTcProdWarps * 32);
        mbar_init(B_(BBE), 1);
        mbar_init(B_(BMD), 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == kTcMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(c.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp >= kTcEpiWarps && warp < kTcMmaWarp) {
        // ------------------------------------------------------------------ producers
        const int g = warp - kTcEpiWarps, pt = tid - kTcProd0;
        uint32_t u = 0;
        int nitem = 0;
        for (int item = blockIdx.x; item < c.nitems; item += gridDim.x, ++nitem) {
            const int la = item % nA, tg = item / nA;
            const int a = d.a_begin + la;
            // dH operands of every bond of the atom, once the MMAs of the previous item are done with them
            if (nitem > 0) wait_or_abort(B_(BBE), (nitem - 1) & 1, abort_flag, status);
            for (int s = 0; s < NB; ++s) {
                const double2* A = dH + ((size_t)a * NB + s) * 3 * nel;
                float m = 0.f;
                for (int i = pt; i < 3 * nel; i += kTcProdWarps * 32) {
                    const double2 v = A[i];
                    m = fmaxf(m, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
                }
                m = warp_max_abs(m);
                if (lane == 0) pmax[g] = m;
                named_bar(2, kTcProdWarps * 32);
                m = fmaxf(fmaxf(pmax[0], pmax[1]), fmaxf(pmax[2], pmax[3]));
                const int eH = scale_exp(m);
                if (pt == 0) ehs[s] = eH;
                named_bar(2, kTcProdWarps * 32);  // pmax is free again
                const uint32_t b1 = sbase + (uint32_t)(c.off_B1 + s * S::B1_BOND);
                const uint32_t b2 = sbase + (uint32_t)(c.off_B2 + s * S::B2_BOND);
                for (int i = pt; i < 3 * nel; i += kTcProdWarps * 32) {
                    const int j = i / nel, e = i - j * nel, n = e / NORB, l = e - n * NORB;
                    const double2 v = A[i];  // dH_j[n][l]
                    const float hr = mul_pow2((float)v.x, eH), hi = mul_pow2((float)v.y, eH);
                    uint32_t h0, l0, h1, l1;
                    // GEMM1 B = dH_j^H in the real embedding: column (j, n, re) holds (Hr, Hi) at K = (l, re/im),
                    // column (j, n, im) holds (-Hi, Hr); hi rows first, lo rows after N1
                    const int r = j * 2 * NORB + 2 * n;
                    const uint32_t k1 = (uint32_t)((2 * l) >> 3) * S::LB1 + (uint32_t)((2 * l) & 7) * 2;
                    split2(hr, hi, h0, l0);
                    split2(-hi, hr, h1, l1);
                    st_shared_b32(b1 + k1 + (uint32_t)r * 16, h0);
                    st_shared_b32(b1 + k1 + (uint32_t)(r + 1) * 16, h1);
                    st_shared_b32(b1 + k1 + (uint32_t)(S::N1 + r) * 16, l0);
                    st_shared_b32(b1 + k1 + (uint32_t)(S::N1 + r + 1) * 16, l1);
                    // GEMM2 B = dH_i^T: the entry dH_i[m'][m] (i = j, m' = n, m = l) sits at K = (m, i, re/im) of
                    // column (m', re) as (Hr, -Hi) and of column (m', im) as (Hi, Hr)
                    const uint32_t k2 = (uint32_t)l * S::LB2 + (uint32_t)(2 * j) * 2;
                    split2(hr, -hi, h0, l0);
                    split2(hi, hr, h1, l1);
                    st_shared_b32(b2 + k2 + (uint32_t)(2 * n) * 16, h0);
                    st_shared_b32(b2 + k2 + (uint32_t)(2 * n + 1) * 16, h1);
                    st_shared_b32(b2 + k2 + (uint32_t)(S::N2 + 2 * n) * 16, l0);
                    st_shared_b32(b2 + k2 + (uint32_t)(S::N2 + 2 * n + 1) * 16, l1);
                }
            }
            fence_async_smem();
            mbar_arrive(B_(BBF));
            named_bar(2, kTcProdWarps * 32);  // ehs written
            const int j0 = tg * kTcTilesPerItem, j1 = min(j0 + kTcTilesPerItem, c.ntiles);
            for (int tile = j0; tile < j1; ++tile) {
                for (int s = 0; s < NB; ++s, ++u) {
                    const int st = (int)(u & 1);
                    const uint32_t par = ((u >> 1) & 1) ^ 1;
                    wait_or_abort(B_(BA1E + st), par, abort_flag, status);  // GEMM1 has read the stage
                    wait_or_abort(B_(BXE + st), par, abort_flag, status);   // the epilogue has read its exponents
                    const int b = nbr[(size_t)a * NB + s];
                    const bool bok = b >= 0 && b < d.NA;
                    if (!bok && pt == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
                    // this warp's group: rows (f', m) for FG frequencies, chunks of 4 complex along l
                    float v[S::CD][8];
                    float m = 0.f;
#pragma unroll
                    for (int it = 0; it < S::CD; ++it) {
                        const int task = lane + 32 * it;
                        const int ch = task / S::R, row = task - ch * S::R;
                        const int fp = row / NORB, mr = row - fp * NORB;
                        const size_t fi = (size_t)tile * S::FT + g * S::FG + fp;
                        const bool ok = bok && ch < S::CD && fi < fm.count;
                        const float2* src = ok ? Ghat + (freq_of(fm, fi) * d.NA + b) * nel + mr * NORB : Ghat;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            const int l = 4 * ch + q;
                            float2 x = make_float2(0.f, 0.f);
                            if (ok && l < NORB) x = src[l];
                            v[it][2 * q] = x.x;
                            v[it][2 * q + 1] = x.y;
                            m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.y)));
                        }
                    }
                    const int e1 = scale_exp(warp_max_abs(m));
                    const uint32_t a1 = sbase + (uint32_t)(c.off_A1 + st * S::A1_STAGE);
#pragma unroll
                    for (int it = 0; it < S::CD; ++it) {
                        const int task = lane + 32 * it;
                        const int ch = task / S::R, row = task - ch * S::R;
                        if (ch < S::CD) {
                            uint32_t h[4], lo[4];
#pragma unroll
                            for (int q = 0; q < 4; ++q)
                                split2(mul_pow2(v[it][2 * q], e1), mul_pow2(v[it][2 * q + 1], e1), h[q], lo[q]);
                            const uint32_t o = a1 + (uint32_t)ch * S::LA1 + (uint32_t)(32 * g + row) * 16;
                            st_shared_v4(o, h[0], h[1], h[2], h[3]);
                            st_shared_v4(o + S::A1_PLANE, lo[0], lo[1], lo[2], lo[3]);
                        }
                    }
                    if (lane == 0) xr[st * 8 + g] = e1;
                    if (pt == 0) xr[st * 8 + 4] = ehs[s];
                    fence_async_smem();
                    mbar_arrive(B_(BA1F + st));
                }
            }
            named_bar(2, kTcProdWarps * 32);  // every producer is done with ehs before the next item rewrites it
        }
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id1w = tc_idesc_f16(2 * S::N1), id1 = tc_idesc_f16(S::N1);
            const uint32_t id2w = tc_idesc_f16(2 * S::N2), id2 = tc_idesc_f16(S::N2);
            uint32_t u1 = 0, u2 = 0;  // units issued to GEMM1 / GEMM2
            int nitem = 0;
            auto gemm1 = [&](int s) {
                const int st = (int)(u1 & 1);
                wait_or_abort(B_(BA1F + st), (u1 >> 1) & 1, abort_flag, status);
                wait_or_abort(B_(BPE + st), ((u1 >> 1) & 1) ^ 1, abort_flag, status);
                tc_fence_after();
                if (!*abort_flag) {
                    const uint32_t dP = tmem + (uint32_t)(st * S::TM_P);
                    const uint32_t ah = sbase + (uint32_t)(c.off_A1 + st * S::A1_STAGE), al = ah + S::A1_PLANE;
                    const uint32_t b = sbase + (uint32_t)(c.off_B1 + s * S::B1_BOND);
#pragma unroll
                    for (int kc = 0; kc < S::K1 / 16; ++kc)
                        umma_f16(dP, smem_desc(ah + 2 * kc * S::LA1, S::LA1, 128), smem_desc(b + 2 * kc * S::LB1, S::LB1, 128),
                                 id1w, kc > 0);
#pragma unroll
                    for (int kc = 0; kc < S::K1 / 16; ++kc)
                        umma_f16(dP, smem_desc(al + 2 * kc * S::LA1, S::LA1, 128), smem_desc(b + 2 * kc * S::LB1, S::LB1, 128),
                                 id1, 1);
                }
                umma_commit(B_(BA1E + st));
                umma_commit(B_(BPF + st));
                ++u1;
            };
            auto gemm2 = [&](int s) {
                const int st = (int)(u2 & 1);
                wait_or_abort(B_(BA2F + st), (u2 >> 1) & 1, abort_flag, status);
                tc_fence_after();
                if (!*abort_flag) {
                    const uint32_t dO = tmem + (uint32_t)(2 * S::TM_P + s * S::TM_O);
                    const uint32_t ah = sbase + (uint32_t)(c.off_A2 + st * S::A2_STAGE), al = ah + S::A2_PLANE;
                    const uint32_t b = sbase + (uint32_t)(c.off_B2 + s * S::B2_BOND);
#pragma unroll
                    for (int kc = 0; kc < S::K2 / 16; ++kc)
                        umma_f16(dO, smem_desc(ah + 2 * kc * S::LA2, S::LA2, 128), smem_desc(b + 2 * kc * S::LB2, S::LB2, 128),
                                 id2w, kc > 0);
#pragma unroll
                    for (int kc = 0; kc < S::K2 / 16; ++kc)
                        umma_f16(dO, smem_desc(al + 2 * kc * S::LA2, S::LA2, 128), smem_desc(b + 2 * kc * S::LB2, S::LB2, 128),
                                 id2, 1);
                }
                umma_commit(B_(BA2E + st));
                ++u2;
            };
            for (int item = blockIdx.x; item < c.nitems; item += gridDim.x, ++nitem) {
                const int tg = item / nA;
                const int j0 = tg * kTcTilesPerItem, j1 = min(j0 + kTcTilesPerItem, c.ntiles);
                const int units = (j1 - j0) * NB;
                wait_or_abort(B_(BBF), nitem & 1, abort_flag, status);  // this item's dH operands
                tc_fence_after();
                gemm1(0);
                for (int v = 0; v < units; ++v) {
                    const int s = v % NB;
                    if (v + 1 < units) gemm1((v + 1) % NB);  // the next bond's GEMM1 overlaps this bond's epilogue
                    gemm2(s);
                    if (s == NB - 1) umma_commit(B_(BOF));  // the tile's bond accumulators are complete
                }
                umma_commit(B_(BBE));  // the dH operands may be replaced
            }
            umma_commit(B_(BMD));
            drain_wait(B_(BMD), 0, status);  // nothing in flight when TMEM is released, also after an abort
        }
    } else {
        // ------------------------------------------------------------------ epilogue
        const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter (= row group), column half
        const int fp = lane / NORB, mr = lane - fp * NORB;
        const bool row_ok = fp < S::FG;
        const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
        const float sc = (float)scale;
        uint32_t u = 0, ntile = 0;
        for (int item = blockIdx.x; item < c.nitems; item += gridDim.x) {
            const int la = item % nA, tg = item / nA;
            const int j0 = tg * kTcTilesPerItem, j1 = min(j0 + kTcTilesPerItem, c.ntiles);
            for (int tile = j0; tile < j1; ++tile, ++ntile) {
                const size_t fi = (size_t)tile * S::FT + q * S::FG + fp;
                const bool fok = row_ok && fi < fm.count;
                const size_t f = fok ? freq_of(fm, fi) : 0;
                int etot[kTcMaxNB] = {0, 0, 0, 0};  // per bond: the exponent that undoes the operand scales
                for (int s = 0; s < NB; ++s, ++u) {
                    const int st = (int)(u & 1);
                    const uint32_t par = (u >> 1) & 1;
                    // exponents of this unit (GEMM1's A scale of this row group, the bond's dH scale)
                    wait_or_abort(B_(BA1F + st), par, abort_flag, status);
                    const int e1 = xr[st * 8 + q], eH = xr[st * 8 + 4];
                    mbar_arrive(B_(BXE + st));
                    float2 k[9];
#pragma unroll
                    for (int ij = 0; ij < 9; ++ij)
                        k[ij] = fok ? Khat[((f * nA + la) * NB + s) * 9 + ij] : make_float2(0.f, 0.f);
                    // P_j rows from TMEM (two parts: hi*B_hi + lo*B_hi, and hi*B_lo), U_i = sum_j K_ij P_j
                    wait_or_abort(B_(BPF + st), par, abort_flag, status);
                    tc_fence_after();
                    float ur[3][S::NH], ui[3][S::NH];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int nn = 0; nn < S::NH; ++nn) ur[i][nn] = ui[i][nn] = 0.f;
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        float p1[2 * S::NH], p2[2 * S::NH];
                        const uint32_t col = (uint32_t)(st * S::TM_P + j * 2 * NORB + 2 * h * S::NH);
                        tmem_ld_half<S::NH>(tq + col, p1);
                        tmem_ld_half<S::NH>(tq + col + S::N1, p2);
                        tmem_wait_ld();
#pragma unroll
                        for (int nn = 0; nn < S::NH; ++nn) {
                            const float pr = p1[2 * nn] + p2[2 * nn], pim = p1[2 * nn + 1] + p2[2 * nn + 1];
#pragma unroll
                            for (int i = 0; i < 3; ++i) {
                                const float2 kk = k[i * 3 + j];
                                ur[i][nn] = fmaf(kk.x, pr, fmaf(-kk.y, pim, ur[i][nn]));
                                ui[i][nn] = fmaf(kk.x, pim, fmaf(kk.y, pr, ui[i][nn]));
                            }
                        }
                    }
                    tc_fence_before();
                    mbar_arrive(B_(BPE + st));  // the P buffer may be overwritten
                    // one scale for the row group: max over both column halves (the partner warp)
                    float m = 0.f;
#pragma unroll
                    for (int nn = 0; nn < S::NH; ++nn)
                        if (h * S::NH + nn < NORB)
#pragma unroll
                            for (int i = 0; i < 3; ++i) m = fmaxf(m, fmaxf(fabsf(ur[i][nn]), fabsf(ui[i][nn])));
                    m = warp_max_abs(m);
                    if (lane == 0) xmax[(st * 4 + q) * 2 + h] = m;
                    named_bar(3 + q, 64);
                    const int e2 = scale_exp(fmaxf(xmax[(st * 4 + q) * 2], xmax[(st * 4 + q) * 2 + 1]));
                    // U^T rows (f', n) into GEMM2's A operand: K chunk m holds (i, re/im) for i = 0..2, then 0, 0
                    wait_or_abort(B_(BA2E + st), par ^ 1, abort_flag, status);
                    if (row_ok) {
                        const uint32_t a2 = sbase + (uint32_t)(c.off_A2 + st * S::A2_STAGE) + (uint32_t)mr * S::LA2;
#pragma unroll
                        for (int nn = 0; nn < S::NH; ++nn) {
                            const int n = h * S::NH + nn;
                            if (n < NORB) {
                                uint32_t hw[3], lw[3];
#pragma unroll
                                for (int i = 0; i < 3; ++i)
                                    split2(mul_pow2(ur[i][nn], e2), mul_pow2(ui[i][nn], e2), hw[i], lw[i]);
                                const uint32_t o = a2 + (uint32_t)(32 * q + fp * NORB + n) * 16;
                                st_shared_v4(o, hw[0], hw[1], hw[2], 0u);
                                st_shared_v4(o + S::A2_PLANE, lw[0], lw[1], lw[2], 0u);
                            }
                        }
                    }
                    fence_async_smem();
                    mbar_arrive(B_(BA2F + st));
#pragma unroll
                    for (int t4 = 0; t4 < kTcMaxNB; ++t4)  // static register indices
                        if (t4 == s) etot[t4] = e1 + 2 * eH + e2;
                }
                // S^(f)^T rows (f', n = mr): sum over bonds of the unscaled accumulators, times i*scale
                wait_or_abort(B_(BOF), ntile & 1, abort_flag, status);
                tc_fence_after();
                float accr[S::NH], acci[S::NH];
#pragma unroll
                for (int mm = 0; mm < S::NH; ++mm) accr[mm] = acci[mm] = 0.f;
#pragma unroll
                for (int s = 0; s < kTcMaxNB; ++s) {
                    if (s < NB) {
                        float p1[2 * S::NH], p2[2 * S::NH];
                        const uint32_t col = (uint32_t)(2 * S::TM_P + s * S::TM_O + 2 * h * S::NH);
                        tmem_ld_half<S::NH>(tq + col, p1);
                        tmem_ld_half<S::NH>(tq + col + S::N2, p2);
                        tmem_wait_ld();
#pragma unroll
                        for (int mm = 0; mm < S::NH; ++mm) {
                            accr[mm] += mul_pow2(p1[2 * mm] + p2[2 * mm], -etot[s]);
                            acci[mm] += mul_pow2(p1[2 * mm + 1] + p2[2 * mm + 1], -etot[s]);
                        }
                    }
                }
                tc_fence_before();
                if (fok) {
                    float2* out = Shat + (f * nA + la) * nel + mr;
#pragma unroll
                    for (int mm = 0; mm < S::NH; ++mm) {
                        const int mp = h * S::NH + mm;
                        if (mp < NORB) out[mp * NORB] = make_float2(-sc * acci[mm], sc * accr[mm]);  // i*scale*S
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kTcMmaWarp) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(c.tmem_cols));
    }
}

template <int NORB>
cudaError_t launch_tc(const sse_dims& d, const FreqMap& fm, const int32_t* nbr, const double2* dH, const float2* Gh,
                      const float2* Kh, float2* Sh, double scale, unsigned* status, cudaStream_t st) {
    const TcCfg c = make_tc_cfg<NORB>(d, fm.count);
    if (c.nitems == 0) return cudaSuccess;
    static int nsm = 0;
    cudaError_t e;
    if (nsm == 0) {
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    }
    if ((e = cudaFuncSetAttribute(spec_prod_tc_kernel<NORB>, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem)) !=
        cudaSuccess)
        return e;
    const int grid = c.nitems < nsm ? c.nitems : nsm;
    SSE_TIMED("spec_prod_tc_kernel", st,
              spec_prod_tc_kernel<NORB><<<grid, kTcThreads, c.smem, st>>>(c, d, fm, nbr, dH, Gh, Kh, Sh, scale, status));
    return cudaGetLastError();
}

template <int NORB>
bool tc_fits(const sse_dims& d) {
    const TcCfg c = make_tc_cfg<NORB>(d, 1);
    return d.NB <= kTcMaxNB && c.smem <= 227 * 1024 && 2 * TcShape<NORB>::TM_P + d.NB * TcShape<NORB>::TM_O <= 512;
}

}  // namespace

bool spectral_prod_tc_supported(const sse_dims& d) {
    switch (d.Norb) {
        case 1: return tc_fits<1>(d);
        case 2: return tc_fits<2>(d);
        case 3: return tc_fits<3>(d);
        case 4: return tc_fits<4>(d);
        case 5: return tc_fits<5>(d);
        case 6: return tc_fits<6>(d);
        case 7: return tc_fits<7>(d);
        case 8: return tc_fits<8>(d);
        case 9: return tc_fits<9>(d);
        case 10: return tc_fits<10>(d);
        default: return false;
    }
}

cudaError_t spectral_prod_tc(const sse_dims& d, const FreqMap& fm, const int32_t* nbr, const double2* dH,
                             const float2* Gh, const float2* Kh, float2* Sh, double scale, unsigned* status,
                             cudaStream_t st) {
    switch (d.Norb) {
        case 1: return launch_tc<1>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 2: return launch_tc<2>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 3: return launch_tc<3>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 4: return launch_tc<4>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 5: return launch_tc<5>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 6: return launch_tc<6>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 7: return launch_tc<7>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 8: return launch_tc<8>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 9: return launch_tc<9>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        case 10: return launch_tc<10>(d, fm, nbr, dH, Gh, Kh, Sh, scale, status, st);
        default: return cudaErrorNotSupported;
    }
}

}  // namespace sse
