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
// Precision: every operand x is scaled by a power of two (per 32-row group, or per warp, for the frequency-stacked
// operands, per bond for dH; exact, undone in the epilogue) and split into FP16 hi = fp16(x), lo = fp16(x - hi).
// GEMM1 accumulates hi*B_hi + lo*B_hi + hi*B_lo in one FP32 accumulator; GEMM2 runs as hi x [B_hi | B_lo] (one MMA
// with N doubled) + lo x B_hi, two accumulators that the epilogue adds. lo*lo (~2^-22 relative) is dropped; the
// result carries about 22 significant bits, the level of the FP32 transforms around it.
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
constexpr int kTcRaw = 3;                   // raw stages: the producers copy up to two units ahead (cp.async)

template <int NORB>
struct TcShape {
    static constexpr int FG = 32 / NORB;                    // frequencies per 32-row group
    static constexpr int FT = 4 * FG;                       // frequencies per 128-row tile
    static constexpr int R = FG * NORB;                     // used rows per group
    static constexpr int CD = (NORB + 3) / 4;               // 16-B chunks of one G^ row (4 complex each)
    static constexpr int KPL = (FG * 9 + 31) / 32;          // K^ entries per producer lane (group of FG frequencies)
    static constexpr int RAW_G = (FG * NORB * NORB + FG * 9 + 1) / 2 * 2;  // float2 per group and raw stage: G^ blocks,
                                                                            // then K^ (even: 16-byte aligned groups)
    static constexpr bool BULK = (NORB * NORB * 8) % 16 == 0;  // a G^ block is whole 16-byte units: one bulk copy
    static constexpr int RAW_STAGE = 4 * RAW_G * 8;          // bytes per raw stage (four groups)
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
    static constexpr int TM_P = N1;                         // TMEM columns per P buffer (two)
    static constexpr int TM_O = 2 * N2;                     // TMEM columns per bond accumulator
};

// Barriers (8 B each) after the operand buffers.
enum { BA1F = 0, BA1E = 2, BPF = 4, BPE = 6, BA2F = 8, BA2E = 10, BXE = 12, BOF = 14, BBF = 15, BBE = 16, BMD = 17,
       BRF = 18,  // raw ring: one barrier per (stage, group), completed by the bulk copies of the G^ blocks
       kTcBars = 18 + 3 * 4 };

struct TcCfg {
    int NB, nA, ntiles, ngroups, nitems;
    int off_A1, off_A2, off_B1, off_B2, off_K, off_raw, off_bar, off_x, smem, tmem_cols;
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
    c.off_K = c.off_B2 + d.NB * S::B2_BOND;  // K^ of the tile's frequencies, two stages: [2][FT][9] float2
    c.off_raw = c.off_K + 2 * S::FT * 9 * 8;  // raw FP32 G^ and K^ of the next units: [kTcRaw][4][RAW_G] float2
    c.off_bar = c.off_raw + kTcRaw * S::RAW_STAGE;
    c.off_x = c.off_bar + kTcBars * 8;
    // exchange area: exponent ring [2][8] int, bond exponents [16] int, producer maxima [2][4][4] float,
    // GEMM2 operand exponents [2][4][4][2] int, TMEM base, abort flag
    c.smem = c.off_x + (16 + 16 + 32 + 64 + 2) * 4;
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

// Exponent e that brings max |x| into [2^13, 2^14) (m = max |x| >= 0, read from its bits: floor(log2 m) is the
// unbiased exponent of a normal float, 31 - clz - 149 of a subnormal); 0 for an all-zero or non-finite group.
__device__ __forceinline__ int scale_exp(float m) {
    const uint32_t b = __float_as_uint(m);
    const int ex = (int)(b >> 23);
    if (b == 0u || ex >= 255) return 0;
    const int lg = ex > 0 ? ex - 127 : (31 - __clz((int)b)) - 149;
    return kTcExpTarget - lg;
}
// 2^e as two normal floats (a * b == 2^e exactly for |e| <= 252): computed once per scale, two FMULs per value.
struct Pow2 {
    float a, b;
};
__device__ __forceinline__ Pow2 pow2_factors(int e) {
    const int e1 = max(-126, min(127, e));
    const int e2 = max(-126, min(127, e - e1));
    return {__int_as_float((e1 + 127) << 23), __int_as_float((e2 + 127) << 23)};
}
__device__ __forceinline__ float scaled(float x, Pow2 f) { return x * f.a * f.b; }

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
// Bulk copy global -> shared through the TMA engine (16-byte aligned addresses, size a multiple of 16), completing
// on an mbarrier's transaction count.
__device__ __forceinline__ void bulk_copy(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// 8-byte asynchronous copy global -> shared; with pred false the destination is zero-filled (nothing is read).
__device__ __forceinline__ void cp_async8(uint32_t dst, const void* src, bool pred) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(dst), "l"(src), "r"(pred ? 8 : 0) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

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
    float* pmax = reinterpret_cast<float*>(ehs + 16);            // [2 items][4 warps][4 bonds] producer maxima
    int* e2s = reinterpret_cast<int*>(pmax + 32);                // [2 tiles][4 bonds][4 groups][2 halves] GEMM2 A scales
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(e2s + 64);
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
        for (int i = 0; i < kTcRaw * 4; ++i) mbar_init(B_(BRF + i), 1);
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
        float2* ks = reinterpret_cast<float2*>(smem + c.off_K);  // [2][FT][9]
        uint32_t u = 0;
        int nitem = 0;
        // One unit (tile, bond) of this warp's row group: the G^ blocks of the group's FG frequencies and their K^
        // entries, copied raw (FP32) into a ring of kTcRaw stages up to two units ahead of their use.
        int bnb[kTcMaxNB] = {-1, -1, -1, -1};  // the item's neighbours (loaded once per item)
        const float2* raw = reinterpret_cast<const float2*>(smem + c.off_raw);
        uint32_t r_issued = 0, r_last = 0;  // raw slots with bulk copies issued; parity of the last use of each
        auto issue_unit = [&](int la, int tile, int s, uint32_t rq) {
            const int rs = (int)(rq % kTcRaw);
            int b = bnb[0];
#pragma unroll
            for (int t4 = 1; t4 < kTcMaxNB; ++t4)
                if (t4 == s) b = bnb[t4];
            const bool bok = b >= 0 && b < d.NA;
            // lane l < FG: the frequency of the group's l-th row block (shared by shuffles below)
            const size_t fi_l = (size_t)tile * S::FT + g * S::FG + lane;
            const bool ok_l = bok && lane < S::FG && fi_l < fm.count;
            const unsigned long long f_l = ok_l ? (unsigned long long)freq_of(fm, fi_l) : ~0ull;
            const uint32_t dst = sbase + (uint32_t)(c.off_raw + rs * S::RAW_STAGE + g * S::RAW_G * 8);
            if (S::BULK) {
                // one bulk copy of its frequency's G^ block per lane l < FG (blocks of invalid frequencies are not
                // copied: the reader takes zeros for them)
                const uint32_t rbar = B_(BRF + rs * 4 + g);
                const unsigned vm = __ballot_sync(0xffffffffu, ok_l);
                if (lane == 0) mbar_expect_tx(rbar, (uint32_t)__popc(vm) * (uint32_t)(nel * 8));
                __syncwarp();
                if (ok_l)
                    bulk_copy(dst + (uint32_t)(lane * nel * 8), Ghat + ((size_t)f_l * d.NA + b) * nel,
                              (uint32_t)(nel * 8), rbar);
                r_issued |= 1u << rs;
                r_last = (r_last & ~(1u << rs)) | (((rq / kTcRaw) & 1u) << rs);
            } else {
#pragma unroll
                for (int it = 0; it < (S::FG * nel + 31) / 32; ++it) {
                    const int idx = lane + 32 * it, fl = idx / nel, e = idx - fl * nel;
                    const unsigned long long f = __shfl_sync(0xffffffffu, f_l, fl < S::FG ? fl : 0);
                    const bool ok = idx < S::FG * nel && f != ~0ull;
                    if (idx < S::FG * nel)
                        cp_async8(dst + (uint32_t)idx * 8, ok ? Ghat + ((size_t)f * d.NA + b) * nel + e : Ghat, ok);
                }
            }
#pragma unroll
            for (int it = 0; it < S::KPL; ++it) {
                const int idx = lane + 32 * it, fl = idx / 9, ij = idx - fl * 9;
                const unsigned long long f = __shfl_sync(0xffffffffu, f_l, fl < S::FG ? fl : 0);
                const bool ok = idx < S::FG * 9 && f != ~0ull;
                if (idx < S::FG * 9)
                    cp_async8(dst + (uint32_t)(S::FG * nel + idx) * 8,
                              ok ? Khat + (((size_t)f * nA + la) * NB + s) * 9 + ij : Khat, ok);
            }
            cp_async_commit();
            if (!bok && pt == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        };
        auto produce = [&](int la, int tile, int s, uint32_t rq) {
            const int rs = (int)(rq % kTcRaw);
            const int st = (int)(u & 1);
            const uint32_t par = ((u >> 1) & 1) ^ 1;
            wait_or_abort(B_(BA1E + st), par, abort_flag, status);  // GEMM1 has read the stage
            wait_or_abort(B_(BXE + st), par, abort_flag, status);   // the epilogue has read its exponents and K^
            int b = bnb[0];
#pragma unroll
            for (int t4 = 1; t4 < kTcMaxNB; ++t4)
                if (t4 == s) b = bnb[t4];
            const bool bok = b >= 0 && b < d.NA;
            if (S::BULK) wait_or_abort(B_(BRF + rs * 4 + g), (rq / kTcRaw) & 1u, abort_flag, status);
            const float2* rg = raw + (size_t)rs * (S::RAW_STAGE / 8) + g * S::RAW_G;
            float v[S::CD][8];
            float m = 0.f;
#pragma unroll
            for (int it = 0; it < S::CD; ++it) {
                const int task = lane + 32 * it;
                const int ch = task / S::R, row = task - ch * S::R;
                const int fp = row / NORB, mr = row - fp * NORB;
                // blocks of frequencies out of range (or of a bad neighbour) were not copied: zeros
                const bool ok = ch < S::CD && (!S::BULK || (bok && (size_t)tile * S::FT + g * S::FG + fp < fm.count));
                if (S::BULK) {  // even Norb: rows are 16-byte aligned, pairs of complex entries as one load
#pragma unroll
                    for (int q = 0; q < 4; q += 2) {
                        const int l = 4 * ch + q;
                        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
                        if (ok && l < NORB) x = *reinterpret_cast<const float4*>(rg + fp * nel + mr * NORB + l);
                        v[it][2 * q] = x.x;
                        v[it][2 * q + 1] = x.y;
                        v[it][2 * q + 2] = x.z;
                        v[it][2 * q + 3] = x.w;
                        m = fmaxf(m, fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w))));
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int l = 4 * ch + q;
                        float2 x = make_float2(0.f, 0.f);
                        if (ok && l < NORB) x = rg[fp * nel + mr * NORB + l];
                        v[it][2 * q] = x.x;
                        v[it][2 * q + 1] = x.y;
                        m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.y)));
                    }
                }
            }
            const int e1 = scale_exp(warp_max_abs(m));
            const Pow2 f1 = pow2_factors(e1);
            const uint32_t a1 = sbase + (uint32_t)(c.off_A1 + st * S::A1_STAGE);
#pragma unroll
            for (int it = 0; it < S::CD; ++it) {
                const int task = lane + 32 * it;
                const int ch = task / S::R, row = task - ch * S::R;
                if (ch < S::CD) {
                    uint32_t h[4], lo[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        split2(scaled(v[it][2 * q], f1), scaled(v[it][2 * q + 1], f1), h[q], lo[q]);
                    const uint32_t o = a1 + (uint32_t)ch * S::LA1 + (uint32_t)(32 * g + row) * 16;
                    st_shared_v4(o, h[0], h[1], h[2], h[3]);
                    st_shared_v4(o + S::A1_PLANE, lo[0], lo[1], lo[2], lo[3]);
                }
            }
#pragma unroll
            for (int r = 0; r < S::KPL; ++r) {
                const int idx = lane + 32 * r;
                if (idx < S::FG * 9) ks[(st * S::FT + g * S::FG) * 9 + idx] = rg[S::FG * nel + idx];
            }
            if (lane == 0) xr[st * 8 + g] = e1;
            if (pt == 0) xr[st * 8 + 4] = ehs[s];
            fence_async_smem();
            mbar_arrive(B_(BA1F + st));
            ++u;
        };
        uint32_t ru = 0;  // units copied into the raw ring
        for (int item = blockIdx.x; item < c.nitems; item += gridDim.x, ++nitem) {
            const int la = item % nA, tg = item / nA;
            const int a = d.a_begin + la;
            const int j0 = tg * kTcTilesPerItem, j1 = min(j0 + kTcTilesPerItem, c.ntiles);
            const int units = (j1 - j0) * NB;
#pragma unroll
            for (int t4 = 0; t4 < kTcMaxNB; ++t4) bnb[t4] = t4 < NB ? nbr[(size_t)a * NB + t4] : -1;
            const uint32_t r0 = ru;  // raw sequence number of the item's first unit
            for (int v = 0; v < 2 && v < units; ++v, ++ru)  // in flight during the dH staging below
                issue_unit(la, j0 + v / NB, v % NB, ru);
            // dH operands of every bond of the atom (all loads issued at once), once the MMAs of the previous item
            // are done with them
            constexpr int RPT = (3 * nel + kTcProdWarps * 32 - 1) / (kTcProdWarps * 32);
            double2 hv[kTcMaxNB][RPT];
            float hm[kTcMaxNB];
#pragma unroll
            for (int t4 = 0; t4 < kTcMaxNB; ++t4) {
                hm[t4] = 0.f;
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int i = pt + r * kTcProdWarps * 32;
                    hv[t4][r] = (t4 < NB && i < 3 * nel) ? dH[((size_t)a * NB + t4) * 3 * nel + i]
                                                          : make_double2(0.0, 0.0);
                }
            }
#pragma unroll
            for (int t4 = 0; t4 < kTcMaxNB; ++t4) {
#pragma unroll
                for (int r = 0; r < RPT; ++r)
                    hm[t4] = fmaxf(hm[t4], fmaxf(fabsf((float)hv[t4][r].x), fabsf((float)hv[t4][r].y)));
                hm[t4] = warp_max_abs(hm[t4]);
                if (lane == 0) pmax[((nitem & 1) * 4 + g) * 4 + t4] = hm[t4];  // two item buffers, no reuse race
            }
            if (nitem > 0) wait_or_abort(B_(BBE), (nitem - 1) & 1, abort_flag, status);
            named_bar(2, kTcProdWarps * 32);  // the four warps' maxima are in place
#pragma unroll
            for (int t4 = 0; t4 < kTcMaxNB; ++t4) {
                if (t4 >= NB) break;
                const float* pm = pmax + (nitem & 1) * 16 + t4;
                const int eH = scale_exp(fmaxf(fmaxf(pm[0], pm[4]), fmaxf(pm[8], pm[12])));
                if (pt == 0) ehs[t4] = eH;
                const Pow2 fH = pow2_factors(eH);
                const uint32_t b1 = sbase + (uint32_t)(c.off_B1 + t4 * S::B1_BOND);
                const uint32_t b2 = sbase + (uint32_t)(c.off_B2 + t4 * S::B2_BOND);
#pragma unroll
                for (int r = 0; r < RPT; ++r) {
                    const int i = pt + r * kTcProdWarps * 32;
                    if (i >= 3 * nel) break;
                    const int j = i / nel, e = i - j * nel, n = e / NORB, l = e - n * NORB;
                    const double2 v = hv[t4][r];  // dH_j[n][l]
                    const float hr = scaled((float)v.x, fH), hi = scaled((float)v.y, fH);
                    uint32_t h0, l0, h1, l1;
                    // GEMM1 B = dH_j^H in the real embedding: column (j, n, re) holds (Hr, Hi) at K = (l, re/im),
                    // column (j, n, im) holds (-Hi, Hr); hi rows first, lo rows after N1
                    const int rr = j * 2 * NORB + 2 * n;
                    const uint32_t k1 = (uint32_t)((2 * l) >> 3) * S::LB1 + (uint32_t)((2 * l) & 7) * 2;
                    split2(hr, hi, h0, l0);
                    split2(-hi, hr, h1, l1);
                    st_shared_b32(b1 + k1 + (uint32_t)rr * 16, h0);
                    st_shared_b32(b1 + k1 + (uint32_t)(rr + 1) * 16, h1);
                    st_shared_b32(b1 + k1 + (uint32_t)(S::N1 + rr) * 16, l0);
                    st_shared_b32(b1 + k1 + (uint32_t)(S::N1 + rr + 1) * 16, l1);
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
            for (int v = 0; v < units; ++v) {
                if (v + 2 < units) {
                    issue_unit(la, j0 + (v + 2) / NB, (v + 2) % NB, ru);
                    ++ru;
                    cp_async_wait<2>();  // this unit's copies are done (the two after it may be in flight)
                } else if (v + 1 < units) {
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncwarp();  // every lane's copies are visible to the warp
                produce(la, j0 + v / NB, v % NB, r0 + v);
            }
        }
        // every bulk copy this warp issued has landed before the CTA releases its shared memory (after an abort the
        // reads above may have skipped their waits)
        if (S::BULK)
            for (int rs = 0; rs < kTcRaw; ++rs)
                if ((r_issued >> rs) & 1u) drain_wait(B_(BRF + rs * 4 + g), (r_last >> rs) & 1u, status);
        cp_async_wait<0>();
    } else if (warp == kTcMmaWarp) {
        // ------------------------------------------------------------------ MMA issuer
        if (lane == 0) {
            const uint32_t id1 = tc_idesc_f16(S::N1);
            const uint32_t id2w = tc_idesc_f16(2 * S::N2), id2 = tc_idesc_f16(S::N2);
            // descriptors of the buffer bases; an operand at byte offset o from its base has descriptor base + o/16
            // (the start-address field holds address/16, and every address stays below 256 KB)
            const uint64_t dA1 = smem_desc(sbase + (uint32_t)c.off_A1, S::LA1, 128);
            const uint64_t dA2 = smem_desc(sbase + (uint32_t)c.off_A2, S::LA2, 128);
            const uint64_t dB1 = smem_desc(sbase + (uint32_t)c.off_B1, S::LB1, 128);
            const uint64_t dB2 = smem_desc(sbase + (uint32_t)c.off_B2, S::LB2, 128);
            uint32_t u1 = 0, u2 = 0;  // units issued to GEMM1 / GEMM2
            int nitem = 0;
            auto gemm1 = [&](int s) {
                const int st = (int)(u1 & 1);
                wait_or_abort(B_(BA1F + st), (u1 >> 1) & 1, abort_flag, status);
                wait_or_abort(B_(BPE + st), ((u1 >> 1) & 1) ^ 1, abort_flag, status);
                tc_fence_after();
                if (!*abort_flag) {
                    const uint32_t dP = tmem + (uint32_t)(st * S::TM_P);
                    const uint64_t ah = dA1 + (uint64_t)((st * S::A1_STAGE) >> 4), al = ah + (S::A1_PLANE >> 4);
                    const uint64_t b = dB1 + (uint64_t)((s * S::B1_BOND) >> 4);
                    // one accumulator: hi*B_hi + lo*B_hi + hi*B_lo (B_lo = the rows after N1 of each chunk plane)
#pragma unroll
                    for (int kc = 0; kc < S::K1 / 16; ++kc) {
                        const uint64_t bh = b + (uint64_t)((2 * kc * S::LB1) >> 4), bl = bh + (uint64_t)S::N1;
                        const uint64_t kofs = (uint64_t)((2 * kc * S::LA1) >> 4);
                        umma_f16(dP, ah + kofs, bh, id1, kc > 0);
                        umma_f16(dP, al + kofs, bh, id1, 1);
                        umma_f16(dP, ah + kofs, bl, id1, 1);
                    }
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
                    const uint64_t ah = dA2 + (uint64_t)((st * S::A2_STAGE) >> 4), al = ah + (S::A2_PLANE >> 4);
                    const uint64_t b = dB2 + (uint64_t)((s * S::B2_BOND) >> 4);
#pragma unroll
                    for (int kc = 0; kc < S::K2 / 16; ++kc)
                        umma_f16(dO, ah + (uint64_t)((2 * kc * S::LA2) >> 4), b + (uint64_t)((2 * kc * S::LB2) >> 4), id2w,
                                 kc > 0);
#pragma unroll
                    for (int kc = 0; kc < S::K2 / 16; ++kc)
                        umma_f16(dO, al + (uint64_t)((2 * kc * S::LA2) >> 4), b + (uint64_t)((2 * kc * S::LB2) >> 4), id2, 1);
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
        const float2* ks = reinterpret_cast<const float2*>(smem + c.off_K);
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
                int e12[kTcMaxNB] = {0, 0, 0, 0};  // per bond: the exponents of GEMM1's operands (G^, dH twice)
                for (int s = 0; s < NB; ++s, ++u) {
                    const int st = (int)(u & 1);
                    const uint32_t par = (u >> 1) & 1;
                    // exponents of this unit (GEMM1's A scale of this row group, the bond's dH scale)
                    wait_or_abort(B_(BA1F + st), par, abort_flag, status);
                    const int e1 = xr[st * 8 + q], eH = xr[st * 8 + 4];
                    float2 k[9];  // K^_ij of this row's frequency (staged by the producers; zero where not in range)
#pragma unroll
                    for (int ij = 0; ij < 9; ++ij)
                        k[ij] = row_ok ? ks[(st * S::FT + q * S::FG + fp) * 9 + ij] : make_float2(0.f, 0.f);
                    mbar_arrive(B_(BXE + st));
                    // P_j rows from TMEM (all three loads, one wait), U_i = sum_j K_ij P_j
                    wait_or_abort(B_(BPF + st), par, abort_flag, status);
                    tc_fence_after();
                    float ur[3][S::NH], ui[3][S::NH];
#pragma unroll
                    for (int i = 0; i < 3; ++i)
#pragma unroll
                        for (int nn = 0; nn < S::NH; ++nn) ur[i][nn] = ui[i][nn] = 0.f;
                    float pv[3][2 * S::NH];
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        tmem_ld_half<S::NH>(tq + (uint32_t)(st * S::TM_P + j * 2 * NORB + 2 * h * S::NH), pv[j]);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
#pragma unroll
                        for (int nn = 0; nn < S::NH; ++nn) {
                            const float pr = pv[j][2 * nn], pim = pv[j][2 * nn + 1];
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
                    // one scale per warp: the rows (f', n) of this half of the group; the final phase reads it back
                    float m = 0.f;
#pragma unroll
                    for (int nn = 0; nn < S::NH; ++nn)
                        if (h * S::NH + nn < NORB)
#pragma unroll
                            for (int i = 0; i < 3; ++i) m = fmaxf(m, fmaxf(fabsf(ur[i][nn]), fabsf(ui[i][nn])));
                    const int e2 = scale_exp(warp_max_abs(m));
                    if (lane == 0) e2s[(((ntile & 1) * kTcMaxNB + s) * 4 + q) * 2 + h] = e2;
                    const Pow2 f2 = pow2_factors(e2);
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
                                    split2(scaled(ur[i][nn], f2), scaled(ui[i][nn], f2), hw[i], lw[i]);
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
                        if (t4 == s) e12[t4] = e1 + 2 * eH;
                }
                // S^(f)^T rows (f', n = mr): sum over bonds of the unscaled accumulators, times i*scale
                named_bar(1, kTcEpiWarps * 32);  // every warp's GEMM2 operand exponents of this tile are in place
                wait_or_abort(B_(BOF), ntile & 1, abort_flag, status);
                tc_fence_after();
                const int hrow = mr >= S::NH;  // the half (warp) that wrote this row (f', n = mr) of U^T
                float accr[S::NH], acci[S::NH];
#pragma unroll
                for (int mm = 0; mm < S::NH; ++mm) accr[mm] = acci[mm] = 0.f;
#pragma unroll
                for (int s = 0; s < kTcMaxNB; ++s) {
                    if (s < NB) {
                        const Pow2 unsc =  // undoes the operand scales of this bond
                            pow2_factors(-(e12[s] + e2s[(((ntile & 1) * kTcMaxNB + s) * 4 + q) * 2 + hrow]));
                        float p1[2 * S::NH], p2[2 * S::NH];
                        const uint32_t col = (uint32_t)(2 * S::TM_P + s * S::TM_O + 2 * h * S::NH);
                        tmem_ld_half<S::NH>(tq + col, p1);
                        tmem_ld_half<S::NH>(tq + col + S::N2, p2);
                        tmem_wait_ld();
#pragma unroll
                        for (int mm = 0; mm < S::NH; ++mm) {
                            accr[mm] = fmaf((p1[2 * mm] + p2[2 * mm]) * unsc.a, unsc.b, accr[mm]);
                            acci[mm] = fmaf((p1[2 * mm + 1] + p2[2 * mm + 1]) * unsc.a, unsc.b, acci[mm]);
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
