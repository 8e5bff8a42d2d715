// Mixed-precision forward of Eq. (3) on the tcgen05 tensor cores (Sec. 4.4, adapted).
//
// Regrouping (the paper's map fission and relayout, Sec. 4.3): per atom a,
// neighbour slot s (b = nbr[a][s]) and type t,
//
//   Y_i(E,k)  = sum_{q,w,sigma} G^t_b(E - sigma(w+1), k - q) W^sigma_i(q,w),
//   W^sigma_i = sum_j D^{tau(t,sigma)}_ij(q,w,a,s) dH_j^H,
//   Sigma^t_a(E,k) = i*scale * sum_s sum_i dH_i Y_i(E,k).
//
// For one (k, q) the first line is a GEMM whose rows are (E, m) -- energies
// stacked into the M dimension -- with K = (w, sigma, l) and N = (i, n). The
// energy shift E - sigma(w+1) moves the A operand by Norb rows, which is a
// start-address offset of the shared-memory descriptor on a window of G rows
// staged with a 16-byte row pitch (K-major, no swizzle). Complex numbers use
// the real embedding [Gr Gi] x [[Wr Wi], [-Wi Wr]] (split-complex, Sec. 4.4).
//
// Precision (Sec. 4.4 adapted to GB300's tensor-core formats):
//   G is scaled by a power of two per (t, b) and W by a power of two per
//   (a, s, t) (the paper's normalisation factors; exact, undone in FP64).
//   TF32  : one K segment [Gr Gi] (TF32, round to nearest) x W (TF32).
//   BF16X3: x = hi + lo with hi = bf16(x), lo = bf16(x - hi); the K dimension
//           holds three segments [G_hi | G_lo | G_hi] x [W_hi ; W_hi ; W_lo],
//           so one accumulation gives hi*hi + lo*hi + hi*lo (lo*lo dropped).
//   FP32 accumulation in TMEM within one qz slice; the slice is drained into
//   FP64 registers (sum over qz in FP64), and the final multiply by dH_i and
//   the sums over i and neighbours run in FP64.
//
// Kernels: (1) per-(t,b) max |G| for the scale, (2) staging of G into split
// planes laid out [t][kz][b][16-byte K chunk][row = E*Norb + m], (3) the
// tcgen05 kernel: CTA = (tile of TE energies = TE*Norb <= 128 rows, kz, atom,
// type); TMA (cp.async.bulk.tensor) loads each shifted window, out-of-range
// rows are zero-filled by the TMA unit (energies outside [0, NE) contribute
// nothing); the W tiles are formed in FP32 on the CUDA cores into shared
// memory; one thread issues the MMAs; every wait is bounded.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {
namespace {

constexpr int kThreads = 128;  // 4 warps: TMEM lanes 0..127 = tile rows
constexpr int kMaxNorb = 10;   // 6*Norb accumulator columns kept in registers
constexpr int kMaxCols = 6 * kMaxNorb;
constexpr uint32_t kWaitIters = 1u << 26;  // bounded waits (about a second)

struct MixCfg {
    int mode, Norb, nel, TE;
    int esz, kpad, nch, npad, kmma;  // element bytes, K per term, 16-B chunks per row, N, MMAs per term
    int wc, wr, rb, nblk, wb;        // window: frequencies, rows (alloc), rows per TMA box, boxes, B tiles per batch
    int tmem_cols, btile;
    int off_B, off_D, off_Ah, off_A64, off_red, smem;
    int nrows;                       // NE * Norb
};

MixCfg make_cfg(const sse_dims& d, int mode) {
    MixCfg c{};
    c.mode = mode;
    c.Norb = d.Norb;
    c.nel = d.Norb * d.Norb;
    c.TE = 128 / d.Norb;
    c.esz = mode == SSE_MODE_BF16X3 ? 2 : 4;
    const int kraw = mode == SSE_MODE_BF16X3 ? 6 * d.Norb : 2 * d.Norb;
    const int kstep = mode == SSE_MODE_BF16X3 ? 16 : 8;  // K per tcgen05.mma
    c.kpad = (kraw + kstep - 1) / kstep * kstep;
    c.kmma = c.kpad / kstep;
    c.nch = c.kpad * c.esz / 16;
    c.npad = (6 * d.Norb + 15) / 16 * 16;
    c.tmem_cols = c.npad <= 32 ? 32 : (c.npad <= 64 ? 64 : 128);
    c.btile = c.npad * c.kpad * c.esz;
    c.nrows = d.NE * d.Norb;
    c.wc = d.Nw < 32 ? d.Nw : 32;
    const int need = 128 + (c.wc - 1) * d.Norb;
    c.nblk = (need + 255) / 256;
    c.rb = ((need + c.nblk - 1) / c.nblk + 7) / 8 * 8;
    c.wr = c.rb * c.nblk;
    c.wb = 4;
    const int win = c.nch * c.wr * 16;
    const int bb = c.wb * c.btile;
    const int yx = 128 * kMaxCols * 8;  // FP64 accumulator exchange for the final multiply (aliases win + B)
    c.off_B = win;
    const int reg0 = (win + bb > yx ? win + bb : yx);
    c.off_D = (reg0 + 127) / 128 * 128;
    c.off_Ah = c.off_D + 2 * d.Nw * 9 * 8;
    c.off_A64 = (c.off_Ah + 3 * c.nel * 8 + 15) / 16 * 16;
    c.off_red = c.off_A64 + 3 * c.nel * 16;
    c.smem = c.off_red + 64 + 128;  // + alignment slack of the dynamic base
    return c;
}

// ---------------------------------------------------------------------------
// PTX helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    // tcgen05 shared-memory matrix descriptor: K-major, no swizzle, base offset 0
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;  // stride between 16-B chunks along K
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;  // stride between 8-row groups along M/N
    d |= (uint64_t)1 << 46;                      // descriptor version
    return d;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(phase)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
    for (uint32_t it = 0; it < kWaitIters; ++it)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2,
                                            uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
        ::"r"(dst), "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
        : "memory");
}

template <int MODE>
__device__ __forceinline__ void umma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    if (MODE == SSE_MODE_BF16X3)
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
    else
        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float to_tf32(float x) {  // round to nearest TF32, kept in an FP32 container
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

// power-of-two exponent e with 2^e <= m < 2^(e+1); 0 for m == 0
__device__ __forceinline__ int floor_log2(float m) {
    if (!(m > 0.f) || !isfinite(m)) return 0;
    int ex;
    frexpf(m, &ex);
    return ex - 1;
}

// ---------------------------------------------------------------------------
// staging
// ---------------------------------------------------------------------------
__global__ void gmax_kernel(sse_dims d, const double2* __restrict__ Gl, const double2* __restrict__ Gg,
                            unsigned* __restrict__ gmax) {
    const int nel = d.Norb * d.Norb;
    const size_t nblocks = (size_t)d.Nkz * d.NE * d.NA;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < 2 * nblocks;
         i += (size_t)gridDim.x * blockDim.x) {
        const int t = i >= nblocks;
        const size_t blk = i - (t ? nblocks : 0);
        const int b = (int)(blk % d.NA);
        const double2* G = (t ? Gg : Gl) + blk * nel;
        double m = 0.0;
        for (int e = 0; e < nel; ++e) {
            const double2 v = G[e];
            m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
        }
        atomicMax(gmax + t * d.NA + b, __float_as_uint(__double2float_ru(m)));
    }
}

template <int MODE>
__global__ void stage_kernel(sse_dims d, MixCfg c, const double2* __restrict__ Gl, const double2* __restrict__ Gg,
                             const unsigned* __restrict__ gmax, uint4* __restrict__ staged) {
    const int N = d.Norb;
    const size_t rows_per_slice = (size_t)c.nrows;
    const size_t total = 2ull * d.Nkz * d.NA * rows_per_slice;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t slice = i / rows_per_slice;  // (t*Nkz + k)*NA + b
        const int row = (int)(i - slice * rows_per_slice);
        const int b = (int)(slice % d.NA);
        const size_t tk = slice / d.NA;
        const int t = (int)(tk / d.Nkz), k = (int)(tk % d.Nkz);
        const int E = row / N, m = row - E * N;
        const double sG = ldexp(1.0, -floor_log2(__uint_as_float(gmax[t * d.NA + b])));
        const double2* src = (t ? Gg : Gl) + ((((size_t)k * d.NE + E) * d.NA + b) * N + m) * N;
        uint32_t w[32];  // up to 128 bytes of the staged row (kpad*esz <= 128 for Norb <= 10)
#pragma unroll
        for (int j = 0; j < 32; ++j) w[j] = 0;
        if (MODE == SSE_MODE_BF16X3) {
            uint16_t* h = reinterpret_cast<uint16_t*>(w);
            for (int l = 0; l < N; ++l) {
                const double2 g = src[l];
                const double xr = g.x * sG, xi = g.y * sG;
                const __nv_bfloat16 hr = __double2bfloat16(xr), hi = __double2bfloat16(xi);
                const __nv_bfloat16 lr = __double2bfloat16(xr - (double)__bfloat162float(hr));
                const __nv_bfloat16 li = __double2bfloat16(xi - (double)__bfloat162float(hi));
                const uint16_t uhr = __bfloat16_as_ushort(hr), uhi = __bfloat16_as_ushort(hi);
                h[0 * 2 * N + l] = uhr;  // segment 0: G_hi
                h[0 * 2 * N + N + l] = uhi;
                h[1 * 2 * N + l] = __bfloat16_as_ushort(lr);  // segment 1: G_lo
                h[1 * 2 * N + N + l] = __bfloat16_as_ushort(li);
                h[2 * 2 * N + l] = uhr;  // segment 2: G_hi
                h[2 * 2 * N + N + l] = uhi;
            }
        } else {
            float* f = reinterpret_cast<float*>(w);
            for (int l = 0; l < N; ++l) {
                const double2 g = src[l];
                f[l] = to_tf32((float)(g.x * sG));
                f[N + l] = to_tf32((float)(g.y * sG));
            }
        }
        uint4* dst = staged + slice * c.nch * rows_per_slice + row;
        for (int ch = 0; ch < c.nch; ++ch)
            dst[(size_t)ch * rows_per_slice] = make_uint4(w[4 * ch], w[4 * ch + 1], w[4 * ch + 2], w[4 * ch + 3]);
    }
}

// ---------------------------------------------------------------------------
// tensor-core kernel
// ---------------------------------------------------------------------------
template <int MODE>
__global__ void __launch_bounds__(kThreads, 2)
sigma_mixed_kernel(const __grid_constant__ CUtensorMap tmap, Problem p, MixCfg c, const unsigned* __restrict__ gmax,
                   double2* __restrict__ S_less, double2* __restrict__ S_greater, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // TMA destinations need 128-byte alignment: round the dynamic base up (the launch adds 128 bytes)
    unsigned char* smem = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
    __shared__ __align__(8) uint64_t bars[2];  // [0] TMA window, [1] MMA batch done
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    const sse_dims& d = p.d;
    const int N = d.Norb, nel = c.nel, TE = c.TE;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int E0 = blockIdx.x * TE;
    const int k = blockIdx.y;
    const int a = d.a_begin + (int)(blockIdx.z >> 1);
    const int t = (int)(blockIdx.z & 1);
    const int row = tid;  // tile row = TMEM lane
    const int le = row / N, mrow = row - le * N;
    const bool row_ok = le < TE && E0 + le < d.NE;

    unsigned char* sWin = smem;
    unsigned char* sB = smem + c.off_B;
    float2* sDw = reinterpret_cast<float2*>(smem + c.off_D);      // [2 sigma][Nw][9] (unscaled weights)
    float2* sAh = reinterpret_cast<float2*>(smem + c.off_Ah);     // [3][l][n] = conj(dH_j[n][l])
    double2* sA64 = reinterpret_cast<double2*>(smem + c.off_A64);  // [3][nel] dH (FP64)
    unsigned* sRed = reinterpret_cast<unsigned*>(smem + c.off_red);
    double* sY = reinterpret_cast<double*>(smem);                  // [128][kMaxCols] (final multiply)
    const uint32_t bar_tma = smem_u32(&bars[0]), bar_mma = smem_u32(&bars[1]);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                     "r"(c.tmem_cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        mbar_init(bar_tma, 1);
        mbar_init(bar_mma, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;
    uint32_t ph_tma = 0, ph_mma = 0;

    const uint32_t idesc = (1u << 4) | (MODE == SSE_MODE_BF16X3 ? (1u << 7) | (1u << 10) : (2u << 7) | (2u << 10)) |
                           ((uint32_t)(c.npad >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t win_addr = smem_u32(sWin), b_addr = smem_u32(sB);
    const uint32_t plane = (uint32_t)c.wr * 16, bplane = (uint32_t)c.npad * 16;
    const int ncols = 6 * N;

    double2 sig[kMaxNorb];
#pragma unroll
    for (int n = 0; n < kMaxNorb; ++n) sig[n] = make_double2(0.0, 0.0);

    for (int s = 0; s < d.NB; ++s) {
        const int b = p.nbr[(size_t)a * d.NB + s];
        if (b < 0 || b >= d.NA) {  // uniform per CTA
            if (tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
            continue;
        }
        __syncthreads();  // previous slot's final multiply is done with sY / sA64
        // the B region is reused: padding entries of every tile must be zero
        for (int i = tid; i < c.wb * c.btile / 16; i += kThreads)
            reinterpret_cast<uint4*>(sB)[i] = make_uint4(0, 0, 0, 0);
        const double2* Ag = p.dH + ((size_t)a * d.NB + s) * 3 * nel;
        float amax = 0.f;
        for (int i = tid; i < 3 * nel; i += kThreads) {
            const double2 v = Ag[i];
            sA64[i] = v;
            const int j = i / nel, e = i - j * nel, nn = e / N, l = e - nn * N;
            sAh[(j * N + l) * N + nn] = make_float2((float)v.x, -(float)v.y);
            amax = fmaxf(amax, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
        }
        float dmax = 0.f;
        for (int i = tid; i < 2 * d.Nqz * d.Nw * 9; i += kThreads) {
            const int tau = i / (d.Nqz * d.Nw * 9), r = i - tau * d.Nqz * d.Nw * 9;
            const int qw = r / 9, ij = r - qw * 9;
            const double2 v = p.D[tau][(((size_t)qw * d.NA + a) * d.NB + s) * 9 + ij];
            dmax = fmaxf(dmax, fmaxf(fabsf((float)v.x), fabsf((float)v.y)));
        }
        if (tid == 0) { sRed[0] = 0; sRed[1] = 0; }
        __syncthreads();
        atomicMax(&sRed[0], __float_as_uint(amax));
        atomicMax(&sRed[1], __float_as_uint(dmax));
        __syncthreads();
        // |W_i[l][n]| <= sum_j |D_ij| |dH_j[n][l]| <= 2 * 3 * dmax * amax (re and im parts)
        const float wbound = 6.f * __uint_as_float(sRed[0]) * __uint_as_float(sRed[1]);
        const int ew = floor_log2(wbound) + 1;
        const float sW = ldexpf(1.f, -ew);
        const int eg = floor_log2(__uint_as_float(gmax[t * d.NA + b]));
        const double unscale = ldexp(1.0, ew + eg);  // 1 / (sG * sW)

        double Y[kMaxCols];
#pragma unroll
        for (int j = 0; j < kMaxCols; ++j) Y[j] = 0.0;

        for (int q = 0; q < d.Nqz; ++q) {
            const int kp = ((k - q) % d.Nkz + d.Nkz) % d.Nkz;
            const int slice = (t * d.Nkz + kp) * d.NA + b;
            __syncthreads();  // all MMAs of the previous slice are complete (waited below)
            for (int i = tid; i < 2 * d.Nw * 9; i += kThreads) {
                const int sg = i / (d.Nw * 9), r = i - sg * d.Nw * 9;
                const int w = r / 9, ij = r - w * 9;
                const int tau = sg == 0 ? t : 1 - t;
                const double2 v = p.D[tau][((((size_t)q * d.Nw + w) * d.NA + a) * d.NB + s) * 9 + ij];
                sDw[i] = make_float2((float)v.x, (float)v.y);
            }
            __syncthreads();
            uint32_t acc_flag = 0;
            for (int sg = 0; sg < 2; ++sg) {
                const int sigma = sg == 0 ? +1 : -1;
                const int wend = min(d.Nw, sigma > 0 ? E0 + TE - 1 : d.NE - 1 - E0);
                for (int w0 = 0; w0 < wend; w0 += c.wc) {
                    const int wn = min(c.wc, wend - w0);
                    const int r0 = E0 * N;
                    const int start = sigma > 0 ? r0 - (w0 + wn) * N : r0 + (w0 + 1) * N;
                    if (tid == 0) {  // the window is free: the last batch of MMAs was waited for
                        mbar_expect_tx(bar_tma, (uint32_t)(c.nch * c.wr * 16));
                        for (int ch = 0; ch < c.nch; ++ch)
                            for (int bk = 0; bk < c.nblk; ++bk)
                                tma_load_3d(win_addr + (uint32_t)(ch * c.wr + bk * c.rb) * 16, &tmap, 0,
                                            start + bk * c.rb, slice * c.nch + ch, bar_tma);
                    }
                    for (int wb0 = 0; wb0 < wn; wb0 += c.wb) {
                        const int nb = min(c.wb, wn - wb0);
                        // W tiles (B operand, K-major: row nn = (i*N + n)*2 + re/im, column kk of the A row)
                        for (int it = tid; it < nb * 3 * nel; it += kThreads) {
                            const int wi = it / (3 * nel), rem = it - wi * 3 * nel;
                            const int i = rem / nel, e = rem - i * nel, l = e / N, n = e - l * N;
                            const float2* Dw = sDw + ((size_t)sg * d.Nw + w0 + wb0 + wi) * 9 + i * 3;
                            float wr = 0.f, wim = 0.f;
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                const float2 dv = Dw[j];
                                const float2 ah = sAh[(j * N + l) * N + n];
                                wr = fmaf(dv.x, ah.x, fmaf(-dv.y, ah.y, wr));
                                wim = fmaf(dv.x, ah.y, fmaf(dv.y, ah.x, wim));
                            }
                            wr *= sW;
                            wim *= sW;
                            unsigned char* tile = sB + (size_t)wi * c.btile;
                            const int nre = (i * N + n) * 2, nim = nre + 1;
                            if (MODE == SSE_MODE_BF16X3) {
                                const __nv_bfloat16 hr = __float2bfloat16_rn(wr), hi = __float2bfloat16_rn(wim);
                                const __nv_bfloat16 lr = __float2bfloat16_rn(wr - __bfloat162float(hr));
                                const __nv_bfloat16 li = __float2bfloat16_rn(wim - __bfloat162float(hi));
                                const __nv_bfloat16 nhi = __hneg(hi), nli = __hneg(li);
                                auto put = [&](int nn, int kk, __nv_bfloat16 v) {
                                    *reinterpret_cast<__nv_bfloat16*>(tile + (kk >> 3) * bplane + nn * 16 +
                                                                      (kk & 7) * 2) = v;
                                };
#pragma unroll
                                for (int seg = 0; seg < 3; ++seg) {
                                    const __nv_bfloat16 vr = seg < 2 ? hr : lr, vi = seg < 2 ? hi : li;
                                    const __nv_bfloat16 nvi = seg < 2 ? nhi : nli;
                                    const int kr = seg * 2 * N + l, ki = kr + N;
                                    put(nre, kr, vr);
                                    put(nre, ki, nvi);
                                    put(nim, kr, vi);
                                    put(nim, ki, vr);
                                }
                            } else {
                                const float vr = to_tf32(wr), vi = to_tf32(wim);
                                auto put = [&](int nn, int kk, float v) {
                                    *reinterpret_cast<float*>(tile + (kk >> 2) * bplane + nn * 16 + (kk & 3) * 4) = v;
                                };
                                put(nre, l, vr);
                                put(nre, N + l, -vi);
                                put(nim, l, vi);
                                put(nim, N + l, vr);
                            }
                        }
                        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                        __syncthreads();
                        int bad = 0;
                        if (tid == 0) {
                            if (wb0 == 0) bad = !mbar_wait(bar_tma, ph_tma);
                            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                            if (!bad) {
                                for (int wi = 0; wi < nb; ++wi) {
                                    const int w = w0 + wb0 + wi;
                                    const int roff = sigma > 0 ? (w0 + wn - w - 1) * N : (w - w0) * N;
                                    for (int kc = 0; kc < c.kmma; ++kc) {
                                        const uint64_t da =
                                            smem_desc(win_addr + (uint32_t)(2 * kc) * plane + (uint32_t)roff * 16, plane, 128);
                                        const uint64_t db =
                                            smem_desc(b_addr + (uint32_t)(wi * c.btile) + (uint32_t)(2 * kc) * bplane, bplane, 128);
                                        umma<MODE>(tmem, da, db, idesc, acc_flag);
                                        acc_flag = 1;
                                    }
                                }
                                umma_commit(bar_mma);
                            }
                        }
                        if (!bad) bad = !mbar_wait(bar_mma, ph_mma);
                        ph_mma ^= 1;
                        if (__syncthreads_or(bad)) {
                            if (tid == 0) atomicOr(status, DEV_TIMEOUT);
                            goto cleanup;
                        }
                        acc_flag = 1;  // every later MMA of this slice accumulates
                    }
                    ph_tma ^= 1;
                }
            }
            // drain the slice: FP32 TMEM -> FP64 registers, undo the scales
            if (acc_flag) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int c0 = 0; c0 < kMaxCols; c0 += 16) {
                    if (c0 < ncols) {
                        float v[16];
                        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < kMaxCols) Y[c0 + j] += (double)v[j] * unscale;
                    }
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            }
        }
        // final multiply in FP64: sig[n'] += sum_i sum_l dH_i[m][l] Y_i[(le, l)][n']
        __syncthreads();  // window / B regions are free (aliased by sY)
#pragma unroll
        for (int j = 0; j < kMaxCols; ++j) sY[(size_t)row * kMaxCols + j] = Y[j];
        __syncthreads();
        if (row_ok) {
            for (int i = 0; i < 3; ++i)
                for (int l = 0; l < N; ++l) {
                    const double2 A = sA64[i * nel + mrow * N + l];
                    const double* Yr = sY + (size_t)(le * N + l) * kMaxCols + i * N * 2;
#pragma unroll
                    for (int n = 0; n < kMaxNorb; ++n)
                        if (n < N) {
                            const double yr = Yr[2 * n], yi = Yr[2 * n + 1];
                            sig[n].x = fma(A.x, yr, fma(-A.y, yi, sig[n].x));
                            sig[n].y = fma(A.x, yi, fma(A.y, yr, sig[n].y));
                        }
                }
        }
    }

    {
        // store Sigma = i*scale*sig, optionally (S - S^H)/2 (FP64)
        const double sc = p.scale;
        double2* out = t == 0 ? S_less : S_greater;
        double2* sS = reinterpret_cast<double2*>(smem);  // [128][kMaxNorb]
        const bool sym = (p.flags & SSE_FLAG_SYMMETRIZE) != 0;
        __syncthreads();
#pragma unroll
        for (int n = 0; n < kMaxNorb; ++n) {
            sig[n] = make_double2(-sc * sig[n].y, sc * sig[n].x);
            sS[(size_t)row * kMaxNorb + n] = sig[n];
        }
        __syncthreads();
        if (row_ok) {
            double2* o = out + ((((size_t)k * d.NE + E0 + le) * d.NA + a) * N + mrow) * N;
#pragma unroll
            for (int n = 0; n < kMaxNorb; ++n)
                if (n < N) {
                    double2 v = sig[n];
                    if (sym) {
                        const double2 u = sS[(size_t)(le * N + n) * kMaxNorb + mrow];
                        v = make_double2(0.5 * (v.x - u.x), 0.5 * (v.y + u.y));
                    }
                    o[n] = v;
                }
        }
    }
cleanup:
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(c.tmem_cols));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    }
    return fn;
}

struct WsLayout {
    size_t gmax_off, staged_off, total;
};

WsLayout ws_layout(const sse_dims& d, const MixCfg& c) {
    WsLayout w;
    w.gmax_off = 0;
    w.staged_off = ((size_t)2 * d.NA * 4 + 255) / 256 * 256;
    w.total = w.staged_off + (size_t)2 * d.Nkz * d.NA * c.nch * c.nrows * 16;
    return w;
}

template <int MODE>
cudaError_t launch(const Problem& p, const MixCfg& c, double2* Sl, double2* Sg, unsigned* status, void* ws,
                   cudaStream_t st) {
    const sse_dims& d = p.d;
    const WsLayout L = ws_layout(d, c);
    unsigned* gmax = reinterpret_cast<unsigned*>(static_cast<char*>(ws) + L.gmax_off);
    uint4* staged = reinterpret_cast<uint4*>(static_cast<char*>(ws) + L.staged_off);
    cudaError_t e = cudaMemsetAsync(gmax, 0, (size_t)2 * d.NA * 4, st);
    if (e != cudaSuccess) return e;
    gmax_kernel<<<152 * 8, 256, 0, st>>>(d, p.G[0], p.G[1], gmax);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    stage_kernel<MODE><<<152 * 16, 256, 0, st>>>(d, c, p.G[0], p.G[1], gmax, staged);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap map;
    const cuuint64_t dims[3] = {16, (cuuint64_t)c.nrows, (cuuint64_t)2 * d.Nkz * d.NA * c.nch};
    const cuuint64_t strides[2] = {16, (cuuint64_t)c.nrows * 16};
    const cuuint32_t box[3] = {16, (cuuint32_t)c.rb, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 3, staged, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(sigma_mixed_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    if (e != cudaSuccess) return e;
    const int nA = d.a_end - d.a_begin;
    dim3 grid((d.NE + c.TE - 1) / c.TE, d.Nkz, 2 * nA);
    sigma_mixed_kernel<MODE><<<grid, kThreads, c.smem, st>>>(map, p, c, gmax, Sl, Sg, status);
    return cudaGetLastError();
}

}  // namespace

size_t mixed_fwd_workspace(const sse_dims& d, int mode) {
    if (d.Norb > kMaxNorb) return 0;
    return ws_layout(d, make_cfg(d, mode)).total;
}

cudaError_t mixed_fwd(const Problem& p, int mode, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                      size_t ws_bytes, cudaStream_t st) {
    if (p.d.Norb > kMaxNorb) return cudaErrorNotSupported;
    const MixCfg c = make_cfg(p.d, mode);
    if (c.smem > 113 * 1024 || ws_bytes < ws_layout(p.d, c).total) return cudaErrorNotSupported;
    if (mode == SSE_MODE_BF16X3) return launch<SSE_MODE_BF16X3>(p, c, S_less, S_greater, status, ws, st);
    return launch<SSE_MODE_TF32>(p, c, S_less, S_greater, status, ws, st);
}

}  // namespace sse
