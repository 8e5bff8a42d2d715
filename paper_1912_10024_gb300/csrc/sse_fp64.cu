// FP64 forward of the electron scattering self-energy, Eq. (3) (Sec. 2).
//
// Regrouping (the paper's map fission, Sec. 4.3, step 1): for one atom a and
// neighbour slot s the double sum over i, j factors as
//
//   Sigma^t_a(E,k) += i*scale * sum_ij dH_i X_ij(E,k) dH_j^H,
//   X_ij(E,k) = sum_{q,w,sigma} D^{tau(t,sigma)}_ij(q,w,a,s) G^t_b(E - sigma(w+1), k - q).
//
// X_ij costs 9 complex MACs per block element per (q, w, sigma) term, against
// 3 Norb^3 for multiplying full blocks, so on GB300 -- where FP64 runs on a
// narrow CUDA-core pipe and tcgen05 has no FP64 kind -- the hot loop is the
// element-wise correlation (sse_fp64_common.cuh) and the block products
// happen once per (E, k, s) in the epilogue.
//
// CTA = (energy tile of TE energies, kz, atom a, type t); it loops over the
// neighbour slots s and keeps Sigma of its tile in registers.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse_fp64_common.cuh"
#include "sse_internal.h"

namespace sse {
namespace {

using namespace fp64;
constexpr int kEpiBlocks = 12;  // X [TE][9] + Y [TE][3]

__global__ void __launch_bounds__(kMaxThreads)
sigma_fp64_fwd_kernel(Problem p, TileCfg c, double2* __restrict__ S_less, double2* __restrict__ S_greater,
                      unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const sse_dims& d = p.d;
    const int Norb = d.Norb, nel = c.nel, nth = c.nthreads, TE = c.TE;
    const int tid = threadIdx.x;
    const int el = tid % nel, grp = tid / nel;
    const int E0 = blockIdx.x * TE;
    const int k = blockIdx.y;
    const int a = d.a_begin + (int)(blockIdx.z >> 1);
    const int t = (int)(blockIdx.z & 1);

    double2* sA = reinterpret_cast<double2*>(smem);            // [3][nel]
    double2* sX = reinterpret_cast<double2*>(smem + c.off_U);  // [TE][9][nel] (epilogue)
    double2* sY = sX + (size_t)TE * 9 * nel;                   // [TE][3][nel]

    double2 accS[kR];
#pragma unroll
    for (int j = 0; j < kR; ++j) accS[j] = make_double2(0.0, 0.0);

    for (int s = 0; s < d.NB; ++s) {
        const int b = p.nbr[(size_t)a * d.NB + s];
        const bool bvalid = b >= 0 && b < d.NA;
        if (!bvalid && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        __syncthreads();  // previous epilogue is done with sA / sX / sY
        const double2* Ag = p.dH + ((size_t)a * d.NB + s) * 3 * nel;
        for (int i = tid; i < 3 * nel; i += nth) sA[i] = Ag[i];

        double K[kR][9][3];
        correlate_tile(p, c, smem, a, s, t, k, E0, b, bvalid, el, grp, K);

        // ---- epilogue of neighbour s: Sigma += sum_i dH_i (sum_j X_ij dH_j^H) ----
        store_x(sX, nel, el, grp, K);
        __syncthreads();
        for (int it = tid; it < TE * 3 * nel; it += nth) {  // Y_i = sum_j X_ij dH_j^H
            const int le = it / (3 * nel), rem = it - le * 3 * nel;
            const int i = rem / nel, mn = rem - i * nel;
            const int m = mn / Norb, n2 = mn - m * Norb;
            double2 acc = make_double2(0.0, 0.0);
            for (int j = 0; j < 3; ++j) {
                const double2* Xr = sX + ((size_t)le * 9 + i * 3 + j) * nel + m * Norb;
                const double2* Ar = sA + j * nel + n2 * Norb;
                for (int n = 0; n < Norb; ++n) acc = cfma_conjb(Xr[n], Ar[n], acc);
            }
            sY[((size_t)le * 3 + i) * nel + mn] = acc;
        }
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kR; ++jj) {  // Sigma += sum_i dH_i Y_i
            const int it = tid + jj * nth;
            const int le = it / nel, mn = it - le * nel;
            const int m2 = mn / Norb, n2 = mn - m2 * Norb;
            double2 acc = accS[jj];
            for (int i = 0; i < 3; ++i) {
                const double2* Ar = sA + i * nel + m2 * Norb;
                const double2* Yc = sY + ((size_t)le * 3 + i) * nel + n2;
                for (int m = 0; m < Norb; ++m) acc = cfma(Ar[m], Yc[m * Norb], acc);
            }
            accS[jj] = acc;
        }
    }

    // ---- store: Sigma = i*scale*acc, optionally (S - S^H)/2 ----
    double2* out = t == 0 ? S_less : S_greater;
    const double sc = p.scale;
    if (p.flags & SSE_FLAG_SYMMETRIZE) {
        __syncthreads();
#pragma unroll
        for (int jj = 0; jj < kR; ++jj) sX[tid + jj * nth] = make_double2(-sc * accS[jj].y, sc * accS[jj].x);
        __syncthreads();
    }
#pragma unroll
    for (int jj = 0; jj < kR; ++jj) {
        const int it = tid + jj * nth;
        const int le = it / nel, mn = it - le * nel;
        const int E = E0 + le;
        if (E >= d.NE) continue;
        double2 v = make_double2(-sc * accS[jj].y, sc * accS[jj].x);
        if (p.flags & SSE_FLAG_SYMMETRIZE) {
            const int m = mn / Norb, n = mn - m * Norb;
            const double2 u = sX[(size_t)le * nel + n * Norb + m];
            v = make_double2(0.5 * (v.x - u.x), 0.5 * (v.y + u.y));
        }
        out[(((size_t)k * d.NE + E) * d.NA + a) * nel + mn] = v;
    }
}

}  // namespace

size_t fp64_fwd_workspace(const sse_dims&) { return 0; }

cudaError_t fp64_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void*, size_t,
                     cudaStream_t st) {
    const TileCfg c = make_tile_cfg(p.d, kEpiBlocks);
    if (c.smem > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(sigma_fp64_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    if (e != cudaSuccess) return e;
    const int nA = p.d.a_end - p.d.a_begin;
    dim3 grid((p.d.NE + c.TE - 1) / c.TE, p.d.Nkz, 2 * nA);
    SSE_TIMED("sigma_fp64_fwd_kernel", st, sigma_fp64_fwd_kernel<<<grid, c.nthreads, c.smem, st>>>(p, c, S_less, S_greater, status));
    return cudaGetLastError();
}

}  // namespace sse
