// FP64 forward of the electron scattering self-energy, Eq. (3) (Sec. 2).
//
// Regrouping (the paper's map fission, Sec. 4.3, step 1): for one atom a and
// neighbour slot s the double sum over i, j factors as
//
//   Sigma^t_a(E,k) += i*scale * sum_ij dH_i X_ij(E,k) dH_j^H,
//   X_ij(E,k) = sum_{q,w,sigma} D^{tau(t,sigma)}_ij(q,w,a,s) G^t_b(E - sigma(w+1), k - q).
//
// X_ij is a 2-D correlation of G_b over (E, kz) with a 3x3 complex kernel per
// (q, w, sigma), separable in the Norb^2 block elements. It costs 9 complex
// MACs per element per term, against 3 Norb^3 for multiplying full blocks, so
// on GB300 -- where FP64 runs on a narrow CUDA-core pipe and FP64 tensor cores
// do not exist in tcgen05 -- the block products are done once per (E,k,s) in
// the epilogue and the hot loop is the element-wise correlation.
//
// The complex MACs use the three-multiplication form (Gauss): with weight
// p+iq and input u+iv, K1 += p(u+v), K2 += (q-p)u, K3 += (p+q)v, and
// Re = K1 - K3, Im = K1 + K2. The weight planes are formed once per tile and
// the input plane u+v once per window element, so the inner loop issues 3 DFMA
// per complex MAC instead of 4.
//
// CTA = (energy tile of TE energies, kz, atom a, type t). Threads = P x Norb^2:
// thread (g, e) owns block element e for energies E0 + g*R + r, r < R, and keeps
// its 9 x 3 x R partial sums in registers. Per (s, q, sigma, frequency chunk)
// the CTA stages the weights and the shifted energy window of G_b in shared
// memory (rows outside [0, NE) are zero: out-of-range energies contribute
// nothing). After all (q, w, sigma) of one neighbour the X blocks go through
// shared memory for the two FP64 block products.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {
namespace {

constexpr int kR = 2;            // energies per thread
constexpr int kMaxThreads = 384;  // P * Norb^2 <= kMaxThreads
constexpr int kSmemBudget = 200 * 1024;

// Three-multiplication weight planes of one complex weight p + iq.
struct __align__(32) Weight3 {
    double x, y, z, pad;  // p, q - p, p + q
};

struct FwdCfg {
    int nel, P, TE, nthreads, wc;
    int off_Dw, off_U, raw_bytes;  // byte offsets in dynamic shared memory
    int smem;
};

__device__ __forceinline__ double2 cfma(double2 a, double2 b, double2 c) {  // a*b + c
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(-a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(a.y, b.x, c.y);
    return c;
}
__device__ __forceinline__ double2 cfma_conjb(double2 a, double2 b, double2 c) {  // a*conj(b) + c
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(a.y, b.x, c.y);
    c.y = fma(-a.x, b.y, c.y);
    return c;
}

__global__ void __launch_bounds__(kMaxThreads)
sigma_fp64_fwd_kernel(Problem p, FwdCfg c, double2* __restrict__ S_less, double2* __restrict__ S_greater,
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

    double2* sA = reinterpret_cast<double2*>(smem);                  // [3][nel]
    Weight3* sDw = reinterpret_cast<Weight3*>(smem + c.off_Dw);      // [wc][9]: (p, q-p, p+q, -)
    double2* sRaw = reinterpret_cast<double2*>(smem + c.off_U);      // [rows][nel]
    double* sSum = reinterpret_cast<double*>(smem + c.off_U + c.raw_bytes);  // [rows][nel]: u+v
    double2* sX = reinterpret_cast<double2*>(smem + c.off_U);        // [TE][9][nel] (epilogue)
    double2* sY = sX + (size_t)TE * 9 * nel;                         // [TE][3][nel]

    double2 accS[kR];
#pragma unroll
    for (int j = 0; j < kR; ++j) accS[j] = make_double2(0.0, 0.0);

    const size_t rowStride = (size_t)d.NA * nel;  // elements between consecutive energies of G
    for (int s = 0; s < d.NB; ++s) {
        const int b = p.nbr[(size_t)a * d.NB + s];
        const bool bvalid = b >= 0 && b < d.NA;
        if (!bvalid && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        __syncthreads();  // previous epilogue is done with sA / sX / sY
        const double2* Ag = p.dH + ((size_t)a * d.NB + s) * 3 * nel;
        for (int i = tid; i < 3 * nel; i += nth) sA[i] = Ag[i];

        double K[kR][9][3];
#pragma unroll
        for (int r = 0; r < kR; ++r)
#pragma unroll
            for (int ij = 0; ij < 9; ++ij) K[r][ij][0] = K[r][ij][1] = K[r][ij][2] = 0.0;

        for (int q = 0; q < d.Nqz; ++q) {
            const int kp = ((k - q) % d.Nkz + d.Nkz) % d.Nkz;
            const double2* Gb = p.G[t] + (size_t)kp * d.NE * rowStride + (size_t)(bvalid ? b : 0) * nel;
#pragma unroll 1
            for (int sg = 0; sg < 2; ++sg) {
                const int sigma = sg == 0 ? +1 : -1;
                const double2* Dt = p.D[sg == 0 ? t : 1 - t];
                // frequencies whose shifted energy is off the grid for every energy of the tile
                // contribute nothing: emission needs E0+TE-1-(w+1) >= 0, absorption E0+w+1 < NE
                const int wend = min(d.Nw, sigma > 0 ? E0 + TE - 1 : d.NE - 1 - E0);
                for (int w0 = 0; w0 < wend; w0 += c.wc) {
                    const int wn = min(c.wc, wend - w0);
                    const int rows = TE + wn - 1;
                    const int Elo = sigma > 0 ? E0 - w0 - wn : E0 + w0 + 1;
                    __syncthreads();  // previous chunk is done with the window and weights
                    for (int i = tid; i < wn * 9; i += nth) {
                        const int wi = i / 9, ij = i - 9 * wi;
                        const double2 v =
                            Dt[((((size_t)q * d.Nw + w0 + wi) * d.NA + a) * d.NB + s) * 9 + ij];
                        sDw[i] = Weight3{v.x, v.y - v.x, v.x + v.y, 0.0};
                    }
                    for (int i = tid; i < rows * nel; i += nth) {
                        const int row = i / nel, e2 = i - row * nel;
                        const int Ep = Elo + row;
                        double2 v = make_double2(0.0, 0.0);
                        if (bvalid && Ep >= 0 && Ep < d.NE) v = __ldg(Gb + (size_t)Ep * rowStride + e2);
                        sRaw[i] = v;
                        sSum[i] = v.x + v.y;
                    }
                    __syncthreads();
#pragma unroll 1
                    for (int wi = 0; wi < wn; ++wi) {
                        double2 x[kR];
                        double xs[kR];
#pragma unroll
                        for (int r = 0; r < kR; ++r) {
                            const int le = grp * kR + r;
                            const int row = sigma > 0 ? le + (wn - 1) - wi : le + wi;
                            x[r] = sRaw[row * nel + el];
                            xs[r] = sSum[row * nel + el];
                        }
#pragma unroll
                        for (int ij = 0; ij < 9; ++ij) {
                            const Weight3 dw = sDw[wi * 9 + ij];
#pragma unroll
                            for (int r = 0; r < kR; ++r) {
                                K[r][ij][0] = fma(dw.x, xs[r], K[r][ij][0]);
                                K[r][ij][1] = fma(dw.y, x[r].x, K[r][ij][1]);
                                K[r][ij][2] = fma(dw.z, x[r].y, K[r][ij][2]);
                            }
                        }
                    }
                }
            }
        }

        // ---- epilogue of neighbour s: Sigma += sum_i dH_i (sum_j X_ij dH_j^H) ----
        __syncthreads();  // all threads done with the window (sX aliases it)
#pragma unroll
        for (int r = 0; r < kR; ++r) {
            const int le = grp * kR + r;
#pragma unroll
            for (int ij = 0; ij < 9; ++ij)
                sX[((size_t)le * 9 + ij) * nel + el] =
                    make_double2(K[r][ij][0] - K[r][ij][2], K[r][ij][0] + K[r][ij][1]);
        }
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

FwdCfg make_cfg(const sse_dims& d) {
    FwdCfg c{};
    c.nel = d.Norb * d.Norb;
    c.P = kMaxThreads / c.nel;
    if (c.P < 1) c.P = 1;
    c.nthreads = c.P * c.nel;
    c.TE = c.P * kR;
    const int a_bytes = 3 * c.nel * 16;
    const int epi_bytes = c.TE * 12 * c.nel * 16;  // X [TE][9] + Y [TE][3]
    // largest frequency chunk whose window + weights fit next to the epilogue buffers
    int wc = d.Nw;
    for (; wc > 1; --wc) {
        const int win = (c.TE + wc - 1) * c.nel * 24;
        const int u = win > epi_bytes ? win : epi_bytes;
        if (a_bytes + wc * 9 * 32 + u <= kSmemBudget) break;
    }
    c.wc = wc;
    c.off_Dw = a_bytes;
    c.off_U = a_bytes + wc * 9 * 32;
    c.raw_bytes = (c.TE + wc - 1) * c.nel * 16;
    const int win = (c.TE + wc - 1) * c.nel * 24;
    c.smem = c.off_U + (win > epi_bytes ? win : epi_bytes);
    return c;
}

}  // namespace

size_t fp64_fwd_workspace(const sse_dims&) { return 0; }

cudaError_t fp64_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void*, size_t,
                     cudaStream_t st) {
    const FwdCfg c = make_cfg(p.d);
    if (c.smem > 227 * 1024) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(sigma_fp64_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    if (e != cudaSuccess) return e;
    const int nA = p.d.a_end - p.d.a_begin;
    dim3 grid((p.d.NE + c.TE - 1) / c.TE, p.d.Nkz, 2 * nA);
    sigma_fp64_fwd_kernel<<<grid, c.nthreads, c.smem, st>>>(p, c, S_less, S_greater, status);
    return cudaGetLastError();
}

}  // namespace sse
