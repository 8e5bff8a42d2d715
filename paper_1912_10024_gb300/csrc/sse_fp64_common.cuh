// Device code shared by the FP64 forward and adjoint kernels of Eq. (3).
//
// Both recompute, for one atom a, neighbour slot s (b = nbr[a][s]), type t,
// momentum kz and an energy tile E0 .. E0+TE-1, the 3x3 blocks
//
//   X_ij(E,k) = sum_{q,w,sigma} D^{tau(t,sigma)}_ij(q,w,a,s) G^t_b(E - sigma(w+1), k - q)
//
// of the regrouped Eq. (3) (Sigma^t_a = i*scale * sum_s sum_ij dH_i X_ij dH_j^H).
// X_ij is a correlation of G_b over (E, kz) with a 3x3 complex kernel per
// (q, w, sigma), separable in the Norb^2 block elements.
//
// Thread layout: P x Norb^2 threads; thread (g, e) owns block element e for
// energies E0 + g*kR + r. Complex MACs use the three-multiplication form:
// weight p+iq, input u+iv: K1 += p(u+v), K2 += (q-p)u, K3 += (p+q)v, and
// Re = K1 - K3, Im = K1 + K2. Shared memory per (q, sigma, frequency chunk):
// the weights as planes (p, q-p, p+q) and the shifted energy window of G_b as
// (u, v) plus the plane u+v; rows outside [0, NE) are zero (out-of-range
// energies contribute nothing).
#pragma once

#include <cuda_runtime.h>

#include "sse_internal.h"

namespace sse {
namespace fp64 {

constexpr int kR = 2;              // energies per thread
constexpr int kMaxThreads = 384;   // P * Norb^2 <= kMaxThreads (keeps <= 168 registers)
constexpr int kSmemBudget = 200 * 1024;

struct __align__(32) Weight3 {
    double x, y, z, pad;  // p, q - p, p + q of one complex weight p + iq
};

struct TileCfg {
    int nel, P, TE, nthreads, wc;
    int off_Dw, off_U, raw_bytes;  // byte offsets in dynamic shared memory
    int smem;
};

// epi_blocks: complex Norb x Norb blocks per energy that the kernel's epilogue keeps in shared memory.
inline TileCfg make_tile_cfg(const sse_dims& d, int epi_blocks) {
    TileCfg c{};
    c.nel = d.Norb * d.Norb;
    c.P = kMaxThreads / c.nel;
    const int reserve = 3 * c.nel * 16 + 9 * 32 * (d.Nw < 8 ? d.Nw : 8);  // dH blocks + a small weight chunk
    const int pmax = (kSmemBudget - reserve) / (epi_blocks * kR * c.nel * 16);
    if (c.P > pmax) c.P = pmax;
    if (c.P < 1) c.P = 1;
    c.nthreads = c.P * c.nel;
    c.TE = c.P * kR;
    const int a_bytes = 3 * c.nel * 16;
    const int epi_bytes = c.TE * epi_blocks * c.nel * 16;
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
__device__ __forceinline__ double2 cfma_conja(double2 a, double2 b, double2 c) {  // conj(a)*b + c
    c.x = fma(a.x, b.x, c.x);
    c.x = fma(a.y, b.y, c.x);
    c.y = fma(a.x, b.y, c.y);
    c.y = fma(-a.y, b.x, c.y);
    return c;
}

// X_ij partial sums (three-multiplication form) of the tile for slot s; see file comment.
// Must be called by all threads of the CTA (it synchronises).
__device__ __forceinline__ void correlate_tile(const Problem& p, const TileCfg& c, unsigned char* smem, int a,
                                               int s, int t, int k, int E0, int b, bool bvalid, int el, int grp,
                                               double (&K)[kR][9][3]) {
    const sse_dims& d = p.d;
    const int nel = c.nel, nth = c.nthreads, TE = c.TE;
    const int tid = threadIdx.x;
    Weight3* sDw = reinterpret_cast<Weight3*>(smem + c.off_Dw);
    double2* sRaw = reinterpret_cast<double2*>(smem + c.off_U);
    double* sSum = reinterpret_cast<double*>(smem + c.off_U + c.raw_bytes);
    const size_t rowStride = (size_t)d.NA * nel;

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
                    const double2 v = Dt[((((size_t)q * d.Nw + w0 + wi) * d.NA + a) * d.NB + s) * 9 + ij];
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
    __syncthreads();  // callers reuse the window region for their epilogue
}

// Writes the X_ij blocks of the tile from the partial sums: sX[(le*9 + ij)*nel + el].
__device__ __forceinline__ void store_x(double2* sX, int nel, int el, int grp, const double (&K)[kR][9][3]) {
#pragma unroll
    for (int r = 0; r < kR; ++r) {
        const int le = grp * kR + r;
#pragma unroll
        for (int ij = 0; ij < 9; ++ij)
            sX[((size_t)le * 9 + ij) * nel + el] = make_double2(K[r][ij][0] - K[r][ij][2], K[r][ij][0] + K[r][ij][1]);
    }
}

}  // namespace fp64
}  // namespace sse
