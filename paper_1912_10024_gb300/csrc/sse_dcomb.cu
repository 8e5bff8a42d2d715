// Bond weights of Eq. (3): Dc_ab = D_ba - D_bb - D_aa + D_ab (Sec. 2), and their adjoint.
//
// Raw phonon Green's functions: [Nqz][Nw][NA][NB+1][3][3], slot s < NB = D_ab for
// b = nbr[a][s], slot NB = the self block D_aa. D_ba is the block atom b stores in
// the slot s' with nbr[b][s'] = a (symmetric neighbour lists). Both kernels are
// memory-bound gathers: one thread per (qz, w, atom, slot) moves 9 complex numbers
// (144 bytes) per block it touches; no atomics, so the results are deterministic.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse_internal.h"

namespace sse {
namespace {

__device__ __forceinline__ int reverse_slot(const int32_t* nbr, int NB, int a, int b) {
    for (int s = 0; s < NB; ++s)
        if (nbr[(size_t)b * NB + s] == a) return s;
    return -1;
}

__device__ __forceinline__ size_t raw_off(const sse_dims& d, int q, int w, int a, int slot) {
    return ((((size_t)q * d.Nw + w) * d.NA + a) * (d.NB + 1) + slot) * 9;
}
__device__ __forceinline__ size_t bond_off(const sse_dims& d, int q, int w, int a, int s) {
    return ((((size_t)q * d.Nw + w) * d.NA + a) * d.NB + s) * 9;
}

// Dc[q][w][a][s] for atoms in range; bonds without a reverse slot (or an out-of-range
// neighbour) get zero and raise the status bit.
__global__ void dcomb_fwd_kernel(sse_dims d, const int32_t* __restrict__ nbr, const double2* __restrict__ raw_l,
                                 const double2* __restrict__ raw_g, double2* __restrict__ Dl,
                                 double2* __restrict__ Dg, unsigned* __restrict__ status) {
    const int nA = d.a_end - d.a_begin;
    const size_t total = (size_t)d.Nqz * d.Nw * nA * d.NB;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int s = (int)(i % d.NB);
        size_t r = i / d.NB;
        const int a = d.a_begin + (int)(r % nA);
        r /= nA;
        const int w = (int)(r % d.Nw), q = (int)(r / d.Nw);
        const int b = nbr[(size_t)a * d.NB + s];
        const int sr = (b >= 0 && b < d.NA) ? reverse_slot(nbr, d.NB, a, b) : -1;
        const size_t o = bond_off(d, q, w, a, s);
        if (sr < 0) {
            atomicOr(status, DEV_BAD_NEIGHBOUR);
            for (int e = 0; e < 9; ++e) Dl[o + e] = Dg[o + e] = make_double2(0.0, 0.0);
            continue;
        }
        const size_t ba = raw_off(d, q, w, b, sr), bb = raw_off(d, q, w, b, d.NB);
        const size_t aa = raw_off(d, q, w, a, d.NB), ab = raw_off(d, q, w, a, s);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const double2* R = t == 0 ? raw_l : raw_g;
            double2* out = t == 0 ? Dl : Dg;
#pragma unroll
            for (int e = 0; e < 9; ++e) {
                const double2 x = R[ba + e], y = R[bb + e], z = R[aa + e], u = R[ab + e];
                out[o + e] = make_double2(x.x - y.x - z.x + u.x, x.y - y.y - z.y + u.y);  // left to right
            }
        }
    }
}

// Adjoint: raw slot s < NB of atom a receives +g(a, s) (its D_ab term) and +g(b, s') (the D_ba term
// of the reverse bond); the self slot receives minus the sum of both over all of a's bonds.
__global__ void dcomb_bwd_kernel(sse_dims d, const int32_t* __restrict__ nbr, const double2* __restrict__ g_l,
                                 const double2* __restrict__ g_g, double2* __restrict__ r_l,
                                 double2* __restrict__ r_g, unsigned* __restrict__ status) {
    const int nA = d.a_end - d.a_begin;
    const size_t total = (size_t)d.Nqz * d.Nw * nA;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int a = d.a_begin + (int)(i % nA);
        const size_t r = i / nA;
        const int w = (int)(r % d.Nw), q = (int)(r / d.Nw);
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const double2* G = t == 0 ? g_l : g_g;
            double2* R = t == 0 ? r_l : r_g;
            double2 self[9];
#pragma unroll
            for (int e = 0; e < 9; ++e) self[e] = make_double2(0.0, 0.0);
            for (int s = 0; s < d.NB; ++s) {
                const int b = nbr[(size_t)a * d.NB + s];
                const int sr = (b >= 0 && b < d.NA) ? reverse_slot(nbr, d.NB, a, b) : -1;
                const size_t o = raw_off(d, q, w, a, s);
                if (sr < 0) {
                    if (t == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
                    for (int e = 0; e < 9; ++e) R[o + e] = make_double2(0.0, 0.0);
                    continue;
                }
                const size_t ga = bond_off(d, q, w, a, s), gb = bond_off(d, q, w, b, sr);
#pragma unroll
                for (int e = 0; e < 9; ++e) {
                    const double2 u = G[ga + e], v = G[gb + e];
                    const double2 sum = make_double2(u.x + v.x, u.y + v.y);
                    R[o + e] = sum;
                    self[e].x -= sum.x;
                    self[e].y -= sum.y;
                }
            }
            const size_t os = raw_off(d, q, w, a, d.NB);
#pragma unroll
            for (int e = 0; e < 9; ++e) R[os + e] = self[e];
        }
    }
}

}  // namespace

cudaError_t dcomb_fwd(const sse_dims& d, const int32_t* nbr, const double2* raw_l, const double2* raw_g,
                      double2* Dl, double2* Dg, unsigned* status, cudaStream_t st) {
    SSE_TIMED("dcomb_fwd_kernel", st, dcomb_fwd_kernel<<<152 * 8, 256, 0, st>>>(d, nbr, raw_l, raw_g, Dl, Dg, status));
    return cudaGetLastError();
}

cudaError_t dcomb_bwd(const sse_dims& d, const int32_t* nbr, const double2* g_l, const double2* g_g, double2* r_l,
                      double2* r_g, unsigned* status, cudaStream_t st) {
    SSE_TIMED("dcomb_bwd_kernel", st, dcomb_bwd_kernel<<<152 * 8, 256, 0, st>>>(d, nbr, g_l, g_g, r_l, r_g, status));
    return cudaGetLastError();
}

}  // namespace sse
