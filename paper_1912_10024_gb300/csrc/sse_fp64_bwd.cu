// FP64 adjoint of Eq. (3) (Sec. 2): gradients of
//   L = sum_t sum_{a,E,k} Re tr( W^t_a(E,k)^H Sigma^t_a(E,k) ),  W = upstream gradient,
// with respect to dH and D^<, D^> (PyTorch convention for complex tensors).
//
// With Sigma^t_a = c * sum_s sum_ij dH_i X_ij dH_j^H, c = i*scale, and
// X_ij(E,k) = sum_{q,w,sigma} D^tau_ij(q,w) G_b(E - sigma(w+1), k - q):
//
//   grad dH_m = sum_{t,E,k} [ conj(c) sum_j W dH_j X_mj^H + c sum_i W^H dH_i X_im ]     (kernel 1)
//   grad D^tau_ij(q,w) = sum_{(t,sigma): tau} sum_{E,k} sum_mn Q_ij(E,k)[mn] conj(G_b(E - sigma(w+1), k - q)[mn]),
//                        Q_ij = conj(c) dH_i^H W dH_j                                       (kernel 2)
//
// Kernel 1 recomputes the X tiles with the forward's correlation
// (sse_fp64_common.cuh): the gathered G windows are recomputed, never stored.
// Each CTA (kz, atom, type) sums its contributions over all energies and
// writes one partial per (a, s, kz, t) to the workspace; a third kernel adds
// the partials in a fixed order, so results are deterministic.
// Kernel 2 runs one CTA per bond (a, s): threads own (frequency, element
// group) pairs, correlate the Q tiles with the shifted G windows and add
// their sums into the bond's gradient entries, which no other CTA touches.
// With SSE_FLAG_SYMMETRIZE the upstream blocks are first projected to
// (W - W^H)/2, the adjoint of the forward's projection.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sse_fp64_common.cuh"
#include "sse_internal.h"

namespace sse {
namespace {

using namespace fp64;
constexpr int kEpiBlocks = 16;  // X [TE][9] + W [TE] + U [TE][3] + V [TE][3]

__device__ __forceinline__ double2 load_w(const double2* W, size_t blk, int m, int n, int Norb, bool sym) {
    const double2 v = W[blk + m * Norb + n];
    if (!sym) return v;
    const double2 u = W[blk + n * Norb + m];
    return make_double2(0.5 * (v.x - u.x), 0.5 * (v.y + u.y));
}

// ---------------------------------------------------------------------------
// kernel 1: partial grad dH per (a, s, kz, t)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kMaxThreads)
grad_dh_partial_kernel(Problem p, TileCfg c, const double2* __restrict__ gS_less,
                       const double2* __restrict__ gS_greater, double2* __restrict__ part,
                       unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const sse_dims& d = p.d;
    const int Norb = d.Norb, nel = c.nel, nth = c.nthreads, TE = c.TE;
    const int tid = threadIdx.x;
    const int el = tid % nel, grp = tid / nel;
    const int k = blockIdx.x;
    const int ai = (int)(blockIdx.y >> 1), a = d.a_begin + ai;
    const int t = (int)(blockIdx.y & 1);
    const bool sym = (p.flags & SSE_FLAG_SYMMETRIZE) != 0;
    const double2* W = t == 0 ? gS_less : gS_greater;

    double2* sA = reinterpret_cast<double2*>(smem);            // [3][nel]
    double2* sX = reinterpret_cast<double2*>(smem + c.off_U);  // [TE][9][nel]
    double2* sW = sX + (size_t)TE * 9 * nel;                   // [TE][nel]
    double2* sU = sW + (size_t)TE * nel;                       // [TE][3][nel]  W dH_j
    double2* sV = sU + (size_t)TE * 3 * nel;                   // [TE][3][nel]  W^H dH_i

    for (int s = 0; s < d.NB; ++s) {
        const int b = p.nbr[(size_t)a * d.NB + s];
        const bool bvalid = b >= 0 && b < d.NA;
        if (!bvalid && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
        __syncthreads();
        const double2* Ag = p.dH + ((size_t)a * d.NB + s) * 3 * nel;
        for (int i = tid; i < 3 * nel; i += nth) sA[i] = Ag[i];

        double2 acc[3];  // items it = tid + j*nth < 3*nel: (direction m, element mn)
#pragma unroll
        for (int j = 0; j < 3; ++j) acc[j] = make_double2(0.0, 0.0);

        for (int E0 = 0; E0 < d.NE; E0 += TE) {
            double K[kR][9][3];
            correlate_tile(p, c, smem, a, s, t, k, E0, b, bvalid, el, grp, K);
            store_x(sX, nel, el, grp, K);
            for (int i = tid; i < TE * nel; i += nth) {
                const int le = i / nel, mn = i - le * nel;
                const int E = E0 + le;
                double2 v = make_double2(0.0, 0.0);
                if (E < d.NE)
                    v = load_w(W, (((size_t)k * d.NE + E) * d.NA + a) * nel, mn / Norb, mn % Norb, Norb, sym);
                sW[i] = v;
            }
            __syncthreads();
            for (int it = tid; it < TE * 3 * nel; it += nth) {  // U_j = W dH_j, V_i = W^H dH_i
                const int le = it / (3 * nel), rem = it - le * 3 * nel;
                const int j = rem / nel, mn = rem - j * nel;
                const int m = mn / Norb, n = mn - m * Norb;
                const double2* Wb = sW + (size_t)le * nel;
                const double2* Ab = sA + j * nel;
                double2 u = make_double2(0.0, 0.0), v = make_double2(0.0, 0.0);
                for (int l = 0; l < Norb; ++l) {
                    u = cfma(Wb[m * Norb + l], Ab[l * Norb + n], u);         // W[m,l] A[l,n]
                    v = cfma_conja(Wb[l * Norb + m], Ab[l * Norb + n], v);   // conj(W[l,m]) A[l,n]
                }
                sU[it] = u;
                sV[it] = v;
            }
            __syncthreads();
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const int it = tid + j * nth;
                if (it >= 3 * nel) break;
                const int md = it / nel, mn = it - md * nel;
                const int pr = mn / Norb, rc = mn - pr * Norb;
                double2 a1 = make_double2(0.0, 0.0), a2 = make_double2(0.0, 0.0);
                for (int le = 0; le < TE; ++le) {
                    for (int jj = 0; jj < 3; ++jj) {
                        // (U_j X_mj^H)[p][r] = sum_n U_j[p,n] conj(X_mj[r,n])
                        const double2* U = sU + ((size_t)le * 3 + jj) * nel + pr * Norb;
                        const double2* Xm = sX + ((size_t)le * 9 + md * 3 + jj) * nel + rc * Norb;
                        for (int n = 0; n < Norb; ++n) a1 = cfma_conjb(U[n], Xm[n], a1);
                        // (V_i X_im)[p][r] = sum_l V_i[p,l] X_im[l,r]   (i = jj)
                        const double2* V = sV + ((size_t)le * 3 + jj) * nel + pr * Norb;
                        const double2* Xi = sX + ((size_t)le * 9 + jj * 3 + md) * nel + rc;
                        for (int l = 0; l < Norb; ++l) a2 = cfma(V[l], Xi[l * Norb], a2);
                    }
                }
                // conj(c) a1 + c a2 with c = i*scale: i*scale*(a2 - a1), applied at the end
                acc[j].x += a2.x - a1.x;
                acc[j].y += a2.y - a1.y;
            }
        }
        const double sc = p.scale;
        double2* out = part + ((((size_t)ai * d.NB + s) * d.Nkz + k) * 2 + t) * 3 * nel;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int it = tid + j * nth;
            if (it < 3 * nel) out[it] = make_double2(-sc * acc[j].y, sc * acc[j].x);
        }
    }
}

// grad dH[a][s] = sum over (kz, t) of the partials, in a fixed order.
__global__ void grad_dh_reduce_kernel(sse_dims d, const double2* __restrict__ part, double2* __restrict__ g_dH) {
    const int nel = d.Norb * d.Norb;
    const size_t per = (size_t)3 * nel;
    const size_t total = (size_t)(d.a_end - d.a_begin) * d.NB * per;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const size_t bond = i / per, e = i - bond * per;  // bond = ai*NB + s
        double2 acc = make_double2(0.0, 0.0);
        for (int kt = 0; kt < 2 * d.Nkz; ++kt) {
            const double2 v = part[(bond * 2 * d.Nkz + kt) * per + e];
            acc.x += v.x;
            acc.y += v.y;
        }
        g_dH[((size_t)d.a_begin * d.NB + bond) * per + e] = acc;
    }
}

// ---------------------------------------------------------------------------
// kernel 2: grad D per bond (a, s)
// ---------------------------------------------------------------------------
constexpr int kThreadsD = 256;
constexpr int kSmemBudgetD = 200 * 1024;

struct DCfg {
    int nel, te, wc, groups;  // energies per Q tile, frequencies per window chunk, element groups
    int off_A, off_W, off_P, off_Q, off_G, off_part, smem;
};

DCfg layout_dcfg(const sse_dims& d, int te, int wc) {
    DCfg c{};
    c.nel = d.Norb * d.Norb;
    c.te = te;
    c.wc = wc;
    c.groups = kThreadsD / c.wc;
    const int blk = c.nel * 16;
    c.off_A = 0;
    c.off_W = c.off_A + 3 * blk;
    c.off_P = c.off_W + te * blk;
    c.off_Q = c.off_P + te * 3 * blk;
    c.off_G = c.off_Q + te * 9 * blk;
    c.off_part = c.off_G + (te + c.wc - 1) * blk;
    c.smem = c.off_part + c.groups * c.wc * 9 * 16;
    return c;
}

// Largest energy tile (4, 2, 1) and frequency chunk (<= 32) whose buffers fit the budget.
DCfg make_dcfg(const sse_dims& d) {
    DCfg c{};
    for (int te = 4; te >= 1; te /= 2)
        for (int wc = d.Nw < 32 ? d.Nw : 32; wc >= 1; --wc) {
            c = layout_dcfg(d, te, wc);
            if (c.smem <= kSmemBudgetD) return c;
        }
    return c;
}

__global__ void __launch_bounds__(kThreadsD)
grad_d_kernel(Problem p, DCfg c, const double2* __restrict__ gS_less, const double2* __restrict__ gS_greater,
              double2* __restrict__ g_D_less, double2* __restrict__ g_D_greater, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const sse_dims& d = p.d;
    const int Norb = d.Norb, nel = c.nel;
    const int tid = threadIdx.x;
    const int wi = tid % c.wc, g = tid / c.wc;
    const bool active = g < c.groups;  // kThreadsD need not be a multiple of wc
    const int a = d.a_begin + (int)(blockIdx.x / d.NB);
    const int s = (int)(blockIdx.x % d.NB);
    const bool sym = (p.flags & SSE_FLAG_SYMMETRIZE) != 0;
    double2* sA = reinterpret_cast<double2*>(smem + c.off_A);     // [3][nel]
    double2* sW = reinterpret_cast<double2*>(smem + c.off_W);     // [TE][nel]
    double2* sP = reinterpret_cast<double2*>(smem + c.off_P);     // [TE][3][nel]  dH_i^H W
    double2* sQ = reinterpret_cast<double2*>(smem + c.off_Q);     // [TE][9][nel]  conj(c) dH_i^H W dH_j
    double2* sG = reinterpret_cast<double2*>(smem + c.off_G);     // [rows][nel]
    double2* sPart = reinterpret_cast<double2*>(smem + c.off_part);  // [groups][wc][9]
    double2* gD[2] = {g_D_less, g_D_greater};

    const int b = p.nbr[(size_t)a * d.NB + s];
    const bool bvalid = b >= 0 && b < d.NA;
    if (!bvalid && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
    const double2* Ag = p.dH + ((size_t)a * d.NB + s) * 3 * nel;
    for (int i = tid; i < 3 * nel; i += kThreadsD) sA[i] = Ag[i];
    // this CTA is the only writer of the bond's gradient entries: zero them first
    for (int i = tid; i < 2 * d.Nqz * d.Nw * 9; i += kThreadsD) {
        const int tau = i / (d.Nqz * d.Nw * 9), r = i - tau * d.Nqz * d.Nw * 9;
        const int qw = r / 9, ij = r - qw * 9;
        gD[tau][(((size_t)qw * d.NA + a) * d.NB + s) * 9 + ij] = make_double2(0.0, 0.0);
    }
    const size_t rowStride = (size_t)d.NA * nel;
    const double sc = p.scale;

    for (int t = 0; t < 2; ++t) {
        const double2* W = t == 0 ? gS_less : gS_greater;
        for (int k = 0; k < d.Nkz; ++k) {
            for (int E0 = 0; E0 < d.NE; E0 += c.te) {
                __syncthreads();  // previous tile is done with sW / sP / sQ
                for (int i = tid; i < c.te * nel; i += kThreadsD) {
                    const int le = i / nel, mn = i - le * nel;
                    const int E = E0 + le;
                    double2 v = make_double2(0.0, 0.0);
                    if (E < d.NE)
                        v = load_w(W, (((size_t)k * d.NE + E) * d.NA + a) * nel, mn / Norb, mn % Norb, Norb, sym);
                    sW[i] = v;
                }
                __syncthreads();
                for (int it = tid; it < c.te * 3 * nel; it += kThreadsD) {  // P_i = dH_i^H W
                    const int le = it / (3 * nel), rem = it - le * 3 * nel;
                    const int i = rem / nel, mn = rem - i * nel;
                    const int m = mn / Norb, n = mn - m * Norb;
                    double2 acc = make_double2(0.0, 0.0);
                    for (int l = 0; l < Norb; ++l)
                        acc = cfma_conja(sA[i * nel + l * Norb + m], sW[(size_t)le * nel + l * Norb + n], acc);
                    sP[it] = acc;
                }
                __syncthreads();
                for (int it = tid; it < c.te * 9 * nel; it += kThreadsD) {  // Q_ij = conj(c) P_i dH_j
                    const int le = it / (9 * nel), rem = it - le * 9 * nel;
                    const int ij = rem / nel, mn = rem - ij * nel;
                    const int i = ij / 3, j = ij - 3 * i;
                    const int m = mn / Norb, n = mn - m * Norb;
                    double2 acc = make_double2(0.0, 0.0);
                    for (int l = 0; l < Norb; ++l)
                        acc = cfma(sP[((size_t)le * 3 + i) * nel + m * Norb + l], sA[j * nel + l * Norb + n], acc);
                    sQ[it] = make_double2(sc * acc.y, -sc * acc.x);  // conj(i*scale) = -i*scale
                }
                for (int q = 0; q < d.Nqz; ++q) {
                    const int kp = ((k - q) % d.Nkz + d.Nkz) % d.Nkz;
                    const double2* Gb = p.G[t] + (size_t)kp * d.NE * rowStride + (size_t)(bvalid ? b : 0) * nel;
                    for (int sg = 0; sg < 2; ++sg) {
                        const int sigma = sg == 0 ? +1 : -1;
                        const int tau = sg == 0 ? t : 1 - t;
                        const int wend = min(d.Nw, sigma > 0 ? E0 + c.te - 1 : d.NE - 1 - E0);
                        for (int w0 = 0; w0 < wend; w0 += c.wc) {
                            const int wn = min(c.wc, wend - w0);
                            const int rows = c.te + wn - 1;
                            const int Elo = sigma > 0 ? E0 - w0 - wn : E0 + w0 + 1;
                            __syncthreads();  // sQ complete; previous chunk done with sG / sPart
                            for (int i = tid; i < rows * nel; i += kThreadsD) {
                                const int row = i / nel, e2 = i - row * nel;
                                const int Ep = Elo + row;
                                double2 v = make_double2(0.0, 0.0);
                                if (bvalid && Ep >= 0 && Ep < d.NE) v = __ldg(Gb + (size_t)Ep * rowStride + e2);
                                sG[i] = v;
                            }
                            __syncthreads();
                            double2 acc[9];
#pragma unroll
                            for (int ij = 0; ij < 9; ++ij) acc[ij] = make_double2(0.0, 0.0);
                            if (active && wi < wn) {
                                for (int le = 0; le < c.te; ++le) {
                                    const int row = sigma > 0 ? le + (wn - 1) - wi : le + wi;
                                    const double2* Gr = sG + (size_t)row * nel;
                                    const double2* Qr = sQ + (size_t)le * 9 * nel;
                                    for (int mn = g; mn < nel; mn += c.groups) {
                                        const double2 x = Gr[mn];
#pragma unroll
                                        for (int ij = 0; ij < 9; ++ij) acc[ij] = cfma_conjb(Qr[ij * nel + mn], x, acc[ij]);
                                    }
                                }
                            }
                            if (active)
#pragma unroll
                                for (int ij = 0; ij < 9; ++ij) sPart[((size_t)g * c.wc + wi) * 9 + ij] = acc[ij];
                            __syncthreads();
                            for (int i = tid; i < wn * 9; i += kThreadsD) {
                                const int w2 = i / 9, ij = i - 9 * w2;
                                double2 sum = make_double2(0.0, 0.0);
                                for (int gg = 0; gg < c.groups; ++gg) {
                                    const double2 v = sPart[((size_t)gg * c.wc + w2) * 9 + ij];
                                    sum.x += v.x;
                                    sum.y += v.y;
                                }
                                double2* o = gD[tau] + ((((size_t)q * d.Nw + w0 + w2) * d.NA + a) * d.NB + s) * 9 + ij;
                                double2 cur = *o;
                                cur.x += sum.x;
                                cur.y += sum.y;
                                *o = cur;
                            }
                        }
                    }
                }
            }
        }
    }
}

}  // namespace

size_t fp64_bwd_workspace(const sse_dims& d) {
    // grad-dH partials: [atoms][NB][Nkz][2][3][Norb^2] complex (sized for the full atom range)
    return (size_t)d.NA * d.NB * d.Nkz * 2 * 3 * d.Norb * d.Norb * 16;
}

cudaError_t fp64_bwd(const Problem& p, const double2* gS_less, const double2* gS_greater, double2* g_dH,
                     double2* g_D_less, double2* g_D_greater, unsigned* status, void* ws, size_t ws_bytes,
                     cudaStream_t st) {
    const sse_dims& d = p.d;
    const int nA = d.a_end - d.a_begin;
    if (ws_bytes < fp64_bwd_workspace(d)) return cudaErrorInvalidValue;
    double2* part = static_cast<double2*>(ws);

    const TileCfg c = make_tile_cfg(d, kEpiBlocks);
    if (c.smem > 227 * 1024) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(grad_dh_partial_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, c.smem);
    if (e != cudaSuccess) return e;
    SSE_TIMED("grad_dh_partial_kernel", st, grad_dh_partial_kernel<<<dim3(d.Nkz, 2 * nA), c.nthreads, c.smem, st>>>(p, c, gS_less, gS_greater, part, status));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    SSE_TIMED("grad_dh_reduce_kernel", st, grad_dh_reduce_kernel<<<1024, 256, 0, st>>>(d, part, g_dH));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;

    const DCfg dc = make_dcfg(d);
    if (dc.smem > 227 * 1024) return cudaErrorNotSupported;
    e = cudaFuncSetAttribute(grad_d_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, dc.smem);
    if (e != cudaSuccess) return e;
    SSE_TIMED("grad_d_kernel", st, grad_d_kernel<<<nA * d.NB, kThreadsD, dc.smem, st>>>(p, dc, gS_less, gS_greater, g_D_less, g_D_greater, status));
    return cudaGetLastError();
}

}  // namespace sse
