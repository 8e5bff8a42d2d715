// Adjoint of Eq. (3) through the transforms: gradients with respect to dH and D (spec_adj_kernel FP64,
// spec_adj32_kernel FP32, the fixed-order reduction of the dH partials) and with respect to G (the incoming-bond
// list, spec_gradg_kernel FP64, spec_gradg32_kernel FP32), with their workspace layouts and drivers.
#include "sse_spectral.cuh"

namespace sse {
namespace {

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
    int ws, us;  // floats per frequency of the W^ and U regions, bank-padded
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
    c.ws = bank_pad16(2 * c.pl);
    c.us = bank_pad16(6 * c.pl);
    c.F = pick_frequencies(c.T, [&](int F) { return (long)6 * pb + F * (4L * (c.ws + c.us) + 9 * 8) + 64; });
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                             // [3 j][2 planes] the current bond's A_j row-major
    c.off_W = a16(c.off_A + 6 * pb);         // [F][ws] W^_a transposed (2 planes): WT[l][m] = W^[m][l]
    c.off_K = a16(c.off_W + c.F * c.ws * 4);  // [F][9] float2
    c.off_U = a16(c.off_K + c.F * 9 * 8);    // [F][us] U_i row-major (3 i x 2 planes)
    c.smem = a16(c.off_U + c.F * c.us * 4);
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
                float* Wp = sW + (size_t)fl * c.ws;
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
                const float* Wp = sW + (size_t)fl * c.ws;
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
                    float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
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
                    const float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
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
    int qs, ss;  // floats per frequency of the W^ / G^ regions (4 planes) and the T_j / V_j regions (6), bank-padded
    int off_A, off_W, off_G, off_K, off_T, off_V, smem;
};

constexpr int kAdj32MaxThreads = 256;
// Each lane adds its frequencies' coupling-gradient terms in FP32; chunks of at most this many terms per lane keep
// that sum short (the chunks are then added in FP64 in a fixed order). At the FinFET workload 269 terms per lane put
// the coupling gradient 2.6e-6 from the FP64 result, 32 terms 7.9e-7.
constexpr int kAdj32LaneTerms = 32;

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
    c.qs = bank_pad16(4 * c.pl);
    c.ss = bank_pad16(6 * c.pl);
    auto smem_of = [&](int F) { return (long)6 * pb + F * (4L * (2 * c.qs + 2 * c.ss) + 9 * 8) + 96; };
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
    c.off_W = a16(c.off_A + 6 * pb);              // [F][qs] W^ row-major (re, im), transposed (re, im)
    c.off_G = a16(c.off_W + c.F * c.qs * 4);      // [F][qs] G^ likewise
    c.off_K = a16(c.off_G + c.F * c.qs * 4);      // [F][9] float2
    c.off_T = a16(c.off_K + c.F * 9 * 8);         // [F][ss] T_j transposed (3 j x 2 planes)
    c.off_V = a16(c.off_T + c.F * c.ss * 4);      // [F][ss] V_j transposed
    c.smem = a16(c.off_V + c.F * c.ss * 4);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    if (fc > (size_t)kAdj32LaneTerms * c.F) fc = (size_t)kAdj32LaneTerms * c.F;
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
                float* Wp = sW + (size_t)fl * c.qs;
                float* Gp = sG + (size_t)fl * c.qs;
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
                const float* Wp = sW + (size_t)fl * c.qs;
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
                    float* Tp = sT + (size_t)fl * c.ss + (size_t)j * 2 * pl;
                    float* Vp = sV + (size_t)fl * c.ss + (size_t)j * 2 * pl;
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
                const float* Gp = sG + (size_t)fl * c.qs;
                float qr[3][4] = {}, qi[3][4] = {}, rr[3][4] = {}, ri[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 yr = ld2(Gp + 2 * pl + l * Np + n0), yi = ld2(Gp + 3 * pl + l * Np + n0);
                    const float2 gr = ld2(Gp + l * Np + n0), gi = ld2(Gp + pl + l * Np + n0);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float* Tp = sT + (size_t)fl * c.ss + (size_t)j * 2 * pl;
                        const float* Vp = sV + (size_t)fl * c.ss + (size_t)j * 2 * pl;
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

}  // namespace

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
        e = launch_fft32("fft_e_kernel(W)", plan, tw,
                       LoadWT<C>{W[t], d.NE, d.Norb, (size_t)d.NA * nel, (size_t)d.a_begin * nel, sym},
                       StoreSpecT<C>{Wh, L, wcols, L}, wcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_dft_k("dft_kz_kernel(W)", Wh, d.Nkz, d.Nkz, (size_t)L * wcols, 0, st)) != cudaSuccess) return e;
        e = launch_fft32("fft_e_kernel(G)", plan, tw, LoadGT<C>{p.G[t], d.NE, gcols}, StoreSpecT<C>{Gh, L, gcols, L},
                       gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_dft_k("dft_kz_kernel(G)", Gh, d.Nkz, d.Nkz, (size_t)L * gcols, 0, st)) != cudaSuccess) return e;
        LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
        e = launch_fft32("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_dft_k("dft_kz_kernel(K)", Kh, d.Nkz, d.Nqz, (size_t)L * kcols, 0, st)) != cudaSuccess) return e;
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
        if ((e = launch_dft_k("dft_kz_kernel(H)", Hh, d.Nkz, d.Nkz, (size_t)L * kcols, 1, st)) != cudaSuccess) return e;
        StoreGDT<C> sg{gD[t], gD[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9,
                       p.scale / (double)nfreq, t, L};
        e = launch_fft32("fft_e_kernel(H)", plan, tw, LoadSpecConjT<C>{Hh, L, kcols}, sg, kcols, d.Nqz, st);
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
// Sizes the FP64 G-gradient's product kernel is configured for: its grid covers every atom b (also those no bond
// reaches: they get zero), and its A region holds one bond's 3 x 4 planes (>= 12 Norb^2 doubles), hence NB >= 2.
sse_dims gradg_prod_dims(const sse_dims& d) {
    sse_dims dall = d;
    dall.a_begin = 0;
    dall.a_end = d.NA;
    dall.NB = d.NB < 2 ? 2 : d.NB;
    return dall;
}
}  // namespace

bool spectral_bwd_g_supported(const sse_dims& d, bool fp32) {
    if (!spectral_supported(d)) return false;
    const size_t nfreq = (size_t)d.Nkz * spectral_length(d);
    const int smem = fp32 ? make_gradg32_cfg(d, nfreq).smem : make_prod_cfg(gradg_prod_dims(d), nfreq, 8).smem;
    return smem <= 227 * 1024;
}

namespace {
// The gradient with respect to G in the real type T: double (FP64_FFT) or float (FP32_FFT: FP32 transforms and
// products, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_bwd_g_t(const Problem& p, const double2* gS_less, const double2* gS_greater,
                             double2* g_G_less, double2* g_G_greater, unsigned* status, void* ws, size_t ws_bytes,
                             cudaStream_t st) {
    using C = typename CX<T>::C;
    constexpr bool fp32 = sizeof(T) == 4;
    const sse_dims& d = p.d;
    if (!spectral_bwd_g_supported(d, fp32)) return cudaErrorNotSupported;
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
    const ProdCfg pc = make_prod_cfg(gradg_prod_dims(d), nfreq, (int)sizeof(T));
    const GradG32Cfg gc = make_gradg32_cfg(d, nfreq);
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
            e = launch_fft32("fft_e_kernel(W)", plan, tw,
                           LoadWT<C>{W[t], d.NE, d.Norb, (size_t)d.NA * nel, (size_t)d.a_begin * nel, sym},
                           StoreSpecT<C>{Wh, L, wcols, L}, wcols, d.Nkz, st);
            if (e != cudaSuccess) return e;
            if ((e = launch_dft_k("dft_kz_kernel(W)", Wh, d.Nkz, d.Nkz, (size_t)L * wcols, 0, st)) != cudaSuccess) return e;
            LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
            e = launch_fft32("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
            if (e != cudaSuccess) return e;
            if ((e = launch_dft_k("dft_kz_kernel(K)", Kh, d.Nkz, d.Nqz, (size_t)L * kcols, 0, st)) != cudaSuccess) return e;
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
        if ((e = launch_dft_k("dft_kz_kernel(R)", Rh, d.Nkz, d.Nkz, (size_t)L * gcols, 1, st)) != cudaSuccess) return e;
        const double inv = 1.0 / ((double)d.Nkz * (double)L);
        e = launch_fft32("fft_e_kernel(R)", plan, tw, LoadSpecConjT<C>{Rh, L, gcols},
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
