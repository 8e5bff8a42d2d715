// Pi of Eq. (4) through the transforms: the per-frequency half products and traces in FP64 (spec_pi_kernel) and
// FP32 (spec_pi32_kernel), the store of the inverse transform, the 3x3 symmetrisation and the driver.
#include "sse_spectral.cuh"

namespace sse {
namespace {

// ---------------------------------------------------------------------------
struct PiCfg {
    int nel, F, threads, fchunk;
    int off_A, off_X, off_Y, off_P, off_R, off_D, off_self, smem;
};

PiCfg make_pi_cfg(const sse_dims& d, size_t nfreq) {
    PiCfg c{};
    c.nel = d.Norb * d.Norb;
    const int pl = c.nel * 8;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    c.F = pick_frequencies(c.nel, [&](int F) {
        return (long)d.NB * 3 * 4 * pl + F * 3 * pl * 2 + F * 6 * pl * 2 + F * 9 * d.Norb * 16 + F * 9 * 16 + 96;
    });
    c.threads = ((c.F * c.nel + 31) / 32) * 32;
    c.off_A = 0;                                     // [NB][3][4 planes: re, im, re+im, re-im]
    c.off_X = a16(c.off_A + d.NB * 3 * 4 * pl);      // [F][3 planes]
    c.off_Y = a16(c.off_X + c.F * 3 * pl);           // [F][3 planes]
    c.off_P = a16(c.off_Y + c.F * 3 * pl);           // [F][3 i][2 planes]
    c.off_R = a16(c.off_P + c.F * 6 * pl);           // [F][3 j][2 planes]
    c.off_D = a16(c.off_R + c.F * 6 * pl);           // [F][9][Norb] complex: diagonal terms
    c.off_self = a16(c.off_D + c.F * 9 * d.Norb * 16);  // [F][9] complex: diagonal-block sums
    c.smem = a16(c.off_self + c.F * 9 * 16);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + 2 * nA - 1) / (nA ? 2 * nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void __launch_bounds__(kProdMaxThreads, 2)
spec_pi_kernel(PiCfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
               const double2* __restrict__ Gl_hat, const double2* __restrict__ Gg_hat, double2* __restrict__ Cl_hat,
               double2* __restrict__ Cg_hat, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const int t = blockIdx.z;
    const double2* X_hat = t == 0 ? Gl_hat : Gg_hat;  // G^t of atom a
    const double2* Y_hat = t == 0 ? Gg_hat : Gl_hat;  // G^t' of the neighbour
    double2* C_hat = t == 0 ? Cl_hat : Cg_hat;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;  // frequency indices of the map
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    double* sA = reinterpret_cast<double*>(smem + c.off_A);
    double* sX = reinterpret_cast<double*>(smem + c.off_X);
    double* sY = reinterpret_cast<double*>(smem + c.off_Y);
    double* sP = reinterpret_cast<double*>(smem + c.off_P);
    double* sR = reinterpret_cast<double*>(smem + c.off_R);
    double2* sD = reinterpret_cast<double2*>(smem + c.off_D);
    double2* sSelf = reinterpret_cast<double2*>(smem + c.off_self);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;
    const int slots = d.NB + 1;
    const int ndiag = c.F * 9 * Norb;

    for (int i = tid; i < d.NB * 3 * nel; i += blockDim.x) {
        const int si = i / nel, ee = i - si * nel;
        const double2 v = dH[((size_t)a * d.NB) * 3 * nel + i];
        double* P = sA + (size_t)si * 4 * nel;
        P[ee] = v.x;
        P[nel + ee] = v.y;
        P[2 * nel + ee] = v.x + v.y;
        P[3 * nel + ee] = v.x - v.y;
    }
    if (tid == 0 && t == 0)
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            if (b < 0 || b >= d.NA) atomicOr(status, DEV_BAD_NEIGHBOUR);
        }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        const size_t fneg = act ? freq_neg(fm, f) : 0;
        if (lane) {
            double2 x = make_double2(0.0, 0.0);
            if (act) x = X_hat[(f * d.NA + a) * nel + e];
            put3(sX + (size_t)fl * 3 * nel, nel, e, x);
        }
        // diagonal-block sums: entry g = (frequency, ij) belongs to thread g mod blockDim for the whole batch
        for (int g = tid; g < c.F * 9; g += blockDim.x) sSelf[g] = make_double2(0.0, 0.0);
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            if (lane) {
                double2 y = make_double2(0.0, 0.0);
                if (act && bok) y = Y_hat[(fneg * d.NA + b) * nel + e];
                put3(sY + (size_t)fl * 3 * nel, nel, e, y);
            }
            __syncthreads();
            // half products P_i = dH_i^H X, R_j = dH_j Y (Gauss 3-multiply MACs)
            if (lane) {
                const double* A = sA + (size_t)s * 12 * nel;
                const double* Xp = sX + (size_t)fl * 3 * nel;
                const double* Yp = sY + (size_t)fl * 3 * nel;
#pragma unroll 1
                for (int i = 0; i < 3; ++i) {
                    const double* Ai = A + (size_t)i * 4 * nel;
                    double t1 = 0.0, u2 = 0.0, t3 = 0.0, r1 = 0.0, r2 = 0.0, r3 = 0.0;
                    for (int l = 0; l < Norb; ++l) {
                        const int lm = l * Norb + m, ml = m * Norb + l, ln = l * Norb + n;
                        t1 = fma(Ai[lm], Xp[ln], t1);                  // conj(A_i[l][m]) X[l][n]
                        u2 = fma(Ai[nel + lm], Xp[nel + ln], u2);
                        t3 = fma(Ai[3 * nel + lm], Xp[2 * nel + ln], t3);
                        r1 = fma(Ai[ml], Yp[ln], r1);                  // A_i[m][l] Y[l][n]
                        r2 = fma(Ai[nel + ml], Yp[nel + ln], r2);
                        r3 = fma(Ai[2 * nel + ml], Yp[2 * nel + ln], r3);
                    }
                    double* P = sP + ((size_t)fl * 3 + i) * 2 * nel;
                    P[e] = t1 + u2;
                    P[nel + e] = t3 - t1 + u2;
                    double* R = sR + ((size_t)fl * 3 + i) * 2 * nel;
                    R[e] = r1 - r2;
                    R[nel + e] = r3 - r1 - r2;
                }
            }
            __syncthreads();
            // diagonal terms D_ij[m] = sum_n P_i[m][n] R_j[n][m]
            for (int g = tid; g < ndiag; g += blockDim.x) {
                const int fi = g / (9 * Norb), rem = g - fi * 9 * Norb;
                const int ij = rem / Norb, mm = rem - ij * Norb;
                const int i = ij / 3, j = ij - 3 * i;
                const double* P = sP + ((size_t)fi * 3 + i) * 2 * nel;
                const double* R = sR + ((size_t)fi * 3 + j) * 2 * nel;
                double re = 0.0, im = 0.0;
                for (int nn = 0; nn < Norb; ++nn) {
                    const double pr = P[mm * Norb + nn], pi = P[nel + mm * Norb + nn];
                    const double rr = R[nn * Norb + mm], ri = R[nel + nn * Norb + mm];
                    re = fma(pr, rr, re);
                    re = fma(-pi, ri, re);
                    im = fma(pr, ri, im);
                    im = fma(pi, rr, im);
                }
                sD[g] = make_double2(re, im);
            }
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {  // fixed-order sums over the rows m
                const int rf = g / 9, ij = g - rf * 9;
                const double2* v = sD + (size_t)g * Norb;
                double2 sum = v[0];
                for (int mm = 1; mm < Norb; ++mm) sum = cadd(sum, v[mm]);
                const double2 self = cadd(sSelf[g], sum);
                sSelf[g] = self;
                if (i0 + rf < i_end) {
                    const size_t ff = freq_of(fm, i0 + rf);
                    C_hat[((ff * nA + la) * slots + s) * 9 + ij] = sum;
                    if (s == d.NB - 1) C_hat[((ff * nA + la) * slots + d.NB) * 9 + ij] = self;
                }
            }
            // the next bond rewrites sY before its first barrier; sP, sR and sD only after it
        }
        __syncthreads();  // sX of the next frequency batch
    }
}

// ---------------------------------------------------------------------------
// FP32 phonon self-energy (mode FP32_FFT): the half products P_i = dH_i^H X^ and R_j = dH_j Y^ three at a time
// on 2 x 2 register tiles (4-multiply MACs on (re, im) planes); R_j goes to shared memory transposed, so each
// thread forms its tile's part of tr(P_i R_j) from P_i in registers; the parts are summed over the tile threads
// in a fixed order.
// ---------------------------------------------------------------------------
constexpr int kPi32MaxThreads = 256;  // <= 128 registers at two CTAs per SM

struct Pi32Cfg {
    int Np, TN, T, pl, F, threads, fchunk;
    int xs, rs;  // floats per frequency of the X^ / Y^ regions and the R_j region, bank-padded
    int off_A, off_X, off_Y, off_R, off_self, smem;
};

Pi32Cfg make_pi32_cfg(const sse_dims& d, size_t nfreq) {
    Pi32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;
    auto a16 = [](int x) { return (x + 15) & ~15; };
    // per CTA: every bond's dH row-major and transposed (12 planes per bond); per frequency X^, Y^ (4 planes),
    // R_j transposed (6 planes; the trace parts reuse them) and the diagonal-block sums (9 float2)
    c.xs = bank_pad16(2 * c.pl);
    c.rs = bank_pad16(6 * c.pl);
    c.F = pick_frequencies(
        c.T, [&](int F) { return (long)d.NB * 12 * pb + F * (4L * (2 * c.xs + c.rs) + 9 * 8) + 96; }, 128,
        kPi32MaxThreads);
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                               // [NB][3][4 planes: re, im row-major; re, im transposed]
    c.off_X = a16(c.off_A + d.NB * 12 * pb);     // [F][xs] X^ row-major (2 planes)
    c.off_Y = a16(c.off_X + c.F * c.xs * 4);     // [F][xs] Y^ row-major
    c.off_R = a16(c.off_Y + c.F * c.xs * 4);     // [F][rs] R_j transposed (3 j x 2 planes)
    c.off_self = a16(c.off_R + c.F * c.rs * 4);  // [F][9] float2
    c.smem = a16(c.off_self + c.F * 9 * 8);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + 2 * nA - 1) / (nA ? 2 * nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void __launch_bounds__(kPi32MaxThreads, 2)
spec_pi32_kernel(Pi32Cfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr, const double2* __restrict__ dH,
                 const float2* __restrict__ Gl_hat, const float2* __restrict__ Gg_hat, float2* __restrict__ Cl_hat,
                 float2* __restrict__ Cg_hat, unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb, T = c.T;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const int t = blockIdx.z;
    const float2* X_hat = t == 0 ? Gl_hat : Gg_hat;  // G^t of atom a
    const float2* Y_hat = t == 0 ? Gg_hat : Gl_hat;  // G^t' of the neighbour
    float2* C_hat = t == 0 ? Cl_hat : Cg_hat;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sX = reinterpret_cast<float*>(smem + c.off_X);
    float* sY = reinterpret_cast<float*>(smem + c.off_Y);
    float* sR = reinterpret_cast<float*>(smem + c.off_R);
    float2* sSelf = reinterpret_cast<float2*>(smem + c.off_self);
    const int tid = threadIdx.x;
    const int fl = tid / T, tt = tid - fl * T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;
    const int slots = d.NB + 1;

    // dH planes of every bond, zero-padded: row-major A[l][n] and transposed AT[l][m] = A[m][l]
    for (int i = tid; i < d.NB * 3 * pl; i += blockDim.x) {
        const int si = i / pl, e = i - si * pl;
        const int r = e / Np, q = e - r * Np;
        double2 v = make_double2(0.0, 0.0), w = make_double2(0.0, 0.0);
        if (r < Norb && q < Norb) {
            v = dH[((size_t)a * d.NB * 3 + si) * nel + r * Norb + q];
            w = dH[((size_t)a * d.NB * 3 + si) * nel + q * Norb + r];
        }
        float* P = sA + (size_t)si * 4 * pl;
        P[e] = (float)v.x;
        P[pl + e] = (float)v.y;
        P[2 * pl + e] = (float)w.x;
        P[3 * pl + e] = (float)w.y;
    }
    if (tid == 0 && t == 0)
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            if (b < 0 || b >= d.NA) atomicOr(status, DEV_BAD_NEIGHBOUR);
        }

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        const size_t fneg = act ? freq_neg(fm, f) : 0;
        __syncthreads();  // the previous batch is done with sX and sSelf
        if (lane) {
            float* Xp = sX + (size_t)fl * c.xs;
#pragma unroll
            for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                for (int dn = 0; dn < 2; ++dn) {
                    const int m = m0 + dm, n = n0 + dn;
                    float2 x = make_float2(0.f, 0.f);
                    if (act && m < Norb && n < Norb) x = X_hat[(f * d.NA + a) * nel + m * Norb + n];
                    Xp[m * Np + n] = x.x;
                    Xp[pl + m * Np + n] = x.y;
                }
        }
        for (int g = tid; g < c.F * 9; g += blockDim.x) sSelf[g] = make_float2(0.f, 0.f);
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            if (lane) {
                float* Yp = sY + (size_t)fl * c.xs;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 y = make_float2(0.f, 0.f);
                        if (act && bok && m < Norb && n < Norb) y = Y_hat[(fneg * d.NA + b) * nel + m * Norb + n];
                        Yp[m * Np + n] = y.x;
                        Yp[pl + m * Np + n] = y.y;
                    }
            }
            __syncthreads();
            const float* A = sA + (size_t)s * 12 * pl;
            // P_i[m][n] = sum_l conj(A_i[l][m]) X[l][n];  R_j[m][n] = sum_l A_j[m][l] Y[l][n] (= AT_j[l][m])
            float pr[3][4] = {}, pim[3][4] = {};
            if (lane) {
                const float* Xp = sX + (size_t)fl * c.xs;
                const float* Yp = sY + (size_t)fl * c.xs;
                float rr[3][4] = {}, ri[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 xr = ld2(Xp + l * Np + n0), xi = ld2(Xp + pl + l * Np + n0);
                    const float2 yr = ld2(Yp + l * Np + n0), yi = ld2(Yp + pl + l * Np + n0);
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        const float* Ai = A + (size_t)i * 4 * pl;
                        cmac2x2<true, false>(pr[i], pim[i], ld2(Ai + l * Np + m0), ld2(Ai + pl + l * Np + m0), xr, xi);
                        cmac2x2<false, false>(rr[i], ri[i], ld2(Ai + 2 * pl + l * Np + m0),
                                              ld2(Ai + 3 * pl + l * Np + m0), yr, yi);
                    }
                }
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    float* Rp = sR + (size_t)fl * c.rs + (size_t)j * 2 * pl;
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {  // transposed: (R[m0][n], R[m0+1][n]) at row n
                        const int o = (n0 + dn) * Np + m0;
                        st2(Rp + o, rr[j][dn], rr[j][2 + dn]);
                        st2(Rp + pl + o, ri[j][dn], ri[j][2 + dn]);
                    }
                }
            }
            __syncthreads();
            // this tile's part of C_ij = sum_{m,n} P_i[m][n] R_j[n][m] = sum_{m,n} P_i[m][n] RT_j[m][n]
            float hp[9][2];
            if (lane) {
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const float* Rp = sR + (size_t)fl * c.rs + (size_t)j * 2 * pl;
                    float tr[4], ti[4];
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        const float2 r2 = ld2(Rp + (m0 + dm) * Np + n0), i2 = ld2(Rp + pl + (m0 + dm) * Np + n0);
                        tr[dm * 2] = r2.x;
                        tr[dm * 2 + 1] = r2.y;
                        ti[dm * 2] = i2.x;
                        ti[dm * 2 + 1] = i2.y;
                    }
#pragma unroll
                    for (int i = 0; i < 3; ++i) {
                        float hr = 0.f, hi = 0.f;
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            hr = fmaf(pr[i][q], tr[q], hr);
                            hr = fmaf(-pim[i][q], ti[q], hr);
                            hi = fmaf(pr[i][q], ti[q], hi);
                            hi = fmaf(pim[i][q], tr[q], hi);
                        }
                        hp[i * 3 + j][0] = hr;
                        hp[i * 3 + j][1] = hi;
                    }
                }
            }
            __syncthreads();  // every read of sR and sY for this bond is done
            float2* sP = reinterpret_cast<float2*>(sR);  // [F][T][9] trace parts (fit in the R_j planes)
            if (lane)
#pragma unroll
                for (int ij = 0; ij < 9; ++ij) sP[((size_t)fl * T + tt) * 9 + ij] = make_float2(hp[ij][0], hp[ij][1]);
            __syncthreads();
            for (int g = tid; g < c.F * 9; g += blockDim.x) {  // fixed-order sums over the tile threads
                const int rf = g / 9, ij = g - rf * 9;
                float2 sum = sP[(size_t)rf * T * 9 + ij];
                for (int u = 1; u < T; ++u) {
                    const float2 v = sP[((size_t)rf * T + u) * 9 + ij];
                    sum.x += v.x;
                    sum.y += v.y;
                }
                const float2 self = make_float2(sSelf[g].x + sum.x, sSelf[g].y + sum.y);
                sSelf[g] = self;
                if (i0 + rf < i_end) {
                    const size_t ff = freq_of(fm, i0 + rf);
                    C_hat[((ff * nA + la) * slots + s) * 9 + ij] = sum;
                    if (s == d.NB - 1) C_hat[((ff * nA + la) * slots + d.NB) * 9 + ij] = self;
                }
            }
            // the next bond writes sY before its first barrier and sR (sP) only after it
        }
    }
}

// Pi^t[q][w][a][slot][ij] = -i*scale * conj(v) * inv for rows l = w+1 in [1, Nw]
template <class C>
struct StorePiT {
    double2* P;
    int Nw, NA, slots;
    size_t col0;
    double inv_scale;  // scale / (Nkz L)
    int rows;
    __device__ void operator()(int q, int r, size_t col, C v) const {
        if (r < 1 || r > Nw) return;
        const size_t rowlen = (size_t)NA * slots * 9;
        // C = conj(v) * inv; Pi = -i * scale * C, in FP64
        P[((size_t)q * Nw + (r - 1)) * rowlen + col0 + col] =
            make_double2(-(double)v.y * inv_scale, -(double)v.x * inv_scale);
    }
};
using StorePi = StorePiT<double2>;

// (P - P^H)/2 on every 3x3 block of the atoms in range
__global__ void symmetrize3_kernel(sse_dims d, double2* __restrict__ P) {
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const int slots = d.NB + 1;
    const size_t nblk = (size_t)d.Nqz * d.Nw * nA * slots;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < nblk; i += (size_t)gridDim.x * blockDim.x) {
        const size_t qw = i / (nA * slots), rem = i - qw * nA * slots;
        double2* B = P + ((qw * d.NA + d.a_begin) * slots + rem) * 9;
        for (int r = 0; r < 3; ++r)
            for (int c2 = r; c2 < 3; ++c2) {
                const double2 x = B[r * 3 + c2], y = B[c2 * 3 + r];
                B[r * 3 + c2] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
                if (r != c2) B[c2 * 3 + r] = make_double2(0.5 * (y.x - x.x), 0.5 * (y.y + x.y));
            }
    }
}

}  // namespace

struct PiLayout {
    int L;
    size_t off_tw, off_G[2], off_C[2], total;
};

PiLayout pi_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    PiLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    l.off_tw = 0;
    l.off_G[0] = align256((size_t)l.L * 16);
    l.off_G[1] = align256(l.off_G[0] + spec * d.NA * nel * csz);
    l.off_C[0] = align256(l.off_G[1] + spec * d.NA * nel * csz);
    l.off_C[1] = align256(l.off_C[0] + spec * nA * (d.NB + 1) * 9 * csz);
    l.total = align256(l.off_C[1] + spec * nA * (d.NB + 1) * 9 * csz);
    return l;
}

size_t spectral_pi_workspace(const sse_dims& d) { return pi_layout(d).total; }
size_t spectral_pi32_workspace(const sse_dims& d) { return pi_layout(d, 8).total; }

bool spectral_pi_supported(const sse_dims& d) {
    const int L = spectral_length(d);
    return d.Nkz <= kMaxNk && L < kFftMaxLength && make_plan(L).smem <= 227 * 1024 && d.NB <= 16 &&
           make_pi_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024 &&
           make_pi32_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024;
}

namespace {
// Pi in the real type T: double (FP64) or float (FP32_FFT: FP32 transforms and products, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_pi_t(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                          const double2* G_greater, double scale, uint32_t flags, double2* P_less,
                          double2* P_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    using C = typename CX<T>::C;
    constexpr bool fp32 = sizeof(T) == 4;
    if (!spectral_pi_supported(d)) return cudaErrorNotSupported;
    const PiLayout lay = pi_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Gh[2] = {reinterpret_cast<C*>(base + lay.off_G[0]), reinterpret_cast<C*>(base + lay.off_G[1])};
    C* Ch[2] = {reinterpret_cast<C*>(base + lay.off_C[0]), reinterpret_cast<C*>(base + lay.off_C[1])};
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, ccols = nA * (d.NB + 1) * 9;
    if (nA == 0) return cudaSuccess;
    cudaError_t e;
    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double2* G[2] = {G_less, G_greater};
    for (int t = 0; t < 2; ++t) {
        e = launch_fft32("fft_e_kernel(G)", plan, tw, LoadGT<C>{G[t], d.NE, gcols}, StoreSpecT<C>{Gh[t], L, gcols, L},
                       gcols, d.Nkz, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_dft_k("dft_kz_kernel(G)", Gh[t], d.Nkz, d.Nkz, (size_t)L * gcols, 0, st)) != cudaSuccess) return e;
    }
    const bool half = (flags & SSE_FLAG_ANTIHERMITIAN) != 0;
    const FreqMap fm = make_freq_map(d.Nkz, L, half);
    if (half && (flags & SSE_FLAG_CHECK))
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nkz * d.NE * d.NA * nel, 256), 256, 0, st>>>(
                          G[t], (size_t)d.Nkz * d.NE * d.NA, d.Norb, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    if constexpr (fp32) {
        const Pi32Cfg pc = make_pi32_cfg(d, fm.count);
        if ((e = cudaFuncSetAttribute(spec_pi32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc.smem)) !=
            cudaSuccess)
            return e;
        const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
        SSE_TIMED("spec_pi_kernel", st,
                  spec_pi32_kernel<<<dim3((unsigned)nA, (unsigned)gy, 2), pc.threads, pc.smem, st>>>(
                      pc, d, fm, nbr, dH, Gh[0], Gh[1], Ch[0], Ch[1], status));
    } else {
        const PiCfg pc = make_pi_cfg(d, fm.count);
        if ((e = cudaFuncSetAttribute(spec_pi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc.smem)) !=
            cudaSuccess)
            return e;
        const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
        SSE_TIMED("spec_pi_kernel", st,
                  spec_pi_kernel<<<dim3((unsigned)nA, (unsigned)gy, 2), pc.threads, pc.smem, st>>>(
                      pc, d, fm, nbr, dH, Gh[0], Gh[1], Ch[0], Ch[1], status));
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (half)
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("mirror_pi_kernel", st,
                      mirror_pi_kernel<<<grid_for(fm.count * nA * (d.NB + 1) * 9, 256), 256, 0, st>>>(
                          fm, nA * (d.NB + 1), Ch[t]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    double2* P[2] = {P_less, P_greater};
    const double inv_scale = scale / ((double)d.Nkz * (double)L);
    for (int t = 0; t < 2; ++t) {
        if ((e = launch_dft_k("dft_kz_kernel(C)", Ch[t], d.Nkz, d.Nkz, (size_t)L * ccols, 1, st)) != cudaSuccess) return e;
        e = launch_fft32("fft_e_kernel(C)", plan, tw, LoadSpecConjT<C>{Ch[t], L, ccols},
                       StorePiT<C>{P[t], d.Nw, d.NA, d.NB + 1, (size_t)d.a_begin * (d.NB + 1) * 9, inv_scale,
                                   d.Nw + 1},
                       ccols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        if (flags & SSE_FLAG_SYMMETRIZE) {
            SSE_TIMED("symmetrize3_kernel", st,
                      symmetrize3_kernel<<<grid_for((size_t)d.Nqz * d.Nw * nA * (d.NB + 1), 256), 256, 0, st>>>(
                          d, P[t]));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t spectral_pi(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                        const double2* G_greater, double scale, uint32_t flags, double2* P_less, double2* P_greater,
                        unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    return spectral_pi_t<double>(d, nbr, dH, G_less, G_greater, scale, flags, P_less, P_greater, status, ws,
                                 ws_bytes, st);
}

cudaError_t spectral_pi32(const sse_dims& d, const int32_t* nbr, const double2* dH, const double2* G_less,
                          const double2* G_greater, double scale, uint32_t flags, double2* P_less,
                          double2* P_greater, unsigned* status, void* ws, size_t ws_bytes, cudaStream_t st) {
    return spectral_pi_t<float>(d, nbr, dH, G_less, G_greater, scale, flags, P_less, P_greater, status, ws,
                                ws_bytes, st);
}

}  // namespace sse
