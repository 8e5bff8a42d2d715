// Sigma of Eq. (3) through the transforms: the per-frequency block products in FP64 (spec_prod_kernel, mode
// FP64_FFT) and FP32 (spec_prod32_kernel, mode FP32_FFT), the symmetrisation, the workspace layout and the
// drivers (device buffers, and the pipelined variant behind the host-buffer entry point). Mode F16X3_FFT runs the
// same FP32 transforms with the block products of sse_spectral_tc.cu on the tensor cores.
#include "sse_spectral.cuh"

namespace sse {
namespace {

template <class T>
__global__ void spec_prod_kernel(ProdCfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr,
                                 const double2* __restrict__ dH, const typename CX<T>::C* __restrict__ Ghat,
                                 const typename CX<T>::C* __restrict__ Khat, typename CX<T>::C* __restrict__ Shat,
                                 double scale, unsigned* __restrict__ status) {
    using C = typename CX<T>::C;
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, nel = c.nel;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;  // frequency indices of the map
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    T* sA = reinterpret_cast<T*>(smem + c.off_A);
    T* sG = reinterpret_cast<T*>(smem + c.off_G);
    C* sK = reinterpret_cast<C*>(smem + c.off_K);
    T* sW = reinterpret_cast<T*>(smem + c.off_W);
    T* sU = reinterpret_cast<T*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / nel, e = tid - fl * nel;
    const int m = e / Norb, n = e - m * Norb;
    const bool lane = fl < c.F;

    for (int i = tid; i < d.NB * 3 * nel; i += blockDim.x) {
        const int si = i / nel, ee = i - si * nel;
        const double2 v = dH[((size_t)a * d.NB) * 3 * nel + i];
        put3(sA + (size_t)si * 3 * nel, nel, ee, CT<C>::mk((T)v.x, (T)v.y));
    }
    int bnb[16];
    for (int s = 0; s < d.NB && s < 16; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        bnb[s] = (b >= 0 && b < d.NA) ? b : -1;
        if (bnb[s] < 0 && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
    }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        T T1 = 0, T2 = 0, T3 = 0;
        for (int s = 0; s < d.NB; ++s) {
            const int b = s < 16 ? bnb[s] : -1;
            // stage G^_b(f) and K^_(a,s)(f)
            if (lane) {
                C g = CT<C>::mk(0, 0);
                if (act && b >= 0) g = Ghat[(f * d.NA + b) * nel + e];
                put3(sG + (size_t)fl * 3 * nel, nel, e, g);
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                C k = CT<C>::mk(0, 0);
                if (i0 + fk < i_end && b >= 0) k = Khat[((freq_of(fm, i0 + fk) * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            // W_i[m][n] = sum_j K_ij conj(dH_j[n][m])
            if (lane) {
                const T* A = sA + (size_t)s * 9 * nel;
                const int et = n * Norb + m;
                T ar[3], ai[3];  // conj(dH_j[n][m]) = (ar, -ai)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    ar[j] = A[(size_t)j * 3 * nel + et];
                    ai[j] = A[(size_t)j * 3 * nel + nel + et];
                }
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    C acc = CT<C>::mk(0, 0);  // plain FMA chains: no separate multiplies or adds
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const C k = sK[fl * 9 + i * 3 + j];
                        acc.x = fma(k.x, ar[j], acc.x);
                        acc.x = fma(k.y, ai[j], acc.x);
                        acc.y = fma(k.y, ar[j], acc.y);
                        acc.y = fma(-k.x, ai[j], acc.y);
                    }
                    put3(sW + ((size_t)fl * 3 + i) * 3 * nel, nel, e, acc);
                }
            }
            __syncthreads();
            // U_i = G^ W_i
            if (lane) {
                const T* Gp = sG + (size_t)fl * 3 * nel;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Wp = sW + ((size_t)fl * 3 + i) * 3 * nel;
                    T t1 = 0, t2 = 0, t3 = 0;
                    for (int l = 0; l < Norb; ++l) {
                        const int ga = m * Norb + l, wb = l * Norb + n;
                        t1 = fma(Gp[ga], Wp[wb], t1);
                        t2 = fma(Gp[nel + ga], Wp[nel + wb], t2);
                        t3 = fma(Gp[2 * nel + ga], Wp[2 * nel + wb], t3);
                    }
                    put3(sU + ((size_t)fl * 3 + i) * 3 * nel, nel, e, CT<C>::mk(t1 - t2, t3 - t1 - t2));
                }
            }
            __syncthreads();
            // acc += sum_i dH_i U_i
            if (lane) {
                const T* A = sA + (size_t)s * 9 * nel;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const T* Ap = A + (size_t)i * 3 * nel;
                    const T* Up = sU + ((size_t)fl * 3 + i) * 3 * nel;
                    for (int l = 0; l < Norb; ++l) {
                        const int aa = m * Norb + l, ub = l * Norb + n;
                        T1 = fma(Ap[aa], Up[ub], T1);
                        T2 = fma(Ap[nel + aa], Up[nel + ub], T2);
                        T3 = fma(Ap[2 * nel + aa], Up[2 * nel + ub], T3);
                    }
                }
            }
        }
        if (act) {
            const T re = T1 - T2, im = T3 - T1 - T2;
            Shat[(f * nA + la) * nel + e] = CT<C>::mk((T)(-scale * (double)im), (T)(scale * (double)re));  // i*scale*(re+i im)
        }
    }
}

// ---------------------------------------------------------------------------
// phonon self-energy, Eq. (4): per (a, slot s, frequency)
//   C^_ij(kappa,eps) = tr( dH_i^H G^t_a(kappa,eps) dH_j G^t'_b(-kappa,-eps) ),
// the transform of the correlation sum_{k,E} tr(dH_i^H G^t_a(E+l, k+q) dH_j G^t'_b(E, k)) over the lags
// (q, l); slot NB (the diagonal block) is the sum over the bonds.
// ---------------------------------------------------------------------------
// FP32 block products with register tiles. The FP32 pipe issues 64x the FP64 rate, so the scalar
// kernel above becomes bound by shared-memory bandwidth (two scalar loads per FMA). Here each
// thread computes a 2 x 2 tile of the (zero-padded, Np = Norb rounded up to even) block for one
// frequency, with G^ and dH stored transposed so that every operand pair is one 8-byte load:
// per reduction step 12 FMA for 6 loads. Same arithmetic as spec_prod_kernel (Gauss MACs).
// ---------------------------------------------------------------------------
struct Prod32Cfg {
    int Np, TN, T, F, threads, fchunk;
    int pl;      // floats per Np x Np plane
    int gs, us;  // floats per frequency of the G^ and U regions, padded to 16 mod 32 (see below)
    int off_A, off_G, off_K, off_U, smem;
};


// FP32 products use the 4-multiply complex MAC on (re, im) planes: with shared-memory bandwidth, not the FP32
// pipe, the limit, two planes per operand (4 loads per 16 FMAs of a 2 x 2 tile) beat the 3-multiply form's
// three planes (6 loads per 12 FMAs). U_i = G^ W_i is formed as sum_j K_ij P_j with P_j = G^ A_j^H, so the
// weight blocks W_i never pass through shared memory.
Prod32Cfg make_prod32_cfg(const sse_dims& d, size_t nfreq) {
    Prod32Cfg c{};
    c.Np = d.Norb + (d.Norb & 1);
    c.TN = c.Np / 2;
    c.T = c.TN * c.TN;
    c.pl = c.Np * c.Np;
    const int pb = c.pl * 4;  // bytes per plane
    auto a16 = [](int x) { return (x + 15) & ~15; };
    c.gs = bank_pad16(2 * c.pl);
    c.us = bank_pad16(6 * c.pl);
    c.F = pick_frequencies(c.T, [&](int F) { return (long)d.NB * 6 * pb + F * (4L * (c.gs + c.us) + 9 * 8) + 64; });
    c.threads = ((c.F * c.T + 31) / 32) * 32;
    c.off_A = 0;                                  // [NB][3 dir][2 planes] dH transposed: AT[l][m] = dH[m][l]
    c.off_G = a16(c.off_A + d.NB * 6 * pb);       // [F][gs] G^ transposed (2 planes): GT[l][m] = G^[m][l]
    c.off_K = a16(c.off_G + c.F * c.gs * 4);      // [F][9] float2
    c.off_U = a16(c.off_K + c.F * 9 * 8);         // [F][us] U_i row-major (3 i x 2 planes)
    c.smem = a16(c.off_U + c.F * c.us * 4);
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    size_t want = (size_t)152 * 2 * 8;
    size_t chunks = (want + nA - 1) / (nA ? nA : 1);
    if (chunks < 1) chunks = 1;
    size_t fc = (nfreq + chunks - 1) / chunks;
    fc = ((fc + c.F - 1) / c.F) * c.F;
    c.fchunk = (int)(fc < 1 ? 1 : fc);
    return c;
}

__global__ void spec_prod32_kernel(Prod32Cfg c, sse_dims d, FreqMap fm, const int32_t* __restrict__ nbr,
                                   const double2* __restrict__ dH, const float2* __restrict__ Ghat,
                                   const float2* __restrict__ Khat, float2* __restrict__ Shat, double scale,
                                   unsigned* __restrict__ status) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int Norb = d.Norb, Np = c.Np, pl = c.pl, nel = Norb * Norb;
    const int la = blockIdx.x;
    const int a = d.a_begin + la;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t i_begin = (size_t)blockIdx.y * c.fchunk;
    const size_t i_end = min(fm.count, i_begin + c.fchunk);
    float* sA = reinterpret_cast<float*>(smem + c.off_A);
    float* sG = reinterpret_cast<float*>(smem + c.off_G);
    float2* sK = reinterpret_cast<float2*>(smem + c.off_K);
    float* sU = reinterpret_cast<float*>(smem + c.off_U);
    const int tid = threadIdx.x;
    const int fl = tid / c.T, tt = tid - fl * c.T;
    const int m0 = 2 * (tt / c.TN), n0 = 2 * (tt % c.TN);
    const bool lane = fl < c.F;

    // dH planes, transposed and zero-padded: AT[s][dir][plane][l][m] = dH(a,s,dir)[m][l]
    for (int i = tid; i < d.NB * 3 * pl; i += blockDim.x) {
        const int sd = i / pl, e = i - sd * pl;
        const int l = e / Np, m = e - l * Np;
        double2 v = make_double2(0.0, 0.0);
        if (l < Norb && m < Norb) v = dH[((size_t)a * d.NB * 3 + sd) * nel + m * Norb + l];
        float* P = sA + (size_t)sd * 2 * pl;
        P[e] = (float)v.x;
        P[pl + e] = (float)v.y;
    }
    for (int s = 0; s < d.NB; ++s) {
        const int b = nbr[(size_t)a * d.NB + s];
        if ((b < 0 || b >= d.NA) && tid == 0) atomicOr(status, DEV_BAD_NEIGHBOUR);
    }
    __syncthreads();

    for (size_t i0 = i_begin; i0 < i_end; i0 += c.F) {
        const bool act = lane && i0 + fl < i_end;
        const size_t f = act ? freq_of(fm, i0 + fl) : 0;
        float accr[4] = {0, 0, 0, 0}, acci[4] = {0, 0, 0, 0};  // the 2 x 2 tile of sum_s sum_i dH_i U_i
        for (int s = 0; s < d.NB; ++s) {
            const int b = nbr[(size_t)a * d.NB + s];
            const bool bok = b >= 0 && b < d.NA;
            // G^_b(f) -> GT planes: element (m, n) goes to GT[n][m]
            if (lane) {
                float* Gp = sG + (size_t)fl * c.gs;
#pragma unroll
                for (int dm = 0; dm < 2; ++dm)
#pragma unroll
                    for (int dn = 0; dn < 2; ++dn) {
                        const int m = m0 + dm, n = n0 + dn;
                        float2 g = make_float2(0.f, 0.f);
                        if (act && bok && m < Norb && n < Norb) g = Ghat[(f * d.NA + b) * nel + m * Norb + n];
                        const int o = n * Np + m;
                        Gp[o] = g.x;
                        Gp[pl + o] = g.y;
                    }
            }
            for (int i = tid; i < c.F * 9; i += blockDim.x) {
                const int fk = i / 9, ij = i - fk * 9;
                float2 k = make_float2(0.f, 0.f);
                if (i0 + fk < i_end && bok) k = Khat[((freq_of(fm, i0 + fk) * nA + la) * d.NB + s) * 9 + ij];
                sK[i] = k;
            }
            __syncthreads();
            const float* A = sA + (size_t)s * 6 * pl;
            // P_j = G^ A_j^H for the three j at once: P_j[m][n] = sum_l GT[l][m] conj(AT_j[l][n]);
            // U_i = G^ W_i = sum_j K_ij P_j
            if (lane) {
                const float* Gp = sG + (size_t)fl * c.gs;
                float pr[3][4] = {}, pim[3][4] = {};
                for (int l = 0; l < Norb; ++l) {
                    const float2 gr = ld2(Gp + l * Np + m0), gi = ld2(Gp + pl + l * Np + m0);
#pragma unroll
                    for (int j = 0; j < 3; ++j)
                        cmac2x2<false, true>(pr[j], pim[j], gr, gi, ld2(A + (size_t)j * 2 * pl + l * Np + n0),
                                             ld2(A + (size_t)j * 2 * pl + pl + l * Np + n0));
                }
                const float2* K = sK + fl * 9;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    float ur[4] = {0, 0, 0, 0}, ui[4] = {0, 0, 0, 0};
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const float2 k = K[i * 3 + j];
#pragma unroll
                        for (int q = 0; q < 4; ++q) {
                            ur[q] = fmaf(k.x, pr[j][q], ur[q]);
                            ur[q] = fmaf(-k.y, pim[j][q], ur[q]);
                            ui[q] = fmaf(k.x, pim[j][q], ui[q]);
                            ui[q] = fmaf(k.y, pr[j][q], ui[q]);
                        }
                    }
                    float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
#pragma unroll
                    for (int dm = 0; dm < 2; ++dm) {
                        float* o = Up + (m0 + dm) * Np + n0;
                        st2(o, ur[dm * 2], ur[dm * 2 + 1]);
                        st2(o + pl, ui[dm * 2], ui[dm * 2 + 1]);
                    }
                }
            }
            __syncthreads();
            // acc += sum_i dH_i U_i: acc[m][n] += sum_l AT_i[l][m] U_i[l][n]
            if (lane) {
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                    const float* Ap = A + (size_t)i * 2 * pl;
                    const float* Up = sU + (size_t)fl * c.us + (size_t)i * 2 * pl;
                    for (int l = 0; l < Norb; ++l) {
                        const float2 ar = ld2(Ap + l * Np + m0), ai = ld2(Ap + pl + l * Np + m0);
                        const float2 vr = ld2(Up + l * Np + n0), vi = ld2(Up + pl + l * Np + n0);
                        cmac2x2<false, false>(accr, acci, ar, ai, vr, vi);
                    }
                }
            }
            __syncthreads();  // sG, sK, sU are rewritten for the next bond
        }
        if (act) {
            const float sc = (float)scale;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int m = m0 + q / 2, n = n0 + (q & 1);
                if (m < Norb && n < Norb)  // i*scale*(re + i im)
                    Shat[(f * nA + la) * nel + m * Norb + n] = make_float2(-sc * acci[q], sc * accr[q]);
            }
        }
    }
}

// (S - S^H)/2 on the blocks of atoms in range
__global__ void symmetrize_kernel(sse_dims d, double2* __restrict__ S) {
    const int Norb = d.Norb, nel = Norb * Norb;
    const size_t nA = (size_t)(d.a_end - d.a_begin);
    const size_t nblk = (size_t)d.Nkz * d.NE * nA;
    const size_t total = nblk * nel;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
        const int e = (int)(i % nel);
        const size_t blk = i / nel;
        const int m = e / Norb, n = e - m * Norb;
        if (n < m) continue;
        const size_t ke = blk / nA, la = blk - ke * nA;
        double2* B = S + (ke * d.NA + d.a_begin + la) * nel;
        const double2 x = B[m * Norb + n], y = B[n * Norb + m];
        B[m * Norb + n] = make_double2(0.5 * (x.x - y.x), 0.5 * (x.y + y.y));
        if (m != n) B[n * Norb + m] = make_double2(0.5 * (y.x - x.x), 0.5 * (y.y + x.y));
    }
}

struct SpecLayout {
    int L;
    size_t off_tw, off_G, off_K, off_S, total;
};

SpecLayout spec_layout(const sse_dims& d, size_t csz = 16) {  // csz: bytes per complex spectrum entry
    SpecLayout l{};
    l.L = spectral_length(d);
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t spec = (size_t)d.Nkz * l.L;
    l.off_tw = 0;
    l.off_G = align256(l.off_tw + (size_t)l.L * 16);
    l.off_K = align256(l.off_G + spec * d.NA * nel * csz);
    l.off_S = align256(l.off_K + spec * nA * d.NB * 9 * csz);
    l.total = align256(l.off_S + spec * nA * nel * csz);
    return l;
}

}  // namespace

int spectral_length(const sse_dims& d) {
    for (int L = d.NE + d.Nw;; ++L) {  // smallest 2^a 3^b: radix-4/2/3 stages only
        int m = L;
        while (m % 2 == 0) m /= 2;
        while (m % 3 == 0) m /= 3;
        if (m == 1) return L;
    }
}

bool spectral_supported(const sse_dims& d) {
    const int L = spectral_length(d);
    return d.Nkz <= kMaxNk && L < kFftMaxLength && make_plan(L).smem <= 227 * 1024 && d.NB <= 16 &&
           make_prod_cfg(d, (size_t)d.Nkz * L).smem <= 227 * 1024;
}

bool spectral_fwd_supported(const sse_dims& d, bool fp32) {
    return spectral_supported(d) && (!fp32 || make_prod32_cfg(d, 1).smem <= 227 * 1024);
}

size_t spectral_fwd_workspace(const sse_dims& d) { return spec_layout(d).total; }
size_t spectral_fwd32_workspace(const sse_dims& d) { return spec_layout(d, 8).total; }

namespace {
// The forward in the real type T: double (FP64_FFT) or float (FP32_FFT: FP32 transforms and block
// products on the FP32 pipe, FP64 inputs and outputs).
template <class T>
cudaError_t spectral_fwd_t(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                           size_t ws_bytes, cudaStream_t st, const FwdPipe* pipe = nullptr, bool tc = false) {
    // With `pipe` (inputs arriving from the host): the lag kernel is transformed first, G^t slice by slice as its
    // kz slices arrive, and the inverse E-transform of Sigma^t runs slice by slice so that each slice's download
    // can start; without it every transform is one launch over all slices.
    using C = typename CX<T>::C;
    const sse_dims& d = p.d;
    // tc: the FP32 transforms with the block products on the tensor cores (mode F16X3_FFT)
    if (tc && sizeof(T) != 4) return cudaErrorNotSupported;
    if (!(tc ? spectral_fwd_tc_supported(d) : spectral_fwd_supported(d, sizeof(T) == 4))) return cudaErrorNotSupported;
    const SpecLayout lay = spec_layout(d, sizeof(C));
    if (ws_bytes < lay.total) return cudaErrorInvalidValue;
    unsigned char* base = static_cast<unsigned char*>(ws);
    double2* tw = reinterpret_cast<double2*>(base + lay.off_tw);
    C* Gh = reinterpret_cast<C*>(base + lay.off_G);
    C* Kh = reinterpret_cast<C*>(base + lay.off_K);
    C* Sh = reinterpret_cast<C*>(base + lay.off_S);
    const int L = lay.L;
    const FftPlan plan = make_plan(L, (int)sizeof(C));
    const size_t nA = (size_t)(d.a_end - d.a_begin), nel = (size_t)d.Norb * d.Norb;
    const size_t gcols = (size_t)d.NA * nel, kcols = nA * d.NB * 9, scols = nA * nel;
    cudaError_t e;
    if (nA == 0) return cudaSuccess;

    SSE_TIMED("twiddle_kernel", st, twiddle_kernel<<<grid_for(L, 256), 256, 0, st>>>(L, tw));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const bool half = (p.flags & SSE_FLAG_ANTIHERMITIAN) != 0;
    const FreqMap fm = make_freq_map(d.Nkz, L, half);
    if (half && (p.flags & SSE_FLAG_CHECK)) {
        if (pipe)  // every input (the copies are issued in order on one stream)
            if ((e = cudaStreamWaitEvent(st, pipe->g[1][d.Nkz - 1], 0)) != cudaSuccess) return e;
        for (int t = 0; t < 2; ++t) {
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nkz * d.NE * d.NA * nel, 256), 256, 0, st>>>(
                          p.G[t], (size_t)d.Nkz * d.NE * d.NA, d.Norb, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            SSE_TIMED("check_antiherm_kernel", st,
                      check_antiherm_kernel<<<grid_for((size_t)d.Nqz * d.Nw * d.NA * d.NB * 9, 256), 256, 0, st>>>(
                          p.D[t], (size_t)d.Nqz * d.Nw * d.NA * d.NB, 3, status));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
    }
    const ProdCfg pc = make_prod_cfg(d, fm.count, (int)sizeof(T));
    const Prod32Cfg pc32 = make_prod32_cfg(d, fm.count);
    const bool tiled = sizeof(T) == 4;  // FP32: register-tiled kernel
    if ((e = tiled ? cudaFuncSetAttribute(spec_prod32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, pc32.smem)
                   : cudaFuncSetAttribute(spec_prod_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          pc.smem)) != cudaSuccess)
        return e;
    double2* S[2] = {S_less, S_greater};
    if (pipe && (e = cudaStreamWaitEvent(st, pipe->inputs, 0)) != cudaSuccess) return e;
    for (int t = 0; t < 2; ++t) {
        // 1. lag kernel -> K^ (needs only D; with `pipe` it runs while G^t is still arriving)
        LoadLagT<C> ll{p.D[t], p.D[1 - t], d.Nw, L, (size_t)d.NA * d.NB * 9, (size_t)d.a_begin * d.NB * 9};
        e = launch_fft32("fft_e_kernel(K)", plan, tw, ll, StoreSpecT<C>{Kh, L, kcols, L}, kcols, d.Nqz, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_dft_k("dft_kz_kernel(K)", Kh, d.Nkz, d.Nqz, (size_t)L * kcols, 0, st)) != cudaSuccess) return e;
        // 2. G^t -> G^ (E-transform per kz slice as the slices arrive, then the kz DFT)
        if (pipe) {
            for (int k = 0; k < d.Nkz; ++k) {
                if ((e = cudaStreamWaitEvent(st, pipe->g[t][k], 0)) != cudaSuccess) return e;
                e = launch_fft32("fft_e_kernel(G)", plan, tw, LoadGT<C>{p.G[t] + (size_t)k * d.NE * gcols, d.NE, gcols},
                               StoreSpecT<C>{Gh + (size_t)k * L * gcols, L, gcols, L}, gcols, 1, st);
                if (e != cudaSuccess) return e;
            }
        } else {
            e = launch_fft32("fft_e_kernel(G)", plan, tw, LoadGT<C>{p.G[t], d.NE, gcols},
                           StoreSpecT<C>{Gh, L, gcols, L}, gcols, d.Nkz, st);
            if (e != cudaSuccess) return e;
        }
        if ((e = launch_dft_k("dft_kz_kernel(G)", Gh, d.Nkz, d.Nkz, (size_t)L * gcols, 0, st)) != cudaSuccess) return e;
        // 3. block products (one frequency of each (f, -f) pair with anti-Hermitian inputs, then the mirror)
        if (tc) {
            e = spectral_prod_tc(d, fm, p.nbr, p.dH, reinterpret_cast<const float2*>(Gh),
                                 reinterpret_cast<const float2*>(Kh), reinterpret_cast<float2*>(Sh), p.scale, status,
                                 st);
            if (e != cudaSuccess) return e;
        } else if (tiled) {
            const size_t gy = (fm.count + pc32.fchunk - 1) / pc32.fchunk;
            SSE_TIMED("spec_prod32_kernel", st,
                      spec_prod32_kernel<<<dim3((unsigned)nA, (unsigned)gy), pc32.threads, pc32.smem, st>>>(
                          pc32, d, fm, p.nbr, p.dH, reinterpret_cast<const float2*>(Gh),
                          reinterpret_cast<const float2*>(Kh), reinterpret_cast<float2*>(Sh), p.scale, status));
        } else {
            const size_t gy = (fm.count + pc.fchunk - 1) / pc.fchunk;
            SSE_TIMED("spec_prod_kernel", st,
                      spec_prod_kernel<T><<<dim3((unsigned)nA, (unsigned)gy), pc.threads, pc.smem, st>>>(
                          pc, d, fm, p.nbr, p.dH, Gh, Kh, Sh, p.scale, status));
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if (half) {
            SSE_TIMED("mirror_sigma_kernel", st,
                      mirror_sigma_kernel<<<grid_for(fm.count * nA * nel, 256), 256, 0, st>>>(fm, nA, d.Norb, Sh));
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        // 4. inverse transforms into Sigma^t
        if ((e = launch_dft_k("dft_kz_kernel(S)", Sh, d.Nkz, d.Nkz, (size_t)L * scols, 1, st)) != cudaSuccess) return e;
        const double inv = 1.0 / ((double)d.Nkz * (double)L);
        const bool sym = (p.flags & SSE_FLAG_SYMMETRIZE) != 0;
        if (pipe) {  // slice by slice, each handed to its download as soon as it is written
            sse_dims dk = d;
            dk.Nkz = 1;
            for (int k = 0; k < d.Nkz; ++k) {
                double2* Sk = S[t] + (size_t)k * d.NE * d.NA * nel;
                e = launch_fft32("fft_e_kernel(S)", plan, tw, LoadSpecConjT<C>{Sh + (size_t)k * L * scols, L, scols},
                               StoreSigmaT<C>{Sk, d.NE, (size_t)d.NA * nel, (size_t)d.a_begin * nel, inv, d.NE},
                               scols, 1, st);
                if (e != cudaSuccess) return e;
                if (sym) {
                    SSE_TIMED("symmetrize_kernel", st,
                              symmetrize_kernel<<<grid_for((size_t)d.NE * nA * nel, 256), 256, 0, st>>>(dk, Sk));
                    if ((e = cudaGetLastError()) != cudaSuccess) return e;
                }
                if ((e = cudaEventRecord(pipe->s[t][k], st)) != cudaSuccess) return e;
            }
        } else {
            e = launch_fft32("fft_e_kernel(S)", plan, tw, LoadSpecConjT<C>{Sh, L, scols},
                           StoreSigmaT<C>{S[t], d.NE, (size_t)d.NA * nel, (size_t)d.a_begin * nel, inv, d.NE}, scols,
                           d.Nkz, st);
            if (e != cudaSuccess) return e;
            if (sym) {
                SSE_TIMED("symmetrize_kernel", st,
                          symmetrize_kernel<<<grid_for((size_t)d.Nkz * d.NE * nA * nel, 256), 256, 0, st>>>(d, S[t]));
                if ((e = cudaGetLastError()) != cudaSuccess) return e;
            }
        }
    }
    return cudaSuccess;
}
}  // namespace

cudaError_t spectral_fwd_pipelined(const Problem& p, int mode, double2* S_less, double2* S_greater, unsigned* status,
                                   void* ws, size_t ws_bytes, cudaStream_t st, const FwdPipe& pipe) {
    if (mode == SSE_MODE_FP64_FFT) return spectral_fwd_t<double>(p, S_less, S_greater, status, ws, ws_bytes, st, &pipe);
    return spectral_fwd_t<float>(p, S_less, S_greater, status, ws, ws_bytes, st, &pipe, mode == SSE_MODE_F16X3_FFT);
}

cudaError_t spectral_fwd(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                         size_t ws_bytes, cudaStream_t st) {
    return spectral_fwd_t<double>(p, S_less, S_greater, status, ws, ws_bytes, st);
}

cudaError_t spectral_fwd32(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                           size_t ws_bytes, cudaStream_t st) {
    return spectral_fwd_t<float>(p, S_less, S_greater, status, ws, ws_bytes, st);
}

bool spectral_fwd_tc_supported(const sse_dims& d) {
    return spectral_fwd_supported(d, true) && spectral_prod_tc_supported(d);
}

cudaError_t spectral_fwd_tc(const Problem& p, double2* S_less, double2* S_greater, unsigned* status, void* ws,
                            size_t ws_bytes, cudaStream_t st) {
    return spectral_fwd_t<float>(p, S_less, S_greater, status, ws, ws_bytes, st, nullptr, true);
}

}  // namespace sse
