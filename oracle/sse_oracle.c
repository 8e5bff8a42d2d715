/*
 * FP64 CPU oracle for the electron and phonon scattering self-energies (SSE)
 * of Ziogas et al., "A Data-Centric Approach to Extreme-Scale Ab initio
 * Dissipative Quantum Transport Simulations" (SC'19), Eqs. (3) and (4), and
 * for the bond-weight combination D_ba - D_bb - D_aa + D_ab of Eq. (3).
 *
 * TEST INFRASTRUCTURE ONLY. This file is the slow, plain reference that the
 * CUDA path is checked against. Only the test suite, the package smoke check
 * and the benchmark's CPU-baseline leg may build, load or call it. It shares
 * no code with the CUDA path and includes none of its headers.
 *
 * Notation (Sec. 2, Eq. 3 and the tensor description that follows it):
 *   G^t   [Nkz][NE][NA][Norb][Norb]   diagonal blocks G^t_bb(E, kz), t in {<,>}
 *   dH    [NA][NB][3][Norb][Norb]     grad_i H_ab for b = nbr[a][s]
 *   Dc^t  [Nqz][Nw][NA][NB][3][3]     phonon weight of the bond (a, slot s):
 *                                     the combination D_ba - D_bb - D_aa + D_ab
 *   Sigma [Nkz][NE][NA][Norb][Norb]   diagonal blocks Sigma^t_aa(E, kz)
 *
 * Eq. (3), with the readings used throughout this project:
 *   Sigma^t_aa(E,k) = i*scale * sum_q sum_{s} sum_{w,sigma} sum_{i,j}
 *        dH_i(a,s) . G^t_bb(E - sigma*(w+1), (k - q) mod Nkz) . dH_j(a,s)^H
 *        * Dc^{tau(t,sigma)}_ij(q, w, a, s)
 *   - b = nbr[a][s]; the l in the printed sum index is the neighbour b.
 *   - grad_j H_ba = (grad_j H_ab)^H.
 *   - sigma = +1 (emission): G at E - (w+1), weight Dc^t;
 *     sigma = -1 (absorption): G at E + (w+1), weight Dc^{other type}.
 *   - energies outside [0, NE) contribute zero (no wrap); kz wraps.
 *   - the integral d(hbar omega)/2pi over the uniform phonon grid is the sum
 *     over w times `scale` (= grid step / 2pi).
 *
 * All arithmetic is IEEE double / double complex, built with
 * -ffp-contract=off so x86 and Arm hosts round identically.
 */
#include <complex.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

typedef struct {
    int32_t NA, NB, Norb, NE, Nkz, Nqz, Nw;
    int32_t a_begin, a_end; /* atoms whose Sigma (or gradients) are computed */
    int32_t E_begin, E_end; /* energies whose Sigma is computed (forward only) */
} sse_oracle_dims;

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1
#define ORACLE_NO_MEM 2

static int check_dims(const sse_oracle_dims* d) {
    if (!d) return 0;
    if (d->NA < 1 || d->NB < 1 || d->Norb < 1 || d->NE < 1 || d->Nkz < 1 || d->Nqz < 1 || d->Nw < 1) return 0;
    if (d->Nqz > d->Nkz) return 0;
    if (d->a_begin < 0 || d->a_end > d->NA || d->a_begin > d->a_end) return 0;
    if (d->E_begin < 0 || d->E_end > d->NE || d->E_begin > d->E_end) return 0;
    return 1;
}

static size_t off_G(const sse_oracle_dims* d, int k, int E, int a) {
    return (((size_t)k * d->NE + E) * d->NA + a) * (size_t)d->Norb * d->Norb;
}
static size_t off_dH(const sse_oracle_dims* d, int a, int s, int i) {
    return (((size_t)a * d->NB + s) * 3 + i) * (size_t)d->Norb * d->Norb;
}
static size_t off_D(const sse_oracle_dims* d, int q, int w, int a, int s) {
    return ((((size_t)q * d->Nw + w) * d->NA + a) * d->NB + s) * 9;
}

/* C = A B */
static void mm(int n, const cplx* A, const cplx* B, cplx* C) {
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            cplx acc = 0;
            for (int l = 0; l < n; ++l) acc += A[r * n + l] * B[l * n + c];
            C[r * n + c] = acc;
        }
}
/* C = A B^H */
static void mm_bh(int n, const cplx* A, const cplx* B, cplx* C) {
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            cplx acc = 0;
            for (int l = 0; l < n; ++l) acc += A[r * n + l] * conj(B[c * n + l]);
            C[r * n + c] = acc;
        }
}
/* C = A^H B */
static void mm_ah(int n, const cplx* A, const cplx* B, cplx* C) {
    for (int r = 0; r < n; ++r)
        for (int c = 0; c < n; ++c) {
            cplx acc = 0;
            for (int l = 0; l < n; ++l) acc += conj(A[l * n + r]) * B[l * n + c];
            C[r * n + c] = acc;
        }
}
/* sum_{mn} conj(X[mn]) Y[mn] = tr(X^H Y) */
static cplx frob(int n, const cplx* X, const cplx* Y) {
    cplx acc = 0;
    for (int e = 0; e < n * n; ++e) acc += conj(X[e]) * Y[e];
    return acc;
}

/* ------------------------------------------------------------------ */
/* forward                                                              */
/* ------------------------------------------------------------------ */

typedef struct {
    const sse_oracle_dims* d;
    const int32_t* nbr;
    const cplx* dH;
    const cplx* D[2]; /* [0] = Dc^<, [1] = Dc^> */
    const cplx* G[2];
    cplx* S[2];
    cplx c; /* i * scale */
    long long n_out, next;
    pthread_mutex_t lock;
    long long terms; /* number of (t,a,E,k,q,s,w,sigma) terms that were in range */
    int fail;
} fwd_job;

/* Sigma^t_aa(E,k) for one output block, following Eq. (3) term by term. */
static long long fwd_one(fwd_job* J, int t, int a, int E, int k, cplx* P, cplx* Q, cplx* S) {
    const sse_oracle_dims* d = J->d;
    const int n = d->Norb, nn = n * n;
    long long terms = 0;
    memset(S, 0, sizeof(cplx) * nn);
    for (int q = 0; q < d->Nqz; ++q) {
        const int kp = ((k - q) % d->Nkz + d->Nkz) % d->Nkz; /* kz - qz, periodic */
        for (int s = 0; s < d->NB; ++s) {
            const int b = J->nbr[(size_t)a * d->NB + s];
            for (int w = 0; w < d->Nw; ++w) {
                for (int sg = 0; sg < 2; ++sg) {
                    const int sigma = sg == 0 ? +1 : -1;
                    const int Ep = E - sigma * (w + 1);
                    if (Ep < 0 || Ep >= d->NE) continue; /* out of range: zero */
                    ++terms;
                    const int tau = sigma == +1 ? t : 1 - t;
                    const cplx* Gp = J->G[t] + off_G(d, kp, Ep, b);
                    const cplx* Dc = J->D[tau] + off_D(d, q, w, a, s);
                    for (int i = 0; i < 3; ++i) {
                        mm(n, J->dH + off_dH(d, a, s, i), Gp, P); /* dH_i(a,b) G_bb */
                        for (int j = 0; j < 3; ++j) {
                            mm_bh(n, P, J->dH + off_dH(d, a, s, j), Q); /* ... dH_j(b,a) */
                            const cplx dij = Dc[i * 3 + j];
                            for (int e = 0; e < nn; ++e) S[e] += dij * Q[e];
                        }
                    }
                }
            }
        }
    }
    cplx* out = J->S[t] + off_G(d, k, E, a);
    for (int e = 0; e < nn; ++e) out[e] = J->c * S[e];
    return terms;
}

static void* fwd_worker(void* arg) {
    fwd_job* J = (fwd_job*)arg;
    const sse_oracle_dims* d = J->d;
    const int nn = d->Norb * d->Norb;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * nn * 3);
    if (!buf) {
        pthread_mutex_lock(&J->lock);
        J->fail = 1;
        pthread_mutex_unlock(&J->lock);
        return NULL;
    }
    const int nA = d->a_end - d->a_begin, nE = d->E_end - d->E_begin;
    long long terms = 0;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        long long o = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (o >= J->n_out) break;
        /* output index -> (t, a, E, k) */
        const int k = (int)(o % d->Nkz);
        long long r = o / d->Nkz;
        const int E = d->E_begin + (int)(r % nE);
        r /= nE;
        const int a = d->a_begin + (int)(r % nA);
        const int t = (int)(r / nA);
        terms += fwd_one(J, t, a, E, k, buf, buf + nn, buf + 2 * nn);
    }
    free(buf);
    pthread_mutex_lock(&J->lock);
    J->terms += terms;
    pthread_mutex_unlock(&J->lock);
    return NULL;
}

static int run_threads(void* (*fn)(void*), void* job, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    int started = 0;
    for (int i = 0; i < nthreads; ++i) {
        if (pthread_create(&th[i], NULL, fn, job) != 0) break;
        ++started;
    }
    if (started == 0) fn(job);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    return 0;
}

/*
 * Sigma^<, Sigma^> of Eq. (3) for atoms [a_begin, a_end) and energies
 * [E_begin, E_end), all kz. Other blocks of S_less / S_greater are untouched.
 * Host pointers, complex128 interleaved. Returns 0 on success. If n_terms is
 * not NULL it receives the number of in-range (t,a,E,k,q,s,w,sigma) terms.
 */
int sse_oracle_fwd(const sse_oracle_dims* d, const int32_t* nbr, const cplx* dH, const cplx* D_less,
                   const cplx* D_greater, const cplx* G_less, const cplx* G_greater, double scale,
                   cplx* S_less, cplx* S_greater, int nthreads, long long* n_terms) {
    if (!check_dims(d) || !nbr || !dH || !D_less || !D_greater || !G_less || !G_greater || !S_less || !S_greater)
        return ORACLE_BAD_ARG;
    for (size_t e = 0; e < (size_t)d->NA * d->NB; ++e)
        if (nbr[e] < 0 || nbr[e] >= d->NA) return ORACLE_BAD_ARG;
    fwd_job J;
    memset(&J, 0, sizeof J);
    J.d = d;
    J.nbr = nbr;
    J.dH = dH;
    J.D[0] = D_less;
    J.D[1] = D_greater;
    J.G[0] = G_less;
    J.G[1] = G_greater;
    J.S[0] = S_less;
    J.S[1] = S_greater;
    J.c = I * scale;
    J.n_out = 2LL * (d->a_end - d->a_begin) * (d->E_end - d->E_begin) * d->Nkz;
    pthread_mutex_init(&J.lock, NULL);
    run_threads(fwd_worker, &J, nthreads);
    pthread_mutex_destroy(&J.lock);
    if (n_terms) *n_terms = J.terms;
    return J.fail ? ORACLE_NO_MEM : ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* adjoint                                                              */
/* ------------------------------------------------------------------ */
/*
 * Loss L = sum_t sum_{a,E,k} Re tr( W^t_a(E,k)^H Sigma^t_a(E,k) ).
 * Gradients follow the PyTorch convention for complex leaves,
 * grad z = dL/dRe z + i dL/dIm z, so for L = Re(alpha z) grad z = conj(alpha)
 * and for L = Re tr(B^H X) grad X = B. With c = i*scale each term
 * c * Dc_ij * dH_i G dH_j^H of Eq. (3) gives
 *   grad Dc_ij     += conj( c * tr(W^H dH_i G dH_j^H) )
 *   grad dH_m      += sum_j conj(c * Dc_mj) * W dH_j G^H      (dH_m on the left)
 *                   + sum_i c * Dc_im * W^H dH_i G            (dH_m^H on the right)
 */

typedef struct {
    const sse_oracle_dims* d;
    const int32_t* nbr;
    const cplx* dH;
    const cplx* D[2];
    const cplx* G[2];
    const cplx* W[2];
    cplx c;
    pthread_mutex_t lock;
    int fail;
} bwd_job;

/* Adds the contributions of energies [E0, E1) of atom a to gdH_a [NB][3][nn] and
 * gD_a[tau] [Nqz][Nw][NB][9] (per-atom packed gradient buffers). */
static void bwd_atom(bwd_job* J, int a, int E0, int E1, cplx* gdH_a, cplx* gD_a0, cplx* gD_a1, cplx* buf) {
    const sse_oracle_dims* d = J->d;
    const int n = d->Norb, nn = n * n;
    cplx* gD_a[2] = {gD_a0, gD_a1};
    cplx* P = buf;           /* dH_i G          */
    cplx* T = buf + nn;      /* scratch         */
    cplx* U = buf + 2 * nn;  /* scratch         */
    cplx* AG = buf + 3 * nn; /* 3 x (dH_i G) or 3 x (W dH_j) */
    for (int t = 0; t < 2; ++t)
        for (int E = E0; E < E1; ++E)
            for (int k = 0; k < d->Nkz; ++k) {
                const cplx* W = J->W[t] + off_G(d, k, E, a);
                for (int q = 0; q < d->Nqz; ++q) {
                    const int kp = ((k - q) % d->Nkz + d->Nkz) % d->Nkz;
                    for (int s = 0; s < d->NB; ++s) {
                        const int b = J->nbr[(size_t)a * d->NB + s];
                        const cplx* A0 = J->dH + off_dH(d, a, s, 0);
                        cplx* gA = gdH_a + (size_t)s * 3 * nn;
                        for (int w = 0; w < d->Nw; ++w)
                            for (int sg = 0; sg < 2; ++sg) {
                                const int sigma = sg == 0 ? +1 : -1;
                                const int Ep = E - sigma * (w + 1);
                                if (Ep < 0 || Ep >= d->NE) continue;
                                const int tau = sigma == +1 ? t : 1 - t;
                                const cplx* Gp = J->G[t] + off_G(d, kp, Ep, b);
                                const cplx* Dc = J->D[tau] + off_D(d, q, w, a, s);
                                cplx* gDc = gD_a[tau] + (((size_t)q * d->Nw + w) * d->NB + s) * 9;
                                /* grad Dc_ij += conj(c tr(W^H dH_i G dH_j^H)) */
                                for (int i = 0; i < 3; ++i) {
                                    mm(n, A0 + (size_t)i * nn, Gp, P);
                                    for (int j = 0; j < 3; ++j) {
                                        mm_bh(n, P, A0 + (size_t)j * nn, T);
                                        gDc[i * 3 + j] += conj(J->c * frob(n, W, T));
                                    }
                                }
                                /* grad dH_m, left occurrences: conj(c Dc_mj) W dH_j G^H */
                                for (int j = 0; j < 3; ++j) {
                                    mm(n, W, A0 + (size_t)j * nn, T); /* W dH_j */
                                    mm_bh(n, T, Gp, AG + (size_t)j * nn);  /* W dH_j G^H */
                                }
                                for (int m = 0; m < 3; ++m)
                                    for (int j = 0; j < 3; ++j) {
                                        const cplx f = conj(J->c * Dc[m * 3 + j]);
                                        for (int e = 0; e < nn; ++e) gA[(size_t)m * nn + e] += f * AG[(size_t)j * nn + e];
                                    }
                                /* grad dH_m, right occurrences: c Dc_im W^H dH_i G */
                                for (int i = 0; i < 3; ++i) {
                                    mm_ah(n, W, A0 + (size_t)i * nn, T); /* W^H dH_i */
                                    mm(n, T, Gp, U);                      /* W^H dH_i G */
                                    memcpy(AG + (size_t)i * nn, U, sizeof(cplx) * nn);
                                }
                                for (int m = 0; m < 3; ++m)
                                    for (int i = 0; i < 3; ++i) {
                                        const cplx f = J->c * Dc[i * 3 + m];
                                        for (int e = 0; e < nn; ++e) gA[(size_t)m * nn + e] += f * AG[(size_t)i * nn + e];
                                    }
                            }
                    }
                }
            }
}

/* Thread `id` of `nthreads` takes the energy chunk [id*NE/n, (id+1)*NE/n) of every atom and
 * accumulates into its own buffers; the chunks are added in thread order afterwards, so the
 * result does not depend on scheduling. */
typedef struct {
    bwd_job* J;
    int id, nthreads;
    cplx *gdH, *gD0, *gD1; /* [atoms][...] private partial sums */
} bwd_part;

static void* bwd_worker(void* arg) {
    bwd_part* P = (bwd_part*)arg;
    bwd_job* J = P->J;
    const sse_oracle_dims* d = J->d;
    const int nn = d->Norb * d->Norb;
    const size_t per_dH = (size_t)d->NB * 3 * nn, per_D = (size_t)d->Nqz * d->Nw * d->NB * 9;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * nn * 6);
    if (!buf) {
        pthread_mutex_lock(&J->lock);
        J->fail = 1;
        pthread_mutex_unlock(&J->lock);
        return NULL;
    }
    const int E0 = (int)((long long)P->id * d->NE / P->nthreads);
    const int E1 = (int)((long long)(P->id + 1) * d->NE / P->nthreads);
    for (int a = d->a_begin; a < d->a_end; ++a) {
        const size_t ai = (size_t)(a - d->a_begin);
        bwd_atom(J, a, E0, E1, P->gdH + ai * per_dH, P->gD0 + ai * per_D, P->gD1 + ai * per_D, buf);
    }
    free(buf);
    return NULL;
}

/*
 * Gradients of L = sum_t Re tr(W^t^H Sigma^t) w.r.t. dH and Dc^<, Dc^> for the
 * atoms [a_begin, a_end) (all energies; E_begin/E_end are ignored). Blocks of
 * other atoms are untouched. W_less / W_greater have the shape of Sigma.
 */
int sse_oracle_bwd(const sse_oracle_dims* d, const int32_t* nbr, const cplx* dH, const cplx* D_less,
                   const cplx* D_greater, const cplx* G_less, const cplx* G_greater, double scale,
                   const cplx* W_less, const cplx* W_greater, cplx* g_dH, cplx* g_D_less, cplx* g_D_greater,
                   int nthreads) {
    if (!check_dims(d) || !nbr || !dH || !D_less || !D_greater || !G_less || !G_greater || !W_less || !W_greater ||
        !g_dH || !g_D_less || !g_D_greater)
        return ORACLE_BAD_ARG;
    for (size_t e = 0; e < (size_t)d->NA * d->NB; ++e)
        if (nbr[e] < 0 || nbr[e] >= d->NA) return ORACLE_BAD_ARG;
    bwd_job J;
    memset(&J, 0, sizeof J);
    J.d = d;
    J.nbr = nbr;
    J.dH = dH;
    J.D[0] = D_less;
    J.D[1] = D_greater;
    J.G[0] = G_less;
    J.G[1] = G_greater;
    J.W[0] = W_less;
    J.W[1] = W_greater;
    J.c = I * scale;
    pthread_mutex_init(&J.lock, NULL);
    int nt = nthreads < 1 ? 1 : (nthreads > 256 ? 256 : nthreads);
    if (nt > d->NE) nt = d->NE;
    const int nA = d->a_end - d->a_begin, nn = d->Norb * d->Norb;
    const size_t per_dH = (size_t)d->NB * 3 * nn, per_D = (size_t)d->Nqz * d->Nw * d->NB * 9;
    const size_t part = (size_t)nA * (per_dH + 2 * per_D);
    cplx* parts = (cplx*)calloc((size_t)nt * part + 1, sizeof(cplx));
    bwd_part P[256];
    pthread_t th[256];
    if (!parts) {
        pthread_mutex_destroy(&J.lock);
        return ORACLE_NO_MEM;
    }
    for (int i = 0; i < nt; ++i) {
        P[i].J = &J;
        P[i].id = i;
        P[i].nthreads = nt;
        P[i].gdH = parts + (size_t)i * part;
        P[i].gD0 = P[i].gdH + (size_t)nA * per_dH;
        P[i].gD1 = P[i].gD0 + (size_t)nA * per_D;
    }
    int started = 0;
    for (int i = 0; i < nt; ++i) {
        if (pthread_create(&th[i], NULL, bwd_worker, &P[i]) != 0) break;
        ++started;
    }
    for (int i = started; i < nt; ++i) bwd_worker(&P[i]);
    for (int i = 0; i < started; ++i) pthread_join(th[i], NULL);
    /* add the energy chunks in thread order and scatter into the caller's layout */
    for (int a = d->a_begin; a < d->a_end; ++a) {
        const size_t ai = (size_t)(a - d->a_begin);
        for (int s = 0; s < d->NB; ++s)
            for (int e = 0; e < 3 * nn; ++e) {
                cplx acc = 0;
                for (int i = 0; i < nt; ++i) acc += P[i].gdH[ai * per_dH + (size_t)s * 3 * nn + e];
                g_dH[off_dH(d, a, s, 0) + e] = acc;
            }
        for (int q = 0; q < d->Nqz; ++q)
            for (int w = 0; w < d->Nw; ++w)
                for (int s = 0; s < d->NB; ++s)
                    for (int e = 0; e < 9; ++e) {
                        const size_t o = ai * per_D + (((size_t)q * d->Nw + w) * d->NB + s) * 9 + e;
                        cplx a0 = 0, a1 = 0;
                        for (int i = 0; i < nt; ++i) {
                            a0 += P[i].gD0[o];
                            a1 += P[i].gD1[o];
                        }
                        g_D_less[off_D(d, q, w, a, s) + e] = a0;
                        g_D_greater[off_D(d, q, w, a, s) + e] = a1;
                    }
    }
    free(parts);
    pthread_mutex_destroy(&J.lock);
    return J.fail ? ORACLE_NO_MEM : ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* phonon weight combination of Eq. (3)                                 */
/* ------------------------------------------------------------------ */
/*
 * The phonon Green's functions are stored as [Nqz][Nw][NA][NB+1][3][3] (Sec. 2):
 * slot s < NB holds D_ab for b = nbr[a][s], slot NB holds the self block D_aa.
 * The weight of the bond (a, s) in Eq. (3) is D_ba - D_bb - D_aa + D_ab, where
 * D_ba is the block stored by atom b in the slot s' with nbr[b][s'] = a (the
 * neighbour lists must be symmetric). Dc has the layout [Nqz][Nw][NA][NB][3][3].
 * Atoms [a_begin, a_end) are written; returns ORACLE_BAD_ARG if a bond has no
 * reverse slot.
 */
static int reverse_slot(const sse_oracle_dims* d, const int32_t* nbr, int a, int b) {
    for (int s = 0; s < d->NB; ++s)
        if (nbr[(size_t)b * d->NB + s] == a) return s;
    return -1;
}

static size_t off_raw(const sse_oracle_dims* d, int q, int w, int a, int slot) {
    return ((((size_t)q * d->Nw + w) * d->NA + a) * (d->NB + 1) + slot) * 9;
}

int sse_oracle_dcomb(const sse_oracle_dims* d, const int32_t* nbr, const cplx* raw_less, const cplx* raw_greater,
                     cplx* Dc_less, cplx* Dc_greater) {
    if (!check_dims(d) || !nbr || !raw_less || !raw_greater || !Dc_less || !Dc_greater) return ORACLE_BAD_ARG;
    const cplx* raw[2] = {raw_less, raw_greater};
    cplx* out[2] = {Dc_less, Dc_greater};
    for (int a = d->a_begin; a < d->a_end; ++a)
        for (int s = 0; s < d->NB; ++s) {
            const int b = nbr[(size_t)a * d->NB + s];
            if (b < 0 || b >= d->NA) return ORACLE_BAD_ARG;
            const int sr = reverse_slot(d, nbr, a, b);
            if (sr < 0) return ORACLE_BAD_ARG;
            for (int t = 0; t < 2; ++t)
                for (int q = 0; q < d->Nqz; ++q)
                    for (int w = 0; w < d->Nw; ++w) {
                        const cplx* Dba = raw[t] + off_raw(d, q, w, b, sr);
                        const cplx* Dbb = raw[t] + off_raw(d, q, w, b, d->NB);
                        const cplx* Daa = raw[t] + off_raw(d, q, w, a, d->NB);
                        const cplx* Dab = raw[t] + off_raw(d, q, w, a, s);
                        cplx* o = out[t] + off_D(d, q, w, a, s);
                        for (int e = 0; e < 9; ++e) o[e] = Dba[e] - Dbb[e] - Daa[e] + Dab[e];
                    }
        }
    return ORACLE_OK;
}

/*
 * Adjoint of sse_oracle_dcomb: each bond (a, s) adds its weight gradient to the
 * four raw blocks it reads (+D_ba, -D_bb, -D_aa, +D_ab). Every bond of every atom
 * is visited; the raw gradient is written for all atoms.
 */
int sse_oracle_dcomb_adj(const sse_oracle_dims* d, const int32_t* nbr, const cplx* g_less, const cplx* g_greater,
                         cplx* graw_less, cplx* graw_greater) {
    if (!check_dims(d) || !nbr || !g_less || !g_greater || !graw_less || !graw_greater) return ORACLE_BAD_ARG;
    const cplx* g[2] = {g_less, g_greater};
    cplx* out[2] = {graw_less, graw_greater};
    const size_t nraw = (size_t)d->Nqz * d->Nw * d->NA * (d->NB + 1) * 9;
    for (int t = 0; t < 2; ++t) memset(out[t], 0, sizeof(cplx) * nraw);
    for (int a = 0; a < d->NA; ++a)
        for (int s = 0; s < d->NB; ++s) {
            const int b = nbr[(size_t)a * d->NB + s];
            if (b < 0 || b >= d->NA) return ORACLE_BAD_ARG;
            const int sr = reverse_slot(d, nbr, a, b);
            if (sr < 0) return ORACLE_BAD_ARG;
            for (int t = 0; t < 2; ++t)
                for (int q = 0; q < d->Nqz; ++q)
                    for (int w = 0; w < d->Nw; ++w) {
                        const cplx* gi = g[t] + off_D(d, q, w, a, s);
                        cplx* Dba = out[t] + off_raw(d, q, w, b, sr);
                        cplx* Dbb = out[t] + off_raw(d, q, w, b, d->NB);
                        cplx* Daa = out[t] + off_raw(d, q, w, a, d->NB);
                        cplx* Dab = out[t] + off_raw(d, q, w, a, s);
                        for (int e = 0; e < 9; ++e) {
                            Dba[e] += gi[e];
                            Dbb[e] -= gi[e];
                            Daa[e] -= gi[e];
                            Dab[e] += gi[e];
                        }
                    }
        }
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* phonon self-energy, Eq. (4)                                          */
/* ------------------------------------------------------------------ */
/*
 * Pi^t_ab(w, q)_ij = -i*scale * sum_k sum_l sum_E
 *        tr{ dH_i(l,a) . G^t_aa(E + (w+1), (k + q) mod Nkz) . dH_j(a,l) . G^{t'}_ll(E, k) }
 * with the readings used throughout this project:
 *   - t' is the other type (G^< pairs with G^>, Eq. 4's lesser/greater order);
 *   - dH_i(l,a) = dH_i(a,l)^H, dH_j(a,l) = dH[a][slot of l][j];
 *   - off-diagonal block b = nbr[a][s] (slot s < NB): the sum over l has the
 *     single term l = b; diagonal block (slot NB): l runs over the NB
 *     neighbours of a;
 *   - energies with E or E + (w+1) outside [0, NE) contribute zero; kz wraps;
 *   - the integral dE/2pi over the uniform energy grid is the sum over E times
 *     `scale` (= grid step / 2pi).
 * Output Pi^t [Nqz][Nw][NA][NB+1][3][3]. Each trace is evaluated as
 * tr{ (dH_i^H G^t_aa)(dH_j G^{t'}_ll) }, the two half products formed once per
 * (E, k) of the bond (associativity of the matrix product).
 */
typedef struct {
    const sse_oracle_dims* d;
    const int32_t* nbr;
    const cplx* dH;
    const cplx* G[2];
    cplx* acc; /* [2][nA][NB][Nqz][Nw][9] unscaled bond sums */
    long long n_jobs, next;
    pthread_mutex_t lock;
    int fail;
} pi_job;

static size_t off_pi(const sse_oracle_dims* d, int q, int w, int a, int slot) {
    return ((((size_t)q * d->Nw + w) * d->NA + a) * (d->NB + 1) + slot) * 9;
}

/* One bond (t, a, s): acc[q][w][i*3+j] = sum_k sum_E tr{ dH_i^H G^t_a(E+w+1, k+q) dH_j G^{t'}_b(E, k) }. */
static void pi_bond(pi_job* J, int t, int a, int s, cplx* P, cplx* R, cplx* acc) {
    const sse_oracle_dims* d = J->d;
    const int n = d->Norb, nn = n * n;
    const int b = J->nbr[(size_t)a * d->NB + s];
    const cplx* A = J->dH + off_dH(d, a, s, 0);
    /* P[k][E][i] = dH_i^H G^t_a(E, k);  R[k][E][j] = dH_j G^{t'}_b(E, k) */
    for (int k = 0; k < d->Nkz; ++k)
        for (int E = 0; E < d->NE; ++E)
            for (int i = 0; i < 3; ++i) {
                const size_t o = (((size_t)k * d->NE + E) * 3 + i) * nn;
                mm_ah(n, A + (size_t)i * nn, J->G[t] + off_G(d, k, E, a), P + o);
                mm(n, A + (size_t)i * nn, J->G[1 - t] + off_G(d, k, E, b), R + o);
            }
    for (int q = 0; q < d->Nqz; ++q)
        for (int w = 0; w < d->Nw; ++w) {
            cplx* o = acc + ((size_t)q * d->Nw + w) * 9;
            for (int e = 0; e < 9; ++e) o[e] = 0;
            for (int k = 0; k < d->Nkz; ++k) {
                const int kp = (k + q) % d->Nkz; /* kz + qz, periodic */
                for (int E = 0; E < d->NE; ++E) {
                    const int Ep = E + (w + 1);
                    if (Ep >= d->NE) continue; /* out of range: zero */
                    for (int i = 0; i < 3; ++i) {
                        const cplx* Pi = P + (((size_t)kp * d->NE + Ep) * 3 + i) * nn;
                        for (int j = 0; j < 3; ++j) {
                            const cplx* Rj = R + (((size_t)k * d->NE + E) * 3 + j) * nn;
                            cplx tr = 0; /* tr(Pi Rj) */
                            for (int m = 0; m < n; ++m)
                                for (int l = 0; l < n; ++l) tr += Pi[m * n + l] * Rj[l * n + m];
                            o[i * 3 + j] += tr;
                        }
                    }
                }
            }
        }
}

static void* pi_worker(void* arg) {
    pi_job* J = (pi_job*)arg;
    const sse_oracle_dims* d = J->d;
    const size_t half = (size_t)d->Nkz * d->NE * 3 * d->Norb * d->Norb;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * 2 * half);
    if (!buf) {
        pthread_mutex_lock(&J->lock);
        J->fail = 1;
        pthread_mutex_unlock(&J->lock);
        return NULL;
    }
    const int nA = d->a_end - d->a_begin;
    for (;;) {
        pthread_mutex_lock(&J->lock);
        long long o = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (o >= J->n_jobs) break;
        const int s = (int)(o % d->NB);
        const int la = (int)((o / d->NB) % nA);
        const int t = (int)(o / ((long long)d->NB * nA));
        pi_bond(J, t, d->a_begin + la, s, buf, buf + half,
                J->acc + (((size_t)t * nA + la) * d->NB + s) * d->Nqz * d->Nw * 9);
    }
    free(buf);
    return NULL;
}

/*
 * Pi^<, Pi^> of Eq. (4) for atoms [a_begin, a_end): all NB+1 slots, all (qz, w).
 * Blocks of other atoms are untouched. Nqz and Nw are the phonon grid sizes of
 * the output. Host pointers, complex128 interleaved. Returns 0 on success.
 */
int sse_oracle_pi(const sse_oracle_dims* d, const int32_t* nbr, const cplx* dH, const cplx* G_less,
                  const cplx* G_greater, double scale, cplx* P_less, cplx* P_greater, int nthreads) {
    if (!check_dims(d) || !nbr || !dH || !G_less || !G_greater || !P_less || !P_greater) return ORACLE_BAD_ARG;
    for (size_t e = 0; e < (size_t)d->NA * d->NB; ++e)
        if (nbr[e] < 0 || nbr[e] >= d->NA) return ORACLE_BAD_ARG;
    const int nA = d->a_end - d->a_begin;
    const size_t per_bond = (size_t)d->Nqz * d->Nw * 9;
    pi_job J;
    memset(&J, 0, sizeof J);
    J.d = d;
    J.nbr = nbr;
    J.dH = dH;
    J.G[0] = G_less;
    J.G[1] = G_greater;
    J.acc = (cplx*)calloc((size_t)2 * nA * d->NB * per_bond + 1, sizeof(cplx));
    if (!J.acc) return ORACLE_NO_MEM;
    J.n_jobs = 2LL * nA * d->NB;
    pthread_mutex_init(&J.lock, NULL);
    run_threads(pi_worker, &J, nthreads);
    pthread_mutex_destroy(&J.lock);
    if (J.fail) {
        free(J.acc);
        return ORACLE_NO_MEM;
    }
    const cplx c = -I * scale;
    cplx* out[2] = {P_less, P_greater};
    for (int t = 0; t < 2; ++t)
        for (int la = 0; la < nA; ++la)
            for (int q = 0; q < d->Nqz; ++q)
                for (int w = 0; w < d->Nw; ++w) {
                    const int a = d->a_begin + la;
                    cplx self[9] = {0};
                    for (int s = 0; s < d->NB; ++s) {
                        const cplx* v = J.acc + ((((size_t)t * nA + la) * d->NB + s) * per_bond) +
                                        ((size_t)q * d->Nw + w) * 9;
                        cplx* o = out[t] + off_pi(d, q, w, a, s);
                        for (int e = 0; e < 9; ++e) {
                            o[e] = c * v[e];  /* l = b */
                            self[e] += v[e];  /* diagonal block: sum over all neighbours l */
                        }
                    }
                    cplx* o = out[t] + off_pi(d, q, w, a, d->NB);
                    for (int e = 0; e < 9; ++e) o[e] = c * self[e];
                }
    free(J.acc);
    return ORACLE_OK;
}

/* ------------------------------------------------------------------ */
/* gradient with respect to G (adjoint of Eq. 3 in its G argument)      */
/* ------------------------------------------------------------------ */
/*
 * For L = sum_t sum_{a in range, E, k} Re tr( W^t_a(E,k)^H Sigma^t_a(E,k) ) each term
 * c * Dc_ij * dH_i G dH_j^H of Eq. (3) gives grad G = conj(c * Dc_ij) dH_i^H W dH_j, so
 *   grad G^t_b(E', k') = sum over bonds (a, s) with nbr[a][s] = b, a in range, and over (q, w, sigma)
 *                        with E = E' + sigma*(w+1) in [0, NE), k = (k' + q) mod Nkz:
 *                        sum_ij conj(c * Dc^{tau(t,sigma)}_ij(q,w,a,s)) dH_i(a,s)^H W^t_a(E,k) dH_j(a,s).
 * Written for every atom b (atoms that no bond in range reaches get zero).
 */
typedef struct {
    const sse_oracle_dims* d;
    const int32_t* nbr;
    const cplx* dH;
    const cplx* D[2];
    const cplx* W[2];
    cplx* gG[2];
    cplx c;
    long long n_out, next;
    pthread_mutex_t lock;
    int fail;
} bwdg_job;

static void bwdg_one(bwdg_job* J, int t, int b, int Ep, int kp, cplx* P, cplx* Q, cplx* acc) {
    const sse_oracle_dims* d = J->d;
    const int n = d->Norb, nn = n * n;
    memset(acc, 0, sizeof(cplx) * nn);
    for (int a = d->a_begin; a < d->a_end; ++a)
        for (int s = 0; s < d->NB; ++s) {
            if (J->nbr[(size_t)a * d->NB + s] != b) continue;
            for (int q = 0; q < d->Nqz; ++q) {
                const int k = (kp + q) % d->Nkz; /* kz - qz = k' */
                for (int w = 0; w < d->Nw; ++w)
                    for (int sg = 0; sg < 2; ++sg) {
                        const int sigma = sg == 0 ? +1 : -1;
                        const int E = Ep + sigma * (w + 1);
                        if (E < 0 || E >= d->NE) continue;
                        const int tau = sigma == +1 ? t : 1 - t;
                        const cplx* Wa = J->W[t] + off_G(d, k, E, a);
                        const cplx* Dc = J->D[tau] + off_D(d, q, w, a, s);
                        for (int i = 0; i < 3; ++i) {
                            mm_ah(n, J->dH + off_dH(d, a, s, i), Wa, P); /* dH_i^H W */
                            for (int j = 0; j < 3; ++j) {
                                mm(n, P, J->dH + off_dH(d, a, s, j), Q); /* ... dH_j */
                                const cplx f = conj(J->c * Dc[i * 3 + j]);
                                for (int e = 0; e < nn; ++e) acc[e] += f * Q[e];
                            }
                        }
                    }
            }
        }
    cplx* out = J->gG[t] + off_G(d, kp, Ep, b);
    for (int e = 0; e < nn; ++e) out[e] = acc[e];
}

static void* bwdg_worker(void* arg) {
    bwdg_job* J = (bwdg_job*)arg;
    const sse_oracle_dims* d = J->d;
    const int nn = d->Norb * d->Norb;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * nn * 3);
    if (!buf) {
        pthread_mutex_lock(&J->lock);
        J->fail = 1;
        pthread_mutex_unlock(&J->lock);
        return NULL;
    }
    for (;;) {
        pthread_mutex_lock(&J->lock);
        long long o = J->next++;
        pthread_mutex_unlock(&J->lock);
        if (o >= J->n_out) break;
        const int kp = (int)(o % d->Nkz);
        long long r = o / d->Nkz;
        const int Ep = (int)(r % d->NE);
        r /= d->NE;
        const int b = (int)(r % d->NA);
        const int t = (int)(r / d->NA);
        bwdg_one(J, t, b, Ep, kp, buf, buf + nn, buf + 2 * nn);
    }
    free(buf);
    return NULL;
}

/* grad G^<, grad G^> (layout of G, every atom overwritten) of the loss above. */
int sse_oracle_bwd_g(const sse_oracle_dims* d, const int32_t* nbr, const cplx* dH, const cplx* D_less,
                     const cplx* D_greater, double scale, const cplx* W_less, const cplx* W_greater, cplx* gG_less,
                     cplx* gG_greater, int nthreads) {
    if (!check_dims(d) || !nbr || !dH || !D_less || !D_greater || !W_less || !W_greater || !gG_less || !gG_greater)
        return ORACLE_BAD_ARG;
    for (size_t e = 0; e < (size_t)d->NA * d->NB; ++e)
        if (nbr[e] < 0 || nbr[e] >= d->NA) return ORACLE_BAD_ARG;
    bwdg_job J;
    memset(&J, 0, sizeof J);
    J.d = d;
    J.nbr = nbr;
    J.dH = dH;
    J.D[0] = D_less;
    J.D[1] = D_greater;
    J.W[0] = W_less;
    J.W[1] = W_greater;
    J.gG[0] = gG_less;
    J.gG[1] = gG_greater;
    J.c = I * scale;
    J.n_out = 2LL * d->NA * d->NE * d->Nkz;
    pthread_mutex_init(&J.lock, NULL);
    run_threads(bwdg_worker, &J, nthreads);
    pthread_mutex_destroy(&J.lock);
    return J.fail ? ORACLE_NO_MEM : ORACLE_OK;
}
