/*
 * sse.h -- C ABI of the GB300 (sm_103a) scattering self-energy library.
 *
 * The library evaluates the electron-phonon scattering self-energies
 * Sigma^<, Sigma^> of Eq. (3) and Pi^<, Pi^> of Eq. (4) of Ziogas et al.,
 * "A Data-Centric Approach to
 * Extreme-Scale Ab initio Dissipative Quantum Transport Simulations"
 * (SC'19, Sec. 2), and the adjoint of that map.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Complex numbers are complex128: two consecutive doubles (re, im), the
 * layout of C99 `double complex`, std::complex<double> and torch.complex128.
 * All tensors are dense, C-contiguous (row-major), in DEVICE memory of the
 * current CUDA device unless stated otherwise:
 *
 *   nbr   int32      [NA][NB]                    neighbour b = nbr[a][s] of atom a
 *   dH    complex128 [NA][NB][3][Norb][Norb]     grad_i H_ab for b = nbr[a][s]
 *                                                (grad_j H_ba is its conjugate transpose)
 *   D^t   complex128 [Nqz][Nw][NA][NB][3][3]     phonon weight of the bond (a,s) at
 *                                                momentum qz and frequency w: the
 *                                                combination D_ba - D_bb - D_aa + D_ab
 *                                                of Eq. (3), t in {<, >}
 *   G^t   complex128 [Nkz][NE][NA][Norb][Norb]   diagonal blocks G^t_bb(E, kz)
 *   S^t   complex128 [Nkz][NE][NA][Norb][Norb]   diagonal blocks Sigma^t_aa(E, kz)
 *
 * Eq. (3) as evaluated (readings of the printed formula):
 *   Sigma^t_aa(E,k) = i*scale * sum_{q<Nqz} sum_{s<NB} sum_{w<Nw} sum_{sigma=+-1} sum_{i,j<3}
 *        dH_i(a,s) G^t_bb(E - sigma*(w+1), (k-q) mod Nkz) dH_j(a,s)^H  D^{tau}_ij(q,w,a,s)
 *   with b = nbr[a][s], tau = t for sigma = +1 (emission) and the other type
 *   for sigma = -1 (absorption). Energies outside [0, NE) contribute zero;
 *   kz is periodic. `scale` is the frequency-integration weight
 *   (grid step / 2 pi; 1/(2 pi) with energies in units of the grid step).
 *
 * Every entry point is asynchronous on `stream` (a cudaStream_t; NULL = the
 * legacy default stream), validates its arguments on the host before
 * launching anything, and returns an sse_status. No entry point throws,
 * exits, prints, allocates device memory or frees caller memory: the caller
 * owns every buffer, including the workspace. The caller keeps all buffers
 * alive until the work queued on `stream` has finished. Calls that share a
 * workspace must be ordered on one stream.
 */
#ifndef SSE_H
#define SSE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SSE_API __attribute__((visibility("default")))
#else
#define SSE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Problem sizes. Atoms [a_begin, a_end) are computed; [0, NA) = all. */
typedef struct sse_dims {
    int32_t NA, NB, Norb, NE, Nkz, Nqz, Nw;
    int32_t a_begin, a_end;
} sse_dims;

/* Arithmetic of the contraction.
 *   FP64   : IEEE double throughout (CUDA-core DFMA).
 *   TF32   : G and the frequency weights rounded to TF32 split-complex planes,
 *            products on the tcgen05 tensor cores with FP32 accumulation over
 *            one qz slice, FP64 sums over qz, neighbours and the final
 *            multiply by dH (Sec. 4.4 adapted to TF32).
 *   BF16X3 : like TF32 but each operand split into bf16 hi + lo parts and the
 *            three products hi*hi + hi*lo + lo*hi accumulated in FP32.
 *            TF32 and BF16X3 need Norb <= 10 and a weight table of 2 Nw taps
 *            per qz in shared memory: Nw <= 286 (TF32) or 194 (BF16X3) at
 *            Norb = 10, more for smaller blocks. sse_sigma_fwd only; beyond
 *            these limits the host checks return SSE_ERR_UNSUPPORTED.
 *   FP64_FFT : IEEE double throughout, evaluated with the convolution theorem:
 *            Eq. (3) is, per bond, a convolution of G^t_b with the phonon
 *            weights over (E, kz) -- cyclic in kz, linear in E -- so G is
 *            transformed (zero-padded in E to L >= NE + Nw, L = 2^a 3^b),
 *            each frequency needs 6 Norb x Norb block products per bond, and
 *            the result is transformed back. Same values as FP64 up to the
 *            rounding of the transforms (normwise ~1e-15), far fewer flops;
 *            workspace Nkz*L*(NA + 2*nA)*Norb^2*16 + Nkz*L*nA*NB*9*16 bytes
 *            (nA = a_end - a_begin). Size limits, the same for FP32_FFT and for
 *            every entry point that runs transforms: Nkz <= 16, L <= 4608
 *            (NE + Nw <= 4608), NB <= 16, and for the widest blocks
 *            NB <= 14, 12, 10 at Norb = 14, 15, 16 (sse_pi_fwd: NB <= 15, 12,
 *            10, 9, 7 at Norb = 12 .. 16). Beyond them the host checks return
 *            SSE_ERR_UNSUPPORTED before any device work.
 *   FP32_FFT : the same transforms and per-frequency block products in FP32 on the
 *            CUDA cores' FP32 pipe (about 60x the FP64 pipe on GB300), FP64 inputs
 *            and outputs; for sse_sigma_fwd, sse_sigma_bwd, sse_sigma_bwd_g and
 *            sse_pi_fwd. Spectra take half of FP64_FFT's workspace. Error (normwise)
 *            a few 1e-7, tested to 2e-6; the adjoint's dH gradient, a sum over
 *            Nkz*L frequencies, to 1e-5.
 *   F16X3_FFT : the FP32 transforms of FP32_FFT with the per-frequency block products on
 *            the tcgen05 tensor cores (Sec. 4.4: split-complex FP16 operands with
 *            power-of-two normalisation, wider accumulation). Frequencies stack into the
 *            rows of two GEMMs per bond whose second operand, dH, is shared by every
 *            frequency; each operand is scaled by a power of two and split into FP16
 *            hi + lo, and hi*hi + hi*lo + lo*hi accumulate in FP32. Error (normwise)
 *            a few 1e-7, tested to 2e-6. sse_sigma_fwd and sse_sigma_fwd_host only;
 *            FP32_FFT's workspace; needs Norb <= 10 and NB <= 4 besides the transform
 *            limits (else SSE_ERR_UNSUPPORTED before any device work). */
typedef enum sse_mode {
    SSE_MODE_FP64 = 0,
    SSE_MODE_TF32 = 1,
    SSE_MODE_BF16X3 = 2,
    SSE_MODE_FP64_FFT = 3,
    SSE_MODE_FP32_FFT = 4,
    SSE_MODE_F16X3_FFT = 5
} sse_mode;

/* SYMMETRIZE: replace each output block S by (S - S^H)/2 in FP64 before the
 *             store (exact Sigma is anti-Hermitian when G and D are; this
 *             removes round-off asymmetry). In the adjoint it projects the
 *             upstream gradient the same way.
 * CHECK     : after the launches, synchronise `stream` and report device-side
 *             input checks (neighbour indices outside [0, NA)) as
 *             SSE_ERR_DEVICE_CHECK. Without CHECK such entries contribute zero
 *             and the call stays asynchronous. With ANTIHERMITIAN it also reports
 *             input blocks that are not anti-Hermitian.
 * PROFILE   : record a pair of CUDA events on `stream` around every kernel the
 *             call launches (no synchronisation, no effect on the results);
 *             sse_profile_read reports the device time per kernel.
 * ANTIHERMITIAN : the caller states that every Norb x Norb block of G^< and G^>
 *             (and, for sse_sigma_fwd, every 3x3 block of D^< and D^>) is exactly
 *             anti-Hermitian, as lesser and greater Green's functions are. The
 *             FP64_FFT forward and sse_pi_fwd then compute one frequency of each
 *             pair (f, -f) and obtain the other from Sigma^(-f) = -Sigma^(f)^H,
 *             C^(-f) = C^(f)^H (half the block products). With CHECK the inputs are
 *             verified bit for bit and a violation is reported as
 *             SSE_ERR_DEVICE_CHECK; without it the results for inputs that are not
 *             anti-Hermitian are unspecified. Ignored by the other modes and entries. */
enum {
    SSE_FLAG_SYMMETRIZE = 1u << 0,
    SSE_FLAG_CHECK = 1u << 1,
    SSE_FLAG_PROFILE = 1u << 2,
    SSE_FLAG_ANTIHERMITIAN = 1u << 3
};

typedef enum sse_status {
    SSE_OK = 0,
    SSE_ERR_INVALID_ARG = 1,  /* null/misaligned pointer, bad size or range     */
    SSE_ERR_UNSUPPORTED = 2,  /* valid but unsupported mode, flag or size       */
    SSE_ERR_CUDA = 3,         /* a CUDA runtime call or launch failed           */
    SSE_ERR_TIMEOUT = 4,      /* a bounded device wait gave up                  */
    SSE_ERR_DEVICE_CHECK = 5, /* device-side input check failed (with CHECK)    */
    SSE_ERR_WORKSPACE = 6     /* workspace missing, misaligned or too small     */
} sse_status;

/* Bytes of device workspace that sse_sigma_fwd and sse_sigma_bwd need for
 * these sizes, mode and flags (the larger of the two). Returns 0 if the
 * arguments are invalid. The workspace must be 256-byte aligned. */
SSE_API size_t sse_workspace_bytes(const sse_dims* d, int mode, uint32_t flags);

/* Sigma^< and Sigma^> of Eq. (3) (Sec. 2) for atoms [a_begin, a_end).
 * Inputs as in the header comment; S_less / S_greater are fully overwritten
 * for atoms in range (all E, kz) and untouched elsewhere.
 * Host checks: non-null, 16-byte aligned complex arrays (4-byte nbr),
 * NA,NB,NE,Nkz,Nqz,Nw >= 1, 1 <= Norb <= 16, Nqz <= Nkz, Nw < NE,
 * 0 <= a_begin <= a_end <= NA, NA <= 32767, finite scale, known mode and flags;
 * in modes TF32, BF16X3, FP64_FFT and FP32_FFT also the size limits stated with the modes. */
SSE_API int sse_sigma_fwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                  const double* D_greater, const double* G_less, const double* G_greater, double scale, int mode,
                  uint32_t flags, double* S_less, double* S_greater, void* workspace, size_t ws_bytes,
                  void* stream);

/* sse_sigma_fwd with every array in HOST memory (page-locked for asynchronous copies):
 * the call copies nbr, dH, D^<, D^>, G^< and G^> into `device_buf` on `copy_stream`,
 * computes on `stream` and copies S^<, S^> (rows of atoms [a_begin, a_end) only) back on
 * `copy_stream`, G and Sigma one kz slice at a time. With modes FP64_FFT and FP32_FFT the
 * lag kernels are transformed while G^< arrives, each kz slice of G is transformed as soon as
 * it is on the device, the upload of G^> overlaps the computation of Sigma^<, and each slice
 * of Sigma is downloaded as soon as its inverse transform has written it; other modes start
 * after the last upload. `device_buf`: caller-owned device memory of
 * sse_sigma_fwd_host_bytes() (256-byte aligned; inputs, outputs and workspace). `stream` and
 * `copy_stream` must differ; all work is ordered after earlier work on `stream`, and `stream`
 * observes the completion of the copies (synchronise it before reading S_less / S_greater).
 * Same checks, flags and status codes as sse_sigma_fwd. */
SSE_API size_t sse_sigma_fwd_host_bytes(const sse_dims* d, int mode, uint32_t flags);
SSE_API int sse_sigma_fwd_host(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                               const double* D_greater, const double* G_less, const double* G_greater, double scale,
                               int mode, uint32_t flags, double* S_less, double* S_greater, void* device_buf,
                               size_t buf_bytes, void* stream, void* copy_stream);

/* Adjoint of sse_sigma_fwd: mode FP64 runs direct FP64 kernels (correlations
 * recomputed from the gathered G windows), mode FP64_FFT the transform-based adjoint
 * in FP64 (per bond and frequency Q_j = W^ dH_j G^^H and R_i = W^^H dH_i G^, the weight
 * gradient from the inverse transform of tr(dH_i^H Q_j), the coupling gradient
 * summed over frequencies in a fixed order), mode FP32_FFT the same steps with FP32
 * transforms and block products, the coupling-gradient partial sums and all inputs and
 * outputs in FP64 (normwise error about 1e-6, bound 1e-5 at the workloads tested);
 * TF32, BF16X3 and F16X3_FFT return SSE_ERR_UNSUPPORTED (after an F16X3_FFT forward,
 * take the FP32_FFT adjoint).
 * For the loss
 *   L = sum_t sum_{a in range, E, k} Re tr( gS^t_a(E,k)^H Sigma^t_a(E,k) )
 * it writes the gradients w.r.t. dH, D^< and D^> in the PyTorch convention
 * for complex tensors (grad z = dL/dRe z + i dL/dIm z):
 *   g_D^tau_ij(q,w,a,s) = sum over (t,sigma) with type tau and (E,k) in range of
 *                         conj( i*scale * tr(gS^H dH_i G dH_j^H) )
 *   g_dH_m(a,s)         = sum_{t,E,k,q,w,sigma} sum_j conj(i*scale*D_mj) gS dH_j G^H
 *                                              + sum_i i*scale*D_im gS^H dH_i G
 * gS_less / gS_greater have the layout of S^t. Gradient blocks of atoms in
 * [a_begin, a_end) are fully overwritten; others are untouched. The gradient with respect
 * to G is sse_sigma_bwd_g's. The gathered G tiles are recomputed, not stored. */
SSE_API int sse_sigma_bwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                  const double* D_greater, const double* G_less, const double* G_greater, double scale, int mode,
                  uint32_t flags, const double* gS_less, const double* gS_greater, double* g_dH, double* g_D_less,
                  double* g_D_greater, void* workspace, size_t ws_bytes, void* stream);

/* Gradient of the same loss as sse_sigma_bwd with respect to G^<, G^> (Sigma is linear in
 * G, so G itself is not an argument):
 *   g_G^t_b(E', k') = sum over bonds (a, s) with nbr[a][s] = b and a in [a_begin, a_end),
 *                     over (q, w, sigma) with E = E' + sigma*(w+1) in [0, NE), k = (k'+q) mod Nkz:
 *                     sum_ij conj(i*scale * D^tau_ij(q,w,a,s)) dH_i(a,s)^H gS^t_a(E,k) dH_j(a,s).
 * g_G_less / g_G_greater have the layout of G and are fully overwritten for every atom (zero where
 * no bond in range reaches). Through the transforms, in FP64 (modes FP64 and FP64_FFT) or with FP32
 * transforms and block products (mode FP32_FFT; FP64 inputs and outputs); TF32, BF16X3 and
 * F16X3_FFT return SSE_ERR_UNSUPPORTED. Per atom and frequency, the bonds into it in (a, s) order from a list built on
 * the device (deterministic sums).
 * SYMMETRIZE projects gS as in sse_sigma_bwd. Workspace: sse_sigma_bwd_g_workspace_bytes(). */
SSE_API size_t sse_sigma_bwd_g_workspace_bytes(const sse_dims* d, int mode, uint32_t flags);
SSE_API int sse_sigma_bwd_g(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                            const double* D_greater, double scale, int mode, uint32_t flags, const double* gS_less,
                            const double* gS_greater, double* g_G_less, double* g_G_greater, void* workspace,
                            size_t ws_bytes, void* stream);

/* Phonon scattering self-energy Pi^<, Pi^> of Eq. (4) (Sec. 2) for atoms [a_begin, a_end):
 *   P^t complex128 [Nqz][Nw][NA][NB+1][3][3]: slot s < NB is the block Pi^t_ab for
 *        b = nbr[a][s], slot NB the diagonal block Pi^t_aa; indices (i, j) of the
 *        3x3 block are the displacement directions.
 *   Pi^t_{a,s}(q, w)_ij = -i*scale * sum_{k<Nkz} sum_E
 *        tr( dH_i(a,s)^H G^t_aa(E+(w+1), (k+q) mod Nkz) dH_j(a,s) G^t'_bb(E, k) ),
 *   t' the other type; energies with E or E+(w+1) outside [0, NE) contribute zero;
 *   the diagonal block sums the NB bond terms (the sum over l of Eq. (4); an
 *   off-diagonal block keeps l = b). `scale` is the energy-integration weight.
 * Modes FP64 and FP64_FFT evaluate it with the convolution theorem in FP64 (per
 * frequency 6 block products and 9 traces per bond, then one inverse transform per
 * (bond, i, j)); mode FP32_FFT takes the same steps with FP32 transforms and block
 * products (FP64 inputs and outputs; normwise error a few 1e-7); TF32, BF16X3 and
 * F16X3_FFT return SSE_ERR_UNSUPPORTED.
 * Flags: SYMMETRIZE replaces each 3x3 block B by (B - B^H)/2; CHECK, PROFILE as above.
 * Rows of other atoms are untouched. Workspace: sse_pi_workspace_bytes(). */
SSE_API size_t sse_pi_workspace_bytes(const sse_dims* d, int mode, uint32_t flags);
SSE_API int sse_pi_fwd(const sse_dims* d, const int32_t* nbr, const double* dH, const double* G_less,
                       const double* G_greater, double scale, int mode, uint32_t flags, double* P_less,
                       double* P_greater, void* workspace, size_t ws_bytes, void* stream);

/* Bond weights of Eq. (3) (Sec. 2) from the raw phonon Green's functions.
 *   Draw^t complex128 [Nqz][Nw][NA][NB+1][3][3]: slot s < NB holds D_ab for b = nbr[a][s],
 *                                                slot NB holds the self block D_aa.
 *   D^t    complex128 [Nqz][Nw][NA][NB][3][3]:   D^t(a,s) = D_ba - D_bb - D_aa + D_ab,
 * where D_ba is the block atom b stores in the slot s' with nbr[b][s'] = a: the
 * neighbour lists must be symmetric. Rows of atoms [a_begin, a_end) are written
 * (NE, Nkz and Norb are not used; they must still pass the checks of sse_dims).
 * A bond without a reverse slot, or with a neighbour outside [0, NA), gets a zero
 * weight; with SSE_FLAG_CHECK it is reported as SSE_ERR_DEVICE_CHECK. Workspace:
 * at least 256 bytes (256-byte aligned) for the status word. Asynchronous on stream. */
SSE_API int sse_dcomb_fwd(const sse_dims* d, const int32_t* nbr, const double* Draw_less, const double* Draw_greater,
                          double* D_less, double* D_greater, uint32_t flags, void* workspace, size_t ws_bytes,
                          void* stream);

/* Adjoint of sse_dcomb_fwd: from the gradients gD^t w.r.t. the bond weights (read for
 * every atom) it writes the gradients gDraw^t w.r.t. the raw blocks of atoms
 * [a_begin, a_end): slot s < NB gets gD(a,s) + gD(b,s'), slot NB gets minus the sum of
 * those over a's bonds. Same checks, workspace and status as sse_dcomb_fwd. */
SSE_API int sse_dcomb_bwd(const sse_dims* d, const int32_t* nbr, const double* gD_less, const double* gD_greater,
                          double* gDraw_less, double* gDraw_greater, uint32_t flags, void* workspace,
                          size_t ws_bytes, void* stream);

/* Size of the library's static device scratch array used by sse_sigma_bwd_static. */
#define SSE_STATIC_SCRATCH_BYTES ((size_t)64 << 20)

/* sse_sigma_bwd_static -- sse_sigma_bwd for callers that cannot allocate device memory.
 * (The paper has no counterpart: this is an interface convenience.)
 * Callers such as a host application whose device memory belongs to its own allocator
 * or pool, code that must not allocate on its hot path, or a foreign-language host that
 * only passes through pointers it was given cannot call cudaMalloc to create the
 * workspace sse_sigma_bwd needs. This entry point takes the same inputs and outputs
 * (and writes the same gradients, FP64 mode only) but no workspace: its scratch (status
 * word and per-bond partial gradients) lives in one static device array of
 * SSE_STATIC_SCRATCH_BYTES that the library holds on every GPU that loads it, until the
 * process exits. It calls no allocation routine.
 * - Sizes whose sse_workspace_bytes(d, SSE_MODE_FP64, flags) exceeds
 *   SSE_STATIC_SCRATCH_BYTES are rejected with SSE_ERR_WORKSPACE before any device work
 *   (the array holds e.g. NA*NB*Nkz*6*Norb^2*16 bytes of partials + 256: NA=256, NB=4,
 *   Norb=10, Nkz=5 fits; NA=1024, Nkz=7 does not).
 * - Argument checks and status codes are those of sse_sigma_bwd: a valid mode other than
 *   SSE_MODE_FP64, or sizes the kernels are not built for, give SSE_ERR_UNSUPPORTED.
 * - Every call looks up the array's device address on the current device (a host-side
 *   query), so a device reset between calls is harmless. The first call on a device may
 *   load the library's device code there: make it before any stream capture.
 * - SSE_FLAG_PROFILE records kernel times as in sse_sigma_bwd.
 * - All calls share the one array and it keeps the last call's contents; the status
 *   word is cleared by each call. Calls that overlap on the GPU (different streams,
 *   different host threads) race on the array: order them on one stream. */
SSE_API int sse_sigma_bwd_static(const sse_dims* d, const int32_t* nbr, const double* dH, const double* D_less,
                                 const double* D_greater, const double* G_less, const double* G_greater,
                                 double scale, int mode, uint32_t flags, const double* gS_less,
                                 const double* gS_greater, double* g_dH, double* g_D_less, double* g_D_greater,
                                 void* stream);

/* Test hook of the bounded device waits (the paper has no counterpart). The next
 * sse_sigma_fwd call in mode TF32 or BF16X3 (and only that call) issues none of the
 * shared-memory window loads of work item `item` of its first energy window -- a
 * work item is (128-row energy tile, kz, type, atom), tile fastest, so item 0 is the first
 * tile of atom a_begin -- and bounds each pipeline wait by `wait_polls` mbarrier polls.
 * The waits that depend on the withheld loads run out, the kernel stops issuing work,
 * still waits (with the full limit) for the loads and matrix products it did issue,
 * and the call reports SSE_ERR_TIMEOUT when made with SSE_FLAG_CHECK. No device fault is
 * involved; the outputs of that call are unspecified and later calls are unaffected.
 * item < 0 disarms the hook. Returns SSE_ERR_INVALID_ARG for item >= 0 with
 * wait_polls = 0, else SSE_OK. Host memory only; not meant for concurrent use. */
SSE_API int sse_test_withhold_window(int item, uint32_t wait_polls);

/* Device time of one kernel over the calls recorded with SSE_FLAG_PROFILE. */
typedef struct sse_profile_entry {
    const char* name; /* static string, e.g. "sigma_fp64_fwd_kernel"      */
    double ms;        /* summed device time of its launches, milliseconds  */
    int32_t launches; /* number of launches recorded                       */
} sse_profile_entry;

/* Kernel times recorded (by any host thread of this process) since the previous
 * call: waits for the recorded events, writes up to `max` entries to `out` (one per
 * kernel name, in first-launch order; `out` may be NULL with max = 0), clears the
 * records and returns the number of kernel names, or -1 if a CUDA event query
 * failed (the records are cleared all the same). At most 65536 launches are kept
 * between reads; later ones are not recorded. Host memory only. */
SSE_API int sse_profile_read(sse_profile_entry* out, int max);

/* Static, NUL-terminated description of a status code (never NULL). */
SSE_API const char* sse_strerror(int status);

#ifdef __cplusplus
}
#endif

#endif /* SSE_H */
