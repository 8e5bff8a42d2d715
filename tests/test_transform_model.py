"""The transform (convolution-theorem) evaluation of Eqs. (3) and (4), written out with numpy FFTs on the CPU and
compared with the FP64 oracle: the algebra behind the FP64_FFT / FP32_FFT modes, independent of the CUDA kernels.

Eq. (3) per bond (a, s), b = nbr[a][s]: Sigma^t_a(E,k) = c sum_ij sum_{q,l} K_ij(q,l) dH_i G^t_b(E-l, k-q) dH_j^H with
the lag kernel K(q, +(w+1)) = D^t(q,w), K(q, -(w+1)) = D^t'(q,w) and c = i*scale. G is zero outside [0, NE) in E and
cyclic in kz, so with G zero-padded to L >= NE + Nw the linear convolution along E equals the cyclic one of period L
on [0, NE); after 2-D DFTs over (kz, E) the convolution is a product per frequency.

Eq. (4): Pi^t_{a,s}(q,w)_ij = -i*scale sum_{k,E} tr(dH_i^H G^t_a(E+l, k+q) dH_j G^t'_b(E, k)), l = w+1, a
cross-correlation: C_ij(q,l) = IDFT[tr(dH_i^H G^_a(f) dH_j G^_b(-f))](q,l); the diagonal slot sums the bonds.

The adjoint of Eq. (3) (gradients with respect to dH, D^< and D^>) and the gradient with respect to G are
correlations of the upstream gradient with G and with the lag kernel, modelled the same way.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1912_10024_gb300.inputs import TINY, Dims, make_inputs, ring_neighbours

SCALE = 1.0 / (2.0 * math.pi)


def smallest_2a3b(n):
    while True:
        m = n
        for p in (2, 3):
            while m % p == 0:
                m //= p
        if m == 1:
            return n
        n += 1


def sigma_by_transforms(nbr, dH, Dl, Dg, Gl, Gg, scale, dt=np.complex128):
    """dt: the complex type of the transforms and products (complex64 models the FP32_FFT arithmetic)."""
    Nkz, NE, NA, Norb, _ = Gl.shape
    Nqz, Nw = Dl.shape[0], Dl.shape[1]
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)
    out = []
    for G, Dt, Dtb in ((Gl, Dl, Dg), (Gg, Dg, Dl)):
        Gp = np.zeros((Nkz, L, NA, Norb, Norb), dt)
        Gp[:, :NE] = G
        Gh = np.fft.fft2(Gp, axes=(0, 1))                        # [kappa][eps][atom]
        K = np.zeros((Nkz, L, NA, NB, 3, 3), dt)                 # lag kernel, q padded to Nkz
        for w in range(Nw):
            K[:Nqz, w + 1] = Dt[:, w]                             # emission: G at E - (w+1), same type
            K[:Nqz, L - (w + 1)] = Dtb[:, w]                      # absorption: G at E + (w+1), other type
        Kh = np.fft.fft2(K, axes=(0, 1))
        Sh = np.zeros((Nkz, L, NA, Norb, Norb), dt)
        for a in range(NA):
            for s in range(NB):
                b = nbr[a, s]
                A = dH[a, s].astype(dt)                           # [3][Norb][Norb]
                for i in range(3):
                    for j in range(3):
                        prod = A[i] @ Gh[:, :, b] @ A[j].conj().T  # per frequency, broadcast over (kappa, eps)
                        Sh[:, :, a] += Kh[:, :, a, s, i, j][..., None, None] * prod
        S = np.fft.ifft2(Sh, axes=(0, 1))[:, :NE].astype(np.complex128)
        out.append(1j * scale * S)
    return out


def pi_by_transforms(nbr, dH, Gl, Gg, scale, Nqz, Nw):
    Nkz, NE, NA, Norb, _ = Gl.shape
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)
    spec = []
    for G in (Gl, Gg):
        Gp = np.zeros((Nkz, L, NA, Norb, Norb), complex)
        Gp[:, :NE] = G
        spec.append(np.fft.fft2(Gp, axes=(0, 1)))
    neg_k = (-np.arange(Nkz)) % Nkz
    neg_e = (-np.arange(L)) % L
    out = []
    for t in range(2):
        X, Y = spec[t], spec[1 - t]                               # G^t of atom a, G^t' of the neighbour
        P = np.zeros((Nqz, Nw, NA, NB + 1, 3, 3), complex)
        for a in range(NA):
            diag = np.zeros((Nkz, L, 3, 3), complex)
            for s in range(NB):
                b = nbr[a, s]
                A = dH[a, s]
                Yneg = Y[neg_k][:, neg_e, b]                      # G^_b(-f)
                Ch = np.zeros((Nkz, L, 3, 3), complex)
                for i in range(3):
                    for j in range(3):
                        Ch[..., i, j] = np.trace(A[i].conj().T @ X[:, :, a] @ A[j] @ Yneg, axis1=-2, axis2=-1)
                diag += Ch
                C = np.fft.ifft2(Ch, axes=(0, 1))                 # C(q, l), positive exponent, 1/(Nkz L)
                P[:, :, a, s] = -1j * scale * C[:Nqz, 1:Nw + 1]
            C = np.fft.ifft2(diag, axes=(0, 1))
            P[:, :, a, NB] = -1j * scale * C[:Nqz, 1:Nw + 1]
        out.append(P)
    return out


CASES = [TINY, Dims(NA=5, NB=2, Norb=3, NE=13, Nkz=4, Nqz=3, Nw=4), Dims(NA=4, NB=1, Norb=2, NE=9, Nkz=1, Nqz=1, Nw=3)]


@pytest.mark.parametrize("d", CASES, ids=lambda d: f"NE{d.NE}_Nkz{d.Nkz}_Nqz{d.Nqz}")
def test_sigma_transform_model_equals_the_oracle(d):
    nbr = None if d is TINY else ring_neighbours(d.NA, d.NB)
    x = make_inputs(d, seed=d.NE + 3, nbr=nbr)
    arrs = [t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater)]
    got = sigma_by_transforms(*arrs, SCALE)
    ref = oracle.sigma(*arrs, SCALE)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("d", CASES, ids=lambda d: f"NE{d.NE}_Nkz{d.Nkz}_Nqz{d.Nqz}")
def test_pi_transform_model_equals_the_oracle(d):
    nbr = None if d is TINY else ring_neighbours(d.NA, d.NB)
    x = make_inputs(d, seed=d.NE + 4, nbr=nbr)
    nb, dH, Gl, Gg = (t.numpy() for t in (x.nbr, x.dH, x.G_less, x.G_greater))
    got = pi_by_transforms(nb, dH, Gl, Gg, SCALE, d.Nqz, d.Nw)
    ref = oracle.pi(nb, dH, Gl, Gg, SCALE, d.Nqz, d.Nw)
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def test_padding_below_ne_plus_nw_aliases():
    """The bound L >= NE + Nw is needed: with L = NE the cyclic wrap of the lags brings energies from the other end
    of the grid into the sum, and the transform result no longer equals Eq. (3)."""
    d = Dims(NA=4, NB=1, Norb=2, NE=9, Nkz=1, Nqz=1, Nw=3)
    x = make_inputs(d, seed=11, nbr=ring_neighbours(4, 1))
    arrs = [t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater)]
    ref = oracle.sigma(*arrs, SCALE)
    global smallest_2a3b
    keep = smallest_2a3b
    try:
        smallest_2a3b = lambda n: d.NE  # noqa: E731  (too short on purpose)
        bad = sigma_by_transforms(*arrs, SCALE)
    finally:
        smallest_2a3b = keep
    assert np.abs(bad[0] - ref[0]).max() > 1e-3 * np.abs(ref[0]).max()


def sigma_grad_by_transforms(nbr, dH, Dl, Dg, Gl, Gg, scale, Wl, Wg, dt=np.complex128):
    """Adjoint of Eq. (3) through the transforms, for L = sum_t Re tr(W^t^H Sigma^t) (PyTorch convention): per bond
    and frequency Q_j = W^ dH_j G^^H and R_i = W^^H dH_i G^; the weight gradient is conj(c) times the inverse
    transform of tr(dH_i^H Q_j) at the emission lags (same type) and the absorption lags (other type); the coupling
    gradient is (scale / N) sum_f sum_j [-i conj(K^_mj) Q_j + i K^_jm R_j]."""
    Nkz, NE, NA, Norb, _ = Gl.shape
    Nqz, Nw = Dl.shape[0], Dl.shape[1]
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)
    N = Nkz * L
    cc = -1j * scale                                              # conj(c)
    g_dH = np.zeros(dH.shape, complex)
    g_D = [np.zeros(Dl.shape, complex), np.zeros(Dg.shape, complex)]

    def spectrum(X):
        Xp = np.zeros((Nkz, L) + X.shape[2:], dt)
        Xp[:, :NE] = X
        return np.fft.fft2(Xp, axes=(0, 1))

    for t, (G, W, Dt, Dtb) in enumerate(((Gl, Wl, Dl, Dg), (Gg, Wg, Dg, Dl))):
        Gh, Wh = spectrum(G), spectrum(W)
        K = np.zeros((Nkz, L, NA, NB, 3, 3), dt)
        for w in range(Nw):
            K[:Nqz, w + 1] = Dt[:, w]
            K[:Nqz, L - (w + 1)] = Dtb[:, w]
        Kh = np.fft.fft2(K, axes=(0, 1))
        for a in range(NA):
            Wa = Wh[:, :, a]
            for s in range(NB):
                b = nbr[a, s]
                A = dH[a, s].astype(dt)
                Gb = Gh[:, :, b]
                Q = [Wa @ A[j] @ np.conj(np.swapaxes(Gb, -1, -2)) for j in range(3)]
                R = [np.conj(np.swapaxes(Wa, -1, -2)) @ A[i] @ Gb for i in range(3)]
                Hh = np.zeros((Nkz, L, 3, 3), complex)
                for i in range(3):
                    for j in range(3):
                        Hh[..., i, j] = np.trace(A[i].conj().T @ Q[j], axis1=-2, axis2=-1)
                H = np.fft.ifft2(Hh, axes=(0, 1))
                for w in range(Nw):
                    g_D[t][:, w, a, s] += cc * H[:Nqz, w + 1]
                    g_D[1 - t][:, w, a, s] += cc * H[:Nqz, L - (w + 1)]
                for m in range(3):  # per-frequency terms in dt, the sum over frequencies in FP64 (as the kernels)
                    acc = np.zeros((Norb, Norb), complex)
                    for j in range(3):
                        tq = (-1j * np.conj(Kh[:, :, a, s, m, j]))[..., None, None] * Q[j]
                        tr = (1j * Kh[:, :, a, s, j, m])[..., None, None] * R[j]
                        acc += (tq + tr).astype(np.complex128).sum(axis=(0, 1))
                    g_dH[a, s, m] += scale / N * acc
    return g_dH, g_D[0], g_D[1]


@pytest.mark.parametrize("d", CASES, ids=lambda d: f"NE{d.NE}_Nkz{d.Nkz}_Nqz{d.Nqz}")
def test_adjoint_transform_model_equals_the_oracle(d):
    from paper_1912_10024_gb300.inputs import make_upstream
    nbr = None if d is TINY else ring_neighbours(d.NA, d.NB)
    x = make_inputs(d, seed=d.NE + 5, nbr=nbr)
    W, V = make_upstream(d, seed=d.NE + 6)
    arrs = [t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater)]
    got = sigma_grad_by_transforms(*arrs, SCALE, W.numpy(), V.numpy())
    ref = oracle.sigma_grad(*arrs, SCALE, W.numpy(), V.numpy())
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def sigma_grad_G_by_transforms(nbr, dH, Dl, Dg, scale, Wl, Wg):
    """Gradient of L = sum_t Re tr(W^t^H Sigma^t) with respect to G^t (PyTorch convention), Sigma being linear in G:
    per atom b and frequency, conj(c) sum over bonds (a, s) into b of sum_i dH_i^H W^_a B_i with
    B_i = sum_j conj(K^_ij) dH_j, then the inverse transforms (rows E < NE)."""
    Nkz, NE, NA, Norb, _ = Wl.shape
    Nqz, Nw = Dl.shape[0], Dl.shape[1]
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)
    cc = -1j * scale
    out = []
    for W, Dt, Dtb in ((Wl, Dl, Dg), (Wg, Dg, Dl)):
        Wp = np.zeros((Nkz, L, NA, Norb, Norb), complex)
        Wp[:, :NE] = W
        Wh = np.fft.fft2(Wp, axes=(0, 1))
        K = np.zeros((Nkz, L, NA, NB, 3, 3), complex)
        for w in range(Nw):
            K[:Nqz, w + 1] = Dt[:, w]
            K[:Nqz, L - (w + 1)] = Dtb[:, w]
        Kh = np.fft.fft2(K, axes=(0, 1))
        Rh = np.zeros((Nkz, L, NA, Norb, Norb), complex)
        for a in range(NA):
            for s in range(NB):
                b = nbr[a, s]
                A = dH[a, s]
                for i in range(3):
                    Bi = sum(np.conj(Kh[:, :, a, s, i, j])[..., None, None] * A[j] for j in range(3))
                    Rh[:, :, b] += cc * (A[i].conj().T @ Wh[:, :, a] @ Bi)
        out.append(np.fft.ifft2(Rh, axes=(0, 1))[:, :NE])
    return out


@pytest.mark.parametrize("d", CASES, ids=lambda d: f"NE{d.NE}_Nkz{d.Nkz}_Nqz{d.Nqz}")
def test_grad_G_transform_model_equals_the_oracle(d):
    from paper_1912_10024_gb300.inputs import make_upstream
    nbr = None if d is TINY else ring_neighbours(d.NA, d.NB)
    x = make_inputs(d, seed=d.NE + 7, nbr=nbr)
    W, V = make_upstream(d, seed=d.NE + 8)
    nb, dH, Dl, Dg = (t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater))
    got = sigma_grad_G_by_transforms(nb, dH, Dl, Dg, SCALE, W.numpy(), V.numpy())
    ref = oracle.sigma_grad_G(nb, dH, Dl, Dg, SCALE, W.numpy(), V.numpy())
    for g, r in zip(got, ref):
        assert np.abs(g - r).max() <= 1e-12 * np.abs(r).max()


def test_fp32_arithmetic_error_is_within_the_stated_bound():
    """The same transforms and products in single precision (numpy complex64 FFTs and products) land a few 1e-7
    from the oracle at Norb = 10: the error level of the FP32_FFT mode, inside its stated bound 2e-6, and clearly
    above FP64 rounding."""
    d = Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11)
    x = make_inputs(d, seed=21, nbr=ring_neighbours(d.NA, d.NB))
    arrs = [t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater)]
    got = sigma_by_transforms(*arrs, SCALE, dt=np.complex64)
    ref = oracle.sigma(*arrs, SCALE)
    errs = [np.abs(g - r).max() / np.abs(r).max() for g, r in zip(got, ref)]
    assert 1e-8 < max(errs) <= 2e-6, errs


def coupling_gradient_terms(nbr, dH, Dl, Dg, Gl, Wl, dt):
    """Per-frequency terms of the coupling gradient of one type (the summand of grad dH_m above), in the complex
    type dt: [bond][m][frequency][Norb][Norb]."""
    Nkz, NE, NA, Norb, _ = Gl.shape
    Nqz, Nw = Dl.shape[0], Dl.shape[1]
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)

    def spectrum(X):
        Xp = np.zeros((Nkz, L) + X.shape[2:], dt)
        Xp[:, :NE] = X
        return np.fft.fft2(Xp, axes=(0, 1))

    Gh, Wh = spectrum(Gl), spectrum(Wl)
    K = np.zeros((Nkz, L, NA, NB, 3, 3), dt)
    for w in range(Nw):
        K[:Nqz, w + 1] = Dl[:, w]
        K[:Nqz, L - (w + 1)] = Dg[:, w]
    Kh = np.fft.fft2(K, axes=(0, 1))
    terms = []
    for a in range(NA):
        for s in range(NB):
            A, Wa, Gb = dH[a, s].astype(dt), Wh[:, :, a], Gh[:, :, nbr[a, s]]
            Q = [Wa @ A[j] @ np.conj(np.swapaxes(Gb, -1, -2)) for j in range(3)]
            R = [np.conj(np.swapaxes(Wa, -1, -2)) @ A[i] @ Gb for i in range(3)]
            terms.append([sum((-1j * np.conj(Kh[:, :, a, s, m, j]))[..., None, None] * Q[j]
                              + (1j * Kh[:, :, a, s, j, m])[..., None, None] * R[j] for j in range(3))
                          .reshape(Nkz * L, Norb, Norb) for m in range(3)])
    return terms


def lane_sums_fp32(x, chunk, lanes):
    """The kernel's order: chunks of `chunk` frequencies; within a chunk lane f adds frequencies f, f + lanes, ...
    one after another in FP32; lanes and chunks are then added in FP64."""
    total = np.zeros(x.shape[1:], np.complex128)
    for c0 in range(0, x.shape[0], chunk):
        for f in range(lanes):
            acc = np.zeros(x.shape[1:], np.complex64)
            for v in x[c0 + f:min(x.shape[0], c0 + chunk):lanes]:
                acc = (acc + v).astype(np.complex64)
            total += acc
    return total


def test_fp32_coupling_gradient_needs_short_lane_sums():
    """On a FinFET-sized frequency grid (Nkz = 7, L = 576, 4032 frequencies) the coupling-gradient terms computed in
    FP32 and added per lane in FP32 drift from the FP64 sums when a lane adds ~270 terms (the chunks of three per atom
    at 1024 atoms, 5 lanes); chunks of at most 32 terms per lane, added in FP64, stay close to the floor set by the
    FP32 terms themselves."""
    from paper_1912_10024_gb300.inputs import make_upstream
    d = Dims(NA=2, NB=2, Norb=10, NE=512, Nkz=7, Nqz=7, Nw=32)
    x = make_inputs(d, seed=41, nbr=ring_neighbours(d.NA, d.NB))
    W, _ = make_upstream(d, seed=42)
    arrs = [t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less)] + [W.numpy()]
    ref = np.array([[t.sum(0) for t in b] for b in coupling_gradient_terms(*arrs, np.complex128)])
    t32 = coupling_gradient_terms(*arrs, np.complex64)
    nfreq = t32[0][0].shape[0]
    lanes = 5

    def err(sums):
        return np.abs(np.array(sums) - ref).max() / np.abs(ref).max()

    floor = err([[t.astype(np.complex128).sum(0) for t in b] for b in t32])
    long_chunks = err([[lane_sums_fp32(t, nfreq // 3, lanes) for t in b] for b in t32])
    short_chunks = err([[lane_sums_fp32(t, 32 * lanes, lanes) for t in b] for b in t32])
    assert long_chunks > 2 * short_chunks, (floor, long_chunks, short_chunks)
    assert short_chunks < 2 * floor, (floor, long_chunks, short_chunks)


def sigma_spectrum(nbr, dH, Dt, Dtb, G, Nw):
    """S^(kappa, eps) of one type before the inverse transform (the product step of the forward model)."""
    Nkz, NE, NA, Norb, _ = G.shape
    Nqz = Dt.shape[0]
    NB = nbr.shape[1]
    L = smallest_2a3b(NE + Nw)
    Gp = np.zeros((Nkz, L, NA, Norb, Norb), complex)
    Gp[:, :NE] = G
    Gh = np.fft.fft2(Gp, axes=(0, 1))
    K = np.zeros((Nkz, L, NA, NB, 3, 3), complex)
    for w in range(Nw):
        K[:Nqz, w + 1] = Dt[:, w]
        K[:Nqz, L - (w + 1)] = Dtb[:, w]
    Kh = np.fft.fft2(K, axes=(0, 1))
    Sh = np.zeros((Nkz, L, NA, Norb, Norb), complex)
    for a in range(NA):
        for s in range(NB):
            A = dH[a, s]
            for i in range(3):
                for j in range(3):
                    Sh[:, :, a] += Kh[:, :, a, s, i, j][..., None, None] * (A[i] @ Gh[:, :, nbr[a, s]] @ A[j].conj().T)
    return 1j * Sh


@pytest.mark.parametrize("Nkz,NE", [(3, 13), (4, 13), (1, 9)])
def test_half_spectrum_mirror_relation(Nkz, NE):
    """With anti-Hermitian G and D blocks (as lesser and greater functions are) the spectrum of Sigma obeys
    S^(-f) = -S^(f)^H, so one frequency of each (f, -f) pair determines the other (the SSE_FLAG_ANTIHERMITIAN path);
    a G block that is not anti-Hermitian breaks the relation."""
    d = Dims(NA=4, NB=2, Norb=3, NE=NE, Nkz=Nkz, Nqz=min(Nkz, 2), Nw=3)
    x = make_inputs(d, seed=NE + Nkz, nbr=ring_neighbours(d.NA, d.NB))
    nb, dH, Dl, Dg, Gl = (t.numpy() for t in (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less))
    L = smallest_2a3b(NE + d.Nw)
    neg = np.ix_((-np.arange(Nkz)) % Nkz, (-np.arange(L)) % L)

    def mirror_error(G):
        Sh = sigma_spectrum(nb, dH, Dl, Dg, G, d.Nw)
        mirrored = -np.conj(np.swapaxes(Sh, -1, -2))[neg]
        return np.abs(Sh - mirrored).max() / np.abs(Sh).max()

    assert mirror_error(Gl) <= 1e-13
    broken = Gl.copy()
    broken[0, 2, 1] += 0.1  # one block gains a Hermitian part
    assert mirror_error(broken) > 1e-4


def test_pi_half_spectrum_mirror_relation():
    """For Eq. (4) with anti-Hermitian G the per-frequency traces obey C^(-f) = C^(f)^H (3x3 blocks)."""
    d = Dims(NA=4, NB=2, Norb=3, NE=13, Nkz=4, Nqz=2, Nw=3)
    x = make_inputs(d, seed=77, nbr=ring_neighbours(d.NA, d.NB))
    nb, dH, Gl, Gg = (t.numpy() for t in (x.nbr, x.dH, x.G_less, x.G_greater))
    L = smallest_2a3b(d.NE + d.Nw)
    spec = []
    for G in (Gl, Gg):
        Gp = np.zeros((d.Nkz, L, d.NA, d.Norb, d.Norb), complex)
        Gp[:, :d.NE] = G
        spec.append(np.fft.fft2(Gp, axes=(0, 1)))
    neg_k, neg_e = (-np.arange(d.Nkz)) % d.Nkz, (-np.arange(L)) % L
    X, Y = spec
    a, s = 1, 0
    A = dH[a, s]
    Yneg = Y[neg_k][:, neg_e, nb[a, s]]
    Ch = np.zeros((d.Nkz, L, 3, 3), complex)
    for i in range(3):
        for j in range(3):
            Ch[..., i, j] = np.trace(A[i].conj().T @ X[:, :, a] @ A[j] @ Yneg, axis1=-2, axis2=-1)
    mirrored = np.conj(np.swapaxes(Ch, -1, -2))[np.ix_(neg_k, neg_e)]
    assert np.abs(Ch - mirrored).max() <= 1e-13 * np.abs(Ch).max()


def test_stage_index_split_by_multiply_high_is_exact():
    """The E-transform's Stockham stages split the butterfly index j = q * Ns + k with q = umulhi(j, floor(2^32/Ns)+1)
    when Ns is not a power of two. For j, Ns < 2^16 the error of the multiplier, below j / 2^32 < 2^-16, never crosses
    an integer (the fractional part of j / Ns is at most 1 - 1/Ns). Enumerated here for every stage of every 2^a 3^b
    length below 2^16, stages in the plan's order (radix 4, then 2, then 3), j over the stage's L / R butterflies."""
    lengths = sorted(2 ** a * 3 ** b for a in range(17) for b in range(11) if 2 <= 2 ** a * 3 ** b < 1 << 16)
    checked = 0
    for L in lengths:
        radices, m = [], L
        for r in (4, 2, 3):
            while m % r == 0:
                radices.append(r)
                m //= r
        ns = 1
        for R in radices:
            if ns & (ns - 1):  # not a power of two: the multiply-high path
                mul = (1 << 32) // ns + 1
                j = np.arange(L // R, dtype=np.uint64)
                assert np.array_equal((j * np.uint64(mul)) >> np.uint64(32), j // np.uint64(ns)), (L, ns)
                checked += 1
            ns *= R
    assert checked > 100
