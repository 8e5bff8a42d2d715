"""Transform-based FP64 forward (sse_sigma_fwd, mode FP64_FFT) against the FP64 CPU oracle.

Same contract as the direct FP64 path: normwise max|gpu - oracle| / max|oracle|
<= 1e-12 per output tensor. The cases cover FFT lengths with every radix
(2, 3, 4), NE + Nw just above and at a 2^a 3^b length, Nqz < Nkz, a
single kz point, every Norb class of the product kernel, atom ranges, the
symmetrisation flag, bad neighbours, and the adjoint and FinFET workloads
(full comparison with the direct FP64 kernel, oracle on sampled blocks).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import Dims, TINY, ADJOINT, FINFET, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def gpu_sigma(inp, **kw):
    g = inp.to("cuda")
    return B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp64_fft", **kw)


def oracle_sigma(inp, scale=SCALE, **kw):
    return oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, scale, **kw)


@pytest.mark.parametrize("scale", [SCALE, 1.0])
def test_tiny_full(scale):
    inp = make_inputs(TINY, seed=0)
    Sl, Sg = gpu_sigma(inp, scale=scale, check=True)
    Ol, Og = oracle_sigma(inp, scale)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL
    assert normwise(Sg.cpu().numpy(), Og) <= TOL


@pytest.mark.parametrize("dims", [
    Dims(NA=9, NB=3, Norb=1, NE=1000, Nkz=2, Nqz=2, Nw=7),    # L = 1024 (radix 4 only), 2 columns per FFT CTA
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nqz < Nkz, L = 72 (4, 2, 3, 3)
    Dims(NA=6, NB=4, Norb=5, NE=47, Nkz=3, Nqz=3, Nw=9),      # L = 64 (4, 4, 4)
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),    # Norb of the workloads, L = 54 (2, 3, 3, 3)
    Dims(NA=4, NB=2, Norb=12, NE=23, Nkz=2, Nqz=1, Nw=6),     # L = 32 (4, 4, 2)
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=40),    # one frequency per product pass, L = 96
    Dims(NA=5, NB=2, Norb=4, NE=70, Nkz=1, Nqz=1, Nw=5),      # single kz point, L = 81 (3, 3, 3, 3)
    Dims(NA=6, NB=3, Norb=2, NE=100, Nkz=9, Nqz=4, Nw=25),    # L = 128 (4, 4, 4, 2), Nkz = 9
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}_Nkz{d.Nkz}")
def test_shapes_full(dims):
    inp = make_inputs(dims, seed=dims.Norb + 100, nbr=ring_neighbours(dims.NA, dims.NB))
    Sl, Sg = gpu_sigma(inp, check=True)
    Ol, Og = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL
    assert normwise(Sg.cpu().numpy(), Og) <= TOL


def test_atom_range_leaves_other_atoms_untouched():
    inp = make_inputs(TINY, seed=3)
    g = inp.to("cuda")
    sentinel = (torch.full(TINY.g_shape(), 7 + 7j, dtype=torch.complex128, device="cuda"),
                torch.full(TINY.g_shape(), 7 + 7j, dtype=torch.complex128, device="cuda"))
    B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, atoms=(5, 11), out=sentinel, mode="fp64_fft")
    Ol, Og = oracle_sigma(inp, a_range=(5, 11))
    for S, O in zip(sentinel, (Ol, Og)):
        S = S.cpu().numpy()
        assert normwise(S[:, :, 5:11], O[:, :, 5:11]) <= TOL
        assert np.all(S[:, :, :5] == 7 + 7j) and np.all(S[:, :, 11:] == 7 + 7j)


def test_symmetrize_flag():
    inp = make_inputs(TINY, seed=4)
    inp.D_less = inp.D_less * (1 + 0.3j)  # break anti-Hermiticity so the projection matters
    Sl, Sg = gpu_sigma(inp, symmetrize=True)
    Ol, Og = oracle_sigma(inp)
    for S, O in ((Sl, Ol), (Sg, Og)):
        P = 0.5 * (O - np.swapaxes(O.conj(), -1, -2))
        assert normwise(S.cpu().numpy(), P) <= TOL


def test_bad_neighbour_is_reported_not_faulted():
    inp = make_inputs(TINY, seed=5)
    inp.nbr[3, 1] = TINY.NA + 5
    with pytest.raises(B.SseError) as e:
        gpu_sigma(inp, check=True)
    assert e.value.status == 5
    torch.cuda.synchronize()
    Sl, _ = gpu_sigma(inp)  # without CHECK the bond contributes zero
    ref = inp.dH.clone()
    ref[3, 1] = 0
    inp.dH = ref
    inp.nbr[3, 1] = 0
    Ol, _ = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL


def test_autograd_forward_spectral_backward_fp64():
    """SigmaFunction with the transform-based forward; the adjoint is the FP64 one."""
    d = Dims(NA=6, NB=2, Norb=3, NE=20, Nkz=3, Nqz=2, Nw=4)
    inp = make_inputs(d, seed=21, nbr=ring_neighbours(6, 2))
    W, V = make_upstream(d, seed=22)
    g = inp.to("cuda")
    dH = g.dH.clone().requires_grad_(True)
    Dl = g.D_less.clone().requires_grad_(True)
    Dg = g.D_greater.clone().requires_grad_(True)
    Sl, Sg = B.sigma_autograd(dH, Dl, Dg, g.G_less, g.G_greater, g.nbr, SCALE, "fp64_fft")
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    o_dH, o_Dl, o_Dg = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater,
                                         SCALE, W, V)
    assert normwise(dH.grad.cpu().numpy(), o_dH) <= TOL
    assert normwise(Dl.grad.cpu().numpy(), o_Dl) <= TOL
    assert normwise(Dg.grad.cpu().numpy(), o_Dg) <= TOL


def _full_vs_direct_and_samples(dims, seed, samples):
    inp = make_inputs(dims, seed=seed, device="cuda")
    args = (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr)
    Fl, Fg = B.sigma(*args, mode="fp64_fft", check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for (a, E0, E1) in samples:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                               a, E0, E1)
        for S, O in ((Fl, Ol), (Fg, Og)):
            worst = max(worst, normwise(S[:, E0:E1, a].cpu().numpy(), O))
    assert worst <= TOL, worst
    return inp, Fl, Fg


def test_adjoint_workload_full_vs_direct():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16: every output against the direct FP64 kernel
    (itself checked against the oracle), and sampled blocks against the oracle."""
    inp, Fl, Fg = _full_vs_direct_and_samples(ADJOINT, 7, [(0, 0, 3), (17, 120, 123), (255, 253, 256)])
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="fp64")
    for F, S in ((Fl, Sl), (Fg, Sg)):
        err = float((F - S).abs().max() / S.abs().max())
        assert err <= TOL, err


def test_finfet_workload_sampled():
    """The benchmark workload (NA=1024, Norb=10, NE=512, Nkz=Nqz=7, Nw=32): oracle on sampled blocks at both
    energy edges and the interior; anti-Hermiticity of the whole output."""
    inp, Fl, Fg = _full_vs_direct_and_samples(FINFET, 0, [(0, 0, 2), (511, 255, 257), (1023, 510, 512),
                                                          (300, 31, 33)])
    for S in (Fl, Fg):
        blk = S[:, ::37, ::61]
        assert float((blk + blk.conj().transpose(-1, -2)).abs().max()) <= 1e-12 * float(S.abs().max())


@pytest.mark.parametrize("dims", [
    TINY,                                                     # L = 36, Nkz = 3
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nkz even, L = 72
    Dims(NA=5, NB=2, Norb=4, NE=70, Nkz=1, Nqz=1, Nw=5),      # L = 81 (odd), one kz point
    Dims(NA=6, NB=3, Norb=2, NE=100, Nkz=9, Nqz=4, Nw=25),    # L = 128
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}")
def test_antihermitian_half_spectrum(dims):
    """SSE_FLAG_ANTIHERMITIAN (inputs are exactly anti-Hermitian by construction): half the frequencies plus the
    mirror S^(-f) = -S^(f)^H give Eq. (3) to the FP64 tolerance; CHECK passes."""
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 600, nbr=nbr)
    Sl, Sg = gpu_sigma(inp, antihermitian=True, check=True)
    Ol, Og = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL
    assert normwise(Sg.cpu().numpy(), Og) <= TOL


def test_antihermitian_check_reports_violations():
    inp = make_inputs(TINY, seed=7)
    inp.G_greater[1, 5, 3, 0, 1] += 1e-3  # one element breaks G^> = -G^>^H
    with pytest.raises(B.SseError) as e:
        gpu_sigma(inp, antihermitian=True, check=True)
    assert e.value.status == 5
    inp = make_inputs(TINY, seed=7)
    inp.D_less[0, 2, 4, 1, 0, 2] += 1e-3j  # one weight block breaks D^< = -D^<^H
    with pytest.raises(B.SseError) as e:
        gpu_sigma(inp, antihermitian=True, check=True)
    assert e.value.status == 5


@pytest.mark.parametrize("dims", [
    Dims(NA=3, NB=2, Norb=2, NE=2000, Nkz=2, Nqz=2, Nw=5),   # L = 2048: one column per FP64 transform CTA
    Dims(NA=4, NB=2, Norb=3, NE=30, Nkz=16, Nqz=16, Nw=4),   # the largest kz grid of the transform path
], ids=lambda d: f"NE{d.NE}_Nkz{d.Nkz}")
def test_maximum_lengths(dims):
    """The transform path at its size limits: a long energy grid (the one-column FFT variant in FP64, column pairs in
    FP32) and Nkz = Nqz = 16 (the kz DFT's largest grid): Sigma in FP64_FFT and FP32_FFT, Pi and the adjoint in
    FP64_FFT, each against the oracle."""
    inp = make_inputs(dims, seed=dims.NE + dims.Nkz, nbr=ring_neighbours(dims.NA, dims.NB))
    W, V = make_upstream(dims, seed=dims.NE + dims.Nkz + 1)
    g = inp.to("cuda")
    Ol, Og = oracle_sigma(inp)
    for mode, bound in (("fp64_fft", TOL), ("fp32_fft", 2e-6)):
        Sl, Sg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode, check=True)
        assert normwise(Sl.cpu().numpy(), Ol) <= bound, mode
        assert normwise(Sg.cpu().numpy(), Og) <= bound, mode
    Pl, Pg = B.pi(g.G_less, g.G_greater, g.dH, g.nbr, dims.Nqz, dims.Nw, check=True)
    Ql, Qg = oracle.pi(inp.nbr, inp.dH, inp.G_less, inp.G_greater, SCALE, dims.Nqz, dims.Nw)
    assert normwise(Pl.cpu().numpy(), Ql) <= TOL and normwise(Pg.cpu().numpy(), Qg) <= TOL
    got = B.sigma_grad(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, W.cuda(), V.cuda(),
                       mode="fp64_fft", check=True)
    ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V)
    for x, y in zip(got, ref):
        assert normwise(x.cpu().numpy(), y) <= TOL


@pytest.mark.parametrize("Nkz", list(range(1, 17)))
def test_every_kz_grid(Nkz):
    """The kz DFT has one kernel instantiation per grid size (1 .. 16, the pairing of k with Nkz - k differs between
    odd and even sizes): Sigma in FP64_FFT and FP32_FFT against the oracle for each, with Nqz < Nkz where possible
    (the lag kernel's zero slices) and L = 36 (the register-codelet FP32 E-transform)."""
    d = Dims(NA=3, NB=2, Norb=2, NE=32, Nkz=Nkz, Nqz=max(1, Nkz - 1), Nw=4)
    inp = make_inputs(d, seed=300 + Nkz, nbr=ring_neighbours(d.NA, d.NB))
    g = inp.to("cuda")
    Ol, Og = oracle_sigma(inp)
    for mode, bound in (("fp64_fft", TOL), ("fp32_fft", 2e-6)):
        Sl, Sg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode, check=True)
        assert max(normwise(Sl.cpu().numpy(), Ol), normwise(Sg.cpu().numpy(), Og)) <= bound, (mode, Nkz)
