"""Phonon self-energy Pi of Eq. (4) (sse_pi_fwd through the convolution theorem, FP64 and FP32_FFT) against the
oracle.

Tolerance: normwise max|gpu - oracle| / max|oracle| <= 1e-12 per output tensor in FP64; the stated FP32_FFT bound
below for the FP32 path.
Cases: every FFT radix (2, 3, 4), Nqz < Nkz, a single kz point, Norb from 1 to 16,
atom ranges, the symmetrisation flag, a bad neighbour index, and the
adjoint and FinFET workloads on sampled atoms (exact sub-problems: the atom
and its neighbours).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import ADJOINT, FINFET, TINY, Dims, make_inputs, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def gpu_pi(inp, d, **kw):
    g = inp.to("cuda")
    return B.pi(g.G_less, g.G_greater, g.dH, g.nbr, d.Nqz, d.Nw, **kw)


def oracle_pi(inp, d, scale=SCALE, **kw):
    return oracle.pi(inp.nbr, inp.dH, inp.G_less, inp.G_greater, scale, d.Nqz, d.Nw, **kw)


@pytest.mark.parametrize("scale", [SCALE, 1.0])
def test_tiny_full(scale):
    inp = make_inputs(TINY, seed=0)
    Pl, Pg = gpu_pi(inp, TINY, scale=scale, check=True)
    Ol, Og = oracle_pi(inp, TINY, scale)
    assert normwise(Pl.cpu().numpy(), Ol) <= TOL
    assert normwise(Pg.cpu().numpy(), Og) <= TOL


@pytest.mark.parametrize("dims", [
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nqz < Nkz, L = 72
    Dims(NA=6, NB=4, Norb=5, NE=47, Nkz=3, Nqz=3, Nw=9),      # L = 64
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),    # L = 54
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=40),    # one frequency per pass, L = 96
    Dims(NA=5, NB=1, Norb=4, NE=70, Nkz=1, Nqz=1, Nw=5),      # single kz point, one neighbour, L = 81
    Dims(NA=6, NB=3, Norb=1, NE=100, Nkz=9, Nqz=4, Nw=25),    # Norb = 1, L = 128, Nkz = 9
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}_Nkz{d.Nkz}")
def test_shapes_full(dims):
    inp = make_inputs(dims, seed=dims.Norb + 200, nbr=ring_neighbours(dims.NA, dims.NB))
    Pl, Pg = gpu_pi(inp, dims, check=True)
    Ol, Og = oracle_pi(inp, dims)
    assert normwise(Pl.cpu().numpy(), Ol) <= TOL
    assert normwise(Pg.cpu().numpy(), Og) <= TOL


def test_atom_range_leaves_other_atoms_untouched():
    inp = make_inputs(TINY, seed=3)
    g = inp.to("cuda")
    shape = (TINY.Nqz, TINY.Nw, TINY.NA, TINY.NB + 1, 3, 3)
    out = (torch.full(shape, 7 + 7j, dtype=torch.complex128, device="cuda"),
           torch.full(shape, 7 + 7j, dtype=torch.complex128, device="cuda"))
    B.pi(g.G_less, g.G_greater, g.dH, g.nbr, TINY.Nqz, TINY.Nw, atoms=(5, 11), out=out)
    Ol, Og = oracle_pi(inp, TINY, a_range=(5, 11))
    for P, O in zip(out, (Ol, Og)):
        P = P.cpu().numpy()
        assert normwise(P[:, :, 5:11], O[:, :, 5:11]) <= TOL
        assert np.all(P[:, :, :5] == 7 + 7j) and np.all(P[:, :, 11:] == 7 + 7j)


def test_symmetrize_flag():
    inp = make_inputs(TINY, seed=4)
    inp.G_less = inp.G_less * (1 + 0.3j)  # break anti-Hermiticity so the projection matters
    Pl, Pg = gpu_pi(inp, TINY, symmetrize=True)
    Ol, Og = oracle_pi(inp, TINY)
    for P, O in ((Pl, Ol), (Pg, Og)):
        S = 0.5 * (O - np.swapaxes(O.conj(), -1, -2))
        assert normwise(P.cpu().numpy(), S) <= TOL


def test_bad_neighbour_is_reported_not_faulted():
    inp = make_inputs(TINY, seed=5)
    inp.nbr[3, 1] = TINY.NA + 5
    with pytest.raises(B.SseError) as e:
        gpu_pi(inp, TINY, check=True)
    assert e.value.status == 5
    torch.cuda.synchronize()
    Pl, _ = gpu_pi(inp, TINY)  # without CHECK the bond contributes zero
    inp.dH[3, 1] = 0
    inp.nbr[3, 1] = 0
    Ol, _ = oracle_pi(inp, TINY)
    assert normwise(Pl.cpu().numpy(), Ol) <= TOL


def _sub_problem(inp, a):
    """Atom a and its neighbours as a small problem in which a is atom 0 (exact: Pi of a only reads
    G of a and of its neighbours and a's couplings)."""
    nb = [int(x) for x in inp.nbr[a].cpu()]
    sub = [a] + nb
    NB = len(nb)
    nbr = torch.zeros((len(sub), NB), dtype=torch.int32)
    nbr[0] = torch.arange(1, NB + 1, dtype=torch.int32)
    idx = torch.tensor(sub, device=inp.G_less.device)
    Gl = inp.G_less.index_select(2, idx).cpu()
    Gg = inp.G_greater.index_select(2, idx).cpu()
    dH = inp.dH.index_select(0, idx).cpu()
    return nbr, dH, Gl, Gg


def _sampled(dims, seed, atoms):
    inp = make_inputs(dims, seed=seed, device="cuda")
    Pl, Pg = B.pi(inp.G_less, inp.G_greater, inp.dH, inp.nbr, dims.Nqz, dims.Nw, check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for a in atoms:
        nbr, dH, Gl, Gg = _sub_problem(inp, a)
        Ol, Og = oracle.pi(nbr, dH, Gl, Gg, SCALE, dims.Nqz, dims.Nw, a_range=(0, 1))
        for P, O in ((Pl, Ol), (Pg, Og)):
            worst = max(worst, normwise(P[:, :, a].cpu().numpy(), O[:, :, 0]))
    assert worst <= TOL, worst
    return Pl, Pg


def test_adjoint_workload_sampled():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16: oracle on three atoms."""
    _sampled(ADJOINT, 7, [0, 131, 255])


def test_finfet_workload_sampled():
    """NA=1024, Norb=10, NE=512, Nkz=Nqz=7, Nw=32: oracle on two atoms; every 3x3 block anti-Hermitian
    (anti-Hermitian G inputs)."""
    Pl, Pg = _sampled(FINFET, 0, [0, 777])
    for P in (Pl, Pg):
        blk = P[:, ::5, ::97]
        assert float((blk + blk.conj().transpose(-1, -2)).abs().max()) <= 1e-12 * float(P.abs().max())


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nkz even, L = 72
    Dims(NA=5, NB=1, Norb=4, NE=70, Nkz=1, Nqz=1, Nw=5),      # L = 81 (odd)
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}")
def test_antihermitian_half_spectrum(dims):
    """SSE_FLAG_ANTIHERMITIAN: half the frequencies plus the mirror C^(-f) = C^(f)^H."""
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 700, nbr=nbr)
    Pl, Pg = gpu_pi(inp, dims, antihermitian=True, check=True)
    Ol, Og = oracle_pi(inp, dims)
    assert normwise(Pl.cpu().numpy(), Ol) <= TOL
    assert normwise(Pg.cpu().numpy(), Og) <= TOL
    inp.G_less[0, 3, 2, 1, 1] += 1e-3  # a diagonal element with a real part breaks anti-Hermiticity
    with pytest.raises(B.SseError) as e:
        gpu_pi(inp, dims, antihermitian=True, check=True)
    assert e.value.status == 5


# mode FP32_FFT: FP32 transforms and products (FP64 inputs and outputs); the per-frequency traces carry a relative
# error of a few unit roundoffs times the transform depth, so a few 1e-7 normwise; stated bound 2e-6 as for the
# FP32_FFT forward of Eq. (3)
FP32_BOUND = 2e-6


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nqz < Nkz, L = 72
    Dims(NA=6, NB=4, Norb=5, NE=47, Nkz=3, Nqz=3, Nw=9),      # odd Norb (padded tiles), L = 64
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),    # L = 54
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=40),    # L = 96
    Dims(NA=6, NB=3, Norb=1, NE=100, Nkz=9, Nqz=4, Nw=25),    # Norb = 1, L = 128
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}_Nkz{d.Nkz}")
@pytest.mark.parametrize("antihermitian", [False, True])
def test_fp32_vs_oracle(dims, antihermitian):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 800, nbr=nbr)
    Pl, Pg = gpu_pi(inp, dims, check=True, mode="fp32_fft", antihermitian=antihermitian)
    Ol, Og = oracle_pi(inp, dims)
    errs = [normwise(Pl.cpu().numpy(), Ol), normwise(Pg.cpu().numpy(), Og)]
    print("fp32 pi", dims, antihermitian, errs)
    assert max(errs) <= FP32_BOUND


def test_fp32_atom_range_and_symmetrize():
    inp = make_inputs(TINY, seed=13)
    g = inp.to("cuda")
    shape = (TINY.Nqz, TINY.Nw, TINY.NA, TINY.NB + 1, 3, 3)
    out = (torch.full(shape, 7 + 7j, dtype=torch.complex128, device="cuda"),
           torch.full(shape, 7 + 7j, dtype=torch.complex128, device="cuda"))
    B.pi(g.G_less, g.G_greater, g.dH, g.nbr, TINY.Nqz, TINY.Nw, atoms=(3, 9), out=out, mode="fp32_fft")
    Ol, Og = oracle_pi(inp, TINY, a_range=(3, 9))
    for P, O in zip(out, (Ol, Og)):
        P = P.cpu().numpy()
        assert normwise(P[:, :, 3:9], O[:, :, 3:9]) <= FP32_BOUND
        assert np.all(P[:, :, :3] == 7 + 7j) and np.all(P[:, :, 9:] == 7 + 7j)
    inp.G_less = inp.G_less * (1 + 0.3j)
    Pl, _ = gpu_pi(inp, TINY, symmetrize=True, mode="fp32_fft")
    Ol, _ = oracle_pi(inp, TINY)
    assert normwise(Pl.cpu().numpy(), 0.5 * (Ol - np.swapaxes(Ol.conj(), -1, -2))) <= FP32_BOUND


def test_fp32_finfet_workload_vs_fp64():
    """NA=1024, Norb=10, NE=512, Nkz=Nqz=7, Nw=32: the FP32_FFT result against the FP64 one (itself pinned to the
    oracle on sampled atoms above)."""
    inp = make_inputs(FINFET, seed=0, device="cuda")
    args = (inp.G_less, inp.G_greater, inp.dH, inp.nbr, FINFET.Nqz, FINFET.Nw)
    ref = B.pi(*args)
    got = B.pi(*args, mode="fp32_fft", check=True)
    errs = [float((x - y).abs().max() / y.abs().max()) for x, y in zip(got, ref)]
    print("fp32 pi at FinFET", errs)
    assert max(errs) <= FP32_BOUND
