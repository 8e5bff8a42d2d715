"""FP32 transform mode (sse_sigma_fwd, mode FP32_FFT) against the FP64 oracle.

FP32 transforms and per-frequency block products (FP64 inputs and outputs). The stated bound is 2e-6
normwise (max |gpu - oracle| / max |oracle| per output tensor); the rounding analysis gives a few 1e-7:
unit roundoff 6e-8 times the log2 of the transform lengths and the Norb-term block products.
"""
import math

import pytest
import torch

import oracle
from conftest import normwise
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import Dims, TINY, FINFET, make_inputs, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
BOUND = 2e-6


def gpu_sigma(inp, **kw):
    g = inp.to("cuda")
    return B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp32_fft", **kw)


def oracle_sigma(inp, **kw):
    return oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, **kw)


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=40),
    Dims(NA=5, NB=2, Norb=4, NE=70, Nkz=1, Nqz=1, Nw=5),
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}")
@pytest.mark.parametrize("antihermitian", [False, True])
def test_shapes(dims, antihermitian):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 800, nbr=nbr)
    Sl, Sg = gpu_sigma(inp, check=True, antihermitian=antihermitian)
    Ol, Og = oracle_sigma(inp)
    errs = [normwise(Sl.cpu().numpy(), Ol), normwise(Sg.cpu().numpy(), Og)]
    print("fp32_fft", dims, antihermitian, errs)
    assert max(errs) <= BOUND


def test_symmetrize_and_atom_range():
    inp = make_inputs(TINY, seed=9)
    g = inp.to("cuda")
    Sl, Sg = gpu_sigma(inp, symmetrize=True)
    Ol, Og = oracle_sigma(inp)
    for S, O in ((Sl, Ol), (Sg, Og)):
        P = 0.5 * (O - O.conj().swapaxes(-1, -2))
        assert normwise(S.cpu().numpy(), P) <= BOUND
    out = (torch.zeros(TINY.g_shape(), dtype=torch.complex128, device="cuda"),
           torch.zeros(TINY.g_shape(), dtype=torch.complex128, device="cuda"))
    B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp32_fft", atoms=(3, 8), out=out)
    Ol, _ = oracle_sigma(inp, a_range=(3, 8))
    assert normwise(out[0][:, :, 3:8].cpu().numpy(), Ol[:, :, 3:8]) <= BOUND
    assert float(out[0][:, :, :3].abs().max()) == 0.0


def test_finfet_sampled():
    inp = make_inputs(FINFET, seed=0, device="cuda")
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="fp32_fft",
                     check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for (a, E0, E1) in [(0, 0, 2), (511, 255, 257), (1023, 510, 512)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                               a, E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            worst = max(worst, normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("fp32_fft finfet sampled", worst)
    assert worst <= BOUND
