"""FP64 CUDA path (sse_sigma_fwd, mode FP64) against the FP64 CPU oracle.

Tolerance: normwise max|gpu - oracle| / max|oracle| <= 1e-12 per output
tensor (the FP64 contract). Sizes span several energy tiles, a ragged last
tile, frequency chunking, Nqz < Nkz and every supported Norb class; the
full-size Si-FinFET-shaped workload is checked on sampled blocks.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import Dims, TINY, ADJOINT, FINFET, make_inputs, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def gpu_sigma(inp, **kw):
    g = inp.to("cuda")
    return B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, **kw)


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
    Dims(NA=9, NB=3, Norb=1, NE=1000, Nkz=2, Nqz=2, Nw=7),    # energy tile larger than NE / ragged
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nqz < Nkz, ragged tail
    Dims(NA=6, NB=4, Norb=5, NE=47, Nkz=3, Nqz=3, Nw=9),
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),    # Norb of the workloads, ragged tiles
    Dims(NA=4, NB=2, Norb=12, NE=23, Nkz=2, Nqz=1, Nw=6),
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=40),    # window split into frequency chunks
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}")
def test_shapes_full(dims):
    inp = make_inputs(dims, seed=dims.Norb, nbr=ring_neighbours(dims.NA, dims.NB))
    Sl, Sg = gpu_sigma(inp, check=True)
    Ol, Og = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL
    assert normwise(Sg.cpu().numpy(), Og) <= TOL


def test_atom_range_leaves_other_atoms_untouched():
    inp = make_inputs(TINY, seed=3)
    g = inp.to("cuda")
    sentinel = (torch.full(TINY.g_shape(), 7 + 7j, dtype=torch.complex128, device="cuda"),
                torch.full(TINY.g_shape(), 7 + 7j, dtype=torch.complex128, device="cuda"))
    B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, atoms=(5, 11), out=sentinel)
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
    torch.cuda.synchronize()  # the context is still usable
    Sl, _ = gpu_sigma(inp)  # without CHECK the bond contributes zero
    ref = inp.dH.clone()
    ref[3, 1] = 0
    inp.dH = ref
    inp.nbr[3, 1] = 0
    Ol, _ = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= TOL


def _sampled(dims, seed, samples, tol=TOL):
    torch.manual_seed(0)
    inp = make_inputs(dims, seed=seed, device="cuda")
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for (a, E0, E1) in samples:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                               a, E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            err = normwise(S[:, E0:E1, a].cpu().numpy(), O)
            worst = max(worst, err)
    assert worst <= tol, worst
    return inp, Sl, Sg


def test_adjoint_workload_sampled():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16 (full run, oracle on sampled blocks)."""
    d = ADJOINT
    samples = [(0, 0, 3), (17, 120, 123), (255, 253, 256), (128, 15, 18)]
    _sampled(d, seed=7, samples=samples)


def test_finfet_workload_sampled():
    """The benchmark workload (NA=1024, Norb=10, NE=512, Nkz=Nqz=7, Nw=32) on sampled blocks:
    both energy edges, the interior, and atoms spread over the diamond slab."""
    d = FINFET
    samples = [(0, 0, 2), (511, 255, 257), (1023, 510, 512), (300, 31, 33)]
    inp, Sl, Sg = _sampled(d, seed=0, samples=samples)
    # anti-Hermiticity holds at any size (anti-Hermitian G and D inputs)
    for S in (Sl, Sg):
        blk = S[:, ::37, ::61]
        assert float((blk + blk.conj().transpose(-1, -2)).abs().max()) <= 1e-12 * float(S.abs().max())
