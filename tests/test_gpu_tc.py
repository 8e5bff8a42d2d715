"""Tensor-core block products on the transform path (sse_sigma_fwd, mode F16X3_FFT) against the FP64 oracle.

FP32 transforms with the per-frequency block products as FP16 hi/lo split GEMMs on tcgen05 (three products,
FP32 accumulation, power-of-two scales). Stated bound: 2e-6 normwise per output tensor (max|gpu - oracle| /
max|oracle|), the FP32_FFT bound: the split keeps ~22 significant bits per operand, so the products add ~2^-22
relative per term to the FP32 transforms' few 1e-7.

Shapes cover every row-group layout of the kernel (Norb = 1 .. 10: 32 down to 3 frequencies per 32-row group, one
to four 16-B chunks per G row, odd Norb with a zero K chunk), ragged last tiles and frequency-tile groups, one to
four bonds, Nqz < Nkz, both flags, atom ranges and the FinFET workload on sampled blocks.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import FINFET, TINY, Dims, make_inputs, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
BOUND = 2e-6


def gpu_sigma(inp, **kw):
    g = inp.to("cuda")
    return B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="f16x3_fft", **kw)


def oracle_sigma(inp, **kw):
    return oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, **kw)


SHAPES = [
    TINY,                                                   # Norb 4: 8 frequencies per group
    Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11),  # the workloads' Norb, ragged tiles, Nqz < Nkz
    Dims(NA=6, NB=3, Norb=1, NE=300, Nkz=2, Nqz=2, Nw=9),   # 32 frequencies per group, several tile groups
    Dims(NA=7, NB=1, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),    # one bond, odd Norb (zero K chunk)
    Dims(NA=4, NB=4, Norb=5, NE=33, Nkz=3, Nqz=3, Nw=6),    # two G chunks
    Dims(NA=3, NB=2, Norb=7, NE=50, Nkz=2, Nqz=1, Nw=13),
    Dims(NA=4, NB=3, Norb=8, NE=29, Nkz=5, Nqz=5, Nw=4),
    Dims(NA=3, NB=4, Norb=9, NE=26, Nkz=3, Nqz=3, Nw=8),    # three G chunks, 27 of 32 rows per group
]


@pytest.mark.parametrize("dims", SHAPES, ids=lambda d: f"Norb{d.Norb}_NB{d.NB}_NE{d.NE}_Nkz{d.Nkz}")
def test_shapes(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 2000, nbr=nbr)
    Sl, Sg = gpu_sigma(inp, check=True)
    Ol, Og = oracle_sigma(inp)
    errs = [normwise(Sl.cpu().numpy(), Ol), normwise(Sg.cpu().numpy(), Og)]
    print("f16x3_fft", dims, errs)
    assert max(errs) <= BOUND


@pytest.mark.parametrize("dims", [TINY, Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11)],
                         ids=["tiny", "norb10"])
def test_antihermitian_half_spectrum(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=2100, nbr=nbr)
    Sl, Sg = gpu_sigma(inp, check=True, antihermitian=True)
    Ol, Og = oracle_sigma(inp)
    assert max(normwise(Sl.cpu().numpy(), Ol), normwise(Sg.cpu().numpy(), Og)) <= BOUND


def test_symmetrize_and_atom_range():
    inp = make_inputs(TINY, seed=2200)
    g = inp.to("cuda")
    Sl, Sg = gpu_sigma(inp, symmetrize=True)
    Ol, Og = oracle_sigma(inp)
    for S, O in ((Sl, Ol), (Sg, Og)):
        assert normwise(S.cpu().numpy(), 0.5 * (O - O.conj().swapaxes(-1, -2))) <= BOUND
    out = (torch.full(TINY.g_shape(), 3 + 3j, dtype=torch.complex128, device="cuda"),
           torch.full(TINY.g_shape(), 3 + 3j, dtype=torch.complex128, device="cuda"))
    B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="f16x3_fft", atoms=(5, 12), out=out)
    Ol, Og = oracle_sigma(inp, a_range=(5, 12))
    for S, O in zip(out, (Ol, Og)):
        S = S.cpu().numpy()
        assert normwise(S[:, :, 5:12], O[:, :, 5:12]) <= BOUND
        assert np.all(S[:, :, :5] == 3 + 3j) and np.all(S[:, :, 12:] == 3 + 3j)


def test_scaled_inputs_keep_the_error():
    """Power-of-two normalisation: inputs scaled by 2^40 and 2^-40 give the same relative error (FP16 alone would
    overflow or flush)."""
    d = Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11)
    inp = make_inputs(d, seed=2300, nbr=ring_neighbours(d.NA, d.NB))
    for f in (2.0 ** 40, 2.0 ** -40):
        big = make_inputs(d, seed=2300, nbr=ring_neighbours(d.NA, d.NB))
        big.G_less, big.G_greater, big.D_less = inp.G_less * f, inp.G_greater * f, inp.D_less / f
        Sl, Sg = gpu_sigma(big)
        Ol, Og = oracle_sigma(big)
        assert max(normwise(Sl.cpu().numpy(), Ol), normwise(Sg.cpu().numpy(), Og)) <= BOUND, f


def test_bad_neighbour_reported_and_contributes_zero():
    inp = make_inputs(TINY, seed=2400)
    inp.nbr[2, 3] = -7
    with pytest.raises(B.SseError) as e:
        gpu_sigma(inp, check=True)
    assert e.value.status == 5
    torch.cuda.synchronize()
    Sl, _ = gpu_sigma(inp)
    ref = inp.dH.clone()
    ref[2, 3] = 0
    inp.dH = ref
    inp.nbr[2, 3] = 0
    Ol, _ = oracle_sigma(inp)
    assert normwise(Sl.cpu().numpy(), Ol) <= BOUND


def test_matches_fp32_fft_at_the_adjoint_workload():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16 (diamond list): the same transforms, products on the tensor
    cores; the two differ by the products' rounding only."""
    from paper_1912_10024_gb300.inputs import ADJOINT
    inp = make_inputs(ADJOINT, seed=7, device="cuda")
    args = (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr)
    tc = B.sigma(*args, mode="f16x3_fft", check=True)
    f32 = B.sigma(*args, mode="fp32_fft")
    f64 = B.sigma(*args, mode="fp64_fft")
    e_tc = max(float((x - y).abs().max() / y.abs().max()) for x, y in zip(tc, f64))
    e_32 = max(float((x - y).abs().max() / y.abs().max()) for x, y in zip(f32, f64))
    print("adjoint workload: f16x3_fft", e_tc, "fp32_fft", e_32)
    assert e_tc <= BOUND


def test_finfet_sampled():
    inp = make_inputs(FINFET, seed=0, device="cuda")
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="f16x3_fft",
                     check=True)
    torch.cuda.synchronize()
    worst = 0.0
    for (a, E0, E1) in [(0, 0, 2), (511, 255, 257), (1023, 510, 512), (77, 100, 101)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                               a, E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            worst = max(worst, normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("f16x3_fft finfet sampled", worst)
    assert worst <= BOUND


def test_host_buffer_entry():
    d = Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11)
    inp = make_inputs(d, seed=2500, nbr=ring_neighbours(d.NA, d.NB))
    pin = [t.pin_memory() for t in (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr)]
    S = B.sigma_host(*pin, mode="f16x3_fft", check=True)
    O = oracle_sigma(inp)
    for s, o in zip(S, O):
        assert normwise(s.numpy(), o) <= BOUND


def test_autograd_after_tensor_core_forward():
    """sigma_autograd in mode f16x3_fft: the forward on the tensor cores, the adjoint in FP32_FFT."""
    d = Dims(NA=6, NB=2, Norb=3, NE=20, Nkz=3, Nqz=2, Nw=4)
    inp = make_inputs(d, seed=2600, nbr=ring_neighbours(6, 2))
    g = inp.to("cuda")
    W = torch.randn(d.g_shape(), dtype=torch.complex128, generator=torch.Generator().manual_seed(1))
    V = torch.randn(d.g_shape(), dtype=torch.complex128, generator=torch.Generator().manual_seed(2))
    leaves = [t.clone().requires_grad_(True) for t in (g.dH, g.D_less, g.D_greater)]
    Sl, Sg = B.sigma_autograd(*leaves, g.G_less, g.G_greater, g.nbr, SCALE, "f16x3_fft")
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V)
    for leaf, r in zip(leaves, ref):
        assert normwise(leaf.grad.cpu().numpy(), r) <= 1e-5
