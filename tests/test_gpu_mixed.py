"""Mixed-precision tensor-core paths (SSE_MODE_TF32, SSE_MODE_BF16X3) against the FP64 oracle.

Stated error bounds (normwise max|gpu - oracle| / max|oracle| per output tensor):
  BF16X3: 2e-5   (three-product bf16 split, FP32 accumulation per qz slice)
  TF32  : 2e-3   (one TF32 product, FP32 accumulation per qz slice)
Both keep the sum over qz, the final multiply by dH and the neighbour sum in FP64.
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
BOUND = {"bf16x3": 2e-5, "tf32": 2e-3}


def run_both(inp, mode, **kw):
    g = inp.to("cuda")
    S = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode, check=True, **kw)
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    return [x.cpu().numpy() for x in S], O


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_tiny_error_bound(mode):
    """Config-3 workload: tiny shapes in each mixed mode, error stated per mode."""
    S, O = run_both(make_inputs(TINY, seed=0), mode)
    errs = [normwise(s, o) for s, o in zip(S, O)]
    print(f"{mode}: normwise error vs FP64 oracle {errs}")
    assert max(errs) <= BOUND[mode]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
@pytest.mark.parametrize("dims", [
    Dims(NA=7, NB=3, Norb=10, NE=61, Nkz=4, Nqz=3, Nw=5),    # ragged tile, Nqz < Nkz
    Dims(NA=5, NB=2, Norb=10, NE=90, Nkz=2, Nqz=2, Nw=40),   # two frequency chunks per window
    Dims(NA=6, NB=4, Norb=4, NE=200, Nkz=3, Nqz=3, Nw=33),
    Dims(NA=4, NB=2, Norb=7, NE=37, Nkz=3, Nqz=1, Nw=9),
    Dims(NA=5, NB=2, Norb=4, NE=700, Nkz=2, Nqz=2, Nw=40),   # three energy windows with halos
    Dims(NA=3, NB=2, Norb=10, NE=600, Nkz=2, Nqz=1, Nw=20),
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}")
def test_shapes(mode, dims):
    inp = make_inputs(dims, seed=dims.NE, nbr=ring_neighbours(dims.NA, dims.NB))
    S, O = run_both(inp, mode)
    assert max(normwise(s, o) for s, o in zip(S, O)) <= BOUND[mode]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_symmetrize_is_exactly_anti_hermitian(mode):
    inp = make_inputs(TINY, seed=2)
    S, O = run_both(inp, mode, symmetrize=True)
    for s, o in zip(S, O):
        assert np.abs(s + np.swapaxes(s.conj(), -1, -2)).max() == 0.0
        assert normwise(s, o) <= BOUND[mode]


def test_atom_range_and_unsupported_norb():
    inp = make_inputs(TINY, seed=3)
    g = inp.to("cuda")
    out = (torch.full(TINY.g_shape(), 3 + 0j, dtype=torch.complex128, device="cuda"),
           torch.full(TINY.g_shape(), 3 + 0j, dtype=torch.complex128, device="cuda"))
    B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="bf16x3", atoms=(4, 9), out=out)
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a_range=(4, 9))
    for s, o in zip(out, O):
        s = s.cpu().numpy()
        assert normwise(s[:, :, 4:9], o[:, :, 4:9]) <= BOUND["bf16x3"]
        assert np.all(s[:, :, :4] == 3) and np.all(s[:, :, 9:] == 3)
    d = Dims(NA=3, NB=2, Norb=12, NE=20, Nkz=2, Nqz=2, Nw=3)
    big = make_inputs(d, seed=4, nbr=ring_neighbours(3, 2)).to("cuda")
    with pytest.raises(B.SseError) as e:
        B.sigma(big.G_less, big.G_greater, big.dH, big.D_less, big.D_greater, big.nbr, mode="tf32")
    assert e.value.status == 2


def test_finfet_bf16x3_sampled():
    """The Si-FinFET-shaped workload in BF16X3 on sampled blocks (edges and interior)."""
    inp = make_inputs(FINFET, seed=0, device="cuda")
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="bf16x3",
                     check=True)
    torch.cuda.synchronize()
    errs = []
    for (a, E0, E1) in [(0, 0, 2), (511, 255, 257), (1023, 510, 512), (77, 40, 42)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a,
                               E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            errs.append(normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("finfet bf16x3 sampled errors", errs)
    assert max(errs) <= BOUND["bf16x3"]


@pytest.mark.parametrize("mode", ["bf16x3", "tf32"])
def test_timed_out_wait_is_reported_and_the_next_call_is_clean(mode):
    """The bounded waits of the tensor-core kernel, made to run out without any device fault: the test hook withholds
    the window loads of one work item, the waits that depend on them give up after a short poll limit, the kernel
    drains the loads and matrix products it did issue and returns, and the call reports SSE_ERR_TIMEOUT. The next
    call on the same stream matches the oracle."""
    inp = make_inputs(TINY, seed=61)
    g = inp.to("cuda")
    args = (g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr)
    assert B.sse_test_withhold_window(0, 1 << 18) == 0
    with pytest.raises(B.SseError) as e:
        B.sigma(*args, mode=mode, check=True)
    assert e.value.status == 4  # SSE_ERR_TIMEOUT
    torch.cuda.synchronize()  # the context is still usable
    S = B.sigma(*args, mode=mode, check=True)  # the hook disarmed itself
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    assert max(normwise(s.cpu().numpy(), o) for s, o in zip(S, O)) <= BOUND[mode]
    assert B.sse_test_withhold_window(0, 0) == 1  # invalid: no poll limit
    assert B.sse_test_withhold_window(-1, 0) == 0  # disarm
