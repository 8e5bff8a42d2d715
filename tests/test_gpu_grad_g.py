"""Gradient of Eq. (3) with respect to G (sse_sigma_bwd_g through the transforms, FP64 and FP32_FFT) against the
oracle.

Tolerance: normwise 1e-12 per gradient tensor in FP64; the stated FP32_FFT bound below for the FP32 path. At the
adjoint workload, where the oracle would take too long for every atom, the identity Re <grad_G, dG> = sum_t Re tr(W^t^H Sigma^t(dG)) (Sigma is linear in G) is
checked with the GPU forward on random dG.
"""
import math

import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import ADJOINT, TINY, Dims, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def gpu(inp, W, V, **kw):
    g = inp.to("cuda")
    return B.sigma_grad_G(g.dH, g.D_less, g.D_greater, g.nbr, W.cuda(), V.cuda(), **kw)


def orc(inp, W, V, scale=SCALE, **kw):
    return oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, scale, W, V, **kw)


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),      # Nqz < Nkz
    Dims(NA=5, NB=1, Norb=4, NE=30, Nkz=2, Nqz=2, Nw=5),      # one neighbour
    Dims(NA=5, NB=2, Norb=10, NE=24, Nkz=3, Nqz=2, Nw=7),
    Dims(NA=6, NB=3, Norb=1, NE=40, Nkz=1, Nqz=1, Nw=9),      # Norb = 1, single kz point
], ids=lambda d: f"NB{d.NB}_Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}")
def test_shapes_vs_oracle(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 500, nbr=nbr)
    W, V = make_upstream(dims, seed=dims.Norb + 501)
    got = gpu(inp, W, V, check=True)
    ref = orc(inp, W, V)
    for x, y in zip(got, ref):
        assert normwise(x.cpu().numpy(), y) <= TOL


def test_atom_range_scale_and_symmetrize():
    inp = make_inputs(TINY, seed=51)
    W, V = make_upstream(TINY, seed=52)
    got = gpu(inp, W, V, atoms=(4, 10), scale=1.0)
    ref = orc(inp, W, V, scale=1.0, a_range=(4, 10))
    for x, y in zip(got, ref):
        assert normwise(x.cpu().numpy(), y) <= TOL
    proj = lambda X: 0.5 * (X - X.conj().transpose(-1, -2))
    got = gpu(inp, W, V, symmetrize=True)
    ref = orc(inp, proj(W), proj(V))
    for x, y in zip(got, ref):
        assert normwise(x.cpu().numpy(), y) <= TOL


def test_bad_neighbour_is_reported():
    inp = make_inputs(TINY, seed=53)
    W, V = make_upstream(TINY, seed=54)
    inp.nbr[2, 1] = -3
    with pytest.raises(B.SseError) as e:
        gpu(inp, W, V, check=True)
    assert e.value.status == 5
    torch.cuda.synchronize()


def test_autograd_all_inputs():
    d = Dims(NA=6, NB=2, Norb=3, NE=20, Nkz=3, Nqz=2, Nw=4)
    inp = make_inputs(d, seed=55, nbr=ring_neighbours(6, 2))
    W, V = make_upstream(d, seed=56)
    g = inp.to("cuda")
    leaves = [t.clone().requires_grad_(True) for t in (g.dH, g.D_less, g.D_greater, g.G_less, g.G_greater)]
    Sl, Sg = B.sigma_autograd(*leaves, g.nbr, SCALE, "fp64_fft")
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V)
    ref = tuple(ref) + tuple(orc(inp, W, V))
    for leaf, r in zip(leaves, ref):
        assert normwise(leaf.grad.cpu().numpy(), r) <= TOL


def test_adjoint_workload_dot_product():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16: Re <grad_G, dG> = L(dG) with the GPU forward."""
    inp = make_inputs(ADJOINT, seed=57, device="cuda")
    W, V = make_upstream(ADJOINT, seed=58, device="cuda")
    gl, gg = B.sigma_grad_G(inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V, check=True)
    gen = torch.Generator(device="cuda").manual_seed(59)
    dl = torch.complex(torch.randn(ADJOINT.g_shape(), generator=gen, dtype=torch.float64, device="cuda"),
                       torch.randn(ADJOINT.g_shape(), generator=gen, dtype=torch.float64, device="cuda"))
    dg = torch.complex(torch.randn(ADJOINT.g_shape(), generator=gen, dtype=torch.float64, device="cuda"),
                       torch.randn(ADJOINT.g_shape(), generator=gen, dtype=torch.float64, device="cuda"))
    Sl, Sg = B.sigma(dl, dg, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="fp64_fft")
    lhs = float((W.conj() * Sl).real.sum() + (V.conj() * Sg).real.sum())
    rhs = float((gl.conj() * dl).real.sum() + (gg.conj() * dg).real.sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs), (lhs, rhs)


# mode FP32_FFT: FP32 transforms and block products (per-frequency relative error ~1e-7); stated bound 1e-5,
# as for the FP32 adjoint of sse_sigma_bwd
FP32_BOUND = 1e-5


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=7, NB=2, Norb=3, NE=61, Nkz=4, Nqz=3, Nw=5),
    Dims(NA=5, NB=2, Norb=10, NE=24, Nkz=3, Nqz=2, Nw=7),
    Dims(NA=6, NB=3, Norb=1, NE=40, Nkz=1, Nqz=1, Nw=9),
], ids=lambda d: f"NB{d.NB}_Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}")
def test_fp32_vs_oracle(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=dims.Norb + 520, nbr=nbr)
    W, V = make_upstream(dims, seed=dims.Norb + 521)
    got = gpu(inp, W, V, check=True, mode="fp32_fft")
    ref = orc(inp, W, V)
    errs = [normwise(x.cpu().numpy(), y) for x, y in zip(got, ref)]
    print("fp32 grad G", dims, errs)
    assert max(errs) <= FP32_BOUND


def test_fp32_adjoint_workload_vs_fp64():
    inp = make_inputs(ADJOINT, seed=60, device="cuda")
    W, V = make_upstream(ADJOINT, seed=61, device="cuda")
    args = (inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V)
    got = B.sigma_grad_G(*args, check=True, mode="fp32_fft")
    ref = B.sigma_grad_G(*args)
    errs = [float((x - y).abs().max() / y.abs().max()) for x, y in zip(got, ref)]
    print("fp32 grad G at the adjoint workload", errs)
    assert max(errs) <= FP32_BOUND
