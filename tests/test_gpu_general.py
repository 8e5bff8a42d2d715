"""Every entry point on GENERAL inputs: G^<, G^> and the 3x3 D blocks with no symmetry at all.

Lesser and greater functions are anti-Hermitian, and most tests feed such inputs. A kernel that quietly
used G^H = -G or D^H = -D (outside SSE_FLAG_ANTIHERMITIAN) would pass those tests and fail these: here
every result is compared element by element with the FP64 oracle, which takes G and D as given.

Bounds (normwise max|gpu - oracle| / max|oracle| per output tensor), the same as each mode's own tests:
FP64 and FP64_FFT 1e-12; FP32_FFT 2e-6 (forward, Pi), 1e-5 (adjoint, G-gradient); F16X3_FFT 2e-6; BF16X3 2e-5;
TF32 2e-3.
Shapes: the tiny workload, and Norb = 10 with ragged energy tiles and Nqz < Nkz.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, Dims, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
NORB10 = Dims(NA=5, NB=2, Norb=10, NE=40, Nkz=3, Nqz=2, Nw=11)
SHAPES = [TINY, NORB10]
FWD_BOUND = {"fp64": 1e-12, "fp64_fft": 1e-12, "fp32_fft": 2e-6, "f16x3_fft": 2e-6, "bf16x3": 2e-5, "tf32": 2e-3}
BWD_BOUND = {"fp64": 1e-12, "fp64_fft": 1e-12, "fp32_fft": 1e-5}


def _general(dims, seed):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=seed, nbr=nbr, general=True)
    # the inputs really are general: neither G nor D is anti-Hermitian
    for X in (inp.G_less, inp.G_greater, inp.D_less, inp.D_greater):
        assert float((X + X.conj().transpose(-1, -2)).abs().max()) > 0.1 * float(X.abs().max())
    return inp


def _ids(d):
    return f"NA{d.NA}_Norb{d.Norb}_NE{d.NE}_Nkz{d.Nkz}_Nqz{d.Nqz}"


@pytest.mark.parametrize("dims", SHAPES, ids=_ids)
@pytest.mark.parametrize("mode", list(FWD_BOUND))
def test_forward(dims, mode):
    inp = _general(dims, seed=1000 + dims.Norb)
    g = inp.to("cuda")
    S = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode, check=True)
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    errs = [normwise(s.cpu().numpy(), o) for s, o in zip(S, O)]
    print(mode, dims, errs)
    assert max(errs) <= FWD_BOUND[mode], errs


@pytest.mark.parametrize("mode", ["fp64_fft", "fp32_fft", "f16x3_fft"])
def test_host_buffer_forward(mode):
    inp = _general(NORB10, seed=1100)
    pin = [t.pin_memory() for t in (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr)]
    S = B.sigma_host(*pin, mode=mode, check=True)
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    for s, o in zip(S, O):
        assert normwise(s.numpy(), o) <= FWD_BOUND[mode]


@pytest.mark.parametrize("dims", SHAPES, ids=_ids)
@pytest.mark.parametrize("mode", list(BWD_BOUND))
def test_adjoint(dims, mode):
    inp = _general(dims, seed=1200 + dims.Norb)
    W, V = make_upstream(dims, seed=1201)
    g = inp.to("cuda")
    got = B.sigma_grad(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, W.cuda(), V.cuda(), mode=mode,
                       check=True)
    ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V)
    errs = [normwise(x.cpu().numpy(), y) for x, y in zip(got, ref)]
    print(mode, dims, errs)
    assert max(errs) <= BWD_BOUND[mode], errs


@pytest.mark.parametrize("dims", SHAPES, ids=_ids)
@pytest.mark.parametrize("mode", ["fp64_fft", "fp32_fft"])
def test_gradient_in_G(dims, mode):
    inp = _general(dims, seed=1300 + dims.Norb)
    W, V = make_upstream(dims, seed=1301)
    g = inp.to("cuda")
    got = B.sigma_grad_G(g.dH, g.D_less, g.D_greater, g.nbr, W.cuda(), V.cuda(), mode=mode, check=True)
    ref = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V)
    errs = [normwise(x.cpu().numpy(), y) for x, y in zip(got, ref)]
    assert max(errs) <= BWD_BOUND[mode], errs


@pytest.mark.parametrize("dims", SHAPES, ids=_ids)
@pytest.mark.parametrize("mode,bound", [("fp64_fft", 1e-12), ("fp32_fft", 2e-6)])
def test_pi(dims, mode, bound):
    inp = _general(dims, seed=1400 + dims.Norb)
    g = inp.to("cuda")
    P = B.pi(g.G_less, g.G_greater, g.dH, g.nbr, dims.Nqz, dims.Nw, mode=mode, check=True)
    O = oracle.pi(inp.nbr, inp.dH, inp.G_less, inp.G_greater, SCALE, dims.Nqz, dims.Nw)
    for p, o in zip(P, O):
        assert normwise(p.cpu().numpy(), o) <= bound


@pytest.mark.parametrize("mode", ["fp64", "fp64_fft"])
def test_autograd_every_input(mode):
    """SigmaFunction on general inputs: gradients for dH, D^<, D^>, G^<, G^> against the oracle."""
    inp = _general(NORB10, seed=1500)
    W, V = make_upstream(NORB10, seed=1501)
    g = inp.to("cuda")
    leaves = [t.clone().requires_grad_(True) for t in (g.dH, g.D_less, g.D_greater, g.G_less, g.G_greater)]
    Sl, Sg = B.sigma_autograd(*leaves, g.nbr, SCALE, mode)
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    ref = tuple(oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V))
    ref += tuple(oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V))
    for name, leaf, r in zip(("dH", "D<", "D>", "G<", "G>"), leaves, ref):
        assert normwise(leaf.grad.cpu().numpy(), r) <= 1e-12, name


def test_antihermitian_flag_rejects_general_inputs():
    """With SSE_FLAG_ANTIHERMITIAN and CHECK, general inputs are reported, not silently mirrored."""
    inp = _general(TINY, seed=1600)
    g = inp.to("cuda")
    with pytest.raises(B.SseError) as e:
        B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp64_fft", check=True,
                antihermitian=True)
    assert e.value.status == 5
    torch.cuda.synchronize()  # the context stays usable
    S = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp64_fft", check=True)
    O = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    assert normwise(S[0].cpu().numpy(), O[0]) <= 1e-12
    assert not np.allclose(O[0], -np.swapaxes(O[0].conj(), -1, -2))  # Sigma itself is not anti-Hermitian
