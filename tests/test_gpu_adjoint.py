"""FP64 adjoint (sse_sigma_bwd) against the oracle's adjoint and finite differences.

Tolerance: normwise 1e-12 per gradient tensor against the oracle (FP64 on
both sides). Finite differences of the GPU forward are exact up to round-off
(L is linear in D and quadratic in dH), checked to 1e-7 of the gradient scale.
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from oracle.subproblem import extract
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import ADJOINT, TINY, Dims, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def oracle_grad(inp, W, V, **kw):
    return oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V,
                             **kw)


def gpu_grad(inp, W, V, **kw):
    g = inp.to("cuda")
    return B.sigma_grad(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, W.cuda(), V.cuda(), scale=SCALE,
                        check=True, **kw)


@pytest.mark.parametrize("dims", [
    TINY,
    Dims(NA=6, NB=3, Norb=3, NE=29, Nkz=4, Nqz=3, Nw=5),
    Dims(NA=5, NB=2, Norb=10, NE=23, Nkz=3, Nqz=2, Nw=7),
    Dims(NA=3, NB=2, Norb=16, NE=45, Nkz=2, Nqz=2, Nw=37),   # frequency chunks in both kernels
], ids=lambda d: f"Norb{d.Norb}_NE{d.NE}_Nw{d.Nw}")
def test_gradients_match_oracle(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=31, nbr=nbr)
    W, V = make_upstream(dims, seed=32)
    ref = oracle_grad(inp, W.numpy(), V.numpy())
    got = gpu_grad(inp, W, V)
    for name, r, g in zip(("dH", "D<", "D>"), ref, got):
        assert normwise(g.cpu().numpy(), r) <= TOL, name


def test_symmetrize_projects_upstream():
    inp = make_inputs(TINY, seed=33)
    W, V = make_upstream(TINY, seed=34)
    proj = [0.5 * (x - x.conj().transpose(-1, -2)) for x in (W, V)]
    ref = oracle_grad(inp, proj[0].numpy(), proj[1].numpy())
    got = gpu_grad(inp, W, V, symmetrize=True)
    for r, g in zip(ref, got):
        assert normwise(g.cpu().numpy(), r) <= TOL


def test_atom_range():
    inp = make_inputs(TINY, seed=35)
    W, V = make_upstream(TINY, seed=36)
    ref = oracle_grad(inp, W.numpy(), V.numpy(), a_range=(3, 9))
    got = gpu_grad(inp, W, V, atoms=(3, 9))
    assert normwise(got[0].cpu().numpy()[3:9], ref[0][3:9]) <= TOL
    assert normwise(got[1].cpu().numpy()[:, :, 3:9], ref[1][:, :, 3:9]) <= TOL
    assert float(got[0][:3].abs().max()) == 0 and float(got[2][:, :, 9:].abs().max()) == 0


def test_autograd_function():
    """SigmaFunction's backward equals the oracle gradient of sum Re <W, S<> + Re <V, S>>."""
    inp = make_inputs(TINY, seed=37)
    W, V = make_upstream(TINY, seed=38)
    g = inp.to("cuda")
    dH = g.dH.clone().requires_grad_(True)
    Dl = g.D_less.clone().requires_grad_(True)
    Dg = g.D_greater.clone().requires_grad_(True)
    Sl, Sg = B.sigma_autograd(dH, Dl, Dg, g.G_less, g.G_greater, g.nbr, SCALE)
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    ref = oracle_grad(inp, W.numpy(), V.numpy())
    for r, t in zip(ref, (dH.grad, Dl.grad, Dg.grad)):
        assert normwise(t.cpu().numpy(), r) <= TOL


def _loss_atom(g, W, V, a):
    Sl, Sg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, scale=SCALE, atoms=(a, a + 1))
    return float((W[:, :, a].conj() * Sl[:, :, a]).real.sum() + (V[:, :, a].conj() * Sg[:, :, a]).real.sum())


def test_adjoint_workload_fd_and_oracle():
    """NA=256, Norb=10, NE=256, Nkz=Nqz=5, Nw=16: GPU gradient vs central differences of
    the GPU forward on 64 random coordinates (h = 1e-6) and vs the oracle gradient of
    sampled atoms."""
    d = ADJOINT
    inp = make_inputs(d, seed=1, device="cuda")
    W, V = make_upstream(d, seed=1, device="cuda")
    g_dH, g_Dl, g_Dg = B.sigma_grad(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V,
                                    scale=SCALE, check=True)
    torch.cuda.synchronize()
    grads = {"dH": g_dH, "D_less": g_Dl, "D_greater": g_Dg}
    gscale = max(float(x.abs().max()) for x in grads.values())
    rng = np.random.default_rng(2)
    sizes = np.array([inp.dH.numel(), inp.D_less.numel(), inp.D_greater.numel()], dtype=np.float64)
    h = 1e-6
    for _ in range(64):
        name = ("dH", "D_less", "D_greater")[rng.choice(3, p=sizes / sizes.sum())]
        base = getattr(inp, name)
        flat = int(rng.integers(base.numel()))
        part = int(rng.integers(2))
        idx = np.unravel_index(flat, tuple(base.shape))
        a = int(idx[0]) if name == "dH" else int(idx[2])
        step = h if part == 0 else 1j * h
        orig = base.view(-1)[flat].item()
        base.view(-1)[flat] = orig + step
        lp = _loss_atom(inp, W, V, a)
        base.view(-1)[flat] = orig - step
        lm = _loss_atom(inp, W, V, a)
        base.view(-1)[flat] = orig
        fd = (lp - lm) / (2 * h)
        an = grads[name].view(-1)[flat].item()
        an = an.real if part == 0 else an.imag
        assert abs(fd - an) <= 1e-7 * gscale, (name, idx, part, fd, an)
    # oracle gradient on sampled atoms (sub-problem: the atom, its neighbours, all energies)
    for a in (0, 131, 255):
        args, _ = extract(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, a, 0, d.NE)
        Wl = torch.zeros_like(args[4])
        Vl = torch.zeros_like(args[5])
        Wl[:, :, 0] = W[:, :, a].cpu()
        Vl[:, :, 0] = V[:, :, a].cpu()
        r_dH, r_Dl, r_Dg = oracle.sigma_grad(*args, SCALE, Wl, Vl, a_range=(0, 1))
        assert normwise(g_dH[a].cpu().numpy(), r_dH[0]) <= TOL
        assert normwise(g_Dl[:, :, a].cpu().numpy(), r_Dl[:, :, 0]) <= TOL
        assert normwise(g_Dg[:, :, a].cpu().numpy(), r_Dg[:, :, 0]) <= TOL
