"""Pins of the oracle's adjoint against its (pinned) forward.

L = sum_t Re tr(W^t^H Sigma^t) is linear in Dc and quadratic in dH, so a
central finite difference in FP64 has no truncation error: it matches the
gradient up to round-off only. Gradients use the PyTorch convention for
complex leaves (grad = dL/dRe z + i dL/dIm z), so for a real perturbation
direction e of Re z the directional derivative is Re(grad) and for Im z it is
Im(grad).
"""
import numpy as np
import pytest

import oracle
from paper_1912_10024_gb300.inputs import Dims, make_inputs, make_upstream, ring_neighbours

SCALE = 1.0 / (2.0 * np.pi)
D = Dims(NA=5, NB=2, Norb=3, NE=8, Nkz=3, Nqz=2, Nw=2)


def loss(inp, W, V):
    Sl, Sg = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    return float(np.real(np.vdot(W, Sl)) + np.real(np.vdot(V, Sg)))


def make_problem(general=False):
    inp = make_inputs(D, seed=21, nbr=ring_neighbours(D.NA, D.NB), general=general)
    W, V = (x.numpy() for x in make_upstream(D, seed=22))
    g = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V)
    return inp, W, V, g


@pytest.fixture(scope="module", params=[False, True], ids=["antihermitian", "general"])
def problem(request):
    return make_problem(request.param)


def test_gradient_central_differences(problem):
    inp, W, V, (g_dH, g_Dl, g_Dg) = problem
    rng = np.random.default_rng(2)
    fields = [("dH", g_dH), ("D_less", g_Dl), ("D_greater", g_Dg)]
    h = 1e-6
    scale_ref = max(np.abs(g).max() for _, g in fields)
    for _ in range(24):
        name, g = fields[rng.integers(3)]
        flat = rng.integers(g.size)
        part = rng.integers(2)  # 0: real part, 1: imaginary part
        step = h if part == 0 else 1j * h
        base = getattr(inp, name)
        plus, minus = base.clone(), base.clone()
        plus.view(-1)[flat] += step
        minus.view(-1)[flat] -= step
        setattr(inp, name, plus)
        lp = loss(inp, W, V)
        setattr(inp, name, minus)
        lm = loss(inp, W, V)
        setattr(inp, name, base)
        fd = (lp - lm) / (2 * h)
        an = g.reshape(-1)[flat]
        an = an.real if part == 0 else an.imag
        assert abs(fd - an) <= 1e-7 * scale_ref, (name, flat, part, fd, an)


def test_dot_product_in_D(problem):
    """L is linear in Dc: L(Dc + dD) - L(Dc) = Re<g_D, dD> exactly (up to round-off)."""
    inp, W, V, (_, g_Dl, g_Dg) = problem
    rng = np.random.default_rng(3)
    dl = rng.standard_normal(g_Dl.shape) + 1j * rng.standard_normal(g_Dl.shape)
    dg = rng.standard_normal(g_Dg.shape) + 1j * rng.standard_normal(g_Dg.shape)
    l0 = loss(inp, W, V)
    import torch
    import copy
    inp2 = copy.copy(inp)  # same G, dH and neighbours
    inp2.D_less = inp.D_less + torch.from_numpy(dl)
    inp2.D_greater = inp.D_greater + torch.from_numpy(dg)
    l1 = loss(inp2, W, V)
    pred = np.real(np.vdot(g_Dl, dl)) + np.real(np.vdot(g_Dg, dg))
    assert abs((l1 - l0) - pred) <= 1e-12 * max(1.0, abs(pred))


def test_dot_product_in_dH(problem):
    """L is a Hermitian quadratic form in dH: L(dH + e) - L(dH - e) = 2 Re<g_dH, e>."""
    inp, W, V, (g_dH, _, _) = problem
    rng = np.random.default_rng(4)
    e = 0.01 * (rng.standard_normal(g_dH.shape) + 1j * rng.standard_normal(g_dH.shape))
    import torch
    base = inp.dH
    inp.dH = base + torch.from_numpy(e)
    lp = loss(inp, W, V)
    inp.dH = base - torch.from_numpy(e)
    lm = loss(inp, W, V)
    inp.dH = base
    pred = 2 * np.real(np.vdot(g_dH, e))
    assert abs((lp - lm) - pred) <= 1e-12 * max(1.0, abs(pred))


def test_atom_range_gradients(problem):
    inp, W, V, (g_dH, g_Dl, g_Dg) = problem
    p = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V,
                          a_range=(1, 3))
    np.testing.assert_array_equal(p[0][1:3], g_dH[1:3])
    np.testing.assert_array_equal(p[1][:, :, 1:3], g_Dl[:, :, 1:3])
    assert np.count_nonzero(p[0][3:]) == 0 and np.count_nonzero(p[2][:, :, :1]) == 0


@pytest.mark.parametrize("d", [
    Dims(NA=4, NB=1, Norb=1, NE=6, Nkz=1, Nqz=1, Nw=5),     # scalar blocks, one kz, Nw = NE - 1
    Dims(NA=7, NB=3, Norb=5, NE=11, Nkz=4, Nqz=2, Nw=3),    # Nqz < Nkz, ragged sizes
    Dims(NA=3, NB=2, Norb=2, NE=2, Nkz=5, Nqz=5, Nw=1),     # the shortest energy grid
], ids=["scalar_all_lags", "ragged", "two_energies"])
@pytest.mark.parametrize("general", [False, True], ids=["antihermitian", "general"])
def test_euler_identities_on_edge_shapes(d, general):
    """L is linear in (D^<, D^>) jointly, linear in (G^<, G^>) jointly and a Hermitian quadratic form in dH, so
    Euler's theorem for homogeneous functions fixes L = Re<g_D, D> = Re<g_G, G> = Re<g_dH, dH> / 2 exactly: every
    gradient entry weighted by its own input, on shapes at the edges of the index ranges."""
    inp = make_inputs(d, seed=77, general=general)
    W, V = (x.numpy() for x in make_upstream(d, seed=78))
    args = (inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE)
    g_dH, g_Dl, g_Dg = oracle.sigma_grad(*args, W, V)
    g_Gl, g_Gg = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V)
    L = loss(inp, W, V)
    dot = lambda g, x: float(np.real(np.vdot(g, x.numpy())))  # noqa: E731
    for got in (dot(g_Dl, inp.D_less) + dot(g_Dg, inp.D_greater), dot(g_Gl, inp.G_less) + dot(g_Gg, inp.G_greater),
                dot(g_dH, inp.dH) / 2):
        assert abs(got - L) <= 1e-12 * abs(L), (got, L)
