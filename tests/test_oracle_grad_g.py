"""Pins of the oracle's gradient with respect to G (adjoint of Eq. 3 in its G argument).

Sigma is linear in G, so L(G) = sum_t Re tr(W^t^H Sigma^t(G)) equals Re <grad_G, G> exactly: the
dot-product test and central differences (no O(h^2) term) check every index of the gradient against the
forward oracle, which is pinned separately.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1912_10024_gb300.inputs import Dims, make_inputs, make_upstream, ring_neighbours

SCALE = 1.0 / (2.0 * np.pi)


def two_way_ring(NA):
    return torch.tensor([[(a + 1) % NA, (a - 1) % NA] for a in range(NA)], dtype=torch.int32)


def loss(inp, Gl, Gg, W, V, a_range=None):
    Sl, Sg = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, Gl, Gg, SCALE, a_range=a_range)
    return float(np.real(np.vdot(W.numpy(), Sl)) + np.real(np.vdot(V.numpy(), Sg)))


@pytest.fixture(scope="module", params=["ring", "two_way_ring"])
def problem(request):
    d = Dims(NA=6, NB=2, Norb=3, NE=11, Nkz=3, Nqz=2, Nw=3)
    nbr = ring_neighbours(6, 2) if request.param == "ring" else two_way_ring(6)
    inp = make_inputs(d, seed=41, nbr=nbr)
    W, V = make_upstream(d, seed=42)
    gGl, gGg = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V)
    return d, inp, W, V, gGl, gGg


def test_dot_product(problem):
    d, inp, W, V, gGl, gGg = problem
    g = torch.Generator().manual_seed(43)
    dl = torch.complex(torch.randn(d.g_shape(), generator=g, dtype=torch.float64),
                       torch.randn(d.g_shape(), generator=g, dtype=torch.float64))
    dg = torch.complex(torch.randn(d.g_shape(), generator=g, dtype=torch.float64),
                       torch.randn(d.g_shape(), generator=g, dtype=torch.float64))
    lhs = loss(inp, dl, dg, W, V)
    rhs = float(np.real(np.vdot(gGl, dl.numpy())) + np.real(np.vdot(gGg, dg.numpy())))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))


def test_central_differences(problem):
    d, inp, W, V, gGl, gGg = problem
    rng = np.random.default_rng(44)
    h = 1e-3  # L is linear in G: the difference quotient is exact up to rounding
    scale = max(np.abs(gGl).max(), np.abs(gGg).max())
    for _ in range(12):
        t = int(rng.integers(2))
        idx = tuple(int(rng.integers(n)) for n in d.g_shape())
        part = int(rng.integers(2))
        step = h if part == 0 else 1j * h
        G = [inp.G_less.clone(), inp.G_greater.clone()]
        G[t][idx] += step
        lp = loss(inp, G[0], G[1], W, V)
        G[t][idx] -= 2 * step
        lm = loss(inp, G[0], G[1], W, V)
        fd = (lp - lm) / (2 * h)
        an = (gGl, gGg)[t][idx]
        an = an.real if part == 0 else an.imag
        assert abs(fd - an) <= 1e-9 * scale, (t, idx, part, fd, an)


def test_atom_range(problem):
    """Only bonds of atoms in range contribute: the gradient of the loss restricted to those rows."""
    d, inp, W, V, _, _ = problem
    gl, gg = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V, a_range=(2, 4))
    g = torch.Generator().manual_seed(45)
    dl = torch.complex(torch.randn(d.g_shape(), generator=g, dtype=torch.float64),
                       torch.randn(d.g_shape(), generator=g, dtype=torch.float64))
    Wr, Vr = torch.zeros_like(W), torch.zeros_like(V)
    Wr[:, :, 2:4], Vr[:, :, 2:4] = W[:, :, 2:4], V[:, :, 2:4]
    lhs = loss(inp, dl, torch.zeros_like(dl), Wr, Vr)
    rhs = float(np.real(np.vdot(gl, dl.numpy())))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, abs(lhs))
