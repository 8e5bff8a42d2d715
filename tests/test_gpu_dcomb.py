"""Bond weights D_ba - D_bb - D_aa + D_ab (sse_dcomb_fwd / sse_dcomb_bwd) against the oracle.

The forward does the same three FP64 subtractions/additions in the same order
as the oracle, so it must match bit for bit; the adjoint adds the same terms in
another order (normwise 1e-15).
"""
import math

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import Dims, diamond_neighbours, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)


def two_way_ring(NA):
    return torch.tensor([[(a + 1) % NA, (a - 1) % NA] for a in range(NA)], dtype=torch.int32)


def rand_raw(shape, seed):
    g = torch.Generator().manual_seed(seed)
    return torch.complex(torch.randn(shape, generator=g, dtype=torch.float64),
                         torch.randn(shape, generator=g, dtype=torch.float64))


@pytest.mark.parametrize("nbr", [diamond_neighbours(2, 2, 4), two_way_ring(9), diamond_neighbours(4, 4, 8)],
                         ids=["diamond128", "two_way_ring", "diamond1024"])
def test_forward_bit_exact_and_adjoint(nbr):
    NA, NB = nbr.shape
    Nqz, Nw = (7, 32) if NA == 1024 else (3, 5)
    raw_l, raw_g = rand_raw((Nqz, Nw, NA, NB + 1, 3, 3), 1), rand_raw((Nqz, Nw, NA, NB + 1, 3, 3), 2)
    Dl, Dg = B.dcomb(raw_l.cuda(), raw_g.cuda(), nbr.cuda(), check=True)
    Ol, Og = oracle.dcomb(nbr, raw_l, raw_g)
    assert np.array_equal(Dl.cpu().numpy(), Ol) and np.array_equal(Dg.cpu().numpy(), Og)
    gl, gg = rand_raw(Ol.shape, 3), rand_raw(Ol.shape, 4)
    rl, rg = B.dcomb_grad(gl.cuda(), gg.cuda(), nbr.cuda(), check=True)
    Rl, Rg = oracle.dcomb_adjoint(nbr, gl, gg)
    assert normwise(rl.cpu().numpy(), Rl) <= 1e-15 and normwise(rg.cpu().numpy(), Rg) <= 1e-15


def test_atom_range():
    nbr = diamond_neighbours(2, 2, 4)
    raw = rand_raw((2, 3, 128, 5, 3, 3), 5)
    Dl, _ = B.dcomb(raw.cuda(), raw.cuda(), nbr.cuda(), atoms=(10, 40))
    Ol, _ = oracle.dcomb(nbr, raw, raw, a_range=(10, 40))
    assert np.array_equal(Dl.cpu().numpy(), Ol)


def test_one_way_list_is_reported():
    nbr = ring_neighbours(8, 2)
    raw = rand_raw((1, 2, 8, 3, 3, 3), 6).cuda()
    with pytest.raises(B.SseError) as e:
        B.dcomb(raw, raw, nbr.cuda(), check=True)
    assert e.value.status == 5


def test_raw_phonon_gf_to_sigma_with_autograd():
    """Raw D -> bond weights -> Sigma (FP64) and the chained gradients w.r.t. the raw D,
    against the oracle's forward and adjoint composed the same way."""
    d = Dims(NA=16, NB=4, Norb=3, NE=20, Nkz=3, Nqz=3, Nw=4)
    # symmetric 4-slot list on 16 atoms (a +- 1, a +- 4)
    nbr = torch.tensor([[(a + 1) % 16, (a - 1) % 16, (a + 4) % 16, (a - 4) % 16] for a in range(16)], dtype=torch.int32)
    inp = make_inputs(d, seed=7, nbr=nbr)
    raw_l, raw_g = rand_raw((3, 4, 16, 5, 3, 3), 8) * 0.01, rand_raw((3, 4, 16, 5, 3, 3), 9) * 0.01
    W, V = make_upstream(d, seed=10)
    g = inp.to("cuda")
    rl = raw_l.cuda().requires_grad_(True)
    rg = raw_g.cuda().requires_grad_(True)
    Dl, Dg = B.DcombFunction.apply(rl, rg, g.nbr)
    Sl, Sg = B.sigma_autograd(g.dH, Dl, Dg, g.G_less, g.G_greater, g.nbr, SCALE)
    loss = (W.cuda().conj() * Sl).real.sum() + (V.cuda().conj() * Sg).real.sum()
    loss.backward()
    ODl, ODg = oracle.dcomb(nbr, raw_l, raw_g)
    OSl, OSg = oracle.sigma(nbr, inp.dH, ODl, ODg, inp.G_less, inp.G_greater, SCALE)
    assert normwise(Sl.detach().cpu().numpy(), OSl) <= 1e-12
    _, gDl, gDg = oracle.sigma_grad(nbr, inp.dH, ODl, ODg, inp.G_less, inp.G_greater, SCALE, W, V)
    Rl, Rg = oracle.dcomb_adjoint(nbr, gDl, gDg)
    assert normwise(rl.grad.cpu().numpy(), Rl) <= 1e-12
    assert normwise(rg.grad.cpu().numpy(), Rg) <= 1e-12
