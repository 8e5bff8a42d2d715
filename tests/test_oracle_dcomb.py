"""Pins of the oracle's bond-weight combination D_ba - D_bb - D_aa + D_ab (Eq. 3).

A hand-derived example, the exchange symmetry of the combination, the
vanishing for uniform blocks, an exact adjoint dot-product test and the
refusal of one-way neighbour lists.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1912_10024_gb300.inputs import diamond_neighbours, ring_neighbours

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_raw(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_worked_example():
    with open(os.path.join(GOLDEN, "dcomb_case.json")) as f:
        g = json.load(f)
    raw = np.zeros((1, 1, 2, 2, 3, 3), np.complex128)  # [q][w][a][slot][i][j]
    raw[0, 0, 0, 0, 0, 0], raw[0, 0, 0, 1, 0, 0], raw[0, 0, 1, 0, 0, 0], raw[0, 0, 1, 1, 0, 0] = 1, 2, 4, 8
    raw[0, 0, 0, 0, 1, 2], raw[0, 0, 0, 1, 1, 2], raw[0, 0, 1, 0, 1, 2], raw[0, 0, 1, 1, 1, 2] = 1j, 3, -2j, 5
    nbr = np.array([[1], [0]], np.int32)
    Dl, Dg = oracle.dcomb(nbr, raw, 2 * raw)
    for a, key in ((0, "Dc_00"), (1, "Dc_10")):
        for (i, j), e in (((0, 0), "e00"), ((1, 2), "e12")):
            want = complex(*g[key][e])
            assert Dl[0, 0, a, 0, i, j] == want
            assert Dg[0, 0, a, 0, i, j] == 2 * want
    mask = np.ones((3, 3), bool)
    mask[0, 0] = mask[1, 2] = False
    assert np.count_nonzero(Dl[0, 0, :, 0][:, mask]) == 0


def two_way_ring(NA):
    """nbr[a] = [a+1, a-1]: the reverse of slot 0 is slot 1 (unlike the diamond slab, where it is the same slot)."""
    return np.array([[(a + 1) % NA, (a - 1) % NA] for a in range(NA)], np.int32)


@pytest.mark.parametrize("kind", ["diamond", "two_way_ring"])
def test_exchange_symmetry(kind):
    """D_ba - D_bb - D_aa + D_ab is symmetric in (a, b): the two bonds of a pair get the same weight."""
    nbr = diamond_neighbours(2, 2, 4).numpy() if kind == "diamond" else two_way_ring(9)
    NA, NB = nbr.shape
    raw = rand_raw((2, 3, NA, NB + 1, 3, 3), 1)
    Dl, _ = oracle.dcomb(nbr, raw, raw)
    for a in range(NA):
        for s in range(NB):
            b = nbr[a, s]
            sr = int(np.where(nbr[b] == a)[0][0])
            np.testing.assert_allclose(Dl[:, :, a, s], Dl[:, :, b, sr], rtol=0, atol=1e-14)


def test_uniform_blocks_cancel():
    nbr = diamond_neighbours(2, 2, 4).numpy()
    block = rand_raw((3, 3), 2)
    raw = np.broadcast_to(block, (2, 2, 128, 5, 3, 3)).copy()
    Dl, Dg = oracle.dcomb(nbr, raw, raw)
    assert np.count_nonzero(Dl) == 0 and np.count_nonzero(Dg) == 0


def test_adjoint_dot_product():
    nbr = diamond_neighbours(2, 2, 4).numpy()
    raw_l, raw_g = rand_raw((2, 3, 128, 5, 3, 3), 3), rand_raw((2, 3, 128, 5, 3, 3), 4)
    gl, gg = rand_raw((2, 3, 128, 4, 3, 3), 5), rand_raw((2, 3, 128, 4, 3, 3), 6)
    Dl, Dg = oracle.dcomb(nbr, raw_l, raw_g)
    rl, rg = oracle.dcomb_adjoint(nbr, gl, gg)
    lhs = np.vdot(gl, Dl).real + np.vdot(gg, Dg).real
    rhs = np.vdot(rl, raw_l).real + np.vdot(rg, raw_g).real
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_one_way_list_is_refused():
    nbr = ring_neighbours(8, 2).numpy()  # a -> a+1, a+2 only
    raw = rand_raw((1, 1, 8, 3, 3, 3), 7)
    with pytest.raises(ValueError):
        oracle.dcomb(nbr, raw, raw)
