"""The sub-problem cutter behind the sampled checks of large workloads: Sigma of one atom on an energy window,
evaluated by the oracle on the cut-out problem (the atom, its neighbours, the window +- Nw), equals the unsharded
oracle's blocks bit for bit (the same terms in the same order), at the grid edges and inside."""
import math

import numpy as np
import pytest

import oracle
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300.inputs import Dims, diamond_neighbours, make_inputs

SCALE = 1.0 / (2.0 * math.pi)


@pytest.mark.parametrize("d,nbr", [
    (Dims(NA=9, NB=3, Norb=2, NE=40, Nkz=3, Nqz=2, Nw=6), None),
    (Dims(NA=16, NB=4, Norb=3, NE=25, Nkz=2, Nqz=2, Nw=4), diamond_neighbours(1, 1, 2)),
], ids=["ring", "diamond16"])
def test_cut_out_blocks_equal_the_full_oracle(d, nbr):
    x = make_inputs(d, seed=33, nbr=nbr)
    args = (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater)
    Sl, Sg = oracle.sigma(*args, SCALE)
    for a, E0, E1 in ((0, 0, 7), (d.NA - 1, d.NE - 5, d.NE), (d.NA // 2, 10, 13), (3, 0, d.NE)):
        bl, bg = oracle_blocks(*args, SCALE, a, E0, E1)
        assert np.array_equal(bl, Sl[:, E0:E1, a]) and np.array_equal(bg, Sg[:, E0:E1, a]), (a, E0, E1)
