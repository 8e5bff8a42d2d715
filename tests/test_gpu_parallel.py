"""The composed sharded calls on the GPU: parallel.sigma_atom_sharded, sigma_grad_atom_sharded,
sigma_grad_G_atom_sharded, pi_atom_sharded and sigma_energy_sharded with their default evaluation (the library calls) on a one-rank process group equal the direct
library calls bit for bit (the local problem is the global one)."""
import math
import socket

import pytest
import torch
import torch.distributed as dist

from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300 import parallel as P
from paper_1912_10024_gb300.inputs import Dims, diamond_neighbours, make_inputs, make_upstream

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)


def test_single_rank_equals_the_library_call():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1)
    try:
        d = Dims(NA=16, NB=4, Norb=3, NE=20, Nkz=3, Nqz=2, Nw=4)
        g = make_inputs(d, seed=81, nbr=diamond_neighbours(1, 1, 2)).to("cuda")
        Sl, Sg = P.sigma_atom_sharded(g.nbr, g.dH, (g.D_less, g.D_greater), (g.G_less, g.G_greater), d.NA, SCALE,
                                      mode="fp64_fft")
        Rl, Rg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, scale=SCALE, mode="fp64_fft")
        assert torch.equal(Sl, Rl) and torch.equal(Sg, Rg)
        W, V = make_upstream(d, seed=82, device="cuda")
        gl, gg = P.sigma_grad_G_atom_sharded(g.nbr, g.dH, (g.D_less, g.D_greater), (W, V), d.NA, SCALE,
                                             mode="fp64_fft")
        rl, rg = B.sigma_grad_G(g.dH, g.D_less, g.D_greater, g.nbr, W, V, scale=SCALE, mode="fp64_fft")
        assert torch.equal(gl, rl) and torch.equal(gg, rg)
        ga = P.sigma_grad_atom_sharded(g.nbr, g.dH, (g.D_less, g.D_greater), (g.G_less, g.G_greater), (W, V), d.NA,
                                       SCALE)
        gr = B.sigma_grad(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, W, V, scale=SCALE)
        assert all(torch.equal(x, y) for x, y in zip(ga, gr))
        Pl, Pg = P.pi_atom_sharded(g.nbr, g.dH, (g.G_less, g.G_greater), d.NA, d.Nqz, d.Nw, SCALE)
        Ql, Qg = B.pi(g.G_less, g.G_greater, g.dH, g.nbr, d.Nqz, d.Nw, scale=SCALE)
        assert torch.equal(Pl, Ql) and torch.equal(Pg, Qg)
        El, Eg = P.sigma_energy_sharded(g.nbr, g.dH, (g.D_less, g.D_greater), (g.G_less, g.G_greater), d.NE, SCALE,
                                        mode="fp64_fft")
        assert torch.equal(El, Rl) and torch.equal(Eg, Rg)
    finally:
        dist.destroy_process_group()
