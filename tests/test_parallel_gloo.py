"""Atom-sharded evaluation with a halo exchange, world sizes 2 and 3 over gloo on the CPU.

Each rank owns a contiguous atom range and only its own G blocks, fetches
the halo blocks with paper_1912_10024_gb300.parallel.exchange_halo, and
evaluates its shard of Sigma (Eq. 3), of Pi (Eq. 4: the same atom halo) and
of the adjoint of Eq. (3) (gradients of its own atoms' dH and D: owned per
atom, so no reduction across ranks) with the CPU oracle. The gathered shards
must equal the unsharded oracle results bit for bit (same arithmetic, same
order).
"""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1912_10024_gb300.inputs import TINY, Dims, diamond_neighbours, make_inputs, make_upstream
from paper_1912_10024_gb300 import parallel as P

SCALE = 0.15915494309189535


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        a0, a1 = P.atom_range(dims.NA, world, rank)
        G_owned = [inp.G_less[:, :, a0:a1].clone(), inp.G_greater[:, :, a0:a1].clone()]
        halo = P.exchange_halo(G_owned, inp.nbr, dims.NA)
        assert sorted(halo) == P.halo_atoms(inp.nbr, a0, a1)
        for b, (gl, gg) in halo.items():  # received blocks are the owners' bytes
            assert torch.equal(gl, inp.G_less[:, :, b]) and torch.equal(gg, inp.G_greater[:, :, b])
        local = P.local_problem(inp.nbr, a0, a1, G_owned, halo, inp.dH[a0:a1],
                                (inp.D_less[:, :, a0:a1], inp.D_greater[:, :, a0:a1]))
        Sl, Sg = oracle.sigma(*local, SCALE, a_range=(0, a1 - a0), nthreads=2)
        Pl, Pg = oracle.pi(local[0], local[1], local[4], local[5], SCALE, dims.Nqz, dims.Nw, a_range=(0, a1 - a0),
                           nthreads=2)
        # adjoint of the shard: the upstream gradient of the owned atoms, zero on the halo atoms
        W, V = make_upstream(dims, seed=seed + 1)
        n_own = a1 - a0
        Wl, Vl = torch.zeros_like(local[4]), torch.zeros_like(local[5])
        Wl[:, :, :n_own], Vl[:, :, :n_own] = W[:, :, a0:a1], V[:, :, a0:a1]
        g_dH, g_Dl, g_Dg = oracle.sigma_grad(*local, SCALE, Wl, Vl, a_range=(0, n_own), nthreads=2)
        shard = [torch.from_numpy(X[:, :, : a1 - a0]).contiguous() for X in (Sl, Sg, Pl, Pg)]
        shard += [torch.from_numpy(g_dH[:n_own]).contiguous()] + [torch.from_numpy(X[:, :, :n_own]).contiguous()
                                                                 for X in (g_Dl, g_Dg)]
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, shard))
        if rank == 0:
            full = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                nthreads=2)
            full = tuple(full) + tuple(oracle.pi(inp.nbr, inp.dH, inp.G_less, inp.G_greater, SCALE, dims.Nqz,
                                                 dims.Nw, nthreads=2))
            grads = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                      W, V, nthreads=2)
            ok = True
            for (b0, b1, sh) in gathered:
                for t in range(4):
                    ok &= np.array_equal(sh[t].numpy(), full[t][:, :, b0:b1])
                ok &= np.array_equal(sh[4].numpy(), grads[0][b0:b1])
                for t in (1, 2):
                    ok &= np.array_equal(sh[4 + t].numpy(), grads[t][:, :, b0:b1])
            q.put(ok)
    finally:
        dist.destroy_process_group()


def _run(dims, world, seed, nbr=None):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_worker, args=(world, _free_port(), dims, seed, nbr, q), nprocs=world, join=True,
                       start_method="spawn")
    return q.get()


def test_two_ranks_ring_list():
    assert _run(TINY, 2, seed=0)


def test_two_ranks_diamond_slab():
    """Symmetric diamond-lattice neighbour list: halo atoms come from both sides."""
    d = Dims(NA=128, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2)  # 2x2x4 cells
    assert _run(d, 2, seed=5, nbr=diamond_neighbours(2, 2, 4))


def test_three_ranks_uneven_tiles():
    """World size 3 on 16 atoms (tiles of 6, 5, 5): with the diamond list each rank's halo has several owners, and
    the G-gradient's halo blocks go back to more than one rank."""
    d = Dims(NA=16, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2)
    nbr = diamond_neighbours(1, 1, 2)  # 1x1x2 cells: 16 atoms
    assert nbr.shape == (16, 4)
    assert _run(d, 3, seed=11, nbr=nbr)
    assert _run_grad_g(d, 3, seed=12, nbr=nbr)


def _composed_worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        a0, a1 = P.atom_range(dims.NA, world, rank)

        def on_cpu(Gl, Gg, dH, Dl, Dg, nbr_l, scale, atoms):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.sigma(nbr_l, dH, Dl, Dg, Gl, Gg, scale, a_range=atoms,
                                                                   nthreads=2))

        Sl, Sg = P.sigma_atom_sharded(inp.nbr, inp.dH[a0:a1], (inp.D_less[:, :, a0:a1], inp.D_greater[:, :, a0:a1]),
                                      (inp.G_less[:, :, a0:a1].clone(), inp.G_greater[:, :, a0:a1].clone()),
                                      dims.NA, SCALE, compute=on_cpu)
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, Sl.contiguous(), Sg.contiguous()))
        if rank == 0:
            full = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                nthreads=2)
            q.put(all(np.array_equal(sl.numpy(), full[0][:, :, b0:b1]) and
                      np.array_equal(sg.numpy(), full[1][:, :, b0:b1]) for b0, b1, sl, sg in gathered))
    finally:
        dist.destroy_process_group()


def test_composed_sharded_sigma():
    """parallel.sigma_atom_sharded (exchange, local problem, evaluation of the owned atoms) with the oracle as the
    evaluation: the gathered shards equal the unsharded oracle bit for bit, at world 3 on 16 atoms (uneven tiles,
    halos with several owners) and on 2 atoms (one rank owns nothing but still takes part in the exchange)."""
    ctx = mp.get_context("spawn")
    for dims, world, nbr in ((Dims(NA=16, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2), 3, diamond_neighbours(1, 1, 2)),
                             (Dims(NA=2, NB=1, Norb=2, NE=6, Nkz=2, Nqz=1, Nw=2), 3, None)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_worker, args=(world, _free_port(), dims, 13, nbr, q), nprocs=world, join=True,
                           start_method="spawn")
        assert q.get()


def _composed_adjoint_worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        W, V = make_upstream(dims, seed=seed + 1)
        a0, a1 = P.atom_range(dims.NA, world, rank)

        def on_cpu(Gl, Gg, dH, Dl, Dg, nbr_l, gl, gg, scale, atoms):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.sigma_grad(nbr_l, dH, Dl, Dg, Gl, Gg, scale, gl, gg,
                                                                        a_range=atoms, nthreads=2))

        g = P.sigma_grad_atom_sharded(inp.nbr, inp.dH[a0:a1], (inp.D_less[:, :, a0:a1], inp.D_greater[:, :, a0:a1]),
                                      (inp.G_less[:, :, a0:a1].clone(), inp.G_greater[:, :, a0:a1].clone()),
                                      (W[:, :, a0:a1], V[:, :, a0:a1]), dims.NA, SCALE, compute=on_cpu)
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, [t.contiguous() for t in g]))
        if rank == 0:
            full = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                     W, V, nthreads=2)
            ok = True
            for b0, b1, sh in gathered:
                ok &= np.array_equal(sh[0].numpy(), full[0][b0:b1])
                for t in (1, 2):
                    ok &= np.array_equal(sh[t].numpy(), full[t][:, :, b0:b1])
            q.put(ok)
    finally:
        dist.destroy_process_group()


def test_composed_sharded_adjoint():
    """parallel.sigma_grad_atom_sharded with the oracle as the evaluation: the gathered dH and D gradient rows equal
    the unsharded oracle's bit for bit (owned per atom, no reduction), at world 3 with a rank that owns nothing."""
    ctx = mp.get_context("spawn")
    for dims, world, nbr in ((Dims(NA=16, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2), 3, diamond_neighbours(1, 1, 2)),
                             (Dims(NA=2, NB=1, Norb=2, NE=6, Nkz=2, Nqz=1, Nw=2), 3, None)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_adjoint_worker, args=(world, _free_port(), dims, 18, nbr, q), nprocs=world,
                           join=True, start_method="spawn")
        assert q.get()


def _composed_pi_worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        a0, a1 = P.atom_range(dims.NA, world, rank)

        def on_cpu(Gl, Gg, dH, nbr_l, Nqz, Nw, scale, atoms):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.pi(nbr_l, dH, Gl, Gg, scale, Nqz, Nw, a_range=atoms,
                                                                nthreads=2))

        Pl, Pg = P.pi_atom_sharded(inp.nbr, inp.dH[a0:a1], (inp.G_less[:, :, a0:a1].clone(),
                                                            inp.G_greater[:, :, a0:a1].clone()),
                                   dims.NA, dims.Nqz, dims.Nw, SCALE, compute=on_cpu)
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, Pl.contiguous(), Pg.contiguous()))
        if rank == 0:
            full = oracle.pi(inp.nbr, inp.dH, inp.G_less, inp.G_greater, SCALE, dims.Nqz, dims.Nw, nthreads=2)
            q.put(all(pl.shape == full[0][:, :, b0:b1].shape and np.array_equal(pl.numpy(), full[0][:, :, b0:b1])
                      and np.array_equal(pg.numpy(), full[1][:, :, b0:b1]) for b0, b1, pl, pg in gathered))
    finally:
        dist.destroy_process_group()


def test_composed_sharded_pi():
    """parallel.pi_atom_sharded with the oracle as the evaluation: the gathered rows of Pi (Eq. 4) equal the
    unsharded oracle bit for bit at world 3, with halos of several owners and with a rank that owns nothing."""
    ctx = mp.get_context("spawn")
    for dims, world, nbr in ((Dims(NA=16, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2), 3, diamond_neighbours(1, 1, 2)),
                             (Dims(NA=2, NB=1, Norb=2, NE=6, Nkz=2, Nqz=1, Nw=2), 3, None)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_pi_worker, args=(world, _free_port(), dims, 17, nbr, q), nprocs=world,
                           join=True, start_method="spawn")
        assert q.get()


def _composed_grad_g_worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        W, V = make_upstream(dims, seed=seed + 1)
        a0, a1 = P.atom_range(dims.NA, world, rank)

        def on_cpu(dH, Dl, Dg, nbr_l, gl, gg, scale):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.sigma_grad_G(nbr_l, dH, Dl, Dg, scale, gl, gg,
                                                                          nthreads=2))

        owned = P.sigma_grad_G_atom_sharded(inp.nbr, inp.dH[a0:a1], (inp.D_less[:, :, a0:a1],
                                                                       inp.D_greater[:, :, a0:a1]),
                                            (W[:, :, a0:a1], V[:, :, a0:a1]), dims.NA, SCALE, compute=on_cpu)
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, [t.contiguous() for t in owned]))
        if rank == 0:
            full = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V, nthreads=2)
            ok = True
            for (b0, b1, sh) in gathered:
                for t in range(2):
                    ref = full[t][:, :, b0:b1]
                    ok &= sh[t].shape == ref.shape
                    if b1 > b0:
                        ok &= bool(np.abs(sh[t].numpy() - ref).max() <= 1e-13 * np.abs(full[t]).max())
            q.put(ok)
    finally:
        dist.destroy_process_group()


def test_composed_sharded_gradient_in_G():
    """parallel.sigma_grad_G_atom_sharded with the oracle as the evaluation equals the unsharded oracle gradient up
    to the order of the additions, at world 3 on 16 atoms and on 2 atoms (one rank owns nothing)."""
    ctx = mp.get_context("spawn")
    for dims, world, nbr in ((Dims(NA=16, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2), 3, diamond_neighbours(1, 1, 2)),
                             (Dims(NA=2, NB=1, Norb=2, NE=6, Nkz=2, Nqz=1, Nw=2), 3, None)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_grad_g_worker, args=(world, _free_port(), dims, 14, nbr, q), nprocs=world,
                           join=True, start_method="spawn")
        assert q.get()


def _composed_energy_worker(rank, world, port, dims, seed, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed)
        E0, E1 = P.energy_range(dims.NE, world, rank)

        def on_cpu(Gl, Gg, dH, Dl, Dg, nbr, scale):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.sigma(nbr, dH, Dl, Dg, Gl, Gg, scale, nthreads=2))

        Sl, Sg = P.sigma_energy_sharded(inp.nbr, inp.dH, (inp.D_less, inp.D_greater),
                                        (inp.G_less[:, E0:E1].clone(), inp.G_greater[:, E0:E1].clone()), dims.NE,
                                        SCALE, compute=on_cpu)
        gathered = [None] * world
        dist.all_gather_object(gathered, (E0, E1, Sl.contiguous(), Sg.contiguous()))
        if rank == 0:
            full = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                nthreads=2)
            q.put(all(np.array_equal(sl.numpy(), full[0][:, b0:b1]) and np.array_equal(sg.numpy(), full[1][:, b0:b1])
                      for b0, b1, sl, sg in gathered))
    finally:
        dist.destroy_process_group()


def _composed_energy_grad_worker(rank, world, port, dims, seed, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed)
        W, V = make_upstream(dims, seed=seed + 1)
        E0, E1 = P.energy_range(dims.NE, world, rank)

        def on_cpu(Gl, Gg, dH, Dl, Dg, nbr, gl, gg, scale):  # the oracle in place of the library call
            return tuple(torch.from_numpy(x) for x in oracle.sigma_grad(nbr, dH, Dl, Dg, Gl, Gg, scale, gl, gg,
                                                                        nthreads=2))

        grads = P.sigma_grad_energy_sharded(inp.nbr, inp.dH, (inp.D_less, inp.D_greater),
                                            (inp.G_less[:, E0:E1].clone(), inp.G_greater[:, E0:E1].clone()),
                                            (W[:, E0:E1], V[:, E0:E1]), dims.NE, SCALE, compute=on_cpu)
        ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, W, V,
                                nthreads=2)
        ok = all(bool(np.abs(g.numpy() - r).max() <= 1e-13 * np.abs(r).max()) for g, r in zip(grads, ref))
        oks = [None] * world
        dist.all_gather_object(oks, ok)
        if rank == 0:
            q.put(all(oks))
    finally:
        dist.destroy_process_group()


def test_composed_energy_sharded_gradients():
    """parallel.sigma_grad_energy_sharded with the oracle as the evaluation: every rank's gradients with respect to
    dH, D^< and D^> equal the unsharded oracle's up to the order of the additions, also with more ranks than
    energies (a rank owns nothing)."""
    ctx = mp.get_context("spawn")
    for dims, world in ((TINY, 3), (Dims(NA=4, NB=2, Norb=2, NE=3, Nkz=2, Nqz=1, Nw=2), 4)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_energy_grad_worker, args=(world, _free_port(), dims, 16, q), nprocs=world,
                           join=True, start_method="spawn")
        assert q.get()


def test_composed_energy_sharded_sigma():
    """parallel.sigma_energy_sharded with the oracle as the evaluation: each rank's rows equal the unsharded oracle
    bit for bit, with windows longer than Nw and shorter than Nw (the halo spans several ranks)."""
    ctx = mp.get_context("spawn")
    for dims, world in ((TINY, 3), (Dims(NA=6, NB=2, Norb=2, NE=12, Nkz=2, Nqz=2, Nw=5), 4)):
        q = ctx.SimpleQueue()
        mp.start_processes(_composed_energy_worker, args=(world, _free_port(), dims, 15, q), nprocs=world, join=True,
                           start_method="spawn")
        assert q.get()


def test_atom_ranges_partition():
    for NA in (1, 7, 16, 1024):
        for world in (1, 2, 3, 8):
            rs = [P.atom_range(NA, world, r) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == NA
            assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
            assert max(b - a for a, b in rs) - min(b - a for a, b in rs) <= 1


def _grad_g_worker(rank, world, port, dims, seed, nbr, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed, nbr=nbr)
        W, V = make_upstream(dims, seed=seed + 1)
        a0, a1 = P.atom_range(dims.NA, world, rank)
        n_own = a1 - a0
        G_owned = [inp.G_less[:, :, a0:a1].clone(), inp.G_greater[:, :, a0:a1].clone()]
        halo = P.exchange_halo(G_owned, inp.nbr, dims.NA)
        local = P.local_problem(inp.nbr, a0, a1, G_owned, halo, inp.dH[a0:a1],
                                (inp.D_less[:, :, a0:a1], inp.D_greater[:, :, a0:a1]))
        Wl, Vl = torch.zeros_like(local[4]), torch.zeros_like(local[5])
        Wl[:, :, :n_own], Vl[:, :, :n_own] = W[:, :, a0:a1], V[:, :, a0:a1]
        # the gradient in G from this rank's bonds only, for owned and halo atoms alike
        gl, gg = oracle.sigma_grad_G(local[0], local[1], local[2], local[3], SCALE, Wl, Vl, a_range=(0, n_own),
                                     nthreads=2)
        owned = P.reduce_halo_grad([torch.from_numpy(gl), torch.from_numpy(gg)], inp.nbr, dims.NA)
        # control: bonds of the other rank reach some of this rank's atoms, so the reduction changes something
        assert float((owned[0] - torch.from_numpy(gl[:, :, :n_own])).abs().max()) > 0
        gathered = [None] * world
        dist.all_gather_object(gathered, (a0, a1, [t.contiguous() for t in owned]))
        if rank == 0:
            full = oracle.sigma_grad_G(inp.nbr, inp.dH, inp.D_less, inp.D_greater, SCALE, W, V, nthreads=2)
            ok = True
            for (b0, b1, sh) in gathered:
                for t in range(2):
                    ref = full[t][:, :, b0:b1]
                    ok &= bool(np.abs(sh[t].numpy() - ref).max() <= 1e-13 * np.abs(full[t]).max())
            q.put(ok)
    finally:
        dist.destroy_process_group()


def _run_grad_g(dims, world, seed, nbr=None):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_grad_g_worker, args=(world, _free_port(), dims, seed, nbr, q), nprocs=world, join=True,
                       start_method="spawn")
    return q.get()


def test_two_ranks_gradient_in_G_reduces_the_halo():
    """The gradient with respect to G, sharded by atoms: each rank's bonds reach halo atoms that other ranks own, and
    reduce_halo_grad returns those contributions to the owners (equal to the unsharded oracle up to the order of the
    additions)."""
    assert _run_grad_g(TINY, 2, seed=3)
    d = Dims(NA=128, NB=4, Norb=2, NE=9, Nkz=2, Nqz=2, Nw=2)
    assert _run_grad_g(d, 2, seed=6, nbr=diamond_neighbours(2, 2, 4))


def _energy_worker(rank, world, port, dims, seed, q):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inp = make_inputs(dims, seed=seed)
        W, V = make_upstream(dims, seed=seed + 1)
        E0, E1 = P.energy_range(dims.NE, world, rank)
        e0, (Gl, Gg) = P.exchange_energy_halo([inp.G_less[:, E0:E1].clone(), inp.G_greater[:, E0:E1].clone()],
                                             dims.NE, dims.Nw)
        e1 = e0 + Gl.shape[1]
        assert torch.equal(Gl, inp.G_less[:, e0:e1]) and torch.equal(Gg, inp.G_greater[:, e0:e1])
        # Sigma on the owned energies from the window and its halo alone
        Sl, Sg = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, Gl, Gg, SCALE, nthreads=2)
        shard = [torch.from_numpy(X[:, E0 - e0:E1 - e0]).contiguous() for X in (Sl, Sg)]
        # adjoint: the loss of the owned energies; gradients summed over energies, then over the ranks
        Wl, Vl = torch.zeros_like(Gl), torch.zeros_like(Gg)
        Wl[:, E0 - e0:E1 - e0], Vl[:, E0 - e0:E1 - e0] = W[:, E0:E1], V[:, E0:E1]
        parts = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, Gl, Gg, SCALE, Wl, Vl, nthreads=2)
        grads = [P.reduce_in_rank_order(torch.from_numpy(g)) for g in parts]
        gathered = [None] * world
        dist.all_gather_object(gathered, (E0, E1, shard))
        if rank == 0:
            full = oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                nthreads=2)
            ref = oracle.sigma_grad(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                    W, V, nthreads=2)
            ok = all(np.array_equal(sh[t].numpy(), full[t][:, b0:b1]) for (b0, b1, sh) in gathered for t in (0, 1))
            for g, r in zip(grads, ref):
                ok &= bool(np.abs(g.numpy() - r).max() <= 1e-13 * np.abs(r).max())
            q.put(ok)
    finally:
        dist.destroy_process_group()


def _run_energy(dims, world, seed):
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    mp.start_processes(_energy_worker, args=(world, _free_port(), dims, seed, q), nprocs=world, join=True,
                       start_method="spawn")
    return q.get()


def test_energy_windows_with_halo():
    """Energy-window sharding: each rank owns [E0, E1), receives the Nw rows on each side from their owners, and
    computes Sigma on its window exactly (bit for bit with the unsharded oracle); the gradients with respect to dH
    and D, sums over energies, are reduced over the ranks in rank order."""
    assert _run_energy(TINY, 2, seed=8)
    assert _run_energy(TINY, 3, seed=9)
    # windows shorter than Nw: the halo of the middle rank comes from both neighbours and beyond
    assert _run_energy(Dims(NA=6, NB=2, Norb=2, NE=12, Nkz=2, Nqz=2, Nw=5), 3, seed=10)
