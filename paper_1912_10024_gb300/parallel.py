"""Atom-tile and energy-window sharding of Eqs. (3) and (4) across ranks with halo exchanges of G.

The communication-avoiding decomposition of Sec. 4.2 tiles the atoms of the
device: a rank that owns atoms [a0, a1) computes Sigma_a for exactly those
atoms and needs, besides its own G blocks, the G blocks of the neighbours of
its atoms that other ranks own (the "+N_b atom halo"). One exchange step
brings those blocks in; Sigma, Pi and the gradients with respect to dH and D
need no reduction afterwards. The gradient with respect to G does: a rank's
bonds also reach the G blocks of its halo atoms, so ``reduce_halo_grad`` sends
those contributions back to their owners. The other axis tiles the energies:
a rank that owns [E0, E1) needs the Nw rows of G on each side (the "+2 N_w
energy halo"); the gradients with respect to dH and D, sums over energies, are
then reduced across the ranks.

The primitives (``exchange_halo``, ``local_problem``, ``reduce_halo_grad``,
``exchange_energy_halo``, ``reduce_in_rank_order``) are composed into one call
per operation: ``sigma_atom_sharded``, ``sigma_grad_atom_sharded``,
``sigma_grad_G_atom_sharded``, ``pi_atom_sharded``, ``sigma_energy_sharded``
and ``sigma_grad_energy_sharded``; each evaluates its local problem with the
library call (or a ``compute`` the caller passes).

On one GPU the shard primitive is sse_sigma_fwd's atom range; across GPUs the
exchanges run over torch.distributed (NCCL for CUDA tensors, gloo for CPU
tensors): one packed point-to-point message of G blocks (or energy rows) per peer, plus the
rank-order chain that sums the energy-summed gradients.
"""
from __future__ import annotations

from typing import Dict, List, Sequence, Tuple

import torch
import torch.distributed as dist


def atom_range(NA: int, world: int, rank: int) -> Tuple[int, int]:
    """Balanced contiguous atom range of ``rank``."""
    base, rem = divmod(NA, world)
    a0 = rank * base + min(rank, rem)
    return a0, a0 + base + (1 if rank < rem else 0)


def owner(a: int, NA: int, world: int) -> int:
    for r in range(world):
        a0, a1 = atom_range(NA, world, r)
        if a0 <= a < a1:
            return r
    raise ValueError(a)


def halo_atoms(nbr: torch.Tensor, a0: int, a1: int) -> List[int]:
    """Neighbours of atoms [a0, a1) that lie outside the range (sorted)."""
    need = set(int(b) for b in nbr[a0:a1].reshape(-1).tolist())
    return sorted(b for b in need if not a0 <= b < a1)


def exchange_halo(G_owned: Sequence[torch.Tensor], nbr: torch.Tensor, NA: int,
                  group=None) -> Dict[int, List[torch.Tensor]]:
    """Fetch the G blocks of this rank's halo atoms from their owners.

    G_owned: the owned slices [Nkz, NE, a1-a0, Norb, Norb] of G^< and G^>.
    Returns {atom: [G^< block, G^> block]} for every halo atom.
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    mine = halo_atoms(nbr, a0, a1)
    wants: List[List[int]] = [None] * world  # type: ignore[list-item]
    dist.all_gather_object(wants, mine, group=group)
    ntype = len(G_owned)
    ops, pending = [], []
    for peer in range(world):
        if peer == rank:
            continue
        # one packed message per peer: the blocks it needs from me, in its (sorted) order, both types
        give = [b - a0 for b in wants[peer] if a0 <= b < a1]
        if give:
            idx = torch.tensor(give, dtype=torch.long, device=G_owned[0].device)
            send = torch.stack([G.index_select(2, idx) for G in G_owned])  # [types, Nkz, NE, len(give), ...]
            ops.append(dist.P2POp(dist.isend, send, peer, group))
        take = [b for b in mine if owner(b, NA, world) == peer]
        if take:
            G = G_owned[0]
            buf = torch.empty((ntype, G.shape[0], G.shape[1], len(take)) + tuple(G.shape[3:]), dtype=G.dtype,
                              device=G.device)
            ops.append(dist.P2POp(dist.irecv, buf, peer, group))
            pending.append((take, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    recv: Dict[int, List[torch.Tensor]] = {}
    for take, buf in pending:
        for i, b in enumerate(take):
            recv[b] = [buf[t, :, :, i] for t in range(ntype)]
    return recv


def _local_neighbours(nbr: torch.Tensor, a0: int, a1: int, halo: Sequence[int]) -> torch.Tensor:
    """Neighbour list [a1-a0+len(halo), NB] (CPU, int32) of the local numbering: atoms [a0, a1) first, then the halo
    atoms in the given order; halo atoms point at themselves (they get zero dH and D)."""
    order = list(range(a0, a1)) + list(halo)
    index = {b: i for i, b in enumerate(order)}
    NB = nbr.shape[1]
    nbr_l = torch.arange(len(order), dtype=torch.int32).unsqueeze(1).repeat(1, NB)
    if a1 > a0:
        nbr_l[:a1 - a0] = torch.tensor([[index[int(b)] for b in row] for row in nbr[a0:a1].tolist()],
                                       dtype=torch.int32)
    return nbr_l


def local_problem(nbr: torch.Tensor, a0: int, a1: int, G_owned: Sequence[torch.Tensor],
                  halo: Dict[int, List[torch.Tensor]], dH_owned: torch.Tensor, D_owned: Sequence[torch.Tensor]):
    """Rank-local problem: atoms [a0, a1) first, then the halo atoms.

    Returns (nbr_local, dH_local, D_less_local, D_greater_local, G_less_local,
    G_greater_local); Sigma of local atoms [0, a1-a0) equals Sigma of global
    atoms [a0, a1). Halo atoms get zero dH/D and point at themselves.
    """
    n_own, n_loc = a1 - a0, a1 - a0 + len(halo)
    nbr_l = _local_neighbours(nbr, a0, a1, sorted(halo))
    Gs = []
    for t, G in enumerate(G_owned):
        blocks = [G] + [halo[b][t].unsqueeze(2) for b in sorted(halo)]
        Gs.append(torch.cat(blocks, dim=2).contiguous())
    dH_l = torch.zeros((n_loc,) + tuple(dH_owned.shape[1:]), dtype=dH_owned.dtype, device=dH_owned.device)
    dH_l[:n_own] = dH_owned
    Ds = []
    for D in D_owned:
        Dl = torch.zeros(D.shape[:2] + (n_loc,) + D.shape[3:], dtype=D.dtype, device=D.device)
        Dl[:, :, :n_own] = D
        Ds.append(Dl)
    return nbr_l.to(dH_owned.device), dH_l, Ds[0], Ds[1], Gs[0], Gs[1]


def sigma_atom_sharded(nbr: torch.Tensor, dH_owned: torch.Tensor, D_owned: Sequence[torch.Tensor],
                       G_owned: Sequence[torch.Tensor], NA: int, scale: float, compute=None, group=None, **kw):
    """Sigma^<, Sigma^> of this rank's atoms [a0, a1) with the one exchange step of the atom tiling.

    nbr: the global neighbour list [NA, NB] (every rank holds it); dH_owned [a1-a0, NB, 3, Norb, Norb],
    D_owned = (D^<, D^>) [Nqz, Nw, a1-a0, NB, 3, 3] and G_owned = (G^<, G^>) [Nkz, NE, a1-a0, Norb, Norb]: the
    rank's slices. The halo G blocks are fetched (``exchange_halo``), the local problem is built
    (``local_problem``) and ``compute`` evaluates Sigma of its first a1-a0 atoms; ``compute`` takes
    (G_less, G_greater, dH, D_less, D_greater, nbr, scale=..., atoms=..., **kw) and returns the pair of full
    local outputs, by default the library call ``binding.sigma`` (CUDA tensors; ``kw`` passes mode and flags).
    Returns the owned slices [Nkz, NE, a1-a0, Norb, Norb]; no reduction follows.
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    halo = exchange_halo(G_owned, nbr, NA, group)  # collective: every rank takes part
    if a1 == a0:  # more ranks than atoms: nothing owned
        return G_owned[0][:, :, :0].clone(), G_owned[1][:, :, :0].clone()
    nbr_l, dH_l, Dl, Dg, Gl, Gg = local_problem(nbr, a0, a1, G_owned, halo, dH_owned, D_owned)
    if compute is None:
        from . import binding
        compute = binding.sigma
    Sl, Sg = compute(Gl, Gg, dH_l, Dl, Dg, nbr_l, scale=scale, atoms=(0, a1 - a0), **kw)
    return Sl[:, :, :a1 - a0], Sg[:, :, :a1 - a0]


def sigma_grad_atom_sharded(nbr: torch.Tensor, dH_owned: torch.Tensor, D_owned: Sequence[torch.Tensor],
                            G_owned: Sequence[torch.Tensor], gS_owned: Sequence[torch.Tensor], NA: int, scale: float,
                            compute=None, group=None, **kw):
    """Gradients of L = sum_t Re tr(gS^t^H Sigma^t) with respect to this rank's dH and D^<, D^> rows: owned per atom,
    so after the halo exchange of G no reduction follows. gS_owned = (gS^<, gS^>) [Nkz, NE, a1-a0, Norb, Norb].
    ``compute`` takes (G_less, G_greater, dH, D_less, D_greater, nbr, gS_less, gS_greater, scale=..., atoms=..., **kw)
    and defaults to ``binding.sigma_grad``. Returns (g_dH [a1-a0, ...], g_D^< and g_D^> [Nqz, Nw, a1-a0, ...])."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    halo = exchange_halo(G_owned, nbr, NA, group)  # collective: every rank takes part
    n_own = a1 - a0
    if n_own == 0:
        return dH_owned.clone(), D_owned[0].clone(), D_owned[1].clone()
    nbr_l, dH_l, Dl, Dg, Gl, Gg = local_problem(nbr, a0, a1, G_owned, halo, dH_owned, D_owned)
    gS = []
    for g in gS_owned:
        x = torch.zeros_like(Gl)
        x[:, :, :n_own] = g
        gS.append(x)
    if compute is None:
        from . import binding
        compute = binding.sigma_grad
    g_dH, g_Dl, g_Dg = compute(Gl, Gg, dH_l, Dl, Dg, nbr_l, gS[0], gS[1], scale=scale, atoms=(0, n_own), **kw)
    return g_dH[:n_own], g_Dl[:, :, :n_own], g_Dg[:, :, :n_own]


def pi_atom_sharded(nbr: torch.Tensor, dH_owned: torch.Tensor, G_owned: Sequence[torch.Tensor], NA: int, Nqz: int,
                    Nw: int, scale: float, compute=None, group=None, **kw):
    """Pi^<, Pi^> of Eq. (4) for this rank's atoms [a0, a1): the same halo as Sigma (the G blocks of the neighbours),
    one exchange, the local problem and ``compute`` on its first a1-a0 atoms. ``compute`` takes (G_less, G_greater,
    dH, nbr, Nqz, Nw, scale=..., atoms=..., **kw) and defaults to the library call ``binding.pi``. Returns the owned
    rows [Nqz, Nw, a1-a0, NB+1, 3, 3]."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    halo = exchange_halo(G_owned, nbr, NA, group)  # collective: every rank takes part
    NB = nbr.shape[1]
    if a1 == a0:
        empty = torch.zeros((Nqz, Nw, 0, NB + 1, 3, 3), dtype=G_owned[0].dtype, device=G_owned[0].device)
        return empty, empty.clone()
    D0 = dH_owned.new_zeros((Nqz, Nw, a1 - a0, NB, 3, 3))  # placeholders: Pi does not read D
    nbr_l, dH_l, _, _, Gl, Gg = local_problem(nbr, a0, a1, G_owned, halo, dH_owned, (D0, D0))
    if compute is None:
        from . import binding
        compute = binding.pi
    Pl, Pg = compute(Gl, Gg, dH_l, nbr_l, Nqz, Nw, scale=scale, atoms=(0, a1 - a0), **kw)
    return Pl[:, :, :a1 - a0], Pg[:, :, :a1 - a0]


def reduce_halo_grad(gG_local: Sequence[torch.Tensor], nbr: torch.Tensor, NA: int,
                     group=None) -> List[torch.Tensor]:
    """The exchange step of the gradient with respect to G: the reverse of ``exchange_halo``.

    gG_local: the rank's gradients with respect to G^< and G^> in the layout of ``local_problem``
    ([Nkz, NE, n_loc, Norb, Norb], owned atoms first, then the halo atoms in sorted order), each computed from the
    rank's own bonds only. A bond (a, s) contributes to the gradient of G_b for b = nbr[a][s], which another rank may
    own: every rank sends the blocks of its halo atoms to their owners, and each owner adds what it receives to its
    own blocks in rank order (deterministic). Returns the owned slices [Nkz, NE, a1-a0, Norb, Norb] with every
    bond's contribution.
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    n_own = a1 - a0
    mine = halo_atoms(nbr, a0, a1)
    halos: List[List[int]] = [None] * world  # type: ignore[list-item]
    dist.all_gather_object(halos, mine, group=group)
    out = [g[:, :, :n_own].clone() for g in gG_local]
    ntype = len(gG_local)
    ops, recv = [], []
    for peer in range(world):
        if peer == rank:
            continue
        # one packed message per peer: my halo blocks that it owns, in my (sorted) halo order, both types
        give = [n_own + i for i, b in enumerate(mine) if owner(b, NA, world) == peer]
        if give:
            idx = torch.tensor(give, dtype=torch.long, device=gG_local[0].device)
            ops.append(dist.P2POp(dist.isend, torch.stack([g.index_select(2, idx) for g in gG_local]), peer, group))
        # the peer's halo blocks that I own, in the peer's order
        take = [b for b in halos[peer] if a0 <= b < a1]
        if take:
            g = gG_local[0]
            buf = torch.empty((ntype, g.shape[0], g.shape[1], len(take)) + tuple(g.shape[3:]), dtype=g.dtype,
                              device=g.device)
            ops.append(dist.P2POp(dist.irecv, buf, peer, group))
            recv.append((peer, take, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    # added in (peer rank, atom) order: deterministic
    adds = sorted(((peer, b, buf, i) for peer, take, buf in recv for i, b in enumerate(take)),
                  key=lambda x: (x[0], x[1]))
    for _peer, b, buf, i in adds:
        for t in range(ntype):
            out[t][:, :, b - a0] += buf[t, :, :, i]
    return out


def sigma_grad_G_atom_sharded(nbr: torch.Tensor, dH_owned: torch.Tensor, D_owned: Sequence[torch.Tensor],
                              gS_owned: Sequence[torch.Tensor], NA: int, scale: float, compute=None, group=None,
                              **kw) -> List[torch.Tensor]:
    """Gradient with respect to this rank's G^<, G^> blocks of L = sum_t Re tr(gS^t^H Sigma^t) summed over every
    rank's atoms, with the atom tiling.

    gS_owned = (gS^<, gS^>) [Nkz, NE, a1-a0, Norb, Norb]: the upstream gradient of the owned atoms' Sigma. The rank
    evaluates the gradient of its own bonds over its local atoms (owned, then halo; Sigma is linear in G, so G itself
    is not needed) with ``compute`` -- by default the library call ``binding.sigma_grad_G``, which takes
    (dH, D_less, D_greater, nbr, gS_less, gS_greater, scale=..., **kw) -- and ``reduce_halo_grad`` returns the halo
    blocks to their owners. Returns the owned slices [Nkz, NE, a1-a0, Norb, Norb].
    """
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    a0, a1 = atom_range(NA, world, rank)
    halo = halo_atoms(nbr, a0, a1)
    n_own, n_loc = a1 - a0, a1 - a0 + len(halo)
    dev = gS_owned[0].device
    if n_loc == 0:  # nothing owned: only the collective of the reduction
        return reduce_halo_grad([g.clone() for g in gS_owned], nbr, NA, group)
    nbr_l = _local_neighbours(nbr, a0, a1, halo).to(dev)
    dH_l = torch.zeros((n_loc,) + tuple(dH_owned.shape[1:]), dtype=dH_owned.dtype, device=dev)
    dH_l[:n_own] = dH_owned
    Ds = []
    for D in D_owned:
        Dl = torch.zeros(D.shape[:2] + (n_loc,) + D.shape[3:], dtype=D.dtype, device=dev)
        Dl[:, :, :n_own] = D
        Ds.append(Dl)
    gS = []
    for g in gS_owned:
        x = torch.zeros(g.shape[:2] + (n_loc,) + g.shape[3:], dtype=g.dtype, device=dev)
        x[:, :, :n_own] = g
        gS.append(x)
    if compute is None:
        from . import binding
        compute = binding.sigma_grad_G
    gG = compute(dH_l, Ds[0], Ds[1], nbr_l, gS[0], gS[1], scale=scale, **kw)
    return reduce_halo_grad(list(gG), nbr, NA, group)


# ---------------------------------------------------------------------------
# Energy windows (the other axis of the Sec. 4.2 tiling). Sigma(E) reads G at E -/+ (w+1), w < Nw, so a rank that
# owns the energy window [E0, E1) needs the Nw rows on each side (the "+2 N_w energy halo"); with them, Sigma on
# [E0, E1) is exact (rows beyond the grid contribute zero as in Eq. (3)). The direct evaluations (FP64 correlation,
# tensor-core windows) shard this way; the transform evaluation needs every energy of a column and shards by atoms.
# ---------------------------------------------------------------------------
def energy_range(NE: int, world: int, rank: int) -> Tuple[int, int]:
    """Balanced contiguous energy window of ``rank``."""
    return atom_range(NE, world, rank)


def energy_owner(E: int, NE: int, world: int) -> int:
    return owner(E, NE, world)


def exchange_energy_halo(G_window: Sequence[torch.Tensor], NE: int, Nw: int, group=None):
    """Extend this rank's energy window of G^< and G^> ([Nkz, E1-E0, ...]) by the Nw rows on each side that other
    ranks own. Returns (e0, [G^< rows e0..e1-1, G^> rows e0..e1-1]) with e0 = max(0, E0-Nw), e1 = min(NE, E1+Nw)."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    E0, E1 = energy_range(NE, world, rank)
    e0, e1 = max(0, E0 - Nw), min(NE, E1 + Nw)
    ranges: List[Tuple[int, int]] = [None] * world  # type: ignore[list-item]
    dist.all_gather_object(ranges, (e0, e1), group=group)
    out = []
    for G in G_window:
        X = torch.empty((G.shape[0], e1 - e0) + tuple(G.shape[2:]), dtype=G.dtype, device=G.device)
        X[:, E0 - e0:E1 - e0] = G
        out.append(X)
    ops, pending = [], []
    for peer in range(world):
        if peer == rank:
            continue
        # my rows inside the peer's extended window, then the peer's rows inside mine (the same interval
        # arithmetic on both sides, so the messages of each direction match in order)
        s0, s1 = max(E0, ranges[peer][0]), min(E1, ranges[peer][1])
        if s0 < s1:
            for G in G_window:
                ops.append(dist.P2POp(dist.isend, G[:, s0 - E0:s1 - E0].contiguous(), peer, group))
        p0, p1 = energy_range(NE, world, peer)
        r0, r1 = max(p0, e0), min(p1, e1)
        if r0 < r1:
            for t in range(len(G_window)):
                buf = torch.empty_like(out[t][:, r0 - e0:r1 - e0])
                ops.append(dist.P2POp(dist.irecv, buf, peer, group))
                pending.append((t, r0 - e0, r1 - e0, buf))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    for t, lo, hi, buf in pending:
        out[t][:, lo:hi] = buf
    return e0, out


def sigma_energy_sharded(nbr: torch.Tensor, dH: torch.Tensor, D: Sequence[torch.Tensor], G_window: Sequence[torch.Tensor],
                         NE: int, scale: float, compute=None, group=None, **kw):
    """Sigma^<, Sigma^> of every atom on this rank's energy window [E0, E1), from its rows of G alone plus the one
    exchange of the +-Nw energy halo.

    G_window = (G^<, G^>) [Nkz, E1-E0, NA, Norb, Norb]: the rank's rows; nbr, dH and D = (D^<, D^>) whole (they do
    not depend on E). ``compute`` evaluates Sigma on the extended window as a problem of its own (energies outside
    it contribute zero, which is exact on [E0, E1)); it takes (G_less, G_greater, dH, D_less, D_greater, nbr,
    scale=..., **kw) and defaults to the library call ``binding.sigma``. Returns Sigma's rows [Nkz, E1-E0, NA, Norb,
    Norb]."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    E0, E1 = energy_range(NE, world, rank)
    Nw = D[0].shape[1]
    e0, (Gl, Gg) = exchange_energy_halo(G_window, NE, Nw, group)  # collective: every rank takes part
    if E1 == E0:
        return G_window[0][:, :0].clone(), G_window[1][:, :0].clone()
    # the extended window has at least Nw + 1 rows (NE > Nw and E1 > E0), so it is a valid problem of its own
    if compute is None:
        from . import binding
        compute = binding.sigma
    Sl, Sg = compute(Gl.contiguous(), Gg.contiguous(), dH, D[0], D[1], nbr, scale=scale, **kw)
    return Sl[:, E0 - e0:E1 - e0], Sg[:, E0 - e0:E1 - e0]


def sigma_grad_energy_sharded(nbr: torch.Tensor, dH: torch.Tensor, D: Sequence[torch.Tensor],
                              G_window: Sequence[torch.Tensor], gS_window: Sequence[torch.Tensor], NE: int,
                              scale: float, compute=None, group=None, **kw) -> List[torch.Tensor]:
    """Gradients (g_dH, g_D^<, g_D^>) of L = sum_t Re tr(gS^t^H Sigma^t) over all energies, with the energy tiling.

    G_window and gS_window: this rank's rows [Nkz, E1-E0, NA, Norb, Norb] of G and of the upstream gradient. The rank
    evaluates the gradient of its own rows' loss on its extended window (upstream zero on the halo rows) with
    ``compute`` -- by default ``binding.sigma_grad``, which takes (G_less, G_greater, dH, D_less, D_greater, nbr,
    gS_less, gS_greater, scale=..., **kw) -- and the sums over energies are completed across the ranks in rank order.
    Every rank returns the full gradients."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    E0, E1 = energy_range(NE, world, rank)
    Nw = D[0].shape[1]
    e0, (Gl, Gg) = exchange_energy_halo(G_window, NE, Nw, group)
    if E1 > E0:
        gS = []
        for g in gS_window:
            x = torch.zeros_like(Gl)
            x[:, E0 - e0:E1 - e0] = g
            gS.append(x)
        if compute is None:
            from . import binding
            compute = binding.sigma_grad
        parts = compute(Gl.contiguous(), Gg.contiguous(), dH, D[0], D[1], nbr, gS[0], gS[1], scale=scale, **kw)
    else:  # nothing owned: zero contributions to the sums
        parts = (torch.zeros_like(dH), torch.zeros_like(D[0]), torch.zeros_like(D[1]))
    return [reduce_in_rank_order(p, group) for p in parts]


def reduce_in_rank_order(x: torch.Tensor, group=None) -> torch.Tensor:
    """Sum of ``x`` over the ranks in rank order, (((x_0 + x_1) + x_2) + ...), returned on every rank (deterministic):
    the reduction that gradients summed over energies (dH, D) need when the energies are split. A chain of
    point-to-point messages (rank r adds its part to the partial sum of ranks < r and passes it on) and a broadcast
    from the last rank: two buffers of x's size per rank, where gathering every rank's part would take world."""
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    if world == 1:
        return x.clone()
    ranks = dist.get_process_group_ranks(group) if group is not None else list(range(world))
    total = x.contiguous().clone()
    if rank > 0:
        prev = torch.empty_like(total)
        dist.recv(prev, src=ranks[rank - 1], group=group)
        total = prev.add_(total)  # partial sum of ranks < r, then x_r
    if rank < world - 1:
        dist.send(total, dst=ranks[rank + 1], group=group)
    dist.broadcast(total, src=ranks[world - 1], group=group)
    return total
