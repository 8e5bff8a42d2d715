"""Cut a small, exact sub-problem out of a large one for the oracle.

TEST INFRASTRUCTURE ONLY (used by tests and the benchmark's CPU-baseline leg).

Sigma^t_a(E, k) for E in [E0, E1) depends only on atom a's dH and D slices and
on G of a's neighbours at energies [E0 - Nw, E1 + Nw) (all kz). This module
copies exactly those slices into a problem with atoms [a, neighbours...] and
that energy window, so the oracle can evaluate sampled outputs of a problem
too large to run whole. Only indexing and copies happen here.
"""
from __future__ import annotations

import torch


def extract(nbr, dH, D_less, D_greater, G_less, G_greater, a: int, E0: int, E1: int):
    """Returns (local arrays as CPU tensors, E_range in local energies)."""
    NE = G_less.shape[1]
    Nw = D_less.shape[1]
    row = nbr[a].to("cpu").tolist()
    atoms = [a] + [b for b in dict.fromkeys(row) if b != a]
    index = {b: i for i, b in enumerate(atoms)}
    NB = len(row)
    nbr_l = torch.zeros((len(atoms), NB), dtype=torch.int32)
    nbr_l[0] = torch.tensor([index[b] for b in row], dtype=torch.int32)
    lo, hi = max(0, E0 - Nw), min(NE, E1 + Nw)
    sel = torch.tensor(atoms, dtype=torch.long, device=G_less.device)
    G_l = G_less[:, lo:hi].index_select(2, sel).to("cpu")
    G_g = G_greater[:, lo:hi].index_select(2, sel).to("cpu")
    dH_l = torch.zeros((len(atoms),) + tuple(dH.shape[1:]), dtype=dH.dtype)
    dH_l[0] = dH[a].to("cpu")
    shape_D = (D_less.shape[0], D_less.shape[1], len(atoms)) + tuple(D_less.shape[3:])
    D_ll = torch.zeros(shape_D, dtype=D_less.dtype)
    D_gl = torch.zeros(shape_D, dtype=D_less.dtype)
    D_ll[:, :, 0] = D_less[:, :, a].to("cpu")
    D_gl[:, :, 0] = D_greater[:, :, a].to("cpu")
    return (nbr_l, dH_l, D_ll, D_gl, G_l, G_g), (E0 - lo, E1 - lo)


def oracle_blocks(nbr, dH, D_less, D_greater, G_less, G_greater, scale, a, E0, E1, nthreads=None):
    """Sigma^<, Sigma^> [Nkz, E1-E0, Norb, Norb] of atom a from the oracle."""
    import oracle
    args, (e0, e1) = extract(nbr, dH, D_less, D_greater, G_less, G_greater, a, E0, E1)
    Sl, Sg = oracle.sigma(*args, scale, a_range=(0, 1), E_range=(e0, e1), nthreads=nthreads)
    return Sl[:, e0:e1, 0], Sg[:, e0:e1, 0]
