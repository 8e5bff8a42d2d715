"""Pins of the FP64 CPU oracle for the phonon self-energy Pi of Eq. (4).

Each test checks the oracle against something other than itself: a closed
form for Green's functions constant in (E, kz), a delta response, the
anti-Hermiticity that Eq. (4) implies for anti-Hermitian G, the quadratic
scaling in the coupling, and an identity with the adjoint of Eq. (3) -- Pi
equals the gradient of a bilinear form of Sigma with respect to the phonon
weights, which the (separately finite-difference-checked) Sigma adjoint
computes. Together they fix the energy and kz shift directions, which type
pairs with which, the conjugate transposes and the prefactor -i*scale.
"""
import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300.inputs import Dims, make_inputs, ring_neighbours

SCALE = 1.0 / (2.0 * np.pi)


def two_way_ring(NA):
    return torch.tensor([[(a + 1) % NA, (a - 1) % NA] for a in range(NA)], dtype=torch.int32)


def rand_c(shape, seed):
    g = np.random.default_rng(seed)
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def run(nbr, dH, Gl, Gg, Nqz, Nw, scale=SCALE, **kw):
    return oracle.pi(nbr, dH, Gl, Gg, scale, Nqz, Nw, **kw)


# --------------------------------------------------------------------------
# closed form: G constant in E and kz
# --------------------------------------------------------------------------

def test_closed_form_constant_G():
    """With G^t_a(E,k) = G0^t_a, Eq. (4) collapses to
    Pi^t_ab(q,w)_ij = -i*scale * Nkz * (NE - (w+1)) * tr(dH_i^H G0^t_a dH_j G0^t'_b)
    (the number of energies with E and E+(w+1) on the grid), independent of q."""
    NA, NB, Norb, NE, Nkz, Nqz, Nw = 7, 3, 4, 11, 4, 3, 5
    nbr = torch.tensor([[(a + 1) % NA, (a + 3) % NA, (a + 6) % NA] for a in range(NA)], dtype=torch.int32)
    dH = rand_c((NA, NB, 3, Norb, Norb), 1) * 0.3
    G0l, G0g = rand_c((NA, Norb, Norb), 2), rand_c((NA, Norb, Norb), 3)
    Gl = np.broadcast_to(G0l, (Nkz, NE) + G0l.shape).copy()
    Gg = np.broadcast_to(G0g, (Nkz, NE) + G0g.shape).copy()
    Pl, Pg = run(nbr, dH, Gl, Gg, Nqz, Nw)
    nb = nbr.numpy()
    count = Nkz * (NE - (np.arange(Nw) + 1))  # [w]
    for P, Ga, Gb in ((Pl, G0l, G0g), (Pg, G0g, G0l)):
        T = np.einsum("asiml,amn,asjnp,aspl->asij", dH.conj(), Ga, dH, Gb[nb])  # tr(dH_i^H Ga dH_j Gb)
        bond = -1j * SCALE * count[None, :, None, None, None, None] * T[None, None]
        bond = np.broadcast_to(bond, (Nqz, Nw, NA, NB, 3, 3))
        assert normwise(P[:, :, :, :NB], bond) < 1e-13
        assert normwise(P[:, :, :, NB], bond.sum(axis=3)) < 1e-13


# --------------------------------------------------------------------------
# delta response: pins the kz and energy shift directions and the type pairing
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k0,E0,k1,E1", [(2, 6, 0, 3), (0, 4, 1, 0), (1, 8, 1, 7)])
def test_delta_response(k0, E0, k1, E1):
    """G^<_a nonzero only at (k0, E0), G^>_b only at (k1, E1): Pi^< of the bond (a, b) is nonzero only at
    w + 1 = E0 - E1 and q = (k0 - k1) mod Nkz; Pi^> of every bond and all other bonds vanish."""
    NA, NB, Norb, NE, Nkz, Nqz, Nw = 5, 2, 3, 9, 3, 3, 4
    nbr = ring_neighbours(NA, NB)
    dH = rand_c((NA, NB, 3, Norb, Norb), 4) * 0.3
    a, s = 1, 1
    b = int(nbr[a, s])
    X, Y = rand_c((Norb, Norb), 5), rand_c((Norb, Norb), 6)
    Gl = np.zeros((Nkz, NE, NA, Norb, Norb), complex)
    Gg = np.zeros_like(Gl)
    Gl[k0, E0, a] = X
    Gg[k1, E1, b] = Y
    Pl, Pg = run(nbr, dH, Gl, Gg, Nqz, Nw)
    expect = np.zeros_like(Pl)
    w, q = E0 - E1 - 1, (k0 - k1) % Nkz
    if 0 <= w < Nw and q < Nqz:
        T = -1j * SCALE * np.einsum("iml,mn,jnp,pl->ij", dH[a, s].conj(), X, dH[a, s], Y)
        expect[q, w, a, s] = T
        expect[q, w, a, NB] = T
    np.testing.assert_allclose(Pl, expect, rtol=0, atol=1e-14 * max(1.0, np.abs(expect).max()))
    assert np.abs(Pg).max() == 0.0


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_anti_hermitian_blocks():
    """For anti-Hermitian G^<, G^> (as physical lesser/greater functions are) tr(dH_i^H G_a dH_j G_b) is
    Hermitian in (i, j), so every 3x3 block of Pi = -i*scale*(...) is anti-Hermitian. Control: a G that is not
    anti-Hermitian breaks it."""
    d = Dims(NA=6, NB=2, Norb=3, NE=10, Nkz=3, Nqz=3, Nw=3)
    inp = make_inputs(d, seed=7, nbr=two_way_ring(6))
    Pl, Pg = run(inp.nbr, inp.dH, inp.G_less, inp.G_greater, d.Nqz, d.Nw)
    for P in (Pl, Pg):
        dev = np.abs(P + np.conj(np.swapaxes(P, -1, -2))).max()
        assert dev <= 1e-14 * np.abs(P).max()
    Gbad = inp.G_less.clone()
    Gbad += 0.3 * torch.complex(torch.ones_like(Gbad.real), torch.zeros_like(Gbad.real))
    Pl, _ = run(inp.nbr, inp.dH, Gbad, inp.G_greater, d.Nqz, d.Nw)
    assert np.abs(Pl + np.conj(np.swapaxes(Pl, -1, -2))).max() > 1e-3 * np.abs(Pl).max()


def test_quadratic_in_coupling():
    """Pi(lambda dH) = |lambda|^2 Pi(dH): one dH enters conjugate-transposed, the other plain."""
    NA, NB, Norb, NE, Nkz, Nqz, Nw = 4, 2, 3, 8, 2, 2, 3
    nbr = ring_neighbours(NA, NB)
    dH = rand_c((NA, NB, 3, Norb, Norb), 8)
    Gl, Gg = rand_c((Nkz, NE, NA, Norb, Norb), 9), rand_c((Nkz, NE, NA, Norb, Norb), 10)
    lam = 0.7 - 1.3j
    P1 = run(nbr, dH, Gl, Gg, Nqz, Nw)
    P2 = run(nbr, lam * dH, Gl, Gg, Nqz, Nw)
    for x, y in zip(P1, P2):
        assert normwise(y, abs(lam) ** 2 * x) < 1e-13


def test_diagonal_block_sums_the_neighbours():
    """Reading of Eq. (4): the diagonal block sums over all neighbours l, an off-diagonal block keeps l = b."""
    d = Dims(NA=5, NB=3, Norb=2, NE=7, Nkz=2, Nqz=2, Nw=2)
    inp = make_inputs(d, seed=12, nbr=ring_neighbours(5, 3))
    for P in run(inp.nbr, inp.dH, inp.G_less, inp.G_greater, d.Nqz, d.Nw):
        assert normwise(P[:, :, :, d.NB], P[:, :, :, :d.NB].sum(axis=3)) < 1e-14


def test_atom_range():
    d = Dims(NA=6, NB=2, Norb=2, NE=6, Nkz=2, Nqz=2, Nw=2)
    inp = make_inputs(d, seed=13, nbr=ring_neighbours(6, 2))
    full = run(inp.nbr, inp.dH, inp.G_less, inp.G_greater, d.Nqz, d.Nw)
    part = run(inp.nbr, inp.dH, inp.G_less, inp.G_greater, d.Nqz, d.Nw, a_range=(2, 4))
    for f, p in zip(full, part):
        np.testing.assert_array_equal(p[:, :, 2:4], f[:, :, 2:4])
        assert np.abs(p[:, :, :2]).max() == 0 and np.abs(p[:, :, 4:]).max() == 0


# --------------------------------------------------------------------------
# identity with the adjoint of Eq. (3)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("nbr_kind", ["ring", "two_way_ring"])
def test_equals_sigma_adjoint_weight_gradient(nbr_kind):
    """Let L = Re sum tr(W^H Sigma^u) with upstream W = G^t (t the type of Pi) on the output of the other type
    u = t', zero upstream on Sigma^t, and feed Eq. (3) the blockwise conjugate transpose of G^u. The gradient
    of L with respect to the weight D^u of the bond (a, s) is conj(i*scale * sum tr(G^t_a(E,k)^H dH_i
    G^u_b(E-(w+1), k-q)^H dH_j^H)) = -i*scale * sum tr(dH_i^H G^t_a(E,k) dH_j G^u_b(E-(w+1), k-q)), which after
    E -> E + (w+1), k -> k + q is Eq. (4)'s off-diagonal block. The Sigma adjoint is pinned separately by
    central differences of the Sigma forward."""
    NA, NB, Norb, NE, Nkz, Nqz, Nw = 6, 2, 3, 9, 3, 2, 3
    nbr = ring_neighbours(NA, NB) if nbr_kind == "ring" else two_way_ring(NA)
    dH = rand_c((NA, NB, 3, Norb, Norb), 14) * 0.5
    Gl, Gg = rand_c((Nkz, NE, NA, Norb, Norb), 15), rand_c((Nkz, NE, NA, Norb, Norb), 16)
    Pl, Pg = run(nbr, dH, Gl, Gg, Nqz, Nw)
    D0 = rand_c((Nqz, Nw, NA, NB, 3, 3), 17)  # the weight gradient does not depend on the weights
    zero = np.zeros_like(Gl)
    herm = lambda G: np.conj(np.swapaxes(G, -1, -2))
    # Pi^<: t = <, u = >
    _, _, gDg = oracle.sigma_grad(nbr, dH, D0, D0, Gl, herm(Gg), SCALE, zero, Gl)
    assert normwise(Pl[:, :, :, :NB], gDg) < 1e-13
    # Pi^>: t = >, u = <
    _, gDl, _ = oracle.sigma_grad(nbr, dH, D0, D0, herm(Gl), Gg, SCALE, Gg, zero)
    assert normwise(Pg[:, :, :, :NB], gDl) < 1e-13


@pytest.mark.parametrize("d", [
    Dims(NA=6, NB=2, Norb=3, NE=10, Nkz=3, Nqz=3, Nw=3),
    Dims(NA=5, NB=3, Norb=2, NE=7, Nkz=4, Nqz=2, Nw=6),   # Nqz < Nkz, Nw = NE - 1 (the last lag pairs one energy)
    Dims(NA=3, NB=1, Norb=1, NE=4, Nkz=1, Nqz=1, Nw=2),   # scalar blocks, one kz
], ids=["square", "ragged_all_lags", "scalar"])
def test_literal_einsum(d):
    """Brute force: Eq. (4) in the layout above, one einsum per (t, q, w) over (kz, E, a, s, i, j) and the orbital
    indices of the trace; the diagonal slot sums the bond slots."""
    x = make_inputs(d, seed=21)
    Pl, Pg = run(x.nbr, x.dH, x.G_less, x.G_greater, d.Nqz, d.Nw)
    A, nbr = x.dH.numpy(), x.nbr.numpy()
    Gs = (x.G_less.numpy(), x.G_greater.numpy())
    k = np.arange(d.Nkz)
    for t, P in enumerate((Pl, Pg)):
        ref = np.zeros_like(P)
        for q in range(d.Nqz):
            for w in range(d.Nw):
                nE = d.NE - (w + 1)  # energies E with E + (w + 1) inside the grid
                X = Gs[t][(k + q) % d.Nkz][:, w + 1:w + 1 + nE]     # G^t_aa(E + w + 1, k + q)  [k, E, a, n, p]
                Y = Gs[1 - t][:, :nE][:, :, nbr]                      # G^t'_bb(E, k)             [k, E, a, s, r, m]
                bond = -1j * SCALE * np.einsum("asinm,kEanp,asjpr,kEasrm->asij", A.conj(), X, A, Y, optimize=True)
                ref[q, w, :, :d.NB] = bond
                ref[q, w, :, d.NB] = bond.sum(axis=1)
        assert normwise(P, ref) < 1e-13
