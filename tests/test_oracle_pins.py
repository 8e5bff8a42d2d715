"""Pins of the FP64 CPU oracle (Eq. 3) to facts other than itself.

Each test checks the oracle against something the paper or the mathematics
fixes: a hand-derived worked example, a closed form, a delta response, an
invariant, or the paper's flop model. Together they catch a dropped term, a
wrong sign or index, a swapped emission/absorption pairing or a transposed
operand anywhere in the oracle.
"""
import dataclasses
import json
import os

import numpy as np
import pytest
import torch

import oracle
from conftest import normwise
from paper_1912_10024_gb300.inputs import Dims, TINY, make_inputs, ring_neighbours

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SCALE = 1.0 / (2.0 * np.pi)
SMALL = Dims(NA=6, NB=2, Norb=3, NE=9, Nkz=3, Nqz=2, Nw=2)


def run(inp, scale=SCALE, **kw):
    return oracle.sigma(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, scale, **kw)


def cplx(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]


# --------------------------------------------------------------------------
# worked example (golden fixture)
# --------------------------------------------------------------------------

def test_scalar_worked_example():
    """Eq. (3) with 1x1 blocks: hand-derived values in tests/golden/scalar_case.json."""
    with open(os.path.join(GOLDEN, "scalar_case.json")) as f:
        g = json.load(f)
    dH = cplx(g["dH"]).reshape(1, 1, 3, 1, 1)
    Dl = cplx(g["D_less"]).reshape(1, 1, 1, 1, 3, 3)
    Dg = cplx(g["D_greater"]).reshape(1, 1, 1, 1, 3, 3)
    Gl = cplx(g["G_less"]).reshape(1, 3, 1, 1, 1)
    Gg = cplx(g["G_greater"]).reshape(1, 3, 1, 1, 1)
    nbr = np.zeros((1, 1), np.int32)
    Sl, Sg = oracle.sigma(nbr, dH, Dl, Dg, Gl, Gg, 1.0)
    np.testing.assert_array_equal(Sl.reshape(3), cplx(g["Sigma_less"]))
    np.testing.assert_array_equal(Sg.reshape(3), cplx(g["Sigma_greater"]))


# --------------------------------------------------------------------------
# closed form: G constant in E and kz
# --------------------------------------------------------------------------

def test_closed_form_constant_G():
    """With G^t_b(E,k) = G0^t_b, Eq. (3) collapses to a weight times dH_i G0 dH_j^H.

    Sigma^t_a(E) = c sum_s sum_ij K^t_ij(a,s,E) dH_i G0_b dH_j^H with
    K^t(a,s,E) = sum_q [ sum_{w: E-(w+1) >= 0} D^t(q,w) + sum_{w: E+(w+1) < NE} D^tbar(q,w) ],
    independent of kz.
    """
    d = Dims(NA=7, NB=3, Norb=4, NE=11, Nkz=4, Nqz=3, Nw=3)
    inp = make_inputs(d, seed=5, nbr=torch.tensor([[(a + 1) % 7, (a + 3) % 7, (a + 6) % 7] for a in range(7)],
                                                  dtype=torch.int32))
    G0l = inp.G_less[0, 0].clone()
    G0g = inp.G_greater[0, 0].clone()
    inp.G_less[:] = G0l
    inp.G_greater[:] = G0g
    Sl, Sg = run(inp)
    E = np.arange(d.NE)[:, None]
    w = np.arange(d.Nw)[None, :]
    em = (E - (w + 1) >= 0).astype(float)  # [E, w] emission term in range
    ab = (E + (w + 1) < d.NE).astype(float)  # [E, w] absorption term in range
    nbr = inp.nbr.numpy()
    A = inp.dH.numpy()
    Dl, Dg = inp.D_less.numpy(), inp.D_greater.numpy()
    c = 1j * SCALE
    for (Dt, Dtb, G0, S) in ((Dl, Dg, G0l.numpy(), Sl), (Dg, Dl, G0g.numpy(), Sg)):
        K = np.einsum("ew,qwasij->easij", em, Dt) + np.einsum("ew,qwasij->easij", ab, Dtb)
        Gb = G0[nbr]  # [a, s, m, n]
        M = np.einsum("asiml,asln,asjpn->asijmp", A, Gb, A.conj())  # dH_i G dH_j^H
        ref = c * np.einsum("easij,asijmp->eamp", K, M)
        for k in range(d.Nkz):
            assert normwise(S[k], ref) < 1e-13


# --------------------------------------------------------------------------
# delta response: pins the kz shift direction, the energy shift direction and
# the emission/absorption type pairing
# --------------------------------------------------------------------------

@pytest.mark.parametrize("k0,q0,E0,w0", [(0, 1, 5, 0), (2, 2, 3, 1), (1, 0, 0, 2)])
def test_delta_response(k0, q0, E0, w0):
    d = Dims(NA=5, NB=2, Norb=3, NE=9, Nkz=3, Nqz=3, Nw=3)
    inp = make_inputs(d, seed=11, nbr=ring_neighbours(5, 2))
    for G in (inp.G_less, inp.G_greater):
        keep = G[k0, E0].clone()
        G.zero_()
        G[k0, E0] = keep
    for D in (inp.D_less, inp.D_greater):
        keep = D[q0, w0].clone()
        D.zero_()
        D[q0, w0] = keep
    Sl, Sg = run(inp)
    kout = (k0 + q0) % d.Nkz  # G(kz - qz) is nonzero only when kz = k0 + q0
    nbr = inp.nbr.numpy()
    A = inp.dH.numpy()
    c = 1j * SCALE
    Dl, Dg = inp.D_less.numpy()[q0, w0], inp.D_greater.numpy()[q0, w0]

    def block(Dw, G0):
        Gb = G0[nbr]
        return c * np.einsum("asij,asiml,asln,asjpn->amp", Dw, A, Gb, A.conj())

    for t, (S, G, Dt, Dtb) in enumerate(((Sl, inp.G_less.numpy(), Dl, Dg), (Sg, inp.G_greater.numpy(), Dg, Dl))):
        expect = np.zeros_like(S)
        Ee = E0 + (w0 + 1)  # emission: E - (w+1) = E0, weight of the same type
        Ea = E0 - (w0 + 1)  # absorption: E + (w+1) = E0, weight of the other type
        if Ee < d.NE:
            expect[kout, Ee] += block(Dt, G[k0, E0])
        if Ea >= 0:
            expect[kout, Ea] += block(Dtb, G[k0, E0])
        assert np.count_nonzero(S[np.abs(expect) == 0]) == 0, "support of the response is wrong"
        assert normwise(S, expect) < 1e-13


# --------------------------------------------------------------------------
# invariants
# --------------------------------------------------------------------------

def test_linearity_in_D_and_G():
    """Sigma(al X1 + be X2) = al Sigma(X1) + be Sigma(X2) for X = (D^<, D^>) and X = (G^<, G^>)."""
    nbr = ring_neighbours(6, 2)
    inp1 = make_inputs(SMALL, seed=1, nbr=nbr)
    inp2 = make_inputs(SMALL, seed=2, nbr=nbr)
    al, be = 0.7 - 1.3j, -0.4 + 0.25j
    S1 = run(inp1)
    for names in (("D_less", "D_greater"), ("G_less", "G_greater")):
        other = dataclasses.replace(inp1, **{n: getattr(inp2, n) for n in names})
        mixed = dataclasses.replace(inp1, **{n: al * getattr(inp1, n) + be * getattr(inp2, n) for n in names})
        S2, Smix = run(other), run(mixed)
        for t in range(2):
            assert normwise(Smix[t], al * S1[t] + be * S2[t]) < 1e-13


def test_sesquilinear_in_dH():
    """dH enters once plain and once conjugate-transposed: Sigma(lam dH) = |lam|^2 Sigma(dH)."""
    inp = make_inputs(SMALL, seed=3, nbr=ring_neighbours(6, 2))
    S = run(inp)
    lam = 0.6 + 0.8j * 1.7
    inp.dH = lam * inp.dH
    S2 = run(inp)
    for t in range(2):
        assert normwise(S2[t], abs(lam) ** 2 * S[t]) < 1e-13


def test_anti_hermitian():
    """Anti-Hermitian G^t and Dc^t blocks give anti-Hermitian Sigma^t.

    sum_ij D_ij A_i G A_j^H is Hermitian when D^H = -D and G^H = -G, so
    i*scale times it is anti-Hermitian. A Hermitian D breaks it (control).
    """
    inp = make_inputs(TINY, seed=0)
    for S in run(inp):
        assert np.abs(S + np.swapaxes(S.conj(), -1, -2)).max() < 1e-15 * 10 * np.abs(S).max() + 1e-18
    inp.D_less = inp.D_less * 1j  # now Hermitian: the property must fail
    Sl, _ = run(inp)
    assert np.abs(Sl + np.swapaxes(Sl.conj(), -1, -2)).max() > 1e-3 * np.abs(Sl).max()


def test_kz_roll_covariance():
    inp = make_inputs(SMALL, seed=4, nbr=ring_neighbours(6, 2))
    S = run(inp)
    inp.G_less = torch.roll(inp.G_less, 1, dims=0)
    inp.G_greater = torch.roll(inp.G_greater, 1, dims=0)
    S2 = run(inp)
    for t in range(2):
        assert normwise(S2[t], np.roll(S[t], 1, axis=0)) < 1e-14


def test_atom_relabel_covariance():
    """On the ring list, shifting every atom label by one shifts Sigma."""
    inp = make_inputs(SMALL, seed=6, nbr=ring_neighbours(6, 2))
    S = run(inp)
    inp.G_less = torch.roll(inp.G_less, 1, dims=2)
    inp.G_greater = torch.roll(inp.G_greater, 1, dims=2)
    inp.dH = torch.roll(inp.dH, 1, dims=0)
    inp.D_less = torch.roll(inp.D_less, 1, dims=2)
    inp.D_greater = torch.roll(inp.D_greater, 1, dims=2)
    S2 = run(inp)
    for t in range(2):
        assert normwise(S2[t], np.roll(S[t], 1, axis=2)) < 1e-14


def test_slot_permutation_invariance():
    inp = make_inputs(SMALL, seed=7, nbr=torch.tensor([[(a + 1) % 6, (a + 4) % 6] for a in range(6)],
                                                      dtype=torch.int32))
    S = run(inp)
    perm = [1, 0]
    inp.nbr = inp.nbr[:, perm].contiguous()
    inp.dH = inp.dH[:, perm].contiguous()
    inp.D_less = inp.D_less[:, :, :, perm].contiguous()
    inp.D_greater = inp.D_greater[:, :, :, perm].contiguous()
    S2 = run(inp)
    for t in range(2):
        assert normwise(S2[t], S[t]) < 1e-14


def test_ranges_compute_only_requested_blocks():
    inp = make_inputs(SMALL, seed=8, nbr=ring_neighbours(6, 2))
    S = run(inp)
    Sp = run(inp, a_range=(2, 5), E_range=(3, 7))
    for t in range(2):
        np.testing.assert_array_equal(Sp[t][:, 3:7, 2:5], S[t][:, 3:7, 2:5])
        mask = np.ones(S[t].shape, bool)
        mask[:, 3:7, 2:5] = False
        assert np.count_nonzero(Sp[t][mask]) == 0


# --------------------------------------------------------------------------
# flop model (Table 3): pins the term structure, not values
# --------------------------------------------------------------------------

def test_term_count_matches_paper_flop_model():
    """The oracle visits 2 (<,>) x 2 (emission, absorption) x Nqz x NB x Nw terms per
    output, minus those whose energy falls off the grid. With 6 products of
    8 Norb^3 flops per term (3 directions x 2 products) that is the paper's
    64 N_a N_b N_3D N_kz N_qz N_E N_w N_orb^3 model; its values for the 'Small'
    structure reproduce Table 3's OMEN row."""
    with open(os.path.join(GOLDEN, "table3_sse_flops.json")) as f:
        g = json.load(f)
    s = g["small_structure"]
    for nkz, ref in zip(g["N_kz"], g["sse_omen_pflop"]):
        model = 64 * s["N_a"] * s["N_b"] * s["N_3D"] * nkz * nkz * s["N_E"] * s["N_omega"] * 12 ** 3 / 1e15
        assert abs(model - ref) / ref < 2e-3
    d = SMALL
    inp = make_inputs(d, seed=9, nbr=ring_neighbours(6, 2))
    _, _, n = run(inp, count_terms=True)
    dropped = sum(1 for E in range(d.NE) for w in range(d.Nw) for Ep in (E - w - 1, E + w + 1) if not 0 <= Ep < d.NE)
    all_terms = 2 * d.NA * d.NB * d.Nkz * d.Nqz * d.NE * 2 * d.Nw
    assert n == all_terms - 2 * d.NA * d.NB * d.Nkz * d.Nqz * dropped
    assert all_terms * 6 * 8 * d.Norb ** 3 == 64 * d.NA * d.NB * 3 * d.Nkz * d.Nqz * d.NE * d.Nw * d.Norb ** 3


# --------------------------------------------------------------------------
# literal 9-term einsum (cross-check, not a pin on its own)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("d", [
    TINY,
    Dims(NA=5, NB=1, Norb=1, NE=7, Nkz=1, Nqz=1, Nw=6),   # scalar blocks, one kz, Nw = NE - 1 (every lag)
    Dims(NA=7, NB=3, Norb=5, NE=11, Nkz=4, Nqz=2, Nw=3),  # Nqz < Nkz, odd orbitals, ragged everything
    Dims(NA=4, NB=2, Norb=2, NE=2, Nkz=5, Nqz=5, Nw=1),   # the shortest energy grid
], ids=["tiny", "scalar_all_lags", "ragged_nqz_lt_nkz", "two_energies"])
@pytest.mark.parametrize("general", [False, True], ids=["antihermitian", "general"])
def test_literal_einsum(d, general):
    """Eq. (3) written out as one einsum per (E, w, sigma) term over the whole (kz, qz, a, s, i, j) index space, on
    shapes that reach its edge cases; with anti-Hermitian inputs and with G, D of no symmetry (where G^H and -G,
    D^H and -D differ, so the oracle may use neither in their place)."""
    inp = make_inputs(d, seed=0, general=general)
    Sl, Sg = run(inp)
    nbr = inp.nbr.numpy()
    A = inp.dH.numpy()
    k = np.arange(d.Nkz)[:, None]
    q = np.arange(d.Nqz)[None, :]
    kp = (k - q) % d.Nkz  # [k, q]
    c = 1j * SCALE
    for t, (G, S) in enumerate(((inp.G_less.numpy(), Sl), (inp.G_greater.numpy(), Sg))):
        Ds = (inp.D_less.numpy(), inp.D_greater.numpy())
        ref = np.zeros_like(S)
        for E in range(d.NE):
            for w in range(d.Nw):
                for sigma in (+1, -1):
                    Ep = E - sigma * (w + 1)
                    if not 0 <= Ep < d.NE:
                        continue
                    Dt = Ds[t if sigma == 1 else 1 - t][:, w]  # [q, a, s, i, j]
                    Gg = G[kp, Ep][:, :, nbr]  # [k, q, a, s, l, p]
                    ref[:, E] += c * np.einsum("qasij,asiml,kqaslp,asjnp->kamn", Dt, A, Gg, A.conj(),
                                               optimize=True)
        assert normwise(S, ref) < 1e-13


def test_oracle_results_do_not_depend_on_the_thread_count():
    """Sigma, Pi and the gradient in G sum every output block in one thread in a fixed order: bit-identical for any
    thread count. The adjoint splits the energies among the threads (private partial sums, then a fixed-order
    reduction), so its summation order follows the thread count: equal to rounding (1e-13 relative)."""
    import math
    from paper_1912_10024_gb300.inputs import make_upstream
    d = TINY
    x = make_inputs(d, seed=91)
    W, V = make_upstream(d, seed=92)
    scale = 1.0 / (2.0 * math.pi)
    args = (x.nbr, x.dH, x.D_less, x.D_greater, x.G_less, x.G_greater, scale)
    runs = {
        "sigma": lambda n: oracle.sigma(*args, nthreads=n),
        "pi": lambda n: oracle.pi(x.nbr, x.dH, x.G_less, x.G_greater, scale, d.Nqz, d.Nw, nthreads=n),
        "grad_G": lambda n: oracle.sigma_grad_G(x.nbr, x.dH, x.D_less, x.D_greater, scale, W, V, nthreads=n),
    }
    for name, run in runs.items():
        for a, b in zip(run(1), run(7)):
            assert np.array_equal(a, b), name
    for a, b in zip(oracle.sigma_grad(*args, W, V, nthreads=1), oracle.sigma_grad(*args, W, V, nthreads=7)):
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


# --------------------------------------------------------------------------
# reading R3 (absorption term) against the bosonic form
# --------------------------------------------------------------------------

def _bosonic_sigma(inp, d):
    """Eq. (3) with the absorption weight in the bosonic form: for sigma = -1 the weight of type t is the other
    type's combined weight transposed in (i, j) at -qz, Dc^{t'}_ji(w, -q) (from D^<_ab(-w, q) = D^>_ba(w, -q) and the
    a <-> b symmetry of the bond combination). Needs the full qz grid (Nqz = Nkz)."""
    nbr = inp.nbr.numpy()
    A = inp.dH.numpy()
    k = np.arange(d.Nkz)[:, None]
    q = np.arange(d.Nqz)[None, :]
    kp = (k - q) % d.Nkz
    qneg = (-np.arange(d.Nqz)) % d.Nkz
    c = 1j * SCALE
    Ds = (inp.D_less.numpy(), inp.D_greater.numpy())
    out = []
    for t, G in enumerate((inp.G_less.numpy(), inp.G_greater.numpy())):
        ref = np.zeros(d.g_shape(), dtype=np.complex128)
        for E in range(d.NE):
            for w in range(d.Nw):
                for sigma in (+1, -1):
                    Ep = E - sigma * (w + 1)
                    if not 0 <= Ep < d.NE:
                        continue
                    if sigma == 1:
                        Dt = Ds[t][:, w]
                    else:
                        Dt = np.swapaxes(Ds[1 - t][qneg, w], -1, -2)
                    Gg = G[kp, Ep][:, :, nbr]
                    ref[:, E] += c * np.einsum("qasij,asiml,kqaslp,asjnp->kamn", Dt, A, Gg, A.conj(), optimize=True)
        out.append(ref)
    return out


def test_absorption_reading_vs_bosonic_form():
    """The library's absorption weight Dc^{t'}_ij(w, qz) equals the bosonic form Dc^{t'}_ji(w, -qz) exactly when the
    combined weights are reciprocal, Dc_ij(w, q) = Dc_ji(w, -q) (phonon functions of a time-reversal-symmetric
    lattice); for weights that are not reciprocal the two readings differ, so the reading is a real choice."""
    d = Dims(NA=5, NB=2, Norb=3, NE=9, Nkz=4, Nqz=4, Nw=3)
    inp = make_inputs(d, seed=41, nbr=ring_neighbours(d.NA, d.NB), general=True)
    qneg = (-np.arange(d.Nqz)) % d.Nkz
    for name in ("D_less", "D_greater"):
        X = getattr(inp, name).numpy()
        recip = 0.5 * (X + np.swapaxes(X[qneg], -1, -2))  # Dc(q)_ij = Dc(-q)_ji
        setattr(inp, name, torch.from_numpy(recip.copy()))
    Sl, Sg = run(inp)
    Bl, Bg = _bosonic_sigma(inp, d)
    assert normwise(Sl, Bl) < 1e-13 and normwise(Sg, Bg) < 1e-13
    general = make_inputs(d, seed=42, nbr=ring_neighbours(d.NA, d.NB), general=True)
    Sl, Sg = run(general)
    Bl, Bg = _bosonic_sigma(general, d)
    assert normwise(Sl, Bl) > 1e-2 and normwise(Sg, Bg) > 1e-2
