"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/sse_oracle.c (on the CPU),
builds it, and checks that at least one pin (tests/test_oracle_pins.py,
tests/test_oracle_adjoint.py, tests/test_oracle_dcomb.py, tests/test_oracle_pi.py,
tests/test_oracle_grad_g.py) fails against the mutated build.
"""
import os

import pytest

import oracle
import test_oracle_adjoint as adj
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "sse_oracle.c")

# (name, original text, mutated text, which pins to run)
FWD = [
    ("emission/absorption types swapped", "const int tau = sigma == +1 ? t : 1 - t;\n                    const cplx* Gp",
     "const int tau = sigma == +1 ? 1 - t : t;\n                    const cplx* Gp"),
    ("energy shift sign", "const int Ep = E - sigma * (w + 1);\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out",
     "const int Ep = E + sigma * (w + 1);\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out"),
    ("frequency offset off by one", "const int Ep = E - sigma * (w + 1);\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out",
     "const int Ep = E - sigma * (w + 0);\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out"),
    ("kz shift sign", "const int kp = ((k - q) % d->Nkz + d->Nkz) % d->Nkz; /* kz - qz",
     "const int kp = ((k + q) % d->Nkz + d->Nkz) % d->Nkz; /* kz - qz"),
    ("absorption term dropped", "for (int sg = 0; sg < 2; ++sg) {\n                    const int sigma = sg == 0 ? +1 : -1;\n                    const int Ep = E - sigma",
     "for (int sg = 0; sg < 1; ++sg) {\n                    const int sigma = sg == 0 ? +1 : -1;\n                    const int Ep = E - sigma"),
    ("right factor not conjugate-transposed", "mm_bh(n, P, J->dH + off_dH(d, a, s, j), Q);",
     "mm(n, P, J->dH + off_dH(d, a, s, j), Q);"),
    ("factor order G dH_i", "mm(n, J->dH + off_dH(d, a, s, i), Gp, P);", "mm(n, Gp, J->dH + off_dH(d, a, s, i), P);"),
    ("weight indices transposed", "const cplx dij = Dc[i * 3 + j];", "const cplx dij = Dc[j * 3 + i];"),
    ("prefactor i dropped", "J.c = I * scale;\n    J.n_out = 2LL * (d->a_end",
     "J.c = scale;\n    J.n_out = 2LL * (d->a_end"),
    ("neighbour G replaced by own atom", "const cplx* Gp = J->G[t] + off_G(d, kp, Ep, b);\n                    const cplx* Dc = J->D[tau]",
     "const cplx* Gp = J->G[t] + off_G(d, kp, Ep, a);\n                    const cplx* Dc = J->D[tau]"),
    # the two below change nothing for anti-Hermitian G and D blocks (the delta-response and closed-form pins,
    # whose inputs are not anti-Hermitian, and the general-input einsum catch them)
    ("G taken as -G^H", "mm(n, J->dH + off_dH(d, a, s, i), Gp, P); /* dH_i(a,b) G_bb */",
     "mm_bh(n, J->dH + off_dH(d, a, s, i), Gp, P); for (int e = 0; e < nn; ++e) P[e] = -P[e];"),
    ("weight taken as -D^H", "const cplx dij = Dc[i * 3 + j];", "const cplx dij = -conj(Dc[j * 3 + i]);"),
    ("edge terms wrapped instead of dropped",
     "const int Ep = E - sigma * (w + 1);\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out",
     "const int Ep = ((E - sigma * (w + 1)) % d->NE + d->NE) % d->NE;\n                    if (Ep < 0 || Ep >= d->NE) continue; /* out"),
]
BWD = [
    ("grad D not conjugated", "gDc[i * 3 + j] += conj(J->c * frob(n, W, T));", "gDc[i * 3 + j] += J->c * frob(n, W, T);"),
    ("grad dH right term uses D_mi", "const cplx f = J->c * Dc[i * 3 + m];", "const cplx f = J->c * Dc[m * 3 + i];"),
    ("grad dH left term not conjugated", "const cplx f = conj(J->c * Dc[m * 3 + j]);", "const cplx f = J->c * Dc[m * 3 + j];"),
    ("grad dH left term misses G^H", "mm_bh(n, T, Gp, AG + (size_t)j * nn);  /* W dH_j G^H */",
     "mm(n, T, Gp, AG + (size_t)j * nn);  /* W dH_j G^H */"),
    # changes nothing for anti-Hermitian G: only the problem with general G and D catches it
    ("grad dH left term takes G^H as -G", "mm_bh(n, T, Gp, AG + (size_t)j * nn);  /* W dH_j G^H */",
     "mm(n, T, Gp, AG + (size_t)j * nn); for (int e = 0; e < nn; ++e) AG[(size_t)j * nn + e] = -AG[(size_t)j * nn + e];"),
]
DCOMB = [
    ("own slot instead of the reverse slot", "const cplx* Dba = raw[t] + off_raw(d, q, w, b, sr);",
     "const cplx* Dba = raw[t] + off_raw(d, q, w, b, s);"),
    ("self block of the wrong atom", "const cplx* Daa = raw[t] + off_raw(d, q, w, a, d->NB);",
     "const cplx* Daa = raw[t] + off_raw(d, q, w, b, d->NB);"),
    ("sign of D_aa", "for (int e = 0; e < 9; ++e) o[e] = Dba[e] - Dbb[e] - Daa[e] + Dab[e];",
     "for (int e = 0; e < 9; ++e) o[e] = Dba[e] - Dbb[e] + Daa[e] + Dab[e];"),
    ("adjoint misses the D_bb term", "                            Dbb[e] -= gi[e];\n", "\n"),
]
PI = [
    ("G_ll of the same type", "mm(n, A + (size_t)i * nn, J->G[1 - t] + off_G(d, k, E, b), R + o);",
     "mm(n, A + (size_t)i * nn, J->G[t] + off_G(d, k, E, b), R + o);"),
    ("energy shift sign", "const int Ep = E + (w + 1);\n                    if (Ep >= d->NE) continue;",
     "const int Ep = E - (w + 1);\n                    if (Ep < 0) continue;"),
    ("frequency offset off by one", "const int Ep = E + (w + 1);\n                    if (Ep >= d->NE) continue;",
     "const int Ep = E + (w + 0);\n                    if (Ep >= d->NE) continue;"),
    ("edge energies wrapped", "const int Ep = E + (w + 1);\n                    if (Ep >= d->NE) continue;",
     "const int Ep = (E + (w + 1)) % d->NE;\n                    if (Ep >= d->NE) continue;"),
    ("kz shift sign", "const int kp = (k + q) % d->Nkz; /* kz + qz, periodic */",
     "const int kp = ((k - q) % d->Nkz + d->Nkz) % d->Nkz; /* kz + qz, periodic */"),
    ("left coupling not conjugate-transposed", "mm_ah(n, A + (size_t)i * nn, J->G[t] + off_G(d, k, E, a), P + o);",
     "mm(n, A + (size_t)i * nn, J->G[t] + off_G(d, k, E, a), P + o);"),
    ("neighbour G replaced by own atom", "mm(n, A + (size_t)i * nn, J->G[1 - t] + off_G(d, k, E, b), R + o);",
     "mm(n, A + (size_t)i * nn, J->G[1 - t] + off_G(d, k, E, a), R + o);"),
    ("(i, j) transposed", "o[i * 3 + j] += tr;", "o[j * 3 + i] += tr;"),
    ("prefactor sign", "const cplx c = -I * scale;", "const cplx c = I * scale;"),
    ("diagonal block misses a neighbour", "self[e] += v[e];  /* diagonal", "if (s > 0) self[e] += v[e];  /* diagonal"),
]
GRADG = [
    ("grad G energy shift sign", "const int E = Ep + sigma * (w + 1);", "const int E = Ep - sigma * (w + 1);"),
    ("grad G kz shift sign", "const int k = (kp + q) % d->Nkz; /* kz - qz = k' */",
     "const int k = ((kp - q) % d->Nkz + d->Nkz) % d->Nkz; /* kz - qz = k' */"),
    ("grad G weight not conjugated", "const cplx f = conj(J->c * Dc[i * 3 + j]);", "const cplx f = J->c * Dc[i * 3 + j];"),
    ("grad G types swapped", "const int tau = sigma == +1 ? t : 1 - t;\n                        const cplx* Wa",
     "const int tau = sigma == +1 ? 1 - t : t;\n                        const cplx* Wa"),
    ("grad G left coupling not conjugate-transposed", "mm_ah(n, J->dH + off_dH(d, a, s, i), Wa, P); /* dH_i^H W */",
     "mm(n, J->dH + off_dH(d, a, s, i), Wa, P); /* dH_i^H W */"),
]


def _gradg_pins():
    import test_oracle_grad_g as gg

    class _Req:
        def __init__(self, p):
            self.param = p

    def run(kind):
        prob = gg.problem.__wrapped__(_Req(kind))
        gg.test_dot_product(prob)
        gg.test_central_differences(prob)
    yield lambda: run("ring")
    yield lambda: run("two_way_ring")


def _pi_pins():
    import test_oracle_pi as pp
    yield pp.test_closed_form_constant_G
    for args in [(2, 6, 0, 3), (0, 4, 1, 0), (1, 8, 1, 7)]:
        yield lambda a=args: pp.test_delta_response(*a)
    yield pp.test_anti_hermitian_blocks
    yield pp.test_quadratic_in_coupling
    yield lambda: pp.test_equals_sigma_adjoint_weight_gradient("ring")
    yield lambda: pp.test_equals_sigma_adjoint_weight_gradient("two_way_ring")


def _dcomb_pins():
    import test_oracle_dcomb as dc
    yield dc.test_worked_example
    yield lambda: dc.test_exchange_symmetry("diamond")
    yield lambda: dc.test_exchange_symmetry("two_way_ring")
    yield dc.test_uniform_blocks_cancel
    yield dc.test_adjoint_dot_product


def _fwd_pins():
    yield pins.test_scalar_worked_example
    yield pins.test_closed_form_constant_G
    for args in [(0, 1, 5, 0), (2, 2, 3, 1), (1, 0, 0, 2)]:
        yield lambda a=args: pins.test_delta_response(*a)
    yield pins.test_anti_hermitian
    yield pins.test_sesquilinear_in_dH
    yield pins.test_term_count_matches_paper_flop_model
    yield lambda: pins.test_literal_einsum(pins.Dims(NA=7, NB=3, Norb=5, NE=11, Nkz=4, Nqz=2, Nw=3), True)


def _bwd_pins():
    def run(general):
        problem = adj.make_problem(general)
        adj.test_gradient_central_differences(problem)
        adj.test_dot_product_in_D(problem)
        adj.test_dot_product_in_dH(problem)
    yield lambda: run(False)
    yield lambda: run(True)


def _build(tmp_path, old, new):
    with open(SRC) as f:
        src = f.read()
    assert src.count(old) == 1, f"mutation anchor not found exactly once: {old!r}"
    path = tmp_path / "mut.c"
    path.write_text(src.replace(old, new))
    return oracle.compile_source(str(path), str(tmp_path / "libmut.so"))


def _caught(so, tests):
    with oracle._library(so):
        for t in tests:
            try:
                t()
            except AssertionError:
                return True
    return False


@pytest.mark.parametrize("name,old,new", FWD, ids=[m[0] for m in FWD])
def test_forward_mutation_is_caught(tmp_path, name, old, new):
    assert _caught(_build(tmp_path, old, new), _fwd_pins()), f"no pin caught: {name}"


@pytest.mark.parametrize("name,old,new", BWD, ids=[m[0] for m in BWD])
def test_adjoint_mutation_is_caught(tmp_path, name, old, new):
    assert _caught(_build(tmp_path, old, new), _bwd_pins()), f"no pin caught: {name}"


@pytest.mark.parametrize("name,old,new", DCOMB, ids=[m[0] for m in DCOMB])
def test_dcomb_mutation_is_caught(tmp_path, name, old, new):
    assert _caught(_build(tmp_path, old, new), _dcomb_pins()), f"no pin caught: {name}"


@pytest.mark.parametrize("name,old,new", PI, ids=[m[0] for m in PI])
def test_pi_mutation_is_caught(tmp_path, name, old, new):
    assert _caught(_build(tmp_path, old, new), _pi_pins()), f"no pin caught: {name}"


@pytest.mark.parametrize("name,old,new", GRADG, ids=[m[0] for m in GRADG])
def test_gradg_mutation_is_caught(tmp_path, name, old, new):
    assert _caught(_build(tmp_path, old, new), _gradg_pins()), f"no pin caught: {name}"


def test_unmutated_source_passes(tmp_path):
    so = _build(tmp_path, "#include <complex.h>", "#include <complex.h>")
    assert not _caught(so, list(_fwd_pins()) + list(_bwd_pins()) + list(_dcomb_pins()) + list(_pi_pins()) +
                       list(_gradg_pins()))
