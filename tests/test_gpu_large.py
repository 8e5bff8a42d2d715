"""Large workload (NA=4096, NB=4, Norb=10, NE=1024, Nkz=Nqz=5, Nw=64).

Mixed-precision (BF16X3) forward processed in energy windows of 256 outputs
with a 2*64 halo and the transform-based FP64 forward (FFT length 1152),
checked against the FP64 oracle on sampled blocks (grid edges, window
boundaries, interior); the phonon self-energy Pi on a sampled atom; the
FP64 adjoint on a subset of atoms checked against central differences of the
FP64 forward; and the transform-based adjoint on a subset of atoms against
the direct one. The FP32_FFT forward, Pi and adjoint, and the F16X3_FFT
(tensor-core) forward, are checked the same way to their stated bounds
(2e-6, 2e-6, 1e-5, 2e-6).
"""
import math

import numpy as np
import pytest
import torch

from conftest import normwise
from oracle.subproblem import oracle_blocks
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import LARGE, make_inputs, make_upstream

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)


@pytest.fixture(scope="module")
def large():
    torch.cuda.empty_cache()
    inp = make_inputs(LARGE, seed=5, device="cuda")
    yield inp
    del inp
    torch.cuda.empty_cache()


def test_large_bf16x3_windows_sampled(large):
    inp = large
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="bf16x3",
                     check=True)
    torch.cuda.synchronize()
    errs = []
    # energies at the grid edges and across the window boundaries 256 and 512
    for (a, E0, E1) in [(0, 0, 2), (4095, 1022, 1024), (2047, 255, 257), (1500, 511, 513), (77, 700, 702)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a,
                               E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            errs.append(normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("large bf16x3 sampled errors", errs)
    assert max(errs) <= 2e-5
    for S in (Sl, Sg):  # anti-Hermitian inputs give anti-Hermitian Sigma, up to the mode's error
        blk = S[:, ::101, ::257]
        assert float((blk + blk.conj().transpose(-1, -2)).abs().max()) <= 2e-5 * float(blk.abs().max())
    del Sl, Sg
    torch.cuda.empty_cache()


def test_large_fp64_fft_sampled(large):
    inp = large
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="fp64_fft",
                     check=True)
    torch.cuda.synchronize()
    errs = []
    for (a, E0, E1) in [(0, 0, 2), (4095, 1022, 1024), (2047, 511, 513), (77, 700, 702)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a,
                               E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            errs.append(normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("large fp64_fft sampled errors", errs)
    assert max(errs) <= 1e-12
    del Sl, Sg
    torch.cuda.empty_cache()


def test_large_pi_sampled(large):
    """Pi of Eq. (4) at the large sizes; the oracle on the exact sub-problem of one atom and its neighbours."""
    import oracle
    inp = large
    Pl, Pg = B.pi(inp.G_less, inp.G_greater, inp.dH, inp.nbr, LARGE.Nqz, LARGE.Nw, check=True)
    torch.cuda.synchronize()
    a = 3001
    nb = [int(x) for x in inp.nbr[a].cpu()]
    idx = torch.tensor([a] + nb, device="cuda")
    nbr = torch.zeros((len(nb) + 1, len(nb)), dtype=torch.int32)
    nbr[0] = torch.arange(1, len(nb) + 1, dtype=torch.int32)
    Ol, Og = oracle.pi(nbr, inp.dH.index_select(0, idx).cpu(), inp.G_less.index_select(2, idx).cpu(),
                       inp.G_greater.index_select(2, idx).cpu(), SCALE, LARGE.Nqz, LARGE.Nw, a_range=(0, 1))
    for P, O in ((Pl, Ol), (Pg, Og)):
        assert normwise(P[:, :, a].cpu().numpy(), O[:, :, 0]) <= 1e-12
    del Pl, Pg
    torch.cuda.empty_cache()


def test_large_fp64_adjoint_atom_subset(large):
    """FP64 gradients for atoms [0, 8) at the large sizes vs central differences (h = 1e-6)."""
    inp = large
    a0, a1 = 0, 8
    W, V = make_upstream(LARGE, seed=6, device="cuda")
    g_dH, g_Dl, g_Dg = B.sigma_grad(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V,
                                    scale=SCALE, atoms=(a0, a1), check=True)
    torch.cuda.synchronize()
    grads = {"dH": g_dH, "D_less": g_Dl, "D_greater": g_Dg}
    gscale = max(float(g_dH[a0:a1].abs().max()), float(g_Dl[:, :, a0:a1].abs().max()),
                 float(g_Dg[:, :, a0:a1].abs().max()))

    out = (torch.zeros_like(inp.G_less), torch.zeros_like(inp.G_greater))  # reused: 2 x 33.5 GB

    def loss(a):
        Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, scale=SCALE,
                         atoms=(a, a + 1), out=out)
        return float((W[:, :, a].conj() * Sl[:, :, a]).real.sum() + (V[:, :, a].conj() * Sg[:, :, a]).real.sum())

    rng = np.random.default_rng(7)
    h = 1e-6
    for _ in range(8):
        name = ("dH", "D_less", "D_greater")[int(rng.integers(3))]
        base = getattr(inp, name)
        a = int(rng.integers(a0, a1))
        sub = base[a] if name == "dH" else base[:, :, a]
        flat = int(rng.integers(sub.numel()))
        part = int(rng.integers(2))
        idx = np.unravel_index(flat, tuple(sub.shape))
        full_idx = (a,) + idx if name == "dH" else idx[:2] + (a,) + idx[2:]
        orig = base[full_idx].item()
        step = h if part == 0 else 1j * h
        base[full_idx] = orig + step
        lp = loss(a)
        base[full_idx] = orig - step
        lm = loss(a)
        base[full_idx] = orig
        fd = (lp - lm) / (2 * h)
        an = grads[name][full_idx].item()
        an = an.real if part == 0 else an.imag
        assert abs(fd - an) <= 1e-7 * gscale, (name, full_idx, part, fd, an)
    # atoms outside the range are untouched (zero-initialised by the binding)
    assert float(g_dH[a1:].abs().max()) == 0.0


def test_large_fp64_fft_adjoint_atom_subset(large):
    """Transform-based adjoint at the large sizes for atoms [100, 108) against the direct FP64 adjoint."""
    inp = large
    W, V = make_upstream(LARGE, seed=9, device="cuda")
    args = (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V)
    got = B.sigma_grad(*args, mode="fp64_fft", atoms=(100, 108), check=True)
    ref = B.sigma_grad(*args, mode="fp64", atoms=(100, 108))
    for x, y, sl in zip(got, ref, (np.s_[100:108], np.s_[:, :, 100:108], np.s_[:, :, 100:108])):
        err = float((x[sl] - y[sl]).abs().max() / y[sl].abs().max())
        assert err <= 1e-12, err
    del W, V
    torch.cuda.empty_cache()


def test_large_fp32_fft_sampled(large):
    """FP32_FFT forward at the large sizes (L = 1152): sampled blocks against the oracle to the mode's bound 2e-6."""
    inp = large
    Sl, Sg = B.sigma(inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, mode="fp32_fft",
                     check=True)
    torch.cuda.synchronize()
    errs = []
    for (a, E0, E1) in [(0, 0, 2), (4095, 1022, 1024), (2047, 511, 513), (77, 700, 702)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a,
                               E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            errs.append(normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("large fp32_fft sampled errors", errs)
    assert max(errs) <= 2e-6
    del Sl, Sg
    torch.cuda.empty_cache()


def test_large_f16x3_fft_sampled(large):
    """F16X3_FFT forward (FP32 transforms, block products on the tensor cores) at the large sizes: sampled blocks
    against the oracle to the mode's bound 2e-6."""
    inp = large
    args = (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr)
    Sl, Sg = B.sigma(*args, mode="f16x3_fft", check=True)
    torch.cuda.synchronize()
    errs = []
    for (a, E0, E1) in [(0, 0, 2), (4095, 1022, 1024), (2047, 511, 513), (1234, 300, 302)]:
        Ol, Og = oracle_blocks(inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE, a,
                               E0, E1)
        for S, O in ((Sl, Ol), (Sg, Og)):
            errs.append(normwise(S[:, E0:E1, a].cpu().numpy(), O))
    print("large f16x3_fft sampled errors", errs)
    assert max(errs) <= 2e-6
    del Sl, Sg
    torch.cuda.empty_cache()


def test_large_fp32_pi_sampled(large):
    """FP32_FFT Pi at the large sizes on one atom against the oracle's exact sub-problem (bound 2e-6)."""
    import oracle
    inp = large
    Pl, Pg = B.pi(inp.G_less, inp.G_greater, inp.dH, inp.nbr, LARGE.Nqz, LARGE.Nw, check=True, mode="fp32_fft")
    torch.cuda.synchronize()
    a = 1234
    nb = [int(x) for x in inp.nbr[a].cpu()]
    idx = torch.tensor([a] + nb, device="cuda")
    nbr = torch.zeros((len(nb) + 1, len(nb)), dtype=torch.int32)
    nbr[0] = torch.arange(1, len(nb) + 1, dtype=torch.int32)
    Ol, Og = oracle.pi(nbr, inp.dH.index_select(0, idx).cpu(), inp.G_less.index_select(2, idx).cpu(),
                       inp.G_greater.index_select(2, idx).cpu(), SCALE, LARGE.Nqz, LARGE.Nw, a_range=(0, 1))
    errs = [normwise(P[:, :, a].cpu().numpy(), O[:, :, 0]) for P, O in ((Pl, Ol), (Pg, Og))]
    print("large fp32 pi errors", errs)
    assert max(errs) <= 2e-6
    del Pl, Pg
    torch.cuda.empty_cache()


def test_large_fp32_fft_adjoint_atom_subset(large):
    """FP32_FFT adjoint at the large sizes for atoms [100, 108) against the direct FP64 adjoint (bound 1e-5)."""
    inp = large
    W, V = make_upstream(LARGE, seed=10, device="cuda")
    args = (inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr, W, V)
    got = B.sigma_grad(*args, mode="fp32_fft", atoms=(100, 108), check=True)
    ref = B.sigma_grad(*args, mode="fp64", atoms=(100, 108))
    errs = []
    for x, y, sl in zip(got, ref, (np.s_[100:108], np.s_[:, :, 100:108], np.s_[:, :, 100:108])):
        errs.append(float((x[sl] - y[sl]).abs().max() / y[sl].abs().max()))
    print("large fp32 adjoint errors", errs)
    assert max(errs) <= 1e-5
    del W, V
    torch.cuda.empty_cache()
