"""Seeded synthetic inputs for the electron scattering self-energy (Eq. 3).

This module is shared by the CUDA path (tests, bench) and by the CPU oracle's
tests. It holds only input generation: neighbour lists and random tensors. It
contains none of the self-energy arithmetic.

The paper's Si FinFET structures (Sec. 5, "Small" and "Large") and their DFT
inputs are not available, so seeded synthetic tensors with the same shapes and
structure stand in for them:

* G^<, G^> : complex128 [Nkz, NE, NA, Norb, Norb]; G^< = i (A A^H),
  G^> = -i (B B^H), with A, B having independent real and imaginary parts
  ~ N(0, 1/Norb) (standard deviation 1/sqrt(Norb)). Both are exactly
  anti-Hermitian (the Hermitian part is symmetrised before multiplying by i).
* dH       : complex128 [NA, NB, 3, Norb, Norb], re/im ~ N(0, 0.1^2).
* D^<, D^> : complex128 [Nqz, Nw, NA, NB, 3, 3], D = (X - X^H)/2 with
  X re/im ~ N(0, 0.01^2) -- exactly anti-Hermitian 3x3 blocks.
* nbr      : int32 [NA, NB] neighbour list (ring or diamond lattice).

With ``general=True`` G^<, G^> are plain complex blocks (re/im ~ N(0, 1/Norb))
and D^<, D^> plain complex 3x3 blocks (re/im ~ N(0, 0.01^2)), with no
symmetry at all: these are the inputs on which a kernel that used G^H = -G or
D^H = -D without being told so would give a different Sigma.

Draw order is G^<, G^>, dH, D^<, D^> from one torch.Generator seeded with
`seed` on the requested device. The same bytes feed the GPU path and the
oracle: whoever generated them copies them to the other side.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import torch


@dataclasses.dataclass(frozen=True)
class Dims:
    """Problem sizes of Eq. (3).

    NA atoms, NB neighbours per atom, Norb orbitals per atom, NE energies,
    Nkz electron momenta, Nqz phonon momenta (Nqz <= Nkz), Nw phonon
    frequencies (energy offsets 1..Nw grid steps).
    """

    NA: int
    NB: int
    Norb: int
    NE: int
    Nkz: int
    Nqz: int
    Nw: int

    def g_shape(self):
        return (self.Nkz, self.NE, self.NA, self.Norb, self.Norb)

    def d_shape(self):
        return (self.Nqz, self.Nw, self.NA, self.NB, 3, 3)

    def dh_shape(self):
        return (self.NA, self.NB, 3, self.Norb, self.Norb)


# Workloads. Shapes follow the paper's OMEN validation structure (Norb=10,
# NB=4) and its Table 2 orders of magnitude: tiny (ring neighbour list), the
# Si-FinFET-shaped problem (4x4x8 diamond cells), the adjoint workload (2x2x8
# cells) and the large workload (8x8x8 cells); values from make_inputs below.
TINY = Dims(NA=16, NB=4, Norb=4, NE=32, Nkz=3, Nqz=3, Nw=4)
FINFET = Dims(NA=1024, NB=4, Norb=10, NE=512, Nkz=7, Nqz=7, Nw=32)
ADJOINT = Dims(NA=256, NB=4, Norb=10, NE=256, Nkz=5, Nqz=5, Nw=16)
LARGE = Dims(NA=4096, NB=4, Norb=10, NE=1024, Nkz=5, Nqz=5, Nw=64)

WORKLOADS = {"tiny": TINY, "finfet": FINFET, "adjoint": ADJOINT, "large": LARGE}


def ring_neighbours(NA: int, NB: int) -> torch.Tensor:
    """nbr[a][s] = (a + s + 1) mod NA (one-way ring list)."""
    a = torch.arange(NA, dtype=torch.int64).unsqueeze(1)
    s = torch.arange(NB, dtype=torch.int64).unsqueeze(0)
    return ((a + s + 1) % NA).to(torch.int32)


# Diamond lattice in units of a/4 (a = cubic lattice constant): the FCC basis
# and the same shifted by (1,1,1). Sublattice A bonds along the four
# directions below, sublattice B along their negatives.
_FCC = ((0, 0, 0), (0, 2, 2), (2, 0, 2), (2, 2, 0))
_BONDS = ((1, 1, 1), (1, -1, -1), (-1, 1, -1), (-1, -1, 1))


def diamond_neighbours(nx: int, ny: int, nz: int) -> torch.Tensor:
    """Nearest-neighbour list of a periodic diamond slab of nx*ny*nz cubic cells.

    8 atoms per cell, so NA = 8*nx*ny*nz; every atom has exactly 4 neighbours,
    slot s = bond direction s (with sign flipped on sublattice B). The list is
    symmetric: b in nbr[a] iff a in nbr[b].
    """
    L = (4 * nx, 4 * ny, 4 * nz)
    pos = []
    for cx in range(nx):
        for cy in range(ny):
            for cz in range(nz):
                for sub in (0, 1):
                    for f in _FCC:
                        pos.append((4 * cx + f[0] + sub, 4 * cy + f[1] + sub, 4 * cz + f[2] + sub, sub))
    index = {(p[0] % L[0], p[1] % L[1], p[2] % L[2]): i for i, p in enumerate(pos)}
    nbr = torch.empty(len(pos), 4, dtype=torch.int32)
    for i, (x, y, z, sub) in enumerate(pos):
        sign = 1 if sub == 0 else -1
        for s, d in enumerate(_BONDS):
            key = ((x + sign * d[0]) % L[0], (y + sign * d[1]) % L[1], (z + sign * d[2]) % L[2])
            nbr[i, s] = index[key]
    return nbr


def default_neighbours(dims: Dims) -> torch.Tensor:
    """Ring list for small NA; a diamond slab when NA = 8*n^2*m fits exactly."""
    if dims.NB == 4:
        for nx, ny, nz in ((4, 4, 8), (8, 8, 8), (2, 2, 8)):
            if 8 * nx * ny * nz == dims.NA:
                return diamond_neighbours(nx, ny, nz)
    return ring_neighbours(dims.NA, dims.NB)


def _cnormal(shape, std: float, gen: torch.Generator, device) -> torch.Tensor:
    re = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    im = torch.randn(shape, generator=gen, dtype=torch.float64, device=device)
    return torch.complex(re * std, im * std)


def _anti_hermitian_gram(shape, sign: float, gen, device) -> torch.Tensor:
    """sign * i * sym(A A^H) with A re/im ~ N(0, 1/Norb)."""
    norb = shape[-1]
    out = torch.empty(shape, dtype=torch.complex128, device=device)
    flat = out.view(-1, norb, norb)
    # Chunked to bound temporary memory at the large workloads.
    chunk = max(1, (1 << 26) // (norb * norb))
    for lo in range(0, flat.shape[0], chunk):
        hi = min(flat.shape[0], lo + chunk)
        a = _cnormal((hi - lo, norb, norb), 1.0 / math.sqrt(norb), gen, device)
        m = a @ a.conj().transpose(-1, -2)
        m = 0.5 * (m + m.conj().transpose(-1, -2))  # exactly Hermitian
        flat[lo:hi] = (1j * sign) * m  # i * Hermitian = exactly anti-Hermitian
    return out


def _anti_hermitian_3x3(shape, std: float, gen, device) -> torch.Tensor:
    x = _cnormal(shape, std, gen, device)
    return 0.5 * (x - x.conj().transpose(-1, -2))


@dataclasses.dataclass
class Inputs:
    dims: Dims
    nbr: torch.Tensor  # int32 [NA, NB]
    dH: torch.Tensor  # complex128 [NA, NB, 3, Norb, Norb]
    D_less: torch.Tensor  # complex128 [Nqz, Nw, NA, NB, 3, 3]
    D_greater: torch.Tensor
    G_less: torch.Tensor  # complex128 [Nkz, NE, NA, Norb, Norb]
    G_greater: torch.Tensor

    def to(self, device) -> "Inputs":
        return Inputs(self.dims, *(t.to(device) for t in (self.nbr, self.dH, self.D_less, self.D_greater,
                                                          self.G_less, self.G_greater)))


def make_inputs(dims: Dims, seed: int = 0, device="cpu", nbr: Optional[torch.Tensor] = None,
                general: bool = False) -> Inputs:
    """Seeded synthetic inputs (draw order G^<, G^>, dH, D^<, D^>).

    general=False: anti-Hermitian G and D blocks (lesser/greater functions);
    general=True: the same draw order with no symmetry in G or D.
    """
    device = torch.device(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    if general:
        g_std = 1.0 / math.sqrt(dims.Norb)
        G_less = _cnormal(dims.g_shape(), g_std, gen, device)
        G_greater = _cnormal(dims.g_shape(), g_std, gen, device)
    else:
        G_less = _anti_hermitian_gram(dims.g_shape(), +1.0, gen, device)
        G_greater = _anti_hermitian_gram(dims.g_shape(), -1.0, gen, device)
    dH = _cnormal(dims.dh_shape(), 0.1, gen, device)
    if general:
        D_less = _cnormal(dims.d_shape(), 0.01, gen, device)
        D_greater = _cnormal(dims.d_shape(), 0.01, gen, device)
    else:
        D_less = _anti_hermitian_3x3(dims.d_shape(), 0.01, gen, device)
        D_greater = _anti_hermitian_3x3(dims.d_shape(), 0.01, gen, device)
    if nbr is None:
        nbr = default_neighbours(dims)
    return Inputs(dims, nbr.to(device=device, dtype=torch.int32).contiguous(), dH, D_less, D_greater,
                  G_less, G_greater)


def make_upstream(dims: Dims, seed: int = 1, device="cpu"):
    """Upstream gradients W, V ~ complex N(0,1) blocks shaped like Sigma."""
    device = torch.device(device)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    return _cnormal(dims.g_shape(), 1.0, gen, device), _cnormal(dims.g_shape(), 1.0, gen, device)
