"""FP64 CPU oracle for the electron and phonon scattering self-energies, Eqs. (3) and (4).

TEST INFRASTRUCTURE ONLY: the plain, slow reference that the CUDA path is
checked against. Only the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package. It shares no code with
the CUDA path (``paper_1912_10024_gb300``) and imports nothing from it.

The arithmetic lives in ``sse_oracle.c`` (plain C99 complex loops, pthreads
over output blocks); this module only compiles it with gcc and marshals
numpy / CPU torch arrays through ctypes.
"""
from __future__ import annotations

import contextlib
import ctypes
import hashlib
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sse_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_lock = threading.Lock()
_lib = None


class _Dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in
                ("NA", "NB", "Norb", "NE", "Nkz", "Nqz", "Nw", "a_begin", "a_end", "E_begin", "E_end")]


def compile_source(src: str, so: str) -> str:
    """gcc flags shared by every build of the oracle (IEEE double, no FMA contraction)."""
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-pthread", "-ffp-contract=off",
                           "-fcx-limited-range", "-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def build() -> str:
    """Compile sse_oracle.c into a shared library (cached by source hash)."""
    with open(_SRC, "rb") as f:
        tag = hashlib.sha1(f.read()).hexdigest()[:12]
    so = os.path.join(_BUILD, f"libsse_oracle_{tag}.so")
    if not os.path.exists(so):
        os.makedirs(_BUILD, exist_ok=True)
        compile_source(_SRC, so)
    return so


def _open(path):
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.sse_oracle_fwd.argtypes = [ctypes.POINTER(_Dims), vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_longlong)]
    lib.sse_oracle_fwd.restype = ctypes.c_int
    lib.sse_oracle_bwd.argtypes = [ctypes.POINTER(_Dims), vp, vp, vp, vp, vp, vp, ctypes.c_double, vp, vp,
                                   vp, vp, vp, ctypes.c_int]
    lib.sse_oracle_bwd.restype = ctypes.c_int
    for name in ("sse_oracle_dcomb", "sse_oracle_dcomb_adj"):
        getattr(lib, name).argtypes = [ctypes.POINTER(_Dims), vp, vp, vp, vp, vp]
        getattr(lib, name).restype = ctypes.c_int
    lib.sse_oracle_bwd_g.argtypes = [ctypes.POINTER(_Dims), vp, vp, vp, vp, ctypes.c_double, vp, vp, vp, vp,
                                     ctypes.c_int]
    lib.sse_oracle_bwd_g.restype = ctypes.c_int
    lib.sse_oracle_pi.argtypes = [ctypes.POINTER(_Dims), vp, vp, vp, vp, ctypes.c_double, vp, vp, ctypes.c_int]
    lib.sse_oracle_pi.restype = ctypes.c_int
    return lib


@contextlib.contextmanager
def _library(path):
    """Temporarily route calls to another build of the oracle (used by the
    test that plants mistakes in a copy of sse_oracle.c)."""
    global _lib
    old = _load()
    _lib = _open(path)
    try:
        yield
    finally:
        _lib = old


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(build())
    return _lib


def _np(x, dtype):
    """numpy view of a CPU torch tensor or array, C-contiguous, given dtype."""
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def _dims(G, D, dH, a_range, E_range):
    Nkz, NE, NA, Norb, _ = G.shape
    Nqz, Nw = D.shape[0], D.shape[1]
    NB = dH.shape[1]
    a0, a1 = a_range if a_range is not None else (0, NA)
    e0, e1 = E_range if E_range is not None else (0, NE)
    return _Dims(NA, NB, Norb, NE, Nkz, Nqz, Nw, a0, a1, e0, e1)


def sigma(nbr, dH, D_less, D_greater, G_less, G_greater, scale, a_range=None, E_range=None, nthreads=None,
          out=None, count_terms=False):
    """Sigma^<, Sigma^> of Eq. (3) in FP64 on the host.

    Arrays may be numpy arrays or CPU torch tensors with the layouts of the
    C-ABI (G/Sigma [Nkz,NE,NA,Norb,Norb], dH [NA,NB,3,Norb,Norb],
    D [Nqz,Nw,NA,NB,3,3], nbr [NA,NB] int32). Only blocks of atoms in
    ``a_range`` and energies in ``E_range`` are computed; the rest of the
    outputs stay zero (or keep the contents of ``out``).
    Returns (S_less, S_greater) as complex128 numpy arrays, plus the number of
    in-range terms if ``count_terms``.
    """
    lib = _load()
    G_l, G_g = _np(G_less, np.complex128), _np(G_greater, np.complex128)
    D_l, D_g = _np(D_less, np.complex128), _np(D_greater, np.complex128)
    dH_, nbr_ = _np(dH, np.complex128), _np(nbr, np.int32)
    d = _dims(G_l, D_l, dH_, a_range, E_range)
    if out is None:
        S_l, S_g = np.zeros_like(G_l), np.zeros_like(G_l)
    else:
        S_l, S_g = out
    n = ctypes.c_longlong(0)
    rc = lib.sse_oracle_fwd(ctypes.byref(d), nbr_.ctypes.data, dH_.ctypes.data, D_l.ctypes.data, D_g.ctypes.data,
                            G_l.ctypes.data, G_g.ctypes.data, float(scale), S_l.ctypes.data, S_g.ctypes.data,
                            int(nthreads or default_threads()), ctypes.byref(n))
    if rc != 0:
        raise ValueError(f"sse_oracle_fwd failed with status {rc}")
    if count_terms:
        return S_l, S_g, int(n.value)
    return S_l, S_g


def sigma_grad(nbr, dH, D_less, D_greater, G_less, G_greater, scale, W_less, W_greater, a_range=None,
               nthreads=None):
    """Gradients of L = sum_t Re tr(W^t^H Sigma^t) w.r.t. dH, Dc^<, Dc^>.

    PyTorch convention for complex leaves (grad = dL/dRe + i dL/dIm).
    Returns (g_dH, g_D_less, g_D_greater); blocks of atoms outside
    ``a_range`` are zero.
    """
    lib = _load()
    G_l, G_g = _np(G_less, np.complex128), _np(G_greater, np.complex128)
    D_l, D_g = _np(D_less, np.complex128), _np(D_greater, np.complex128)
    dH_, nbr_ = _np(dH, np.complex128), _np(nbr, np.int32)
    W_l, W_g = _np(W_less, np.complex128), _np(W_greater, np.complex128)
    d = _dims(G_l, D_l, dH_, a_range, None)
    g_dH = np.zeros_like(dH_)
    g_Dl, g_Dg = np.zeros_like(D_l), np.zeros_like(D_g)
    rc = lib.sse_oracle_bwd(ctypes.byref(d), nbr_.ctypes.data, dH_.ctypes.data, D_l.ctypes.data, D_g.ctypes.data,
                            G_l.ctypes.data, G_g.ctypes.data, float(scale), W_l.ctypes.data, W_g.ctypes.data,
                            g_dH.ctypes.data, g_Dl.ctypes.data, g_Dg.ctypes.data, int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError(f"sse_oracle_bwd failed with status {rc}")
    return g_dH, g_Dl, g_Dg


def _raw_dims(raw, nbr, a_range):
    Nqz, Nw, NA = raw.shape[0], raw.shape[1], raw.shape[2]
    NB = nbr.shape[1]
    a0, a1 = a_range if a_range is not None else (0, NA)
    # the energy/kz fields are unused by the combination; any valid values pass the checks
    return _Dims(NA, NB, 1, 1, Nqz, Nqz, Nw, a0, a1, 0, 1)


def dcomb(nbr, raw_less, raw_greater, a_range=None):
    """Bond weights D_ba - D_bb - D_aa + D_ab of Eq. (3) from raw [Nqz,Nw,NA,NB+1,3,3] tensors.

    Returns (Dc_less, Dc_greater) [Nqz,Nw,NA,NB,3,3]; atoms outside ``a_range`` stay zero.
    """
    lib = _load()
    r_l, r_g = _np(raw_less, np.complex128), _np(raw_greater, np.complex128)
    nbr_ = _np(nbr, np.int32)
    d = _raw_dims(r_l, nbr_, a_range)
    shape = r_l.shape[:3] + (nbr_.shape[1], 3, 3)
    D_l, D_g = np.zeros(shape, np.complex128), np.zeros(shape, np.complex128)
    rc = lib.sse_oracle_dcomb(ctypes.byref(d), nbr_.ctypes.data, r_l.ctypes.data, r_g.ctypes.data,
                              D_l.ctypes.data, D_g.ctypes.data)
    if rc != 0:
        raise ValueError(f"sse_oracle_dcomb failed with status {rc}")
    return D_l, D_g


def dcomb_adjoint(nbr, g_less, g_greater):
    """Gradient w.r.t. the raw tensors given the gradient w.r.t. the bond weights (all atoms)."""
    lib = _load()
    g_l, g_g = _np(g_less, np.complex128), _np(g_greater, np.complex128)
    nbr_ = _np(nbr, np.int32)
    d = _raw_dims(g_l, nbr_, None)
    shape = g_l.shape[:3] + (nbr_.shape[1] + 1, 3, 3)
    r_l, r_g = np.zeros(shape, np.complex128), np.zeros(shape, np.complex128)
    rc = lib.sse_oracle_dcomb_adj(ctypes.byref(d), nbr_.ctypes.data, g_l.ctypes.data, g_g.ctypes.data,
                                  r_l.ctypes.data, r_g.ctypes.data)
    if rc != 0:
        raise ValueError(f"sse_oracle_dcomb_adj failed with status {rc}")
    return r_l, r_g


def pi(nbr, dH, G_less, G_greater, scale, Nqz, Nw, a_range=None, nthreads=None):
    """Pi^<, Pi^> of Eq. (4) in FP64 on the host.

    G [Nkz,NE,NA,Norb,Norb], dH [NA,NB,3,Norb,Norb], nbr [NA,NB] int32.
    Returns (P_less, P_greater) [Nqz,Nw,NA,NB+1,3,3] complex128: slot s < NB is
    the block Pi_ab for b = nbr[a][s], slot NB the diagonal block Pi_aa.
    Atoms outside ``a_range`` stay zero.
    """
    lib = _load()
    G_l, G_g = _np(G_less, np.complex128), _np(G_greater, np.complex128)
    dH_, nbr_ = _np(dH, np.complex128), _np(nbr, np.int32)
    Nkz, NE, NA, Norb, _ = G_l.shape
    NB = dH_.shape[1]
    a0, a1 = a_range if a_range is not None else (0, NA)
    d = _Dims(NA, NB, Norb, NE, Nkz, int(Nqz), int(Nw), a0, a1, 0, NE)
    shape = (int(Nqz), int(Nw), NA, NB + 1, 3, 3)
    P_l, P_g = np.zeros(shape, np.complex128), np.zeros(shape, np.complex128)
    rc = lib.sse_oracle_pi(ctypes.byref(d), nbr_.ctypes.data, dH_.ctypes.data, G_l.ctypes.data, G_g.ctypes.data,
                           float(scale), P_l.ctypes.data, P_g.ctypes.data, int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError(f"sse_oracle_pi failed with status {rc}")
    return P_l, P_g


def sigma_grad_G(nbr, dH, D_less, D_greater, scale, W_less, W_greater, a_range=None, nthreads=None):
    """Gradients w.r.t. G^<, G^> of L = sum_t Re tr(W^t^H Sigma^t) over atoms in ``a_range``.

    PyTorch convention for complex tensors. Returns (gG_less, gG_greater) shaped like G (every atom).
    """
    lib = _load()
    D_l, D_g = _np(D_less, np.complex128), _np(D_greater, np.complex128)
    dH_, nbr_ = _np(dH, np.complex128), _np(nbr, np.int32)
    W_l, W_g = _np(W_less, np.complex128), _np(W_greater, np.complex128)
    d = _dims(W_l, D_l, dH_, a_range, None)
    gG_l, gG_g = np.zeros_like(W_l), np.zeros_like(W_g)
    rc = lib.sse_oracle_bwd_g(ctypes.byref(d), nbr_.ctypes.data, dH_.ctypes.data, D_l.ctypes.data, D_g.ctypes.data,
                              float(scale), W_l.ctypes.data, W_g.ctypes.data, gG_l.ctypes.data, gG_g.ctypes.data,
                              int(nthreads or default_threads()))
    if rc != 0:
        raise ValueError(f"sse_oracle_bwd_g failed with status {rc}")
    return gG_l, gG_g
