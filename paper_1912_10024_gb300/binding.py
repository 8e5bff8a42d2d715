"""Thin ctypes binding of libsse (include/sse.h).

The functions named like the C entry points only marshal arguments: every
step of the computation runs in the CUDA kernels of libsse. There is no CPU
fallback: if the library cannot be built or loaded, or no CUDA device is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import math
import threading
from typing import Optional, Sequence

import torch

from . import build as _build

SSE_MODE_FP64, SSE_MODE_TF32, SSE_MODE_BF16X3, SSE_MODE_FP64_FFT, SSE_MODE_FP32_FFT, SSE_MODE_F16X3_FFT = 0, 1, 2, 3, 4, 5
SSE_FLAG_SYMMETRIZE, SSE_FLAG_CHECK, SSE_FLAG_PROFILE, SSE_FLAG_ANTIHERMITIAN = 1, 2, 4, 8
MODES = {"fp64": SSE_MODE_FP64, "tf32": SSE_MODE_TF32, "bf16x3": SSE_MODE_BF16X3, "fp64_fft": SSE_MODE_FP64_FFT,
         "fp32_fft": SSE_MODE_FP32_FFT, "f16x3_fft": SSE_MODE_F16X3_FFT}
EXPORTED = ("sse_workspace_bytes", "sse_sigma_fwd", "sse_sigma_bwd", "sse_sigma_bwd_static", "sse_test_withhold_window",
            "sse_dcomb_fwd",
            "sse_dcomb_bwd", "sse_pi_workspace_bytes", "sse_pi_fwd", "sse_sigma_bwd_g_workspace_bytes",
            "sse_sigma_bwd_g",
            "sse_sigma_fwd_host_bytes", "sse_sigma_fwd_host", "sse_profile_read", "sse_strerror")
SSE_STATIC_SCRATCH_BYTES = 64 << 20


class sse_profile_entry(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char_p), ("ms", ctypes.c_double), ("launches", ctypes.c_int32)]


class sse_dims(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int32) for n in ("NA", "NB", "Norb", "NE", "Nkz", "Nqz", "Nw", "a_begin", "a_end")]


class SseError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {sse_strerror(status)} (status {status})")
        self.status = status


_lock = threading.Lock()
_lib: Optional[ctypes.CDLL] = None


def library_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Build (if the sources changed) and load libsse.so from the package tree."""
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(_build.build())
            vp, i32, u32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_double
            pd = ctypes.POINTER(sse_dims)
            lib.sse_workspace_bytes.argtypes = [pd, i32, u32]
            lib.sse_workspace_bytes.restype = ctypes.c_size_t
            lib.sse_sigma_fwd.argtypes = [pd, vp, vp, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, ctypes.c_size_t, vp]
            lib.sse_sigma_fwd.restype = i32
            lib.sse_sigma_bwd.argtypes = [pd, vp, vp, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, vp, vp, vp,
                                          ctypes.c_size_t, vp]
            lib.sse_sigma_bwd.restype = i32
            lib.sse_sigma_bwd_static.argtypes = [pd, vp, vp, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, vp, vp, vp]
            lib.sse_sigma_bwd_static.restype = i32
            for name in ("sse_dcomb_fwd", "sse_dcomb_bwd"):
                getattr(lib, name).argtypes = [pd, vp, vp, vp, vp, vp, u32, vp, ctypes.c_size_t, vp]
                getattr(lib, name).restype = i32
            lib.sse_strerror.argtypes = [i32]
            lib.sse_strerror.restype = ctypes.c_char_p
            lib.sse_pi_workspace_bytes.argtypes = [pd, i32, u32]
            lib.sse_pi_workspace_bytes.restype = ctypes.c_size_t
            lib.sse_pi_fwd.argtypes = [pd, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, ctypes.c_size_t, vp]
            lib.sse_pi_fwd.restype = i32
            lib.sse_sigma_bwd_g_workspace_bytes.argtypes = [pd, i32, u32]
            lib.sse_sigma_bwd_g_workspace_bytes.restype = ctypes.c_size_t
            lib.sse_sigma_bwd_g.argtypes = [pd, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
            lib.sse_sigma_bwd_g.restype = i32
            lib.sse_sigma_fwd_host_bytes.argtypes = [pd, i32, u32]
            lib.sse_sigma_fwd_host_bytes.restype = ctypes.c_size_t
            lib.sse_sigma_fwd_host.argtypes = [pd, vp, vp, vp, vp, vp, vp, f64, i32, u32, vp, vp, vp, ctypes.c_size_t,
                                               vp, vp]
            lib.sse_sigma_fwd_host.restype = i32
            lib.sse_test_withhold_window.argtypes = [i32, u32]
            lib.sse_test_withhold_window.restype = i32
            lib.sse_profile_read.argtypes = [ctypes.POINTER(sse_profile_entry), i32]
            lib.sse_profile_read.restype = i32
            _lib = lib
    return _lib


def _p(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, torch.Tensor):
        return x.data_ptr()
    return int(x)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


# ---- the C entry points, one to one -------------------------------------

def sse_workspace_bytes(d: sse_dims, mode: int, flags: int) -> int:
    return int(load().sse_workspace_bytes(ctypes.byref(d), int(mode), int(flags)))


def sse_sigma_fwd(d: sse_dims, nbr, dH, D_less, D_greater, G_less, G_greater, scale: float, mode: int, flags: int,
                  S_less, S_greater, workspace, ws_bytes: int, stream=None) -> int:
    return int(load().sse_sigma_fwd(ctypes.byref(d), _p(nbr), _p(dH), _p(D_less), _p(D_greater), _p(G_less),
                                    _p(G_greater), float(scale), int(mode), int(flags), _p(S_less), _p(S_greater),
                                    _p(workspace), int(ws_bytes), _stream(stream)))


def sse_pi_workspace_bytes(d: sse_dims, mode: int, flags: int) -> int:
    return int(load().sse_pi_workspace_bytes(ctypes.byref(d), int(mode), int(flags)))


def sse_pi_fwd(d: sse_dims, nbr, dH, G_less, G_greater, scale: float, mode: int, flags: int, P_less, P_greater,
               workspace, ws_bytes: int, stream=None) -> int:
    return int(load().sse_pi_fwd(ctypes.byref(d), _p(nbr), _p(dH), _p(G_less), _p(G_greater), float(scale),
                                 int(mode), int(flags), _p(P_less), _p(P_greater), _p(workspace), int(ws_bytes),
                                 _stream(stream)))


def sse_sigma_bwd_g_workspace_bytes(d: sse_dims, mode: int, flags: int) -> int:
    return int(load().sse_sigma_bwd_g_workspace_bytes(ctypes.byref(d), int(mode), int(flags)))


def sse_sigma_bwd_g(d: sse_dims, nbr, dH, D_less, D_greater, scale: float, mode: int, flags: int, gS_less,
                    gS_greater, g_G_less, g_G_greater, workspace, ws_bytes: int, stream=None) -> int:
    return int(load().sse_sigma_bwd_g(ctypes.byref(d), _p(nbr), _p(dH), _p(D_less), _p(D_greater), float(scale),
                                      int(mode), int(flags), _p(gS_less), _p(gS_greater), _p(g_G_less),
                                      _p(g_G_greater), _p(workspace), int(ws_bytes), _stream(stream)))


def sse_sigma_fwd_host_bytes(d: sse_dims, mode: int, flags: int) -> int:
    return int(load().sse_sigma_fwd_host_bytes(ctypes.byref(d), int(mode), int(flags)))


def sse_sigma_fwd_host(d: sse_dims, nbr, dH, D_less, D_greater, G_less, G_greater, scale: float, mode: int,
                       flags: int, S_less, S_greater, device_buf, buf_bytes: int, stream=None, copy_stream=None) -> int:
    return int(load().sse_sigma_fwd_host(ctypes.byref(d), _p(nbr), _p(dH), _p(D_less), _p(D_greater), _p(G_less),
                                         _p(G_greater), float(scale), int(mode), int(flags), _p(S_less), _p(S_greater),
                                         _p(device_buf), int(buf_bytes), _stream(stream), _stream(copy_stream)))


def sse_sigma_bwd(d: sse_dims, nbr, dH, D_less, D_greater, G_less, G_greater, scale: float, mode: int, flags: int,
                  gS_less, gS_greater, g_dH, g_D_less, g_D_greater, workspace, ws_bytes: int, stream=None) -> int:
    return int(load().sse_sigma_bwd(ctypes.byref(d), _p(nbr), _p(dH), _p(D_less), _p(D_greater), _p(G_less),
                                    _p(G_greater), float(scale), int(mode), int(flags), _p(gS_less), _p(gS_greater),
                                    _p(g_dH), _p(g_D_less), _p(g_D_greater), _p(workspace), int(ws_bytes),
                                    _stream(stream)))


def sse_sigma_bwd_static(d: sse_dims, nbr, dH, D_less, D_greater, G_less, G_greater, scale: float, mode: int,
                         flags: int, gS_less, gS_greater, g_dH, g_D_less, g_D_greater, stream=None) -> int:
    """sse_sigma_bwd without a workspace, for callers that cannot allocate device memory
    (scratch in the library's static device array; see include/sse.h)."""
    return int(load().sse_sigma_bwd_static(ctypes.byref(d), _p(nbr), _p(dH), _p(D_less), _p(D_greater),
                                           _p(G_less), _p(G_greater), float(scale), int(mode), int(flags),
                                           _p(gS_less), _p(gS_greater), _p(g_dH), _p(g_D_less), _p(g_D_greater),
                                           _stream(stream)))


def sse_dcomb_fwd(d: sse_dims, nbr, Draw_less, Draw_greater, D_less, D_greater, flags: int, workspace,
                  ws_bytes: int, stream=None) -> int:
    return int(load().sse_dcomb_fwd(ctypes.byref(d), _p(nbr), _p(Draw_less), _p(Draw_greater), _p(D_less),
                                    _p(D_greater), int(flags), _p(workspace), int(ws_bytes), _stream(stream)))


def sse_dcomb_bwd(d: sse_dims, nbr, gD_less, gD_greater, gDraw_less, gDraw_greater, flags: int, workspace,
                  ws_bytes: int, stream=None) -> int:
    return int(load().sse_dcomb_bwd(ctypes.byref(d), _p(nbr), _p(gD_less), _p(gD_greater), _p(gDraw_less),
                                    _p(gDraw_greater), int(flags), _p(workspace), int(ws_bytes), _stream(stream)))


def sse_test_withhold_window(item: int, wait_polls: int) -> int:
    """Arm the test hook of the bounded device waits for the next TF32 / BF16X3 forward (see include/sse.h)."""
    return load().sse_test_withhold_window(int(item), int(wait_polls))


def sse_profile_read(max_entries: int = 64):
    """Kernel device times recorded by calls made with SSE_FLAG_PROFILE since the last read:
    a list of (name, total ms, launches); clears the records."""
    buf = (sse_profile_entry * max_entries)()
    n = int(load().sse_profile_read(buf, max_entries))
    if n < 0:
        raise RuntimeError("sse_profile_read: a CUDA event query failed")
    return [(buf[i].name.decode(), float(buf[i].ms), int(buf[i].launches)) for i in range(min(n, max_entries))]


def sse_strerror(status: int) -> str:
    return load().sse_strerror(int(status)).decode()


# ---- tensor-level helpers ------------------------------------------------

def dims_of(G: torch.Tensor, D: torch.Tensor, dH: torch.Tensor, atoms: Optional[Sequence[int]] = None) -> sse_dims:
    Nkz, NE, NA, Norb, _ = G.shape
    a0, a1 = (0, NA) if atoms is None else atoms
    return sse_dims(NA, dH.shape[1], Norb, NE, Nkz, D.shape[0], D.shape[1], a0, a1)


def _check_tensor(name, x, dtype, shape, cuda: bool = True, contiguous: bool = True, device=None):
    """Every pointer the library receives covers exactly the bytes of its documented layout: right place (a CUDA
    tensor on the inputs' device, or a host tensor for the host-buffer entry point), dtype, shape and contiguity."""
    if not isinstance(x, torch.Tensor) or x.is_cuda != cuda:
        raise TypeError(f"{name} must be a {'CUDA' if cuda else 'host'} tensor")
    if device is not None and x.device != device:
        raise ValueError(f"{name} is on {x.device}, the inputs on {device}")
    if x.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {x.dtype}")
    if tuple(x.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")
    if contiguous and not x.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def check_inputs(G_less, G_greater, dH, D_less, D_greater, nbr, cuda: bool = True):
    for name, x, rank in (("G_less", G_less, 5), ("dH", dH, 5), ("D_less", D_less, 6)):
        if not isinstance(x, torch.Tensor) or x.dim() != rank:
            raise ValueError(f"{name} must be a tensor of rank {rank}")
    Nkz, NE, NA, Norb, _ = G_less.shape
    NB = dH.shape[1]
    Nqz, Nw = D_less.shape[0], D_less.shape[1]
    c128 = torch.complex128
    dev = G_less.device if cuda else None
    _check_tensor("G_less", G_less, c128, (Nkz, NE, NA, Norb, Norb), cuda)
    _check_tensor("G_greater", G_greater, c128, (Nkz, NE, NA, Norb, Norb), cuda, device=dev)
    _check_tensor("dH", dH, c128, (NA, NB, 3, Norb, Norb), cuda, device=dev)
    _check_tensor("D_less", D_less, c128, (Nqz, Nw, NA, NB, 3, 3), cuda, device=dev)
    _check_tensor("D_greater", D_greater, c128, (Nqz, Nw, NA, NB, 3, 3), cuda, device=dev)
    _check_tensor("nbr", nbr, torch.int32, (NA, NB), cuda, device=dev)


def _check_grads(gS_less, gS_greater, G_shape, device):
    """Upstream gradients shaped like G (any strides: autograd may hand over expanded views); returns contiguous
    copies where needed."""
    out = []
    for name, g in (("gS_less", gS_less), ("gS_greater", gS_greater)):
        _check_tensor(name, g, torch.complex128, G_shape, contiguous=False, device=device)
        out.append(g.contiguous())
    return out


def _check_outputs(out, shape, device=None, cuda: bool = True):
    if not isinstance(out, (tuple, list)) or len(out) != 2:
        raise TypeError("out must be a pair of tensors")
    for name, x in zip(("out[0]", "out[1]"), out):
        _check_tensor(name, x, torch.complex128, shape, cuda, device=device)


def _buffer_bytes(name, buf, device) -> int:
    """Size in bytes of a caller-provided workspace: a contiguous CUDA tensor on the inputs' device."""
    if not isinstance(buf, torch.Tensor) or not buf.is_cuda or buf.device != device:
        raise TypeError(f"{name} must be a CUDA tensor on {device}")
    if not buf.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return buf.numel() * buf.element_size()


def workspace(d: sse_dims, mode: int, flags: int, device) -> torch.Tensor:
    n = sse_workspace_bytes(d, mode, flags)
    if n == 0:
        raise ValueError("invalid or unsupported problem sizes for libsse")
    # torch's caching allocator returns >= 512-byte aligned blocks
    return torch.empty(n, dtype=torch.uint8, device=device)


def sigma(G_less, G_greater, dH, D_less, D_greater, nbr, scale: float = 1.0 / (2.0 * math.pi), mode: str = "fp64",
          symmetrize: bool = False, check: bool = False, atoms=None, out=None, ws: Optional[torch.Tensor] = None,
          stream=None, profile: bool = False, antihermitian: bool = False):
    """Sigma^<, Sigma^> of Eq. (3) on the current CUDA device via sse_sigma_fwd.

    Returns (S_less, S_greater), complex128 tensors shaped like G. With
    ``atoms=(a0, a1)`` only those atoms are written (the rest of ``out``, or
    of the freshly allocated zero outputs, is left as is).
    """
    check_inputs(G_less, G_greater, dH, D_less, D_greater, nbr)
    d = dims_of(G_less, D_less, dH, atoms)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    flags = (SSE_FLAG_SYMMETRIZE if symmetrize else 0) | (SSE_FLAG_CHECK if check else 0)
    flags |= (SSE_FLAG_PROFILE if profile else 0) | (SSE_FLAG_ANTIHERMITIAN if antihermitian else 0)
    dev = G_less.device
    if out is None:
        alloc = torch.empty if atoms is None else torch.zeros
        out = (alloc(G_less.shape, dtype=torch.complex128, device=dev),
               alloc(G_less.shape, dtype=torch.complex128, device=dev))
    _check_outputs(out, G_less.shape, dev)
    if ws is None:
        ws = workspace(d, m, flags, dev)
    with torch.cuda.device(dev):  # the library works on the current device
        rc = sse_sigma_fwd(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, m, flags, out[0], out[1], ws,
                           _buffer_bytes("ws", ws, dev), stream)
    if rc != 0:
        raise SseError(rc, "sse_sigma_fwd")
    return out


def sigma_grad(G_less, G_greater, dH, D_less, D_greater, nbr, gS_less, gS_greater,
               scale: float = 1.0 / (2.0 * math.pi), mode: str = "fp64", symmetrize: bool = False,
               check: bool = False, atoms=None, ws: Optional[torch.Tensor] = None, stream=None):
    """Gradients (g_dH, g_D_less, g_D_greater) of sum_t Re tr(gS^t^H Sigma^t) via sse_sigma_bwd."""
    check_inputs(G_less, G_greater, dH, D_less, D_greater, nbr)
    d = dims_of(G_less, D_less, dH, atoms)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    flags = (SSE_FLAG_SYMMETRIZE if symmetrize else 0) | (SSE_FLAG_CHECK if check else 0)
    dev = G_less.device
    gSl, gSg = _check_grads(gS_less, gS_greater, G_less.shape, dev)
    alloc = torch.empty if atoms is None else torch.zeros
    g_dH = alloc(dH.shape, dtype=torch.complex128, device=dev)
    g_Dl = alloc(D_less.shape, dtype=torch.complex128, device=dev)
    g_Dg = alloc(D_greater.shape, dtype=torch.complex128, device=dev)
    if ws is None:
        ws = workspace(d, m, flags, dev)
    with torch.cuda.device(dev):
        rc = sse_sigma_bwd(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, m, flags, gSl, gSg, g_dH, g_Dl,
                           g_Dg, ws, _buffer_bytes("ws", ws, dev), stream)
    if rc != 0:
        raise SseError(rc, "sse_sigma_bwd")
    return g_dH, g_Dl, g_Dg


def sigma_host(G_less, G_greater, dH, D_less, D_greater, nbr, scale: float = 1.0 / (2.0 * math.pi),
               mode: str = "fp64_fft", symmetrize: bool = False, check: bool = False, atoms=None, out=None,
               device_buf: Optional[torch.Tensor] = None, stream=None, copy_stream=None, device=None,
               antihermitian: bool = False):
    """Sigma^<, Sigma^> from HOST (CPU, ideally pinned) tensors via sse_sigma_fwd_host: uploads, compute and
    downloads overlap on two streams. Returns host tensors (S_less, S_greater); synchronises the stream."""
    c128 = torch.complex128
    check_inputs(G_less, G_greater, dH, D_less, D_greater, nbr, cuda=False)
    if out is not None:
        _check_outputs(out, G_less.shape, cuda=False)
    d = dims_of(G_less, D_less, dH, atoms)
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    flags = (SSE_FLAG_SYMMETRIZE if symmetrize else 0) | (SSE_FLAG_CHECK if check else 0)
    flags |= SSE_FLAG_ANTIHERMITIAN if antihermitian else 0
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out is None:
        out = (torch.zeros(G_less.shape, dtype=c128).pin_memory(), torch.zeros(G_less.shape, dtype=c128).pin_memory())
    if device_buf is None:
        n = sse_sigma_fwd_host_bytes(d, m, flags)
        if n == 0:
            raise ValueError("invalid or unsupported problem sizes for libsse")
        device_buf = torch.empty(n, dtype=torch.uint8, device=dev)
    nbuf = _buffer_bytes("device_buf", device_buf, dev)
    st = torch.cuda.current_stream(dev) if stream is None else stream
    cp = torch.cuda.Stream(device=dev) if copy_stream is None else copy_stream
    with torch.cuda.device(dev):
        rc = sse_sigma_fwd_host(d, nbr, dH, D_less, D_greater, G_less, G_greater, scale, m, flags, out[0], out[1],
                                device_buf, nbuf, st, cp)
    if rc != 0:
        raise SseError(rc, "sse_sigma_fwd_host")
    st.synchronize()
    return out


def pi(G_less, G_greater, dH, nbr, Nqz: int, Nw: int, scale: float = 1.0 / (2.0 * math.pi),
       symmetrize: bool = False, check: bool = False, atoms=None, out=None, ws: Optional[torch.Tensor] = None,
       stream=None, profile: bool = False, antihermitian: bool = False, mode="fp64"):
    """Pi^<, Pi^> of Eq. (4) on the current CUDA device via sse_pi_fwd (modes fp64 / fp64_fft: FP64 transforms;
    fp32_fft: FP32 transforms and products, FP64 inputs and outputs).

    Returns (P_less, P_greater), complex128 [Nqz, Nw, NA, NB+1, 3, 3]: slot s < NB is the block for
    b = nbr[a][s], slot NB the diagonal block.
    """
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    c128 = torch.complex128
    for name, x, rank in (("G_less", G_less, 5), ("dH", dH, 5)):
        if not isinstance(x, torch.Tensor) or x.dim() != rank:
            raise ValueError(f"{name} must be a tensor of rank {rank}")
    Nkz, NE, NA, Norb, _ = G_less.shape
    NB = dH.shape[1]
    _check_tensor("G_less", G_less, c128, (Nkz, NE, NA, Norb, Norb))
    dev = G_less.device
    _check_tensor("G_greater", G_greater, c128, (Nkz, NE, NA, Norb, Norb), device=dev)
    _check_tensor("dH", dH, c128, (NA, NB, 3, Norb, Norb), device=dev)
    _check_tensor("nbr", nbr, torch.int32, (NA, NB), device=dev)
    a0, a1 = (0, NA) if atoms is None else atoms
    d = sse_dims(NA, NB, Norb, NE, Nkz, int(Nqz), int(Nw), a0, a1)
    flags = (SSE_FLAG_SYMMETRIZE if symmetrize else 0) | (SSE_FLAG_CHECK if check else 0)
    flags |= (SSE_FLAG_PROFILE if profile else 0) | (SSE_FLAG_ANTIHERMITIAN if antihermitian else 0)
    shape = (int(Nqz), int(Nw), NA, NB + 1, 3, 3)
    if out is None:
        alloc = torch.empty if atoms is None else torch.zeros
        out = (alloc(shape, dtype=c128, device=dev), alloc(shape, dtype=c128, device=dev))
    _check_outputs(out, shape, dev)
    if ws is None:
        n = sse_pi_workspace_bytes(d, m, flags)
        if n == 0:
            raise ValueError("invalid or unsupported problem sizes for libsse")
        ws = torch.empty(n, dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        rc = sse_pi_fwd(d, nbr, dH, G_less, G_greater, scale, m, flags, out[0], out[1], ws,
                        _buffer_bytes("ws", ws, dev), stream)
    if rc != 0:
        raise SseError(rc, "sse_pi_fwd")
    return out


def sigma_grad_G(dH, D_less, D_greater, nbr, gS_less, gS_greater, scale: float = 1.0 / (2.0 * math.pi),
                 symmetrize: bool = False, check: bool = False, atoms=None, ws: Optional[torch.Tensor] = None,
                 stream=None, profile: bool = False, mode="fp64_fft"):
    """Gradients (g_G_less, g_G_greater) of sum_t Re tr(gS^t^H Sigma^t) with respect to G via sse_sigma_bwd_g
    (mode fp64_fft: FP64 transforms; fp32_fft: FP32 transforms and products)."""
    m = MODES[mode] if isinstance(mode, str) else int(mode)
    c128 = torch.complex128
    for name, x, rank in (("gS_less", gS_less, 5), ("dH", dH, 5), ("D_less", D_less, 6)):
        if not isinstance(x, torch.Tensor) or x.dim() != rank:
            raise ValueError(f"{name} must be a tensor of rank {rank}")
    NA, NB, _, Norb, _ = dH.shape
    Nqz, Nw = D_less.shape[0], D_less.shape[1]
    _check_tensor("dH", dH, c128, (NA, NB, 3, Norb, Norb))
    dev = dH.device
    _check_tensor("D_less", D_less, c128, (Nqz, Nw, NA, NB, 3, 3), device=dev)
    _check_tensor("D_greater", D_greater, c128, (Nqz, Nw, NA, NB, 3, 3), device=dev)
    _check_tensor("nbr", nbr, torch.int32, (NA, NB), device=dev)
    G_shape = (gS_less.shape[0], gS_less.shape[1], NA, Norb, Norb)
    gSl, gSg = _check_grads(gS_less, gS_greater, G_shape, dev)
    d = dims_of(gSl, D_less, dH, atoms)
    flags = (SSE_FLAG_SYMMETRIZE if symmetrize else 0) | (SSE_FLAG_CHECK if check else 0)
    flags |= SSE_FLAG_PROFILE if profile else 0
    g_Gl, g_Gg = torch.empty_like(gSl), torch.empty_like(gSg)
    if ws is None:
        n = sse_sigma_bwd_g_workspace_bytes(d, m, flags)
        if n == 0:
            raise ValueError("invalid or unsupported problem sizes for libsse")
        ws = torch.empty(n, dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        rc = sse_sigma_bwd_g(d, nbr, dH, D_less, D_greater, scale, m, flags, gSl, gSg, g_Gl, g_Gg, ws,
                             _buffer_bytes("ws", ws, dev), stream)
    if rc != 0:
        raise SseError(rc, "sse_sigma_bwd_g")
    return g_Gl, g_Gg


class SigmaFunction(torch.autograd.Function):
    """(dH, D^<, D^>, G^<, G^>) -> (Sigma^<, Sigma^>) with the hand-written adjoints.

    Gradients for G^<, G^> are computed only when requested (sse_sigma_bwd_g); nbr and the
    scalar options are not differentiated.
    """

    @staticmethod
    def forward(ctx, dH, D_less, D_greater, G_less, G_greater, nbr, scale, mode, symmetrize):
        S = sigma(G_less, G_greater, dH, D_less, D_greater, nbr, scale=scale, mode=mode, symmetrize=symmetrize)
        ctx.save_for_backward(dH, D_less, D_greater, G_less, G_greater, nbr)
        ctx.scale, ctx.symmetrize = scale, symmetrize
        # transform-based adjoint after a transform-based forward (FP32 products after an FP32_FFT
        # forward), the direct FP64 adjoint otherwise
        if mode in ("fp32_fft", SSE_MODE_FP32_FFT, "f16x3_fft", SSE_MODE_F16X3_FFT):
            ctx.bwd_mode = "fp32_fft"  # the tensor-core forward's adjoint: FP32 transforms and products
        elif mode in ("fp64_fft", SSE_MODE_FP64_FFT):
            ctx.bwd_mode = "fp64_fft"
        else:
            ctx.bwd_mode = "fp64"
        return S

    @staticmethod
    def backward(ctx, gSl, gSg):
        dH, D_less, D_greater, G_less, G_greater, nbr = ctx.saved_tensors
        if gSl is None:
            gSl = torch.zeros_like(G_less)
        if gSg is None:
            gSg = torch.zeros_like(G_greater)
        g = sigma_grad(G_less, G_greater, dH, D_less, D_greater, nbr, gSl, gSg, scale=ctx.scale,
                       symmetrize=ctx.symmetrize, mode=ctx.bwd_mode)
        gG = (None, None)
        if ctx.needs_input_grad[3] or ctx.needs_input_grad[4]:
            gG = sigma_grad_G(dH, D_less, D_greater, nbr, gSl, gSg, scale=ctx.scale, symmetrize=ctx.symmetrize,
                              mode="fp32_fft" if ctx.bwd_mode == "fp32_fft" else "fp64_fft")
        return g[0], g[1], g[2], gG[0], gG[1], None, None, None, None


def sigma_autograd(dH, D_less, D_greater, G_less, G_greater, nbr, scale=1.0 / (2.0 * math.pi), mode="fp64",
                   symmetrize=False):
    return SigmaFunction.apply(dH, D_less, D_greater, G_less, G_greater, nbr, scale, mode, symmetrize)


# ---- bond weights from raw phonon Green's functions ---------------------

def _dcomb_dims(raw_or_bond: torch.Tensor, nbr: torch.Tensor, atoms=None) -> sse_dims:
    Nqz, Nw, NA = raw_or_bond.shape[:3]
    a0, a1 = (0, NA) if atoms is None else atoms
    # NE, Nkz, Norb are unused by the combination; values that pass the checks
    return sse_dims(NA, nbr.shape[1], 1, Nw + 1, Nqz, Nqz, Nw, a0, a1)


def dcomb(Draw_less, Draw_greater, nbr, check: bool = False, atoms=None, stream=None):
    """D^t(a,s) = D_ba - D_bb - D_aa + D_ab of Eq. (3) from raw [Nqz,Nw,NA,NB+1,3,3] tensors."""
    if not isinstance(nbr, torch.Tensor) or nbr.dim() != 2 or not isinstance(Draw_less, torch.Tensor) or \
            Draw_less.dim() != 6:
        raise ValueError("nbr must be a tensor of rank 2 and Draw_less of rank 6")
    NB = nbr.shape[1]
    _check_tensor("nbr", nbr, torch.int32, (Draw_less.shape[2], NB))
    dev = nbr.device
    _check_tensor("Draw_less", Draw_less, torch.complex128, Draw_less.shape[:3] + (NB + 1, 3, 3), device=dev)
    _check_tensor("Draw_greater", Draw_greater, torch.complex128, Draw_less.shape[:3] + (NB + 1, 3, 3), device=dev)
    d = _dcomb_dims(Draw_less, nbr, atoms)
    shape = tuple(Draw_less.shape[:3]) + (NB, 3, 3)
    alloc = torch.empty if atoms is None else torch.zeros
    out = (alloc(shape, dtype=torch.complex128, device=dev), alloc(shape, dtype=torch.complex128, device=dev))
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        rc = sse_dcomb_fwd(d, nbr, Draw_less, Draw_greater, out[0], out[1], SSE_FLAG_CHECK if check else 0, ws, 256,
                           stream)
    if rc != 0:
        raise SseError(rc, "sse_dcomb_fwd")
    return out


def dcomb_grad(gD_less, gD_greater, nbr, check: bool = False, stream=None):
    """Gradients w.r.t. the raw tensors from the gradients w.r.t. the bond weights."""
    if not isinstance(nbr, torch.Tensor) or nbr.dim() != 2 or not isinstance(gD_less, torch.Tensor) or \
            gD_less.dim() != 6:
        raise ValueError("nbr must be a tensor of rank 2 and gD_less of rank 6")
    NB = nbr.shape[1]
    _check_tensor("nbr", nbr, torch.int32, (gD_less.shape[2], NB))
    dev = nbr.device
    # autograd may hand over expanded gradients: any strides, copied contiguous below
    _check_tensor("gD_less", gD_less, torch.complex128, gD_less.shape[:3] + (NB, 3, 3), contiguous=False, device=dev)
    _check_tensor("gD_greater", gD_greater, torch.complex128, gD_less.shape[:3] + (NB, 3, 3), contiguous=False,
                  device=dev)
    d = _dcomb_dims(gD_less, nbr)
    shape = tuple(gD_less.shape[:3]) + (NB + 1, 3, 3)
    out = (torch.empty(shape, dtype=torch.complex128, device=dev), torch.empty(shape, dtype=torch.complex128, device=dev))
    ws = torch.empty(256, dtype=torch.uint8, device=dev)
    with torch.cuda.device(dev):
        rc = sse_dcomb_bwd(d, nbr, gD_less.contiguous(), gD_greater.contiguous(), out[0], out[1],
                           SSE_FLAG_CHECK if check else 0, ws, 256, stream)
    if rc != 0:
        raise SseError(rc, "sse_dcomb_bwd")
    return out


class DcombFunction(torch.autograd.Function):
    """(Draw^<, Draw^>) -> (D^<, D^>) bond weights, with the gather adjoint."""

    @staticmethod
    def forward(ctx, Draw_less, Draw_greater, nbr):
        ctx.save_for_backward(nbr)
        return dcomb(Draw_less, Draw_greater, nbr)

    @staticmethod
    def backward(ctx, gl, gg):
        (nbr,) = ctx.saved_tensors
        if gl is None:
            gl = torch.zeros_like(gg)
        if gg is None:
            gg = torch.zeros_like(gl)
        r = dcomb_grad(gl, gg, nbr)
        return r[0], r[1], None
