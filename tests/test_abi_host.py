"""Host-side checks of the C ABI (no GPU needed: nothing here launches work).

The library must load, export every symbol include/sse.h declares, and
reject invalid arguments before touching the device.
"""
import os
import re

import pytest

from paper_1912_10024_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as f:
                names |= set(re.findall(r"SSE_API\s+[\w\s\*]+?\b(sse_\w+)\s*\(", f.read()))
    return names


def test_header_declares_the_entry_points():
    assert {"sse_workspace_bytes", "sse_sigma_fwd", "sse_sigma_bwd", "sse_strerror"} <= declared_symbols()


def test_library_exports_every_declared_symbol():
    lib = B.load()
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(B.EXPORTED) <= declared_symbols()


def good_dims():
    return B.sse_dims(16, 4, 4, 32, 3, 3, 4, 0, 16)


def test_strerror_covers_all_codes():
    for s in range(7):
        assert B.sse_strerror(s) and B.sse_strerror(s) != "unknown status"
    assert B.sse_strerror(99) == "unknown status"


def test_workspace_bytes_validation():
    d = good_dims()
    assert B.sse_workspace_bytes(d, B.SSE_MODE_FP64, 0) >= 256
    for field, value in (("NA", 0), ("Nqz", 4), ("Nw", 32), ("a_end", 17), ("a_begin", 5), ("Norb", 0)):
        bad = good_dims()
        setattr(bad, field, value)
        if field == "a_begin":
            bad.a_end = 4
        assert B.sse_workspace_bytes(bad, B.SSE_MODE_FP64, 0) == 0, field
    assert B.sse_workspace_bytes(d, 7, 0) == 0
    assert B.sse_workspace_bytes(d, 0, 1 << 7) == 0
    big = good_dims()
    big.Norb = 17
    assert B.sse_workspace_bytes(big, 0, 0) == 0


FAKE = 1 << 20  # 16-byte aligned fake device address: never dereferenced on these paths


def call_fwd(d, **over):
    args = dict(nbr=FAKE, dH=FAKE, D_less=FAKE, D_greater=FAKE, G_less=FAKE, G_greater=FAKE, scale=0.1, mode=0,
                flags=0, S_less=FAKE, S_greater=FAKE, workspace=FAKE, ws_bytes=1 << 20)
    args.update(over)
    return B.sse_sigma_fwd(d, stream=0, **args)


@pytest.mark.parametrize("over,status", [
    (dict(G_less=0), 1), (dict(S_greater=0), 1), (dict(dH=FAKE + 8), 1), (dict(nbr=FAKE + 2), 1),
    (dict(scale=float("nan")), 1), (dict(mode=9), 1), (dict(flags=1 << 5), 1),
    (dict(workspace=0), 6), (dict(workspace=FAKE + 16), 6), (dict(ws_bytes=16), 6),
])
def test_fwd_rejects_bad_arguments_on_host(over, status):
    assert call_fwd(good_dims(), **over) == status


@pytest.mark.parametrize("field,value,status", [("Nqz", 4, 1), ("Nw", 32, 1), ("a_end", 17, 1), ("NB", 0, 1),
                                                ("Norb", 17, 2), ("NA", 40000, 1)])
def test_fwd_rejects_bad_dims_on_host(field, value, status):
    d = good_dims()
    setattr(d, field, value)
    if field == "NA":
        d.a_end = 16
        status = 2  # valid but larger than the kernels support
    assert call_fwd(d) == status


def test_empty_atom_range_is_a_noop():
    d = good_dims()
    d.a_begin = d.a_end = 3
    assert call_fwd(d) == 0


def test_bwd_rejects_non_fp64_and_nulls():
    d = good_dims()
    args = [FAKE] * 6
    assert B.sse_sigma_bwd(d, *args, 0.1, 1, 0, FAKE, FAKE, FAKE, FAKE, FAKE, FAKE, 1 << 20, 0) == 2
    assert B.sse_sigma_bwd(d, *args, 0.1, 0, 0, 0, FAKE, FAKE, FAKE, FAKE, FAKE, 1 << 20, 0) == 1


def test_profile_read_without_records():
    assert B.sse_profile_read() == []


def call_pi(d, **over):
    args = dict(nbr=FAKE, dH=FAKE, G_less=FAKE, G_greater=FAKE, scale=0.1, mode=0, flags=0, P_less=FAKE,
                P_greater=FAKE, workspace=FAKE, ws_bytes=1 << 20)
    args.update(over)
    return B.sse_pi_fwd(d, stream=0, **args)


@pytest.mark.parametrize("over,status", [
    (dict(G_less=0), 1), (dict(P_greater=0), 1), (dict(dH=FAKE + 8), 1), (dict(nbr=FAKE + 2), 1),
    (dict(scale=float("inf")), 1), (dict(mode=9), 1), (dict(flags=1 << 5), 1), (dict(mode=1), 2),
    (dict(mode=2), 2), (dict(workspace=0), 6), (dict(workspace=FAKE + 16), 6), (dict(ws_bytes=16), 6),
])
def test_pi_rejects_bad_arguments_on_host(over, status):
    assert call_pi(good_dims(), **over) == status


def test_pi_workspace_bytes():
    d = good_dims()
    assert B.sse_pi_workspace_bytes(d, B.SSE_MODE_FP64, 0) > 256
    bad = good_dims()
    bad.Nw = bad.NE
    assert B.sse_pi_workspace_bytes(bad, B.SSE_MODE_FP64, 0) == 0


def test_bwd_g_rejects_bad_arguments_on_host():
    d = good_dims()
    base = dict(nbr=FAKE, dH=FAKE, D_less=FAKE, D_greater=FAKE, scale=0.1, mode=3, flags=0, gS_less=FAKE,
                gS_greater=FAKE, g_G_less=FAKE, g_G_greater=FAKE, workspace=FAKE, ws_bytes=1 << 20)
    for over, status in ((dict(dH=0), 1), (dict(g_G_less=FAKE + 8), 1), (dict(mode=2), 2), (dict(flags=1 << 5), 1),
                         (dict(workspace=0), 6), (dict(ws_bytes=8), 6)):
        args = dict(base)
        args.update(over)
        assert B.sse_sigma_bwd_g(d, stream=0, **args) == status, over
    assert B.sse_sigma_bwd_g_workspace_bytes(d, 3, 0) > 256


def test_fwd_host_checks_before_any_device_work():
    d = good_dims()
    n = B.sse_sigma_fwd_host_bytes(d, 3, 0)
    assert n > 256
    base = dict(nbr=FAKE, dH=FAKE, D_less=FAKE, D_greater=FAKE, G_less=FAKE, G_greater=FAKE, scale=0.1, mode=3,
                flags=0, S_less=FAKE, S_greater=FAKE, device_buf=FAKE, buf_bytes=n)
    for over, status in ((dict(S_less=0), 1), (dict(G_less=FAKE + 4), 1), (dict(buf_bytes=n - 1), 6),
                         (dict(device_buf=FAKE + 64), 6), (dict(mode=9), 1)):
        args = dict(base)
        args.update(over)
        assert B.sse_sigma_fwd_host(d, stream=0, copy_stream=1, **args) == status, over
    assert B.sse_sigma_fwd_host(d, stream=0, copy_stream=0, **base) == 1  # the overlap needs two streams


def test_fp32_workspaces_are_smaller_and_tensor_modes_unsupported():
    """FP32_FFT keeps its spectra in complex64: every transform workspace is smaller than the FP64 one, about half
    where the spectra are all of it."""
    d = B.sse_dims(256, 4, 10, 256, 5, 5, 16, 0, 256)
    fft64, fft32 = B.SSE_MODE_FP64_FFT, B.SSE_MODE_FP32_FFT
    for fn in (B.sse_workspace_bytes, B.sse_pi_workspace_bytes, B.sse_sigma_bwd_g_workspace_bytes,
               B.sse_sigma_fwd_host_bytes):
        w64, w32 = fn(d, fft64, 0), fn(d, fft32, 0)
        assert 0 < w32 < w64, fn
    # the spectra dominate: FP32 needs a little over half (the FP64 partial sums of the adjoint stay FP64)
    assert B.sse_pi_workspace_bytes(d, fft32, 0) < 0.51 * B.sse_pi_workspace_bytes(d, fft64, 0)
    assert B.sse_sigma_bwd_g_workspace_bytes(d, fft32, 0) < 0.51 * B.sse_sigma_bwd_g_workspace_bytes(d, fft64, 0)


def test_bwd_g_refuses_tensor_modes():
    d = good_dims()
    for mode in (B.SSE_MODE_TF32, B.SSE_MODE_BF16X3):
        rc = B.sse_sigma_bwd_g(d, FAKE, FAKE, FAKE, FAKE, 0.1, mode, 0, FAKE, FAKE, FAKE, FAKE, FAKE, 1 << 30, 0)
        assert rc == 2, mode  # SSE_ERR_UNSUPPORTED, before any device work


# Largest NB the transform kernels take per Norb = 1 .. 16 (their shared-memory configurations): the limits the
# header documents for FP64_FFT and FP32_FFT.
NB_MAX = [16] * 13 + [14, 12, 10]
NB_MAX_PI = [16] * 11 + [15, 12, 10, 9, 7]


def transform_entries():
    """Every entry point that runs transforms, called with a 16-byte workspace: SSE_ERR_WORKSPACE (6) means the sizes
    passed the support checks (which come first), SSE_ERR_UNSUPPORTED (2) that they did not; neither touches the
    device."""
    fwd = lambda d, m: call_fwd(d, mode=m, ws_bytes=16)  # noqa: E731
    host = lambda d, m: B.sse_sigma_fwd_host(  # noqa: E731
        d, nbr=FAKE, dH=FAKE, D_less=FAKE, D_greater=FAKE, G_less=FAKE, G_greater=FAKE, scale=0.1, mode=m, flags=0,
        S_less=FAKE, S_greater=FAKE, device_buf=FAKE, buf_bytes=16, stream=0, copy_stream=1)
    bwd = lambda d, m: B.sse_sigma_bwd(d, *[FAKE] * 6, 0.1, m, 0, *[FAKE] * 6, 16, 0)  # noqa: E731
    pi = lambda d, m: call_pi(d, mode=m, ws_bytes=16)  # noqa: E731
    bwd_g = lambda d, m: B.sse_sigma_bwd_g(  # noqa: E731
        d, nbr=FAKE, dH=FAKE, D_less=FAKE, D_greater=FAKE, scale=0.1, mode=m, flags=0, gS_less=FAKE, gS_greater=FAKE,
        g_G_less=FAKE, g_G_greater=FAKE, workspace=FAKE, ws_bytes=16, stream=0)
    return [("fwd", fwd, NB_MAX), ("fwd_host", host, NB_MAX), ("bwd", bwd, NB_MAX), ("pi", pi, NB_MAX_PI),
            ("bwd_g", bwd_g, NB_MAX)]


@pytest.mark.parametrize("mode", [B.SSE_MODE_FP64_FFT, B.SSE_MODE_FP32_FFT])
def test_transform_size_limits_are_checked_on_host(mode):
    """The transform evaluations' limits (Nkz <= 16 for the kz DFT pass, L = NE + Nw rounded up to 2^a 3^b <= 4608
    for the shared-memory FFT, NB by Norb for the product kernels) are refused with SSE_ERR_UNSUPPORTED before any
    device work, by every entry point, and sizes inside them pass."""
    for name, fn, nb_max in transform_entries():
        for Norb in range(1, 17):
            for NB in (nb_max[Norb - 1], nb_max[Norb - 1] + 1):
                want = 6 if NB == nb_max[Norb - 1] else 2
                assert fn(B.sse_dims(16, NB, Norb, 64, 4, 1, 4, 0, 16), mode) == want, (name, Norb, NB)
        assert fn(B.sse_dims(16, 4, 10, 64, 16, 1, 4, 0, 16), mode) == 6, name
        assert fn(B.sse_dims(16, 4, 10, 64, 17, 1, 4, 0, 16), mode) == 2, name
        assert fn(B.sse_dims(16, 4, 10, 4576, 4, 1, 32, 0, 16), mode) == 6, name  # L = 4608 = 2^9 3^2
        assert fn(B.sse_dims(16, 4, 10, 4577, 4, 1, 32, 0, 16), mode) == 2, name  # L = 5184


def test_tensor_core_transform_mode_limits_are_checked_on_host():
    """Mode F16X3_FFT (FP32 transforms, block products on tcgen05): the forward entries take Norb <= 10 and NB <= 4
    (one TMEM accumulator and one pair of staged dH operands per bond) inside the transform limits; the adjoint, Pi
    and the G-gradient refuse the mode. All of it before any device work."""
    m = B.SSE_MODE_F16X3_FFT
    entries = dict((n, f) for n, f, _ in transform_entries())
    for name in ("fwd", "fwd_host"):
        fn = entries[name]
        for Norb in range(1, 12):
            for NB in range(1, 6):
                want = 6 if Norb <= 10 and NB <= 4 else 2
                assert fn(B.sse_dims(16, NB, Norb, 64, 4, 1, 4, 0, 16), m) == want, (name, Norb, NB)
        assert fn(B.sse_dims(16, 4, 10, 64, 17, 1, 4, 0, 16), m) == 2, name  # the kz DFT pass
        assert fn(B.sse_dims(16, 4, 10, 4577, 4, 1, 32, 0, 16), m) == 2, name  # the FFT length
    for name in ("bwd", "pi", "bwd_g"):
        assert entries[name](B.sse_dims(16, 4, 10, 64, 4, 1, 4, 0, 16), m) == 2, name
    # the FP32_FFT forward's spectra (FP32_FFT's own figure also covers its adjoint, which needs more here)
    d = B.sse_dims(256, 4, 10, 256, 5, 5, 16, 0, 256)
    assert 0 < B.sse_workspace_bytes(d, m, 0) < B.sse_workspace_bytes(d, B.SSE_MODE_FP32_FFT, 0)


def test_direct_fp64_adjoint_has_no_transform_limits():
    """Mode FP64 of sse_sigma_bwd runs the direct kernels: no kz, length or NB limit beyond the common ones."""
    bwd = dict((n, f) for n, f, _ in transform_entries())["bwd"]
    for d in (B.sse_dims(16, 17, 16, 64, 4, 1, 4, 0, 16), B.sse_dims(16, 4, 10, 64, 17, 1, 4, 0, 16),
              B.sse_dims(16, 4, 10, 6000, 4, 1, 32, 0, 16)):
        assert bwd(d, B.SSE_MODE_FP64) == 6


@pytest.mark.parametrize("mode,nw_max", [(B.SSE_MODE_TF32, 286), (B.SSE_MODE_BF16X3, 194)])
def test_tensor_core_mode_limits_are_checked_on_host(mode, nw_max):
    """The tcgen05 forward keeps 6 Norb accumulator columns in epilogue registers (Norb <= 10) and the weight rows of
    2 Nw taps per qz in shared memory: sizes beyond are SSE_ERR_UNSUPPORTED before any device work (a 16-byte
    workspace makes every size inside the limits stop at SSE_ERR_WORKSPACE instead)."""
    def fwd(d):
        return call_fwd(d, mode=mode, ws_bytes=16)
    assert fwd(B.sse_dims(16, 4, 10, 512, 4, 1, 4, 0, 16)) == 6
    assert fwd(B.sse_dims(16, 4, 11, 512, 4, 1, 4, 0, 16)) == 2
    assert fwd(B.sse_dims(16, 4, 10, 4096, 4, 1, nw_max, 0, 16)) == 6
    assert fwd(B.sse_dims(16, 4, 10, 4096, 4, 1, nw_max + 1, 0, 16)) == 2


def test_static_entry_point_status_codes_match_sse_sigma_bwd():
    """sse_sigma_bwd_static returns sse_sigma_bwd's status codes, all decided on the host: unsupported valid modes
    and sizes give SSE_ERR_UNSUPPORTED, invalid arguments SSE_ERR_INVALID_ARG, problems too large for the static
    array SSE_ERR_WORKSPACE. The fake pointers are never dereferenced."""
    fake = 1 << 20
    scale = 0.159

    def call(d, mode, ptr=fake):
        return B.sse_sigma_bwd_static(d, ptr, fake, fake, fake, fake, fake, scale, mode, 0, fake, fake, fake, fake,
                                      fake, 0)

    d = good_dims()
    for mode in (B.SSE_MODE_TF32, B.SSE_MODE_BF16X3, B.SSE_MODE_FP64_FFT, B.SSE_MODE_FP32_FFT):
        assert call(d, mode) == 2, mode
    assert call(d, 7) == 1
    assert call(d, B.SSE_MODE_FP64, ptr=0) == 1
    wide = good_dims()
    wide.Norb = 17
    assert call(wide, B.SSE_MODE_FP64) == 2
    bad = good_dims()
    bad.Nqz = 4
    assert call(bad, B.SSE_MODE_FP64) == 1
    big = B.sse_dims(1024, 4, 10, 512, 7, 7, 32, 0, 1024)
    assert call(big, B.SSE_MODE_FP64) == 6


def test_withhold_window_hook_arguments():
    """The bounded-wait test hook checks its arguments on the host and disarms with item < 0."""
    assert B.sse_test_withhold_window(0, 0) == 1
    assert B.sse_test_withhold_window(-1, 0) == 0
    assert B.sse_test_withhold_window(3, 1 << 16) == 0
    assert B.sse_test_withhold_window(-1, 0) == 0  # leave it disarmed
