"""Host-buffer forward (sse_sigma_fwd_host): uploads, compute and downloads on two streams, G and Sigma handed over
one kz slice at a time, give the same bytes as the device-pointer entry point, for every kind of mode and with the
symmetrisation and anti-Hermitian flags, and write only the rows of the atom range."""
import pytest
import torch

from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, Dims, make_inputs, ring_neighbours

pytestmark = pytest.mark.gpu


def host_inputs(inp, pin):
    t = [inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr]
    return [x.contiguous().pin_memory() if pin else x.contiguous() for x in t]


@pytest.mark.parametrize("mode", ["fp64_fft", "fp32_fft", "fp64", "bf16x3"])
@pytest.mark.parametrize("pin", [True, False])
def test_same_bytes_as_device_entry(mode, pin):
    d = Dims(NA=9, NB=3, Norb=5, NE=40, Nkz=3, Nqz=2, Nw=6)
    inp = make_inputs(d, seed=61, nbr=ring_neighbours(9, 3))
    Gl, Gg, dH, Dl, Dg, nbr = host_inputs(inp, pin)
    Hl, Hg = B.sigma_host(Gl, Gg, dH, Dl, Dg, nbr, mode=mode, check=True)
    g = inp.to("cuda")
    Sl, Sg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode)
    assert torch.equal(Hl, Sl.cpu()) and torch.equal(Hg, Sg.cpu())


def test_atom_range_rows_only():
    inp = make_inputs(TINY, seed=62)
    Gl, Gg, dH, Dl, Dg, nbr = host_inputs(inp, True)
    out = (torch.full(TINY.g_shape(), 5 + 5j, dtype=torch.complex128).pin_memory(),
           torch.full(TINY.g_shape(), 5 + 5j, dtype=torch.complex128).pin_memory())
    B.sigma_host(Gl, Gg, dH, Dl, Dg, nbr, atoms=(4, 9), out=out)
    g = inp.to("cuda")
    Sl, _ = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode="fp64_fft", atoms=(4, 9))
    assert torch.equal(out[0][:, :, 4:9], Sl.cpu()[:, :, 4:9])
    assert bool((out[0][:, :, :4] == 5 + 5j).all()) and bool((out[0][:, :, 9:] == 5 + 5j).all())


def test_one_stream_is_refused():
    inp = make_inputs(TINY, seed=63)
    Gl, Gg, dH, Dl, Dg, nbr = host_inputs(inp, True)
    s = torch.cuda.current_stream()
    with pytest.raises(B.SseError) as e:
        B.sigma_host(Gl, Gg, dH, Dl, Dg, nbr, stream=s, copy_stream=s)
    assert e.value.status == 1


@pytest.mark.parametrize("mode", ["fp64_fft", "fp32_fft"])
@pytest.mark.parametrize("flags", [("symmetrize",), ("antihermitian",), ("symmetrize", "antihermitian")])
def test_flags_same_bytes_many_slices(mode, flags):
    """Nkz = 9 kz slices: the per-slice transforms, symmetrisation and downloads match the device call bit for bit."""
    d = Dims(NA=7, NB=2, Norb=3, NE=50, Nkz=9, Nqz=4, Nw=7)
    inp = make_inputs(d, seed=64, nbr=ring_neighbours(7, 2))
    Gl, Gg, dH, Dl, Dg, nbr = host_inputs(inp, True)
    kw = {f: True for f in flags}
    Hl, Hg = B.sigma_host(Gl, Gg, dH, Dl, Dg, nbr, mode=mode, check=True, **kw)
    g = inp.to("cuda")
    Sl, Sg = B.sigma(g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr, mode=mode, check=True, **kw)
    assert torch.equal(Hl, Sl.cpu()) and torch.equal(Hg, Sg.cpu())
