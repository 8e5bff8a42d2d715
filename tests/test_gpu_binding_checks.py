"""The binding's checks on the CUDA side: outputs, workspaces and upstream gradients that do not cover the documented
layout are refused on the host, before any launch; workspaces of any dtype count in bytes; the expanded (stride-0)
gradients autograd hands to the backward are accepted."""
import pytest
import torch

from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, make_inputs

pytestmark = pytest.mark.gpu
SCALE = 0.15915494309189535


@pytest.fixture(scope="module")
def g():
    return make_inputs(TINY, seed=71).to("cuda")


def args(g):
    return (g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr)


def test_outputs_of_the_wrong_layout_are_refused(g):
    shape = TINY.g_shape()
    good = torch.empty(shape, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):
        B.sigma(*args(g), out=(good, torch.empty(shape[:-1] + (1,), dtype=torch.complex128, device="cuda")))
    with pytest.raises(TypeError):
        B.sigma(*args(g), out=(good, torch.empty(shape, dtype=torch.complex64, device="cuda")))
    with pytest.raises(ValueError):
        B.sigma(*args(g), out=(good, torch.empty(shape, dtype=torch.complex128, device="cuda").transpose(3, 4)))
    pshape = (TINY.Nqz, TINY.Nw, TINY.NA, TINY.NB, 3, 3)  # one slot short of NB + 1
    with pytest.raises(ValueError):
        B.pi(g.G_less, g.G_greater, g.dH, g.nbr, TINY.Nqz, TINY.Nw,
             out=tuple(torch.empty(pshape, dtype=torch.complex128, device="cuda") for _ in range(2)))


def test_workspace_counts_bytes_and_must_be_contiguous(g):
    d = B.dims_of(g.G_less, g.D_less, g.dH)
    n = B.sse_workspace_bytes(d, B.SSE_MODE_FP64_FFT, 0)
    ref = B.sigma(*args(g), scale=SCALE, mode="fp64_fft")
    ws8 = torch.empty((n + 7) // 8, dtype=torch.float64, device="cuda")  # n bytes as doubles
    got = B.sigma(*args(g), scale=SCALE, mode="fp64_fft", ws=ws8)
    assert torch.equal(got[0], ref[0]) and torch.equal(got[1], ref[1])
    strided = torch.empty(2 * n, dtype=torch.uint8, device="cuda")[::2]
    with pytest.raises(ValueError):
        B.sigma(*args(g), scale=SCALE, mode="fp64_fft", ws=strided)
    with pytest.raises(TypeError):
        B.sigma(*args(g), scale=SCALE, mode="fp64_fft", ws=torch.empty(n, dtype=torch.uint8))  # host memory


def test_upstream_gradients_are_checked(g):
    gl = torch.ones(TINY.g_shape(), dtype=torch.complex128, device="cuda")
    with pytest.raises(TypeError):
        B.sigma_grad(*args(g), gl, gl.to(torch.complex64), scale=SCALE)
    with pytest.raises(ValueError):
        B.sigma_grad(*args(g), gl, gl[:, :-1], scale=SCALE)
    with pytest.raises(TypeError):
        B.sigma_grad_G(g.dH, g.D_less, g.D_greater, g.nbr, gl, gl.cpu(), scale=SCALE)


def test_autograd_expanded_gradients(g):
    """loss = sum Re S^< + 2 sum Re S^>: autograd passes constant (expanded) upstream gradients 1 and 2."""
    dH = g.dH.clone().requires_grad_(True)
    Sl, Sg = B.sigma_autograd(dH, g.D_less, g.D_greater, g.G_less, g.G_greater, g.nbr, SCALE)
    (Sl.real.sum() + 2 * Sg.real.sum()).backward()
    one = torch.ones(TINY.g_shape(), dtype=torch.complex128, device="cuda")
    ref = B.sigma_grad(*args(g), one, 2 * one, scale=SCALE)
    assert torch.equal(dH.grad, ref[0])
