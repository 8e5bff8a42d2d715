"""Host-side checks of the Python binding (no GPU): every pointer it hands to libsse must cover the documented
layout, so tensors in the wrong place, of the wrong dtype, shape or rank, or not contiguous are refused before any
CUDA call (none of these calls initialises CUDA)."""
import pytest
import torch

from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, make_inputs


@pytest.fixture(scope="module")
def inp():
    return make_inputs(TINY, seed=5)


def host_args(inp):
    return [inp.G_less, inp.G_greater, inp.dH, inp.D_less, inp.D_greater, inp.nbr]


def test_device_entry_points_refuse_host_tensors(inp):
    G, Gg, dH, Dl, Dg, nbr = host_args(inp)
    with pytest.raises(TypeError, match="CUDA"):
        B.sigma(G, Gg, dH, Dl, Dg, nbr)
    with pytest.raises(TypeError, match="CUDA"):
        B.sigma_grad(G, Gg, dH, Dl, Dg, nbr, G, Gg)
    with pytest.raises(TypeError, match="CUDA"):
        B.pi(G, Gg, dH, nbr, TINY.Nqz, TINY.Nw)
    with pytest.raises(TypeError, match="CUDA"):
        B.sigma_grad_G(dH, Dl, Dg, nbr, G, Gg)


def test_rank_is_checked_before_shapes_are_read(inp):
    G, Gg, dH, Dl, Dg, nbr = host_args(inp)
    with pytest.raises(ValueError, match="rank"):
        B.sigma(G[0], Gg, dH, Dl, Dg, nbr)
    with pytest.raises(ValueError, match="rank"):
        B.pi(G, Gg, dH[0], nbr, TINY.Nqz, TINY.Nw)
    with pytest.raises(ValueError, match="rank"):
        B.sigma_grad_G(dH, Dl[0], Dg, nbr, G, Gg)
    with pytest.raises(ValueError, match="rank"):
        B.sigma_host(G, Gg, dH, Dl[..., 0], Dg, nbr)


@pytest.mark.parametrize("which,bad,err", [
    (5, lambda x: x.to(torch.int64), TypeError),                      # nbr must be int32
    (1, lambda x: x.to(torch.complex64), TypeError),                  # G^> must be complex128
    (2, lambda x: x[:, :-1].contiguous(), ValueError),                # dH with a slot missing
    (4, lambda x: x[:, :-1].contiguous(), ValueError),                # D^> with a frequency missing
    (0, lambda x: x.transpose(3, 4), ValueError),                     # G^< not contiguous
    (3, lambda x: x.to(torch.complex64), TypeError),                  # D^< must be complex128
])
def test_host_entry_checks_every_input(inp, which, bad, err):
    """sse_sigma_fwd_host copies whole host arrays: each must be a contiguous host tensor of its exact layout."""
    args = host_args(inp)
    args[which] = bad(args[which])
    with pytest.raises(err):
        B.sigma_host(*args)


def test_host_entry_checks_the_outputs(inp):
    args = host_args(inp)
    shape = TINY.g_shape()
    for out, err in (((torch.zeros(shape, dtype=torch.complex128),), TypeError),
                     ((torch.zeros(shape, dtype=torch.complex128), torch.zeros(shape, dtype=torch.complex64)),
                      TypeError),
                     ((torch.zeros(shape, dtype=torch.complex128), torch.zeros(shape[:-1] + (1,),
                                                                                dtype=torch.complex128)), ValueError)):
        with pytest.raises(err):
            B.sigma_host(*args, out=out)


def test_dcomb_refuses_host_tensors_and_wrong_ranks():
    nbr = torch.tensor([[1], [0]], dtype=torch.int32)
    raw = torch.zeros((1, 2, 2, 2, 3, 3), dtype=torch.complex128)
    with pytest.raises(TypeError, match="CUDA"):
        B.dcomb(raw, raw, nbr)
    with pytest.raises(TypeError, match="CUDA"):
        B.dcomb_grad(raw[:, :, :, :1], raw[:, :, :, :1], nbr)
    with pytest.raises(ValueError, match="rank"):
        B.dcomb(raw[0], raw[0], nbr)
    with pytest.raises(ValueError, match="rank"):
        B.dcomb_grad(raw, raw, nbr[0])
