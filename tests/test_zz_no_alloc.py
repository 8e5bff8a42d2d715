"""sse_sigma_bwd_static: the adjoint for callers that cannot allocate device memory.

Callers whose device memory is owned by another allocator, or that must not
allocate on their hot path, call this entry point instead of sse_sigma_bwd:
it takes no workspace and keeps its scratch in the library's static device
array. Its gradients must equal sse_sigma_bwd's (same kernels, FP64, normwise
1e-12 -- the tolerance of the other FP64 tests) on two calls in a row, and
problems too large for the array must be refused before any device work.

This file is collected last so that a failure here cannot hide other tests.
"""
import math

import pytest
import torch

from conftest import normwise
from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, Dims, make_inputs, make_upstream, ring_neighbours

pytestmark = pytest.mark.gpu
SCALE = 1.0 / (2.0 * math.pi)
TOL = 1e-12


def _outputs(inp):
    return (torch.empty_like(inp.dH), torch.empty_like(inp.D_less), torch.empty_like(inp.D_greater))


def _with_workspace(inp, d, W, V):
    ws = B.workspace(d, B.SSE_MODE_FP64, 0, "cuda")
    out = _outputs(inp)
    rc = B.sse_sigma_bwd(d, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                         B.SSE_MODE_FP64, 0, W, V, *out, ws, ws.numel())
    assert rc == 0, B.sse_strerror(rc)
    return out


def _static(inp, d, W, V):
    out = _outputs(inp)
    rc = B.sse_sigma_bwd_static(d, inp.nbr, inp.dH, inp.D_less, inp.D_greater, inp.G_less, inp.G_greater, SCALE,
                                B.SSE_MODE_FP64, B.SSE_FLAG_CHECK, W, V, *out)
    assert rc == 0, B.sse_strerror(rc)
    return out


@pytest.mark.parametrize("dims", [TINY, Dims(NA=64, NB=4, Norb=10, NE=64, Nkz=5, Nqz=5, Nw=16)],
                         ids=["tiny", "norb10"])
def test_static_scratch_matches_workspace_entry_point(dims):
    nbr = None if dims is TINY else ring_neighbours(dims.NA, dims.NB)
    inp = make_inputs(dims, seed=41, nbr=nbr).to("cuda")
    d = B.dims_of(inp.G_less, inp.D_less, inp.dH)
    assert B.sse_workspace_bytes(d, B.SSE_MODE_FP64, 0) <= B.SSE_STATIC_SCRATCH_BYTES
    for call, seed in enumerate((42, 43)):  # two calls in a row share the static array
        W, V = make_upstream(dims, seed=seed, device="cuda")
        ref = _with_workspace(inp, d, W, V)
        got = _static(inp, d, W, V)
        torch.cuda.synchronize()
        for r, g in zip(ref, got):
            assert normwise(g.cpu().numpy(), r.cpu().numpy()) <= TOL, f"call {call}"


def test_too_large_for_the_static_array_is_refused():
    d = B.sse_dims(1024, 4, 10, 512, 7, 7, 32, 0, 1024)  # needs 275 MB of partials
    assert B.sse_workspace_bytes(d, B.SSE_MODE_FP64, 0) > B.SSE_STATIC_SCRATCH_BYTES
    fake = 1 << 20  # never dereferenced: the size check comes before any device work
    rc = B.sse_sigma_bwd_static(d, fake, fake, fake, fake, fake, fake, SCALE, B.SSE_MODE_FP64, 0, fake, fake, fake,
                                fake, fake, 0)
    assert rc == 6  # SSE_ERR_WORKSPACE
