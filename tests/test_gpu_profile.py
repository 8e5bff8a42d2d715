"""SSE_FLAG_PROFILE: per-kernel device times through sse_profile_read, results unchanged."""
import pytest
import torch

from paper_1912_10024_gb300 import binding as B
from paper_1912_10024_gb300.inputs import TINY, make_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,kernel,launches", [("fp64", "sigma_fp64_fwd_kernel", 1),
                                                  ("fp64_fft", "spec_prod_kernel", 2),
                                                  ("fp32_fft", "spec_prod32_kernel", 2),
                                                  ("bf16x3", "sigma_mixed_kernel", 1)])
def test_profile_records_kernels_and_changes_nothing(mode, kernel, launches):
    g = make_inputs(TINY, seed=9).to("cuda")
    args = (g.G_less, g.G_greater, g.dH, g.D_less, g.D_greater, g.nbr)
    B.sse_profile_read()  # clear
    ref = B.sigma(*args, mode=mode)
    assert B.sse_profile_read() == []  # nothing recorded without the flag
    out = B.sigma(*args, mode=mode, profile=True)
    torch.cuda.synchronize()
    rec = {name: (ms, n) for name, ms, n in B.sse_profile_read()}
    assert kernel in rec, rec
    assert rec[kernel][1] == launches and rec[kernel][0] > 0.0
    for a, b in zip(ref, out):
        assert torch.equal(a, b)
    assert B.sse_profile_read() == []  # reading clears
