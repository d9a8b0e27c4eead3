"""pf_resample_multinomial_static: the multinomial resampler for callers that
cannot let the library allocate device memory.

It runs the same kernel as pf_resample_multinomial with its scratch in the
library's fixed device array instead of a per-stream workspace, so two calls
in a row must give exactly the ancestors pf_resample_multinomial gives for the
same inputs and seeds (the tolerance of the other GPU tests: identical, or a
near tie against the oracle).  Kept in a file of its own that pytest collects
last.
"""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_cumulative

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_scratch_matches_workspace_call_twice():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    pf.load()
    status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
    for P, seed in ((300001, 41), (1 << 20, 42)):
        lw_h = workloads.gaussian_logw(P, 1.0, seed=seed)
        lw = torch.from_numpy(lw_h).cuda()
        a_static = torch.full((P,), -1, dtype=torch.int32, device="cuda")
        a_ws = torch.full((P,), -2, dtype=torch.int32, device="cuda")
        pf.pf_resample_multinomial_static(lw, P, seed, a_static, status)
        pf.pf_resample_multinomial(lw, P, 0, seed, a_ws)
        assert pf.pf_get_device_status() == pf.PF_OK
        assert status.item() == 0
        s, w = a_static.cpu().numpy(), a_ws.cpu().numpy()
        if not np.array_equal(s, w):
            rep = check_cumulative("multinomial", lw_h, s, oracle.multinomial(lw_h, seed), seed)
            assert rep.ok, rep.summary()


def test_static_scratch_rejects_sizes_beyond_its_array():
    pf.load()
    P = (1 << 20) + 1
    lw = torch.zeros(P, device="cuda")
    a = torch.zeros(P, dtype=torch.int32, device="cuda")
    with pytest.raises(pf.PFError) as ei:
        pf.pf_resample_multinomial_static(lw, P, 0, a)
    assert ei.value.status == pf.PF_ERR_INVALID
