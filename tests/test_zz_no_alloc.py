"""pf_resample_multinomial_static: the multinomial resampler for callers that
cannot let the library allocate device memory (an allocator that owns all of
it, a deadline that a first-call cudaMalloc would break, a no-allocation rule
after start-up).

It keeps its scratch in the library's fixed device array instead of a
per-stream workspace and searches each draw directly, so two calls in a row
must give exactly the ancestors pf_resample_multinomial gives for the same
inputs and seeds, and both must pass the oracle comparison (the near-tie rule
of the other GPU tests).  Its own status word reports device-side errors and
starts from zero at every call, and a call after the first allocates nothing.
Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_cumulative

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    pf.load()
    yield


def test_static_scratch_matches_workspace_call_twice():
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
        assert np.array_equal(s, w)
        rep = check_cumulative("multinomial", lw_h, s, oracle.multinomial(lw_h, seed), seed)
        assert rep.ok, rep.summary()


def test_static_status_word_and_no_allocation_after_the_first_call():
    P = 5000
    lw_h = workloads.gaussian_logw(P, 1.0, seed=3)
    bad_h = lw_h.copy()
    bad_h[123] = np.inf
    lw, bad = torch.from_numpy(lw_h).cuda(), torch.from_numpy(bad_h).cuda()
    a = torch.empty(P, dtype=torch.int32, device="cuda")
    status = torch.full((1,), 77, dtype=torch.int32, device="cuda")
    pf.pf_resample_multinomial_static(lw, P, 8, a, status)  # set-up call on this device
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    pf.pf_resample_multinomial_static(bad, P, 8, a, status)
    torch.cuda.synchronize()
    assert status.item() == pf.PF_ERR_DOMAIN  # +inf log-weight, reported in this call's word
    pf.pf_resample_multinomial_static(lw, P, 8, a, status)
    torch.cuda.synchronize()
    assert status.item() == 0  # the next call starts from zero
    assert torch.cuda.mem_get_info()[0] == free0  # nothing allocated by the later calls
    rep = check_cumulative("multinomial", lw_h, a.cpu().numpy(), oracle.multinomial(lw_h, 8), 8)
    assert rep.ok, rep.summary()


def test_static_scratch_rejects_sizes_beyond_its_array():
    P = (1 << 20) + 1
    lw = torch.zeros(P, device="cuda")
    a = torch.zeros(P, dtype=torch.int32, device="cuda")
    with pytest.raises(pf.PFError) as ei:
        pf.pf_resample_multinomial_static(lw, P, 0, a)
    assert ei.value.status == pf.PF_ERR_INVALID
