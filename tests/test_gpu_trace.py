"""The phase trace of the tile kernels (pf_set_trace_buffer), and the ordering
properties of the kernels' waits that it makes visible: no CTA of a
single-launch call leaves the grid-wide wait before the last CTA has published
its tile records, and no tile of a split batched filter leaves its wait before
the filter's last tile has published."""
import numpy as np
import pytest

from paper_1202_6163_gb300 import pf, workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
W = pf.PF_TRACE_WORDS


def traced(call, cap=4096):
    buf = torch.zeros(cap * W, dtype=torch.int64, device="cuda")
    pf.pf_set_trace_buffer(buf, cap)
    try:
        call()
        torch.cuda.synchronize()
    finally:
        pf.pf_set_trace_buffer(None)
    rec = buf.view(cap, W).cpu().numpy()
    return rec[rec[:, 0] != 0]


@pytest.mark.parametrize("fn", [pf.pf_resample_systematic, pf.pf_resample_stratified, pf.pf_resample_multinomial])
def test_single_launch_phases_and_grid_wait(fn):
    P = 1 << 20
    lw = torch.from_numpy(workloads.gaussian_logw(P, 1.0, seed=3)).cuda()
    anc = torch.empty(P, dtype=torch.int32, device="cuda")
    rec = traced(lambda: fn(lw, P, 0, 5, anc))
    assert pf.pf_get_device_status() == pf.PF_OK
    G = len(rec)
    assert G >= 1 and sorted(rec[:, 5]) == list(range(G))  # one record per CTA
    t = rec[:, :5]
    assert np.all(np.diff(t, axis=1) >= 0), "phases out of order"
    assert t[:, 2].min() >= t[:, 1].max(), "a CTA left the grid-wide wait before every CTA had published"
    assert rec[:, 7].min() >= 1  # every CTA owned at least one tile


def test_trace_off_writes_nothing_and_capacity_is_respected():
    P = 1 << 18
    lw = torch.from_numpy(workloads.gaussian_logw(P, 1.0, seed=4)).cuda()
    anc = torch.empty(P, dtype=torch.int32, device="cuda")
    buf = torch.zeros(64 * W, dtype=torch.int64, device="cuda")
    pf.pf_set_trace_buffer(buf, 2)
    try:
        pf.pf_resample_systematic(lw, P, 0, 1, anc)
        torch.cuda.synchronize()
    finally:
        pf.pf_set_trace_buffer(None)
    rec = buf.view(64, W).cpu().numpy()
    assert np.all(rec[:2, 0] != 0) and np.all(rec[2:] == 0)
    buf.zero_()
    pf.pf_resample_systematic(lw, P, 0, 1, anc)
    torch.cuda.synchronize()
    assert np.all(buf.cpu().numpy() == 0)
    with pytest.raises(RuntimeError):
        pf.pf_set_trace_buffer(buf, -1)


def test_batched_items_and_split_filter_waits():
    off, sf = workloads.batched_layout(F=300, seed=2)
    lw = torch.from_numpy(workloads.batched_logw(off, sf, seed=2)).cuda()
    d_off = torch.from_numpy(off).cuda()
    seeds = torch.from_numpy(workloads.batched_seeds(300, base=7).view(np.int64)).cuda()
    anc = torch.empty(lw.numel(), dtype=torch.int32, device="cuda")
    for kind in (pf.PF_SYSTEMATIC, pf.PF_MULTINOMIAL, pf.PF_METROPOLIS):
        B = 8 if kind == pf.PF_METROPOLIS else 0
        rec = traced(lambda: pf.pf_resample_batched(kind, lw, d_off, 300, B, seeds, anc))
        assert pf.pf_get_device_status() == pf.PF_OK
        assert np.all(np.diff(rec[:, :5], axis=1) >= 0)
        assert sorted(set(rec[:, 6].tolist())) == list(range(300))  # every filter was an item
        if kind == pf.PF_SYSTEMATIC:
            split = rec[rec[:, 7] != 31]
            assert len(split) > 0
            for f in np.unique(split[:, 6]):
                r = split[split[:, 6] == f]
                lead = int(off[f]) % 4  # floats before the filter in its 16-byte aligned window
                Tf = int(-(-(off[f + 1] - off[f] + lead) // 8192))
                assert len(r) == Tf >= 2 and sorted(r[:, 7]) == list(range(Tf))
                assert r[:, 2].min() >= r[:, 1].max(), f"filter {f}: a tile left its wait early"
