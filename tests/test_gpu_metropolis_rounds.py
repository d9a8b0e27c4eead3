"""The opt-in Metropolis stream (Section 3, closing paragraph: the resampler's
speed hinges on the random-number rate): Philox-4x32-7 in place of
Philox-4x32-10, same counters.  With the setting at 7, single and batched
Metropolis calls -- staged in shared memory or reading L2, filters shared by
several CTAs included -- equal the oracle on the seven-round stream under the
near-tie rule; the setting goes back to 10 and the default stream returns."""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_metropolis

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture
def seven_rounds():
    pf.load()
    assert pf.pf_get_metropolis_philox_rounds() == 10
    pf.pf_set_metropolis_philox_rounds(7)
    try:
        yield
    finally:
        pf.pf_set_metropolis_philox_rounds(10)
    assert pf.pf_get_metropolis_philox_rounds() == 10


@pytest.mark.parametrize("P,B", [(1024, 64), (49152, 33), (60001, 32), (1 << 20, 32)])
def test_single_call_on_the_seven_round_stream(seven_rounds, P, B):
    lw = workloads.gaussian_logw(P, 1.0, seed=P)
    d = torch.from_numpy(lw).cuda()
    a = torch.full((P,), -1, dtype=torch.int32, device="cuda")
    pf.pf_resample_metropolis(d, P, B, 21, a)
    assert pf.pf_get_device_status() == pf.PF_OK
    idx = np.unique(np.random.default_rng(P).integers(0, P, size=min(P, 3000)))
    got = a.cpu().numpy()[idx]
    rep = check_metropolis(lw, B, got, oracle.metropolis(lw, B, 21, chains=idx, rounds=7), 21, chains=idx, rounds=7)
    assert rep.ok, rep.summary()
    # and it is a different stream from the default one
    assert not np.array_equal(got, oracle.metropolis(lw, B, 21, chains=idx))


def test_batched_on_the_seven_round_stream(seven_rounds):
    # small filters, a staged filter shared by several CTAs (P_f B >= 2^22) and an L2 one
    sizes = [700, 57344, 3000, 70001, 1]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = workloads.batched_logw(off, np.array([1.0, 0.8, 2.0, 1.1, 0.5]), seed=8)
    seeds = workloads.batched_seeds(len(sizes), base=40)
    B = 80
    anc = torch.full((lw.size,), -1, dtype=torch.int32, device="cuda")
    pf.pf_resample_batched(pf.PF_METROPOLIS, torch.from_numpy(lw).cuda(), torch.from_numpy(off).cuda(), len(sizes),
                           B, torch.from_numpy(seeds.view(np.int64)).cuda(), anc)
    assert pf.pf_get_device_status() == pf.PF_OK
    a = anc.cpu().numpy()
    for f in range(len(sizes)):
        lo, hi = off[f], off[f + 1]
        l = lw[lo:hi]
        idx = np.unique(np.random.default_rng(f).integers(0, hi - lo, size=min(hi - lo, 2500)))
        rep = check_metropolis(l, B, a[lo:hi][idx], oracle.metropolis(l, B, int(seeds[f]), f, chains=idx, rounds=7),
                               int(seeds[f]), chains=idx, filter_id=f, rounds=7)
        assert rep.ok, (f, rep.summary())


def test_setting_rejects_other_round_counts():
    pf.load()
    for r in (0, 6, 8, 12):
        with pytest.raises(pf.PFError):
            pf.pf_set_metropolis_philox_rounds(r)
    assert pf.pf_get_metropolis_philox_rounds() == 10
