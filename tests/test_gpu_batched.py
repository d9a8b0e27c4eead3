"""GPU parity of the batched call (many independent filters in one launch)
against the oracle run filter by filter (filter f: key seeds[f], filter id f)."""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_cumulative, check_metropolis

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"multinomial": (pf.PF_MULTINOMIAL, oracle.multinomial),
         "stratified": (pf.PF_STRATIFIED, oracle.stratified),
         "systematic": (pf.PF_SYSTEMATIC, oracle.systematic)}


def run_batched(kind, lw, off, seeds, B=0):
    d_lw = torch.from_numpy(lw).cuda()
    d_off = torch.from_numpy(off.astype(np.int64)).cuda()
    d_seeds = torch.from_numpy(seeds.astype(np.uint64).view(np.int64)).cuda()
    anc = torch.full((lw.size,), -9, dtype=torch.int32, device="cuda")
    pf.pf_resample_batched(kind, d_lw, d_off, off.size - 1, B, d_seeds, anc)
    return anc.cpu().numpy(), pf.pf_get_device_status()


def ragged_layout(seed=0):
    off, sf = workloads.batched_layout(F=40, seed=seed)
    # 57344 / 57345: the largest filter the batched Metropolis stages in shared memory, and one more
    sizes = list(np.diff(off)) + [0, 1, 2, 3, 5, 4096, 8189, 8190, 8192, 8193, 16384 + 7, 57344, 57345, 131069 - 8]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sf = np.concatenate([sf, np.full(len(sizes) - sf.size, 1.3)])
    return off, sf


@pytest.mark.parametrize("name", list(KINDS))
def test_batched_ragged_filters(name):
    kind, orc = KINDS[name]
    off, sf = ragged_layout(1)
    lw = workloads.batched_logw(off, sf, seed=2)
    seeds = workloads.batched_seeds(off.size - 1, base=1000)
    a, st = run_batched(kind, lw, off, seeds)
    assert st == pf.PF_OK, pf.pf_status_string(st)
    for f in range(off.size - 1):
        lo, hi = off[f], off[f + 1]
        if hi == lo:
            continue
        l = lw[lo:hi]
        rep = check_cumulative(name, l, a[lo:hi], orc(l, int(seeds[f]), f), int(seeds[f]), filter_id=f)
        assert rep.ok, (f, hi - lo, rep.summary(), rep.failures[:3])


def test_batched_metropolis_ragged_filters():
    off, sf = ragged_layout(3)
    lw = workloads.batched_logw(off, sf, seed=4)
    seeds = workloads.batched_seeds(off.size - 1, base=77)
    B = 12
    a, st = run_batched(pf.PF_METROPOLIS, lw, off, seeds, B=B)
    assert st == pf.PF_OK
    for f in range(off.size - 1):
        lo, hi = off[f], off[f + 1]
        if hi == lo:
            continue
        l = lw[lo:hi]
        rep = check_metropolis(l, B, a[lo:hi], oracle.metropolis(l, B, int(seeds[f]), f), int(seeds[f]), filter_id=f)
        assert rep.ok, (f, rep.summary())


def test_batched_metropolis_wide_range():
    # spreads of 40: most staged weights fall below 2^-100 and those states decide
    # from the log-weights (filters of 3000 and 57000 are staged, 60000 is not)
    sizes = [3000, 57000, 60000, 1]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = workloads.batched_logw(off, np.full(len(sizes), 40.0), seed=6)
    lw[np.random.default_rng(6).random(lw.size) < 0.05] = -np.inf
    seeds = workloads.batched_seeds(len(sizes), base=90)
    B = 20
    a, st = run_batched(pf.PF_METROPOLIS, lw, off, seeds, B=B)
    assert st == pf.PF_OK
    for f in range(len(sizes)):
        l = lw[off[f]:off[f + 1]]
        rep = check_metropolis(l, B, a[off[f]:off[f + 1]], oracle.metropolis(l, B, int(seeds[f]), f), int(seeds[f]),
                               filter_id=f)
        assert rep.ok, (f, rep.summary())


def test_batched_bad_filters_are_reported_and_others_resampled():
    sizes = [1000, 2000, 150000, 500]  # the third exceeds the per-filter limit
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = workloads.gaussian_logw(int(off[-1]), 1.0, seed=5)
    lw[off[1]:off[2]] = -np.inf  # a filter with every weight zero
    seeds = workloads.batched_seeds(4, base=3)
    a, st = run_batched(pf.PF_SYSTEMATIC, lw, off, seeds)
    assert st in (pf.PF_ERR_DOMAIN, pf.PF_ERR_INVALID)
    for f in (0, 3):
        l = lw[off[f]:off[f + 1]]
        rep = check_cumulative("systematic", l, a[off[f]:off[f + 1]], oracle.systematic(l, int(seeds[f]), f),
                               int(seeds[f]), filter_id=f)
        assert rep.ok


@pytest.mark.parametrize("name", list(KINDS))
def test_batched_4096_filters_sampled(name):
    # F = 4096, P_f log-uniform in [256, 65536], s_f ~ U[0.5, 3]; 64 filters checked in full
    kind, orc = KINDS[name]
    off, sf = workloads.batched_layout(F=4096, seed=0)
    lw = workloads.batched_logw(off, sf, seed=0)
    seeds = workloads.batched_seeds(4096, base=0)
    a, st = run_batched(kind, lw, off, seeds)
    assert st == pf.PF_OK
    for f in np.random.default_rng(1).choice(4096, size=64, replace=False):
        lo, hi = off[f], off[f + 1]
        l = lw[lo:hi]
        rep = check_cumulative(name, l, a[lo:hi], orc(l, int(seeds[f]), int(f)), int(seeds[f]), filter_id=int(f))
        assert rep.ok, (f, rep.summary())
    # every ancestor is filter-local and in range
    sizes = np.repeat(np.diff(off), np.diff(off))
    assert np.all((a >= 0) & (a < sizes))


def test_batched_repeatable():
    off, sf = ragged_layout(5)
    lw = workloads.batched_logw(off, sf, seed=6)
    seeds = workloads.batched_seeds(off.size - 1, base=9)
    a1, _ = run_batched(pf.PF_STRATIFIED, lw, off, seeds)
    a2, _ = run_batched(pf.PF_STRATIFIED, lw, off, seeds)
    assert np.array_equal(a1, a2)


def test_split_filter_timeout_is_reported_and_recovered():
    # filters of several tiles are split over CTAs that wait for each other's
    # records; a withheld record makes the waits run out (bounded), the call
    # reports PF_ERR_TIMEOUT, and the next call is correct again
    sizes = np.array([30000, 100, 70000, 9000], dtype=np.int64)
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = workloads.gaussian_logw(int(off[-1]), 1.0, seed=4)
    seeds = workloads.batched_seeds(sizes.size, base=3)
    d_lw, d_off = torch.from_numpy(lw).cuda(), torch.from_numpy(off).cuda()
    d_seeds = torch.from_numpy(seeds.view(np.int64)).cuda()
    anc = torch.empty(lw.size, dtype=torch.int32, device="cuda")
    pf.pf_set_wait_limit_ns(5_000_000)
    try:
        pf.pf_debug_skip_publish(1)
        pf.pf_resample_batched(pf.PF_SYSTEMATIC, d_lw, d_off, sizes.size, 0, d_seeds, anc)
        assert pf.pf_get_device_status() == pf.PF_ERR_TIMEOUT
    finally:
        pf.pf_debug_skip_publish(-1)
        pf.pf_set_wait_limit_ns(1_000_000_000)
    pf.pf_resample_batched(pf.PF_SYSTEMATIC, d_lw, d_off, sizes.size, 0, d_seeds, anc)
    assert pf.pf_get_device_status() == pf.PF_OK
    a = anc.cpu().numpy()
    for f in range(sizes.size):
        l = lw[off[f]:off[f + 1]]
        rep = check_cumulative("systematic", l, a[off[f]:off[f + 1]], oracle.systematic(l, int(seeds[f]), f),
                               int(seeds[f]), filter_id=f)
        assert rep.ok, (f, rep.summary())


def test_batched_metropolis_takes_each_filters_own_bound():
    # B < 0: every filter takes B from Eq. 5 with its own largest normalised weight.
    # The B the device chose equals the host bound of the FP64 w_max (one step off at
    # most, and only where the bound sits at an integer), and each filter's chains equal
    # the oracle's for that B; the plain batched call with B = -1 is the same call at
    # eps = 0.01.  Filters staged in shared memory and larger ones (read from L2), a
    # one-particle filter, an all-equal filter (w_max = 1/P, so lambda = 0 and B = 1)
    # and an empty one.
    sizes = [3000, 1, 777, 0, 20000, 57344, 57345, 70001, 12, 4096]
    spreads = [1.0, 0.5, 2.0, 1.0, 0.7, 1.2, 1.2, 0.9, 3.0, 0.0]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = workloads.batched_logw(off, np.array(spreads), seed=5)
    seeds = workloads.batched_seeds(len(sizes), base=900)
    F = len(sizes)
    d_lw = torch.from_numpy(lw).cuda()
    d_off = torch.from_numpy(off).cuda()
    d_seeds = torch.from_numpy(seeds.view(np.int64)).cuda()
    for eps in (0.01, 0.1):
        anc = torch.full((lw.size,), -9, dtype=torch.int32, device="cuda")
        B_out = torch.full((F,), -5, dtype=torch.int32, device="cuda")
        pf.pf_resample_batched_metropolis_bound(d_lw, d_off, F, eps, d_seeds, anc, B_out)
        assert pf.pf_get_device_status() == pf.PF_OK
        a, Bg = anc.cpu().numpy(), B_out.cpu().numpy()
        off_by_one = 0
        for f in range(F):
            lo, hi = off[f], off[f + 1]
            if hi == lo:
                assert Bg[f] == -5  # skipped: left untouched
                continue
            l = lw[lo:hi]
            w = np.exp(l.astype(np.float64) - l.max())
            B_host = pf.pf_metropolis_B(hi - lo, w.max() / w.sum(), eps)
            assert abs(int(Bg[f]) - B_host) <= 1, (f, Bg[f], B_host)
            off_by_one += int(Bg[f]) != B_host
            rep = check_metropolis(l, int(Bg[f]), a[lo:hi], oracle.metropolis(l, int(Bg[f]), int(seeds[f]), f),
                                   int(seeds[f]), filter_id=f)
            assert rep.ok, (f, rep.summary())
        assert off_by_one <= 1
        print(f"\neps={eps}: per-filter B {Bg.tolist()}")
        if eps == 0.01:
            anc2 = torch.full((lw.size,), -9, dtype=torch.int32, device="cuda")
            pf.pf_resample_batched(pf.PF_METROPOLIS, d_lw, d_off, F, -1, d_seeds, anc2)
            assert pf.pf_get_device_status() == pf.PF_OK
            assert torch.equal(anc, anc2)


@pytest.mark.parametrize("name", ["systematic", "stratified"])
def test_batched_whole_filters_when_they_fill_the_grid(name):
    # with at least as many several-tile filters as resident CTAs (304 on GB300) the plan keeps
    # each filter whole in one CTA (no wait on other CTAs); ragged sizes around tile boundaries,
    # unaligned offsets, one-tile filters between them, every filter against the oracle
    kind, orc = KINDS[name]
    cycle = [8193, 9001, 16384 + 7, 20000, 8189 + 8, 65536, 131069 - 8, 12345, 300, 8192]
    sizes = [cycle[i % len(cycle)] for i in range(480)]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    sf = np.resize(np.array([0.5, 1.0, 2.0, 3.0]), len(sizes))
    lw = workloads.batched_logw(off, sf, seed=12)
    seeds = workloads.batched_seeds(len(sizes), base=70)
    a, st = run_batched(kind, lw, off, seeds)
    assert st == pf.PF_OK
    for f in range(len(sizes)):
        l = lw[off[f]:off[f + 1]]
        rep = check_cumulative(name, l, a[off[f]:off[f + 1]], orc(l, int(seeds[f]), f), int(seeds[f]), filter_id=f)
        assert rep.ok, (f, sizes[f], rep.summary())
