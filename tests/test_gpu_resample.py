"""GPU parity: libpf (through its C ABI) against the FP64 oracle.

Ancestors must match the oracle's exactly except at near-tie decisions (see
tests/parity.py); gathered states bit for bit; ESS within the tolerance derived
from the arithmetic (2e-6 relative: per-weight error of a few float ulps,
compensated sums, an FP64 combine).
"""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_cumulative, check_metropolis

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CUMULATIVE = {
    "systematic": (pf.pf_resample_systematic, oracle.systematic),
    "stratified": (pf.pf_resample_stratified, oracle.stratified),
    "multinomial": (pf.pf_resample_multinomial, oracle.multinomial),
}


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("a CUDA device is required for -m gpu tests")
    pf.load()
    yield
    torch.cuda.synchronize()


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_resample(fn, lw, seed, B=0):
    t = to_dev(lw)
    a = torch.full((lw.size,), -7, dtype=torch.int32, device="cuda")
    fn(t, lw.size, B, seed, a)
    st = pf.pf_get_device_status()
    return a.cpu().numpy(), st


def assert_cumulative(kind, lw, seed):
    fn, orc = CUMULATIVE[kind]
    a, st = gpu_resample(fn, lw, seed)
    assert st == pf.PF_OK, pf.pf_status_string(st)
    rep = check_cumulative(kind, lw, a, orc(lw, seed), seed)
    assert rep.ok, rep.summary() + f" first failures: {rep.failures[:5]}"
    if kind != "multinomial":
        assert np.all(np.diff(a) >= 0)
    return rep


# ------------------------------------------------------------------ workload: P = 1024
def test_single_resample_P1024_all_four_and_gather():
    P = 1024
    lw = workloads.gaussian_logw(P, 1.0, seed=0)
    states = workloads.states(P, 4, seed=1)
    for kind in CUMULATIVE:
        assert_cumulative(kind, lw, 0)
    a, st = gpu_resample(pf.pf_resample_metropolis, lw, 0, B=64)
    assert st == pf.PF_OK
    rep = check_metropolis(lw, 64, a, oracle.metropolis(lw, 64, 0), 0)
    assert rep.ok, rep.summary()
    src = to_dev(states)
    dst = torch.empty_like(src)
    anc = to_dev(a.astype(np.int32))
    pf.pf_gather(src, P, 16, anc, P, dst)
    assert pf.pf_get_device_status() == pf.PF_OK
    assert np.array_equal(dst.cpu().numpy(), oracle.gather(states, a))


# ------------------------------------------------------------------ sizes, tiles, ragged tails
SIZES = [1, 2, 3, 4, 5, 31, 1000, 2048, 4097, 65539, 300001]


@pytest.mark.parametrize("kind", list(CUMULATIVE))
@pytest.mark.parametrize("P", SIZES)
@pytest.mark.parametrize("s", [0.25, 1.0, 4.0])
def test_cumulative_sizes(kind, P, s):
    lw = workloads.gaussian_logw(P, s, seed=P + int(10 * s))
    assert_cumulative(kind, lw, seed=P * 7 + 1)


@pytest.mark.parametrize("kind", list(CUMULATIVE))
@pytest.mark.parametrize("s", [0.25, 1.0, 2.0, 4.0])
def test_cumulative_P2e20(kind, s):
    P = 1 << 20
    lw = workloads.gaussian_logw(P, s, seed=int(100 * s))
    rep = assert_cumulative(kind, lw, seed=11)
    print(kind, s, rep.summary())


@pytest.mark.parametrize("P", [1, 3, 1000, 65539])
@pytest.mark.parametrize("B", [0, 1, 7, 64])
def test_metropolis_sizes(P, B):
    lw = workloads.gaussian_logw(P, 1.0, seed=P + B)
    a, st = gpu_resample(pf.pf_resample_metropolis, lw, 5, B=B)
    assert st == pf.PF_OK
    rep = check_metropolis(lw, B, a, oracle.metropolis(lw, B, 5), 5)
    assert rep.ok, rep.summary()


@pytest.mark.parametrize("s,B", [(0.25, 8), (1.0, 32), (2.0, 128), (4.0, 512)])
def test_metropolis_P2e20_sampled(s, B):
    P = 1 << 20
    lw = workloads.gaussian_logw(P, s, seed=int(100 * s))
    a, st = gpu_resample(pf.pf_resample_metropolis, lw, 21, B=B)
    assert st == pf.PF_OK
    idx = np.random.default_rng(0).choice(P, size=2000, replace=False)
    idx = np.concatenate([idx, [0, 1, P - 1]])
    rep = check_metropolis(lw, B, a[idx], oracle.metropolis(lw, B, 21, chains=idx), 21, chains=idx)
    assert rep.ok, rep.summary()
    print("metropolis", s, B, rep.summary())


# ------------------------------------------------------------------ edge cases
def test_zero_weights_never_selected():
    rng = np.random.default_rng(3)
    for P in (7, 5000, 100003):
        lw = rng.standard_normal(P).astype(np.float32)
        lw[rng.random(P) < 0.3] = -np.inf
        for kind in CUMULATIVE:
            assert_cumulative(kind, lw, seed=P)
        a, st = gpu_resample(pf.pf_resample_metropolis, lw, 1, B=16)
        assert st == pf.PF_OK
        assert check_metropolis(lw, 16, a, oracle.metropolis(lw, 16, 1), 1).ok


def test_metropolis_staged_weights_over_a_wide_range():
    # log-weights N(0, 40^2): most staged weights exp(lw - max) fall below 2^-100 or
    # underflow, so chains in those states decide from the log-weights; P = 3000 and
    # 40000 are staged in shared memory, 60000 is read through L2
    rng = np.random.default_rng(11)
    for P in (3000, 40000, 60000):
        lw = (40.0 * rng.standard_normal(P)).astype(np.float32)
        lw[rng.random(P) < 0.05] = -np.inf
        a, st = gpu_resample(pf.pf_resample_metropolis, lw, 4, B=24)
        assert st == pf.PF_OK
        rep = check_metropolis(lw, 24, a, oracle.metropolis(lw, 24, 4), 4)
        assert rep.ok, rep.summary()


def test_one_hot_and_equal_weights():
    for P in (1, 9, 70001):
        lw = np.full(P, -np.inf, np.float32)
        lw[P // 3] = 1.5
        for kind, (fn, _) in CUMULATIVE.items():
            a, st = gpu_resample(fn, lw, 2)
            assert st == pf.PF_OK and np.all(a == P // 3), kind
        # equal weights: the oracle gives the identity; the GPU may differ only at
        # strata whose offset lies within the near-tie band of a stratum edge
        eq = np.full(P, -3.25, np.float32)
        for kind in ("systematic", "stratified"):
            a, st = gpu_resample(CUMULATIVE[kind][0], eq, 4)
            assert st == pf.PF_OK
            assert np.array_equal(CUMULATIVE[kind][1](eq, 4), np.arange(P))
            rep = check_cumulative(kind, eq, a, np.arange(P), 4)
            assert rep.ok and rep.mismatches <= max(2, P // 1000), (kind, rep.summary())


def test_extreme_log_weights():
    rng = np.random.default_rng(5)
    P = 200003
    for lw in (rng.standard_normal(P).astype(np.float32) - 5000.0,
               (30.0 * rng.standard_normal(P)).astype(np.float32),
               np.linspace(-80, 80, P).astype(np.float32)):
        for kind in CUMULATIVE:
            assert_cumulative(kind, lw, seed=9)


def test_deterministic_and_seed_sensitive():
    lw = workloads.gaussian_logw(100000, 1.0, seed=8)
    for kind, (fn, _) in CUMULATIVE.items():
        a1, _ = gpu_resample(fn, lw, 123)
        a2, _ = gpu_resample(fn, lw, 123)
        a3, _ = gpu_resample(fn, lw, 124)
        assert np.array_equal(a1, a2)
        assert not np.array_equal(a1, a3)


def test_philox_streams_visible_through_equal_weights():
    # with equal weights and P = 2^k the multinomial pick is floor(u_j P) and the
    # Metropolis pick is the last proposal: both expose the raw Philox words
    P = 1 << 12
    lw = np.zeros(P, np.float32)
    a, _ = gpu_resample(pf.pf_resample_multinomial, lw, 77)
    u = oracle.stream_uniforms(77, 0, oracle.TAG_MULTI, P, kind=1)
    assert np.array_equal(a, np.floor(u * P).astype(np.int64))
    a, _ = gpu_resample(pf.pf_resample_metropolis, lw, 78, B=5)
    last = [oracle.metropolis_draws(78, 0, P, i, 5)[0][-1] for i in range(P)]
    assert np.array_equal(a, last)


# ------------------------------------------------------------------ errors
@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_domain_errors(bad):
    lw = workloads.gaussian_logw(50000, 1.0, seed=1)
    lw[1234] = bad
    for kind, (fn, _) in CUMULATIVE.items():
        _, st = gpu_resample(fn, lw, 0)
        assert st == pf.PF_ERR_DOMAIN, kind
    _, st = gpu_resample(pf.pf_resample_metropolis, lw, 0, B=4)
    assert st == pf.PF_ERR_DOMAIN
    e = torch.zeros(1, device="cuda")
    pf.pf_ess(to_dev(lw), lw.size, e)
    assert pf.pf_get_device_status() == pf.PF_ERR_DOMAIN


def test_all_zero_weights_is_domain_error():
    lw = np.full(3000, -np.inf, np.float32)
    for kind, (fn, _) in CUMULATIVE.items():
        _, st = gpu_resample(fn, lw, 0)
        assert st == pf.PF_ERR_DOMAIN, kind


def test_invalid_arguments():
    t = torch.zeros(17, device="cuda")
    a = torch.zeros(17, dtype=torch.int32, device="cuda")
    for fn in list(pf.RESAMPLERS.values()):
        with pytest.raises(pf.PFError) as ei:
            fn(t, 0, 1, 0, a)
        assert ei.value.status == pf.PF_ERR_INVALID
        with pytest.raises(pf.PFError):
            fn(t.data_ptr() + 2, 16, 1, 0, a)  # log-weights not 4-byte aligned
        with pytest.raises(pf.PFError):
            fn(0, 16, 1, 0, a)
    with pytest.raises(pf.PFError):
        pf.pf_gather(t, 17, 6, a, 1, torch.zeros(17, device="cuda"))
    with pytest.raises(pf.PFError):
        pf.pf_gather(t, 17, 4, a, 4, t)  # overlapping


def test_timeout_is_reported_and_recovered():
    P = 1 << 20
    lw = workloads.gaussian_logw(P, 1.0, seed=2)
    pf.pf_set_wait_limit_ns(20_000_000)
    try:
        pf.pf_debug_skip_publish(3)
        _, st = gpu_resample(pf.pf_resample_systematic, lw, 1)
        assert st == pf.PF_ERR_TIMEOUT
    finally:
        pf.pf_debug_skip_publish(-1)
        pf.pf_set_wait_limit_ns(1_000_000_000)
    assert_cumulative("systematic", lw, 1)


# ------------------------------------------------------------------ ESS and gather
@pytest.mark.parametrize("P", [1, 5, 4096, 4099, 1 << 20])
@pytest.mark.parametrize("s", [0.25, 1.0, 4.0])
def test_ess(P, s):
    lw = workloads.gaussian_logw(P, s, seed=P)
    e = torch.zeros(1, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    pf.pf_ess(to_dev(lw), P, e, ls)
    assert pf.pf_get_device_status() == pf.PF_OK
    ess, log_sum = oracle.ess(lw)
    assert e.item() == pytest.approx(ess, rel=2e-6)
    assert ls.item() == pytest.approx(log_sum, rel=1e-12, abs=2e-6)


@pytest.mark.parametrize("case", ["gauss_2_6M", "heavy_2e24", "dead_tiles_2e23"])
def test_ess_large_and_dead_tiles(case):
    # thousands of tile records in the final combine; dead_tiles has whole
    # runs of tiles with no mass (lw = -inf) and the largest exponent reached
    # in a single late tile; a NaN in the last tile then gives PF_ERR_DOMAIN
    if case == "gauss_2_6M":
        lw = workloads.gaussian_logw(2_600_007, 2.0, seed=41)
    elif case == "heavy_2e24":
        lw = workloads.heavy_tail_logw(1 << 24, shift=10.0, frac=0.01, seed=3)
    else:
        lw = workloads.gaussian_logw(1 << 23, 1.0, seed=42)
        lw[: 3 << 20] = -np.inf
        lw[(5 << 20):(6 << 20)] = -np.inf
        lw[(7 << 20) + 12345] = 40.0
    e = torch.zeros(1, device="cuda")
    ls = torch.zeros(1, dtype=torch.float64, device="cuda")
    pf.pf_ess(to_dev(lw), lw.size, e, ls)
    assert pf.pf_get_device_status() == pf.PF_OK
    ess, log_sum = oracle.ess(lw)
    assert e.item() == pytest.approx(ess, rel=2e-6)
    assert ls.item() == pytest.approx(log_sum, rel=1e-12, abs=2e-6)
    lw[lw.size - 7] = np.nan
    pf.pf_ess(to_dev(lw), lw.size, e, ls)
    assert pf.pf_get_device_status() == pf.PF_ERR_DOMAIN
    assert np.isnan(e.item()) and np.isnan(ls.item())


@pytest.mark.parametrize("row_bytes", [4, 12, 16, 64, 68, 256])
@pytest.mark.parametrize("P", [1, 1000, 70001])
def test_gather_bit_exact(row_bytes, P):
    rng = np.random.default_rng(row_bytes + P)
    src = rng.integers(0, 2**31, size=(P, row_bytes // 4), dtype=np.int64).astype(np.int32)
    P_dst = P + 3
    anc = rng.integers(0, P, size=P_dst).astype(np.int32)
    d_src = to_dev(src)
    d_dst = torch.zeros((P_dst, row_bytes // 4), dtype=torch.int32, device="cuda")
    pf.pf_gather(d_src, P, row_bytes, to_dev(anc), P_dst, d_dst)
    assert pf.pf_get_device_status() == pf.PF_OK
    assert np.array_equal(d_dst.cpu().numpy(), oracle.gather(src, anc))


def test_gather_rejects_out_of_range_ancestor():
    src = torch.arange(40, dtype=torch.int32, device="cuda").reshape(10, 4)
    dst = torch.full((3, 4), -1, dtype=torch.int32, device="cuda")
    anc = torch.tensor([2, 10, 0], dtype=torch.int32, device="cuda")
    pf.pf_gather(src, 10, 16, anc, 3, dst)
    assert pf.pf_get_device_status() == pf.PF_ERR_INVALID
    out = dst.cpu().numpy()
    assert np.array_equal(out[0], [8, 9, 10, 11]) and np.all(out[1] == -1) and np.array_equal(out[2], [0, 1, 2, 3])


def test_metropolis_autotuned_B():
    P = 4096
    lw = workloads.gaussian_logw(P, 1.0, seed=6)
    ess, log_sum = oracle.ess(lw)
    w_max = float(np.exp(np.float64(lw.max()) - log_sum))
    B = oracle.metropolis_B(P, w_max, 0.01)
    a, st = gpu_resample(pf.pf_resample_metropolis, lw, 3, B=-1)
    assert st == pf.PF_OK
    # the device derives w_max from its own float sums: B may differ by one at a rounding edge
    matches = [b for b in (B - 1, B, B + 1) if np.array_equal(a, gpu_resample(pf.pf_resample_metropolis, lw, 3, b)[0])]
    assert matches, (B, matches)
    assert check_metropolis(lw, B, gpu_resample(pf.pf_resample_metropolis, lw, 3, B)[0],
                            oracle.metropolis(lw, B, 3), 3).ok


# ------------------------------------------------------------------ several tiles per CTA (large P)
@pytest.mark.parametrize("kind", list(CUMULATIVE))
def test_cumulative_multi_tile_2_6M(kind):
    P = 2_600_007  # more tiles than resident CTAs
    lw = workloads.gaussian_logw(P, 1.5, seed=77)
    rep = assert_cumulative(kind, lw, seed=5)
    print(kind, "2.6M", rep.summary())


@pytest.mark.parametrize("case", ["dead_runs", "one_heavy", "spread4", "ragged_unaligned", "dirichlet_0.01",
                                  "equal_4M", "two_level"])
def test_multinomial_guide_table_cases(case):
    # above one tile per resident CTA the multinomial draws go through the guide
    # table first: runs of zero-weight particles (whole tiles without mass, where
    # the guide's tile has no positive element), a handful of particles holding
    # almost all the weight (buckets spanning thousands of light particles, the
    # three-level fallback), a wide spread, a ragged unaligned view, the paper's
    # Dirichlet law at alpha = .01, equal weights (every bucket exactly four
    # particles) and alternating runs of heavy and light particles
    rng = np.random.default_rng(31)
    P = 3_000_017
    lw = workloads.gaussian_logw(P, 1.0, seed=32)
    if case == "dead_runs":
        for start in rng.integers(0, P - 40000, size=12):
            lw[start:start + int(rng.integers(100, 40000))] = -np.inf
        lw[: 8192 * 3 + 5] = -np.inf
    elif case == "one_heavy":
        lw[rng.integers(0, P, size=7)] += 25.0
    elif case == "spread4":
        lw = workloads.gaussian_logw(P, 4.0, seed=33)
    elif case == "dirichlet_0.01":  # the paper's weight law at its smallest alpha: log-weights spread over thousands
        lw = workloads.dirichlet_logw(P, 0.01, seed=34)
    elif case == "equal_4M":  # every bucket holds exactly four particles
        P = 1 << 22
        lw = np.full(P, -1.5, np.float32)
    elif case == "two_level":  # alternating runs of heavy and light particles
        lw = np.where((np.arange(P) // 1000) % 2 == 0, 3.0, -3.0).astype(np.float32)
    a_ref = oracle.multinomial(lw if case != "ragged_unaligned" else lw[3:], 41)
    if case == "ragged_unaligned":
        base = to_dev(lw)
        view = base[3:]
        a = torch.full((P - 3,), -7, dtype=torch.int32, device="cuda")
        pf.pf_resample_multinomial(view, P - 3, 0, 41, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative("multinomial", lw[3:], a.cpu().numpy(), a_ref, 41)
    else:
        a, st = gpu_resample(pf.pf_resample_multinomial, lw, 41)
        assert st == pf.PF_OK
        rep = check_cumulative("multinomial", lw, a, a_ref, 41)
    assert rep.ok, rep.summary() + f" first failures: {rep.failures[:5]}"
    print(case, rep.summary())


@pytest.mark.parametrize("kind", list(CUMULATIVE))
def test_offsets_beyond_2e24_in_one_launch(kind):
    # 2^24 < P <= 2^25 in the single cooperative launch: offset counts above 2^24
    # have no exact float, so each tile's offset map takes its origin from the
    # exact pair minus the integer count; the mismatches stay rare near ties
    P = (1 << 24) + (1 << 23) + 5
    lw = workloads.gaussian_logw(P, 1.0, seed=93)
    rep = assert_cumulative(kind, lw, seed=21)
    assert rep.mismatches <= P // 1000, rep.summary()
    print(kind, "2^24 + 2^23 + 5", rep.summary())


@pytest.mark.parametrize("kind", list(CUMULATIVE))
def test_cumulative_beyond_one_launch(kind):
    # P + lead above 4096 tiles of 8192: the tile scans, one CTA forming every
    # tile's carry, then the assignment or the draws, as three ordinary launches
    P = (1 << 25) + 12345
    lw = workloads.gaussian_logw(P, 1.0, seed=91)
    rep = assert_cumulative(kind, lw, seed=13)
    assert rep.mismatches <= P // 1000, rep.summary()
    print(kind, "2^25 + 12345", rep.summary())


def test_multinomial_ordinary_launches_below_the_tile_limit():
    # 3400 tiles of 8192: the tile table and its level-1 samples no longer fit
    # shared memory, so the multinomial takes the ordinary launches and their
    # guide table although one cooperative launch could hold the tiles
    P = 3400 * 8192 - 11
    lw = workloads.gaussian_logw(P, 2.0, seed=94)
    rep = assert_cumulative("multinomial", lw, seed=23)
    assert rep.mismatches <= P // 1000, rep.summary()
    print("multinomial", P, rep.summary())


def test_cumulative_beyond_one_launch_unaligned_heavy_tail_and_errors():
    P = (1 << 25) + 3
    lw = workloads.heavy_tail_logw(P + 1, shift=10.0, frac=0.01, seed=92)
    base = to_dev(lw)
    view = base[1:]  # a lead of one float: P + lead = 2^25 + 4
    for kind, (fn, orc) in CUMULATIVE.items():
        a = torch.full((P,), -7, dtype=torch.int32, device="cuda")
        fn(view, P, 0, 17, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative(kind, lw[1:], a.cpu().numpy(), orc(lw[1:], 17), 17)
        assert rep.ok, (kind, rep.summary())
    bad = lw[1:].copy()
    bad[P - 2] = np.nan
    zero = np.full(P, -np.inf, np.float32)
    for arr in (bad, zero):
        for kind, (fn, _) in CUMULATIVE.items():
            a, st = gpu_resample(fn, arr, 3)
            assert st == pf.PF_ERR_DOMAIN, kind
            assert np.all(a == -7), kind  # no ancestor written


def test_multinomial_guide_after_other_kinds():
    # the guide's second grid-wide arrival uses its own pair of epoch-alternating
    # counters; every single-launch call resets the one the next call may use, so
    # a guided multinomial call right after systematic or stratified calls (an odd
    # or even number of them) still waits for every CTA's guide entries
    P = 3_000_017
    lw = workloads.gaussian_logw(P, 1.0, seed=36)
    others = [pf.pf_resample_systematic, pf.pf_resample_stratified]
    for gap in (0, 1, 2, 3, 4):
        for k in range(gap):
            gpu_resample(others[k % 2], lw, 50 + k)
        a, st = gpu_resample(pf.pf_resample_multinomial, lw, 60 + gap)
        assert st == pf.PF_OK
        rep = check_cumulative("multinomial", lw, a, oracle.multinomial(lw, 60 + gap), 60 + gap)
        assert rep.ok, (gap, rep.summary())


@pytest.mark.parametrize("kind", list(CUMULATIVE))
def test_cumulative_P2e24_heavy_tail(kind):
    # log-weights N(0,1) with 1% of entries shifted by +10
    P = 1 << 24
    lw = workloads.heavy_tail_logw(P, shift=10.0, frac=0.01, seed=3)
    rep = assert_cumulative(kind, lw, seed=9)
    print(kind, "2^24", rep.summary())


def test_config3_P2e24_metropolis_autotuned_B_and_gather():
    # P = 2^24 heavy tail, Metropolis with B from the Eq. 5 bound on the device
    # (eps = 0.01; P w_max is about 1.2e4, so B is about 5e4), then the gather
    # of P x 8 float32 states by its ancestors
    P = 1 << 24
    lw = workloads.heavy_tail_logw(P, shift=10.0, frac=0.01, seed=3)
    ess, log_sum = oracle.ess(lw)
    w_max = float(np.exp(np.float64(lw.max()) - log_sum))
    B = oracle.metropolis_B(P, w_max, 0.01)
    assert 20000 < B < 200000
    d = torch.from_numpy(lw).cuda()
    a_auto = torch.empty(P, dtype=torch.int32, device="cuda")
    pf.pf_resample_metropolis(d, P, -1, 8, a_auto)
    assert pf.pf_get_device_status() == pf.PF_OK
    a_B = torch.empty(P, dtype=torch.int32, device="cuda")
    pf.pf_resample_metropolis(d, P, B, 8, a_B)
    assert pf.pf_get_device_status() == pf.PF_OK
    # the device's w_max comes from its own float sums: B may differ by one at a rounding edge
    same = bool(torch.equal(a_auto, a_B))
    if not same:
        for b in (B - 1, B + 1):
            pf.pf_resample_metropolis(d, P, b, 8, a_B)
            same = same or bool(torch.equal(a_auto, a_B))
    assert same
    chains = np.unique(np.random.default_rng(1).integers(0, P, size=48))
    a = a_auto.cpu().numpy()
    rep = check_metropolis(lw, B, a[chains], oracle.metropolis(lw, B, 8, chains=chains), 8, chains=chains)
    assert rep.ok, rep.summary()
    # most chains end on a shifted particle: the heavy tail holds ~0.99 of the weight
    shifted = lw[a] > 5
    assert shifted.mean() > 0.97
    st = torch.from_numpy(workloads.states(P, 8, seed=4)).cuda()
    dst = torch.empty_like(st)
    pf.pf_gather(st, P, 32, a_auto, P, dst)
    assert pf.pf_get_device_status() == pf.PF_OK
    rows = np.random.default_rng(2).integers(0, P, size=20000)
    np.testing.assert_array_equal(dst[torch.from_numpy(rows).cuda()].cpu().numpy(),
                                  st[torch.from_numpy(a[rows]).long().cuda()].cpu().numpy())


def test_cumulative_one_past_single_launch_capacity_is_served():
    # one particle past 4096 tiles of 8192: the ordinary launches, with equal
    # weights every particle keeps one offspring (systematic, stratified), and
    # P beyond PF_MAX_PARTICLES is still rejected on the host
    P = (1 << 25) + 1
    t = torch.zeros(P, device="cuda")
    for fn in (pf.pf_resample_systematic, pf.pf_resample_stratified):
        a = torch.full((P,), -7, dtype=torch.int32, device="cuda")
        fn(t, P, 0, 0, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        counts = torch.bincount(a.long(), minlength=P)
        assert counts.numel() == P and int((counts != 1).sum()) <= P // 1000
    a = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    pf.pf_resample_multinomial(t, P, 0, 0, a)
    assert pf.pf_get_device_status() == pf.PF_OK
    assert int(a.min()) >= 0 and int(a.max()) < P
    with pytest.raises(pf.PFError) as ei:
        pf.pf_resample_systematic(t, 1 << 31, 0, 0, a)
    assert ei.value.status == pf.PF_ERR_INVALID


@pytest.mark.parametrize("kind", list(CUMULATIVE))
@pytest.mark.parametrize("off", [1, 2, 3])
def test_unaligned_inputs(kind, off):
    # log-weights and ancestors that start 4, 8 or 12 bytes past a 16-byte boundary
    fn, orc = CUMULATIVE[kind]
    for P in (5, 4099, 300001):
        lw = workloads.gaussian_logw(P, 1.0, seed=P + off)
        buf = torch.zeros(P + 8, device="cuda")
        buf[off:off + P] = torch.from_numpy(lw).cuda()
        abuf = torch.full((P + 8,), -5, dtype=torch.int32, device="cuda")
        fn(buf.data_ptr() + 4 * off, P, 0, 3, abuf.data_ptr() + 4 * ((off + 1) % 4))
        assert pf.pf_get_device_status() == pf.PF_OK
        out = abuf.cpu().numpy()
        o = (off + 1) % 4
        a = out[o:o + P]
        assert np.all(out[:o] == -5) and np.all(out[o + P:] == -5)
        rep = check_cumulative(kind, lw, a, orc(lw, 3), 3)
        assert rep.ok, rep.summary()


def test_gather_with_host_resident_states():
    # page-locked host memory is device-accessible at the same address: the
    # gather reads the source rows and writes the result over the CPU-GPU link
    P, D = 70001, 16
    st = torch.from_numpy(workloads.states(P, D, seed=8)).pin_memory()
    out = torch.full((P, D), -1.0).pin_memory()
    assert pf.pf_is_device_accessible(st.data_ptr()) and pf.pf_is_device_accessible(out.data_ptr())
    assert pf.pf_is_device_accessible(torch.zeros(4, device="cuda").data_ptr())
    assert not pf.pf_is_device_accessible(np.zeros(1024, np.float32).ctypes.data)
    assert not pf.pf_is_device_accessible(None)
    lw = workloads.gaussian_logw(P, 1.0, seed=9)
    a, st_code = gpu_resample(pf.pf_resample_systematic, lw, 5)
    assert st_code == pf.PF_OK
    pf.pf_gather(st.data_ptr(), P, 4 * D, torch.from_numpy(a).cuda(), P, out.data_ptr())
    torch.cuda.synchronize()
    assert pf.pf_get_device_status() == pf.PF_OK
    np.testing.assert_array_equal(out.numpy(), st.numpy()[a])


@pytest.mark.parametrize("P", [1, 7, 4096, 4097, 100003, 1 << 20])
def test_permute_matches_oracle_and_inplace_gather(P):
    rng = np.random.default_rng(P)
    cases = [rng.integers(0, P, size=P).astype(np.int32),
             np.sort(rng.integers(0, P, size=P)).astype(np.int32),
             np.full(P, P // 2, np.int32), np.arange(P, dtype=np.int32)]
    lw = workloads.gaussian_logw(P, 2.0, seed=P)
    a, st = gpu_resample(pf.pf_resample_systematic, lw, 3)
    assert st == pf.PF_OK
    cases.append(a)
    for anc in cases:
        d_anc = torch.from_numpy(anc).cuda()
        perm = torch.full((P,), -9, dtype=torch.int32, device="cuda")
        pf.pf_permute(d_anc, P, perm)
        assert pf.pf_get_device_status() == pf.PF_OK
        np.testing.assert_array_equal(perm.cpu().numpy(), oracle.permute(anc))
    # in-place move of the states equals the out-of-place gather by the permuted ancestors
    D = 8
    x = torch.from_numpy(workloads.states(P, D, seed=1)).cuda()
    ref = x[perm.long()].clone()
    pf.pf_gather_inplace(x, P, 4 * D, perm)
    assert pf.pf_get_device_status() == pf.PF_OK
    assert torch.equal(x, ref)


def test_permute_and_inplace_gather_errors():
    P = 1000
    bad = torch.arange(P, dtype=torch.int32, device="cuda")
    bad[5] = P
    out = torch.empty(P, dtype=torch.int32, device="cuda")
    pf.pf_permute(bad, P, out)
    assert pf.pf_get_device_status() == pf.PF_ERR_INVALID
    with pytest.raises(pf.PFError):
        pf.pf_permute(bad, P, bad)  # overlapping
    # a vector not in the in-place form: entry 3 reads row 4, which is itself overwritten
    perm = torch.arange(P, dtype=torch.int32, device="cuda")
    perm[3], perm[4] = 4, 5
    x = torch.arange(P * 4, dtype=torch.float32, device="cuda").view(P, 4)
    x0 = x.clone()
    pf.pf_gather_inplace(x, P, 16, perm)
    assert pf.pf_get_device_status() == pf.PF_ERR_INVALID
    assert torch.equal(x[3], x0[3])  # left untouched
    assert torch.equal(x[4], x0[5])


def test_single_filter_calls_in_a_cuda_graph():
    # the single-launch kernels keep their barrier counters on the device
    # (alternating epochs), so a captured step replays without host resets
    P, D = 300007, 16
    lw = to_dev(workloads.gaussian_logw(P, 1.0, seed=12))
    src = torch.from_numpy(workloads.states(P, D, seed=13)).cuda()
    s = torch.cuda.Stream()
    pf.pf_reserve(P, 0, 0, s)
    anc = [torch.empty(P, dtype=torch.int32, device="cuda") for _ in range(4)]
    dst = torch.empty_like(src)
    ess = torch.zeros(1, device="cuda")

    def step():
        pf.pf_ess(lw, P, ess, None, s)
        pf.pf_resample_systematic(lw, P, 0, 21, anc[0], s)
        pf.pf_resample_stratified(lw, P, 0, 21, anc[1], s)
        pf.pf_resample_multinomial(lw, P, 0, 21, anc[2], s)
        pf.pf_resample_metropolis(lw, P, 16, 21, anc[3], s)
        pf.pf_gather(src, P, 4 * D, anc[0], P, dst, s)

    with torch.cuda.stream(s):
        step()
    s.synchronize()
    assert pf.pf_get_device_status(s) == pf.PF_OK
    eager = [a.clone() for a in anc] + [dst.clone(), ess.clone()]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        step()
    for _ in range(3):
        for a in anc:
            a.fill_(-1)
        dst.zero_()
        with torch.cuda.stream(s):
            g.replay()
        s.synchronize()
        assert pf.pf_get_device_status(s) == pf.PF_OK
        for x, y in zip(anc + [dst, ess], eager):
            assert torch.equal(x, y)


def test_trailing_zero_mass_tiles_get_no_offsets():
    # The systematic uniform of seed 1472623 (filter 0) is 1 - 3 * 2^-24, the
    # largest that can shift an offset across the boundary at the total mass W;
    # every tile after the last positive weight has boundary W at both ends and
    # must receive no offset, whatever the rounding of B P / W.
    seed = 1472623
    assert oracle.stream_uniforms(seed, 0, oracle.TAG_SYS, 1)[0] > 1 - 2.0 ** -21
    rng = np.random.default_rng(12)
    for P, live in (((1 << 25) - 3, 20_000_000), (131069, 60000)):
        lw = np.full(P, -np.inf, np.float32)
        lw[:live] = rng.standard_normal(live).astype(np.float32)
        a, st = gpu_resample(pf.pf_resample_systematic, lw, seed)
        assert st == pf.PF_OK
        assert a.min() >= 0 and a.max() < live
        rep = check_cumulative("systematic", lw, a, oracle.systematic(lw, seed), seed)
        assert rep.ok, rep.summary()
        # the same filter through the batched call (filter 0, key = seed)
        if P <= 1 << 17:
            off = np.array([0, P], np.int64)
            d_off = torch.from_numpy(off).cuda()
            seeds = torch.tensor([seed], dtype=torch.int64, device="cuda")
            b = torch.full((P,), -7, dtype=torch.int32, device="cuda")
            pf.pf_resample_batched(pf.PF_SYSTEMATIC, to_dev(lw), d_off, 1, 0, seeds, b)
            assert pf.pf_get_device_status() == pf.PF_OK
            bb = b.cpu().numpy()
            assert bb.min() >= 0 and bb.max() < live
            assert check_cumulative("systematic", lw, bb, oracle.systematic(lw, seed), seed).ok
