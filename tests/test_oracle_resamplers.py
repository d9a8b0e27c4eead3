"""Pins for the oracle's resamplers, ESS, gather and the Metropolis B bound.

Nothing here compares the oracle with itself: each check is a property the
paper or the mathematics fixes (identity under equal weights, exact offspring
expectations, exact laws at tiny P by enumeration or chi-square, closed forms
of Eqs. 1-5, brute-force reformulations via library search routines), chosen so
that a dropped term, a wrong index or a transposed operand fails one of them.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1202_6163_gb300 import workloads


def _w(lw):
    lw = np.asarray(lw, dtype=np.float64)
    return np.exp(lw - lw.max())


def _lw(*vals):
    return np.array(vals, dtype=np.float32)


# ---------------------------------------------------------------- systematic
@pytest.mark.parametrize("P", [1, 2, 7, 64, 1000])
def test_systematic_equal_weights_identity(P):
    for seed in range(5):
        assert np.array_equal(oracle.systematic(np.full(P, 0.3, np.float32), seed), np.arange(P))


def test_systematic_one_hot_and_zero_weights():
    lw = np.full(50, -np.inf, np.float32)
    lw[17] = 2.0
    assert np.all(oracle.systematic(lw, 3) == 17)
    lw[40] = 2.0
    a = oracle.systematic(lw, 3)
    assert set(a.tolist()) == {17, 40} and np.sum(a == 17) == 25


def test_systematic_offspring_bounds_and_order():
    for seed in range(20):
        lw = workloads.gaussian_logw(500, s=1.5, seed=seed)
        a = oracle.systematic(lw, seed)
        assert np.all(np.diff(a) >= 0)
        o = oracle.offspring(a, lw.size)
        assert o.sum() == lw.size
        w = _w(lw)
        e = lw.size * w / w.sum()
        assert np.all((o == np.floor(e)) | (o == np.ceil(e)))


def _systematic_pieces(lw):
    """Breakpoints of the systematic ancestor vector as a function of u (from a
    numpy cumulative sum) and the midpoints of the pieces."""
    w = _w(lw)
    c = np.cumsum(w)
    W = c[-1]
    P = len(lw)
    bps = set([0.0, 1.0])
    for i in range(P):
        for j in range(P):
            x = P * c[i] / W - j
            if 0.0 < x < 1.0:
                bps.add(float(x))
    bps = np.array(sorted(bps))
    return bps, 0.5 * (bps[1:] + bps[:-1]), c, W


@pytest.mark.parametrize("seed", range(6))
def test_systematic_exact_expectation_and_bruteforce(seed):
    # E_u[o_i] = P w_i / W exactly (unbiasedness), integrating the piecewise-constant output
    rng = np.random.default_rng(seed)
    P = int(rng.integers(2, 6))
    lw = (2 * rng.standard_normal(P)).astype(np.float32)
    bps, mids, c, W = _systematic_pieces(lw)
    eo = np.zeros(P)
    for lo, hi, u in zip(bps[:-1], bps[1:], mids):
        a = oracle.systematic_u(lw, u)
        # brute force: a_j = #{i : c_i <= (j+u) W / P}
        t = (np.arange(P) + u) * W / P
        assert np.array_equal(a, np.searchsorted(c, t, side="right"))
        eo += (hi - lo) * np.bincount(a, minlength=P)
    np.testing.assert_allclose(eo, P * _w(lw) / _w(lw).sum(), rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------- stratified
@pytest.mark.parametrize("P", [1, 3, 64, 999])
def test_stratified_equal_weights_identity(P):
    for seed in range(5):
        assert np.array_equal(oracle.stratified(np.zeros(P, np.float32), seed), np.arange(P))


def test_stratified_position_law():
    # P(a_j = i) = |[j, j+1) ∩ [P c_{i-1}/W, P c_i/W)| for each stratum j
    lw = _lw(0.0, 1.2, -0.7, 0.4, -2.0)
    P = lw.size
    w = _w(lw)
    c = np.concatenate([[0.0], np.cumsum(w)]) * P / w.sum()
    grid = (np.arange(4000) + 0.5) / 4000
    for j in range(P):
        counts = np.zeros(P)
        for u in grid:
            uu = np.full(P, 0.5)
            uu[j] = u
            counts[oracle.stratified_u(lw, uu)[j]] += 1
        law = np.array([max(0.0, min(j + 1, c[i + 1]) - max(j, c[i])) for i in range(P)])
        np.testing.assert_allclose(counts / grid.size, law, atol=2.0 / grid.size)


def test_stratified_offspring_bounds_and_unbiased():
    lw = workloads.gaussian_logw(300, s=1.0, seed=4)
    w = _w(lw)
    e = lw.size * w / w.sum()
    total = np.zeros(lw.size)
    n = 400
    for seed in range(n):
        a = oracle.stratified(lw, seed)
        assert np.all(np.diff(a) >= 0)
        o = oracle.offspring(a, lw.size)
        assert o.sum() == lw.size
        assert np.all(o >= np.floor(e) - 1) and np.all(o <= np.ceil(e) + 1)
        total += o
    # mean offspring -> P w / W; stratified variance per particle is at most 1/4 per stratum touched
    z = (total / n - e) / np.sqrt(np.maximum(e, 1e-3) / n)
    assert np.max(np.abs(z)) < 6


# ---------------------------------------------------------------- multinomial
def test_multinomial_exact_law_chisquare():
    lw = _lw(0.0, -0.9, 0.6)
    p = _w(lw) / _w(lw).sum()
    n = 30000
    outcomes = {}
    for seed in range(n):
        a = tuple(oracle.multinomial(lw, seed).tolist())
        outcomes[a] = outcomes.get(a, 0) + 1
    keys = list(itertools.product(range(3), repeat=3))
    obs = np.array([outcomes.get(k, 0) for k in keys])
    exp = np.array([n * np.prod(p[list(k)]) for k in keys])
    assert obs.sum() == n
    assert stats.chisquare(obs, exp).pvalue > 1e-4


def test_multinomial_bruteforce_search():
    rng = np.random.default_rng(7)
    lw = rng.standard_normal(257).astype(np.float32)
    lw[[3, 100, 256]] = -np.inf
    u = rng.random(257)
    a = oracle.multinomial_u(lw, u)
    c = np.cumsum(_w(lw))
    assert np.array_equal(a, np.searchsorted(c, u * c[-1], side="right"))
    assert not np.isin(a, [3, 100, 256]).any()


def test_multinomial_pooled_offspring():
    lw = workloads.gaussian_logw(16, s=1.0, seed=2)
    p = _w(lw) / _w(lw).sum()
    counts = np.zeros(16)
    for seed in range(3000):
        counts += oracle.offspring(oracle.multinomial(lw, seed), 16)
    assert stats.chisquare(counts, counts.sum() * p).pvalue > 1e-4


def test_multinomial_one_hot():
    lw = np.full(33, -np.inf, np.float32)
    lw[5] = -3.0
    assert np.all(oracle.multinomial(lw, 1) == 5)


# ---------------------------------------------------------------- Metropolis
def test_metropolis_zero_steps_identity():
    lw = workloads.gaussian_logw(100, seed=1)
    assert np.array_equal(oracle.metropolis(lw, 0, 5), np.arange(100))


def test_metropolis_equal_weights_takes_last_proposal():
    P, B = 50, 7
    a = oracle.metropolis(np.zeros(P, np.float32), B, 9)
    for i in range(P):
        prop, _ = oracle.metropolis_draws(9, 0, P, i, B)
        assert a[i] == prop[-1]


def test_metropolis_matrix_is_reversible_for_w():
    # a Metropolis chain with uniform proposals targets w/W: rows sum to one,
    # detailed balance pi_k M_kj = pi_j M_jk, and a heavier proposal is always taken
    lw = _lw(0.3, -1.0, 2.0, 0.0, -0.5)
    M = oracle.metropolis_matrix(lw)
    P = lw.size
    pi = _w(lw) / _w(lw).sum()
    np.testing.assert_allclose(M.sum(1), 1.0, atol=1e-14)
    np.testing.assert_allclose(pi[:, None] * M, (pi[:, None] * M).T, atol=1e-15)
    np.testing.assert_allclose(pi @ M, pi, atol=1e-14)
    for k in range(P):
        for j in range(P):
            if j != k and lw[j] >= lw[k]:
                assert M[k, j] == 1.0 / P


@pytest.mark.parametrize("B", [1, 3])
def test_metropolis_law_matches_matrix_power(B):
    lw = _lw(0.0, 1.0, -1.0, 0.5)
    P = lw.size
    MB = np.linalg.matrix_power(oracle.metropolis_matrix(lw), B)
    n = 20000
    counts = np.zeros((P, P))
    for seed in range(n):
        a = oracle.metropolis(lw, B, seed)
        counts[np.arange(P), a] += 1
    for i in range(P):
        exp = n * MB[i]
        keep = exp > 0
        assert counts[i][~keep].sum() == 0
        assert stats.chisquare(counts[i][keep], exp[keep]).pvalue > 1e-4


def _lumped(P, w_max, l):
    """Eq. 3 in the invariant labelling: beta = 1/P (into the heaviest particle),
    alpha = (1 - w_max)/(P w_max) (out of it), lambda = 1 - alpha - beta.
    Returns (P(on | started on), P(on | started off)) after l steps."""
    beta = 1.0 / P
    alpha = (1.0 - w_max) / (P * w_max)
    lam = 1.0 - alpha - beta
    stay = (beta + lam ** l * alpha) / (alpha + beta)
    enter = beta * (1.0 - lam ** l) / (alpha + beta)
    return stay, enter


@pytest.mark.parametrize("lw", [[0.0, 1.0, -1.0, 0.5, 2.5], [3.0, 0.0, 0.0, 0.0], [0.1, 0.2, 0.3]])
def test_eq3_closed_form_matches_exact_chain(lw):
    # the 0-1 process "chain is on p_max" is exactly Markov (from any other state
    # p_max is proposed w.p. 1/P and always accepted), so Eq. 3 must equal M^l
    lw = np.array(lw, np.float32)
    P = lw.size
    pmax = int(np.argmax(lw))
    w_max = _w(lw).max() / _w(lw).sum()
    M = oracle.metropolis_matrix(lw)
    for l in range(0, 12):
        Ml = np.linalg.matrix_power(M, l)
        stay, enter = _lumped(P, w_max, l)
        assert Ml[pmax, pmax] == pytest.approx(stay, abs=1e-13)
        for k in range(P):
            if k != pmax:
                assert Ml[k, pmax] == pytest.approx(enter, abs=1e-13)


@pytest.mark.parametrize("lw,eps", [([0.0, 1.0, -1.0, 0.5, 2.5, 0.0, -0.3, 1.1], 0.01),
                                    ([4.0, 0.0, 0.0, 0.0, 0.0, 0.0], 0.001),
                                    ([0.2, 0.1, 0.0, -0.1], 0.05)])
def test_B_bound_is_tight_on_exact_chain(lw, eps):
    # Eq. 5: at B every start is within eps of w_max on p_max; at B-1 some start is not
    lw = np.array(lw, np.float32)
    P = lw.size
    pmax = int(np.argmax(lw))
    w_max = _w(lw).max() / _w(lw).sum()
    B = oracle.metropolis_B(P, w_max, eps)
    assert B >= 1
    M = oracle.metropolis_matrix(lw)
    dev = lambda l: np.max(np.abs(np.linalg.matrix_power(M, l)[:, pmax] - w_max))
    assert dev(B) <= eps * (1 + 1e-12)
    assert dev(B - 1) > eps


def test_B_bound_large_P_values():
    # Eq. 5 with the paper's quantities at sizes the tests cannot enumerate:
    # a heavier p_max (larger P w_max) or a smaller eps needs more steps,
    # and lambda^B <= target < lambda^(B-1)
    for P, wm, eps in [(1024, 0.01, 0.01), (1 << 20, 1e-4, 0.01), (65536, 0.3, 1e-3)]:
        B = oracle.metropolis_B(P, wm, eps)
        lam = 1 - 1 / (P * wm)
        target = eps / max(wm, 1 - wm)
        assert lam ** B <= target * (1 + 1e-12) and lam ** (B - 1) > target
        assert oracle.metropolis_B(P, min(2 * wm, 0.5), eps) > B
        assert oracle.metropolis_B(P, wm, eps / 10) > B
    assert oracle.metropolis_B(8, 1.0 / 8, 0.01) == 1    # equal weights: one step mixes exactly
    assert oracle.metropolis_B(8, 0.5, 0.0) == -1


# ---------------------------------------------------------------- ESS, gather, errors
def test_ess_closed_forms():
    P = 1000
    e, ls = oracle.ess(np.full(P, 1.5, np.float32))
    assert e == pytest.approx(P, rel=1e-12)
    assert ls == pytest.approx(1.5 + math.log(P), rel=1e-12)
    lw = np.full(P, -np.inf, np.float32)
    lw[10] = 4.0
    assert oracle.ess(lw)[0] == pytest.approx(1.0, rel=1e-15)
    r = float(np.exp(np.float64(np.float32(-1.25))))
    lw = np.zeros(P, np.float32)
    lw[P // 2:] = -1.25
    assert oracle.ess(lw)[0] == pytest.approx(P * (1 + r) ** 2 / (2 * (1 + r * r)), rel=1e-12)


def test_ess_lognormal_expectation():
    # Gaussian log-weights N(0, s^2): ESS/P -> exp(-s^2)
    for s in (0.25, 0.5, 1.0):
        lw = workloads.gaussian_logw(1 << 20, s=s, seed=3)
        assert oracle.ess(lw)[0] / lw.size == pytest.approx(math.exp(-s * s), rel=0.02)


def test_gather_rows():
    src = workloads.states(100, 7, seed=2)
    anc = np.random.default_rng(0).integers(0, 100, size=130).astype(np.int32)
    assert np.array_equal(oracle.gather(src, anc), src[anc])
    with pytest.raises(oracle.OracleError):
        oracle.gather(src, np.array([100], np.int32))


def test_domain_errors():
    lw = np.zeros(10, np.float32)
    for bad in (np.nan, np.inf):
        x = lw.copy()
        x[4] = bad
        for fn in (oracle.systematic, oracle.stratified, oracle.multinomial):
            with pytest.raises(oracle.OracleError):
                fn(x, 0)
        with pytest.raises(oracle.OracleError):
            oracle.metropolis(x, 4, 0)
        with pytest.raises(oracle.OracleError):
            oracle.ess(x)
    allneg = np.full(10, -np.inf, np.float32)
    for fn in (oracle.systematic, oracle.stratified, oracle.multinomial):
        with pytest.raises(oracle.OracleError):
            fn(allneg, 0)
    # Metropolis has no collective step: zero weights everywhere just move to the proposals
    assert np.array_equal(oracle.metropolis(allneg, 1, 0),
                          [oracle.metropolis_draws(0, 0, 10, i, 1)[0][0] for i in range(10)])


# ---------------------------------------------------------------- Figure 2 protocol
def test_error_metric_ordering():
    # mean of sum_i (o_i/P - w_i/W)^2 over resamplings (Figure 2, top row):
    # multinomial has the exact expectation (1 - sum p^2)/P; stratified and
    # systematic are lower (Section 3); Metropolis approaches multinomial as B grows.
    P, n = 256, 600
    lw = workloads.gaussian_logw(P, s=1.0, seed=11)
    p = _w(lw) / _w(lw).sum()

    def err(fn):
        return np.mean([np.sum((oracle.offspring(fn(s), P) / P - p) ** 2) for s in range(n)])

    e_multi = err(lambda s: oracle.multinomial(lw, s))
    e_strat = err(lambda s: oracle.stratified(lw, s))
    e_sys = err(lambda s: oracle.systematic(lw, s))
    e_met = err(lambda s: oracle.metropolis(lw, 200, s))
    e_met_1 = err(lambda s: oracle.metropolis(lw, 1, s))
    e_met_4 = err(lambda s: oracle.metropolis(lw, 4, s))
    assert e_multi == pytest.approx((1 - np.sum(p * p)) / P, rel=0.1)
    assert e_sys < e_strat < e_multi
    assert e_met == pytest.approx(e_multi, rel=0.15)
    # too few steps leaves the sample biased towards the starting particles
    assert e_met_1 > e_met_4 > e_met and e_met_1 > 1.3 * e_multi


# ---------------------------------------------------------------- batched loop
def test_orc_batched_is_the_per_filter_calls_with_their_filter_ids():
    """The batched oracle resamples filter f on its own slice with key seeds[f] and
    filter id f: each slice equals the single-filter call with that id, its ancestors
    are filter-local, a filter of equal weights keeps the systematic identity, the
    systematic offspring of every filter stay within floor/ceil of P_f w_i / W_f, and
    two filters with the same weights and seed but different ids draw different
    streams.  Empty filters are skipped."""
    rng = np.random.default_rng(7)
    sizes = [5, 0, 300, 1, 64, 64, 1000]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = rng.standard_normal(int(off[-1])).astype(np.float32)
    lw[off[3]:off[4]] = 0.5                          # a one-particle filter
    lw[off[6]:off[7]] = 1.25                         # equal weights
    lw[off[5]:off[6]] = lw[off[4]:off[5]]            # same weights as filter 4 ...
    seeds = np.array([3, 9, 11, 2, 5, 5, 8], dtype=np.uint64)  # ... and the same seed
    single = {0: oracle.multinomial, 1: oracle.stratified, 2: oracle.systematic}
    for kind in (0, 1, 2, 3):
        a = oracle.batched(kind, lw, off, 16, seeds)
        for f in range(len(sizes)):
            lo, hi = off[f], off[f + 1]
            if hi == lo:
                continue
            seg = lw[lo:hi]
            want = (oracle.metropolis(seg, 16, int(seeds[f]), f) if kind == 3
                    else single[kind](seg, int(seeds[f]), f))
            assert np.array_equal(a[lo:hi], want), (kind, f)
            assert a[lo:hi].min() >= 0 and a[lo:hi].max() < hi - lo
        if kind == 2:
            assert np.array_equal(a[off[6]:off[7]], np.arange(sizes[6]))
            for f in range(len(sizes)):
                lo, hi = off[f], off[f + 1]
                if hi == lo:
                    continue
                w = _w(lw[lo:hi])
                e = (hi - lo) * w / w.sum()
                o = np.bincount(a[lo:hi], minlength=hi - lo)
                assert np.all(o >= np.floor(e - 1e-9)) and np.all(o <= np.ceil(e + 1e-9)), f
        if kind in (0, 3):
            assert not np.array_equal(a[off[4]:off[5]], a[off[5]:off[6]])


# ----------------------------------------------- Metropolis on the seven-round stream
def test_seven_round_metropolis_identity_and_last_proposal():
    lw = workloads.gaussian_logw(100, seed=1)
    assert np.array_equal(oracle.metropolis(lw, 0, 5, rounds=7), np.arange(100))
    P, B = 50, 7
    a = oracle.metropolis(np.zeros(P, np.float32), B, 9, rounds=7)
    for i in range(P):
        prop, _ = oracle.metropolis_draws(9, 0, P, i, B, rounds=7)
        assert a[i] == prop[-1]
    assert not np.array_equal(a, oracle.metropolis(np.zeros(P, np.float32), B, 9))  # another stream


@pytest.mark.parametrize("B", [1, 3])
def test_seven_round_metropolis_law_matches_matrix_power(B):
    lw = _lw(0.0, 1.0, -1.0, 0.5)
    P = lw.size
    MB = np.linalg.matrix_power(oracle.metropolis_matrix(lw), B)
    n = 20000
    counts = np.zeros((P, P))
    for seed in range(n):
        a = oracle.metropolis(lw, B, seed, rounds=7)
        counts[np.arange(P), a] += 1
    for i in range(P):
        exp = n * MB[i]
        keep = exp > 0
        assert counts[i][~keep].sum() == 0
        assert stats.chisquare(counts[i][keep], exp[keep]).pvalue > 1e-4
