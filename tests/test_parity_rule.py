"""The near-tie rule itself: it excuses only disagreements at thresholds the
uniform lies within 1e-6 (relative) of, and nothing else."""
import numpy as np

import oracle
from parity import check_cumulative, check_metropolis


def test_exact_match_passes():
    lw = np.random.default_rng(0).standard_normal(500).astype(np.float32)
    a = oracle.systematic(lw, 3)
    rep = check_cumulative("systematic", lw, a, a, seed=3)
    assert rep.ok and rep.mismatches == 0


def test_shifted_pick_far_from_threshold_fails():
    lw = np.random.default_rng(1).standard_normal(500).astype(np.float32)
    a = oracle.multinomial(lw, 4)
    bad = a.copy()
    bad[10] = (bad[10] + 1) % 500
    rep = check_cumulative("multinomial", lw, bad, a, seed=4)
    assert not rep.ok and rep.mismatches == 1


def test_near_tie_is_excused_and_listed():
    P = 64
    lw = np.random.default_rng(2).standard_normal(P).astype(np.float32)
    theta = oracle.normalised_cumsum(lw)
    # a uniform just below threshold theta_20: the oracle picks 20, a pick of 21 is a near tie
    x = np.full(P, 0.5)
    x[7] = theta[20] * (1 - 3e-7)
    a_orc = oracle.multinomial_u(lw, x)
    assert a_orc[7] == 20
    a_gpu = a_orc.copy()
    a_gpu[7] = 21
    rep = check_cumulative("multinomial", lw, a_gpu, a_orc, x=x)
    assert rep.ok and len(rep.excused) == 1 and rep.excused[0][0] == 7
    # the same disagreement with the uniform 1e-5 away is not excused
    x[7] = theta[20] * (1 - 1e-5)
    a_orc = oracle.multinomial_u(lw, x)
    rep = check_cumulative("multinomial", lw, a_gpu, a_orc, x=x)
    assert not rep.ok


def test_zero_weight_pick_never_excused():
    lw = np.zeros(8, np.float32)
    lw[3] = -np.inf
    theta = oracle.normalised_cumsum(lw)
    x = np.full(8, 0.9)
    x[0] = theta[2] * (1 + 1e-8)   # lands on particle 4 (3 has zero weight)
    a_orc = oracle.multinomial_u(lw, x)
    assert a_orc[0] == 4
    a_gpu = a_orc.copy()
    a_gpu[0] = 3
    assert not check_cumulative("multinomial", lw, a_gpu, a_orc, x=x).ok


def test_metropolis_wrong_chain_fails():
    lw = np.random.default_rng(3).standard_normal(100).astype(np.float32)
    a = oracle.metropolis(lw, 16, 9)
    bad = a.copy()
    bad[5] = (bad[5] + 1) % 100
    rep = check_metropolis(lw, 16, bad, a, 9)
    assert not rep.ok and rep.mismatches == 1
    assert check_metropolis(lw, 16, a, a, 9).ok
