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
    e = rep.excused[0]
    assert (e.gpu, e.orc, e.gap, e.between) == (21, 20, 1, 0)
    assert 2e-7 < e.rel < 4e-7 and rep.worst_rel == e.rel and rep.non_adjacent == 0
    # the same disagreement with the uniform 1e-5 away is not excused
    x[7] = theta[20] * (1 - 1e-5)
    a_orc = oracle.multinomial_u(lw, x)
    rep = check_cumulative("multinomial", lw, a_gpu, a_orc, x=x)
    assert not rep.ok


def test_skipped_particles_between_the_picks_are_counted():
    # particle 21 holds e^-30 of a unit weight: thresholds theta_20 and theta_21 both lie
    # within 1e-6 of the position, so a GPU pick of 22 against the oracle's 20 is a near
    # tie that skips one positive-weight particle (not adjacent), and the report says so
    P = 64
    lw = np.random.default_rng(2).standard_normal(P).astype(np.float32)
    lw[21] = -30.0
    theta = oracle.normalised_cumsum(lw)
    x = np.full(P, 0.5)
    x[7] = theta[20] * (1 - 3e-7)
    a_orc = oracle.multinomial_u(lw, x)
    assert a_orc[7] == 20
    a_gpu = a_orc.copy()
    a_gpu[7] = 22
    rep = check_cumulative("multinomial", lw, a_gpu, a_orc, x=x)
    assert rep.ok and rep.mismatches == 1
    e = rep.excused[0]
    assert (e.gap, e.between) == (2, 1) and rep.worst_gap == 2 and rep.worst_between == 1
    assert rep.non_adjacent == 1
    # a zero-weight particle in between is not counted
    lw[21] = -np.inf
    theta = oracle.normalised_cumsum(lw)
    x[7] = theta[20] * (1 - 3e-7)
    a_orc = oracle.multinomial_u(lw, x)
    rep = check_cumulative("multinomial", lw, a_gpu, a_orc, x=x)
    assert rep.ok and rep.excused[0].between == 0 and rep.non_adjacent == 0


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


def test_metropolis_declined_move_to_a_barely_heavier_particle_is_a_near_tie():
    # chain 0 proposes particle 1, whose log-weight is two float ulps above its own:
    # r = exp(lw_1 - lw_0) = 1 + 2.4e-7 and u = 1 - 2^-24 lies within 1e-6 r of r, so a
    # GPU that rounds the ratio below u and stays at 0 is excused; 1e-5 above is not
    base = np.float32(1.0)
    for step, ok in ((2, True), (84, False)):
        lw = np.array([base, np.nextafter(base, np.float32(2), dtype=np.float32), 0.0, 0.0], np.float32)
        for _ in range(step - 1):
            lw[1] = np.nextafter(lw[1], np.float32(2), dtype=np.float32)
        prop = np.array([[1], [1], [2], [3]], np.int32)
        unif = np.full((4, 1), 1.0 - 2.0 ** -24)
        a_orc = oracle.metropolis_u(lw, 1, prop, unif)
        assert a_orc[0] == 1
        a_gpu = a_orc.copy()
        a_gpu[0] = 0
        rep = check_metropolis(lw, 1, a_gpu, a_orc, 0, draws=(prop, unif))
        assert rep.ok == ok and rep.mismatches == 1
        if ok:  # the excused chain names the step the replay flipped
            assert (rep.excused[0].chain, rep.excused[0].first_step, rep.excused[0].flips) == (0, 0, 1)
