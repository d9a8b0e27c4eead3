"""Pins for the oracle's Philox-4x32-10 generator and its stream layout.

The generator itself is not in the paper (which used a Tausworthe generator,
Section 3); both sides of this project implement Philox-4x32-10 from Salmon et
al. (SC'11).  These tests pin the oracle's copy to the published known answers
and to the statistical properties every later pin relies on.
"""
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_known_answers(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_stream_layout_words():
    # element j of a stream is word j%4 of counter (j/4, 0, filter, tag), key = seed halves
    seed = 0x0123456789ABCDEF
    w = oracle.stream_words(seed, 7, oracle.TAG_STRAT, 10)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for q in range(3):
        block = oracle.philox4x32_10([q, 0, 7, oracle.TAG_STRAT], key)
        n = min(4, 10 - 4 * q)
        assert list(w[4 * q:4 * q + n]) == list(block[:n])


def test_metropolis_draw_layout():
    seed, f, P, i, B = 99, 3, 1000, 17, 5
    prop, unif = oracle.metropolis_draws(seed, f, P, i, B)
    key = [seed, 0]
    for b in range(B):
        r = oracle.philox4x32_10([i, b // 2, f, oracle.TAG_METRO], key)
        x_j, x_u = (r[0], r[1]) if b % 2 == 0 else (r[2], r[3])
        assert prop[b] == (int(x_j) * P) >> 32
        assert unif[b] == oracle.u23(int(x_u))


def test_uniform_conversions_edges():
    # u23 takes the odd multiples of 2^-24 strictly inside (0, 1); u32 those of 2^-33
    assert oracle.u23(0) == 2.0 ** -24
    assert oracle.u23(0xFFFFFFFF) == 1.0 - 2.0 ** -24
    assert oracle.u23(0x1FF) == 2.0 ** -24          # low 9 bits are dropped
    assert oracle.u23(0x200) == 3 * 2.0 ** -24
    assert np.float32(oracle.u23(0xFFFFFFFF)) == oracle.u23(0xFFFFFFFF)  # exact in float32
    assert oracle.u32(0) == 2.0 ** -33
    assert oracle.u32(0xFFFFFFFF) == 1.0 - 2.0 ** -33
    assert oracle.index(0xFFFFFFFF, 1000) == 999
    assert oracle.index(0, 1000) == 0
    assert oracle.index(1 << 31, 8) == 4


def test_uniformity_and_independence():
    n = 1 << 18
    u = oracle.stream_uniforms(5, 0, oracle.TAG_MULTI, n, kind=1)
    counts, _ = np.histogram(u, bins=64, range=(0, 1))
    assert stats.chisquare(counts).pvalue > 1e-4
    # successive pairs fill the unit square evenly (catches a repeated or shifted word)
    pairs = np.histogram2d(u[0::2], u[1::2], bins=16, range=[[0, 1], [0, 1]])[0].ravel()
    assert stats.chisquare(pairs).pvalue > 1e-4
    # different tags and filters give unrelated streams
    v = oracle.stream_uniforms(5, 0, oracle.TAG_STRAT, n, kind=1)
    g = oracle.stream_uniforms(5, 1, oracle.TAG_MULTI, n, kind=1)
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.01
    assert abs(np.corrcoef(u, g)[0, 1]) < 0.01


def test_index_draws_uniform():
    P = 37
    prop = np.concatenate([oracle.metropolis_draws(11, 0, P, i, 64)[0] for i in range(2000)])
    counts = np.bincount(prop, minlength=P)
    assert counts.size == P
    assert stats.chisquare(counts).pvalue > 1e-4
