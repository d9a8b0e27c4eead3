"""Pins for the oracle's Philox-4x32-10 generator and its stream layout.

The generator itself is not in the paper (which used a Tausworthe generator,
Section 3); both sides of this project implement Philox-4x32-10 from Salmon et
al. (SC'11).  The oracle's copy is pinned to an independent implementation run
as a black box -- cuRAND's host-side Philox-4x32-10 generator, whose output
block i for a seed is the generator applied to counter (0, 0, i, 0) under the
key (seed low word, seed high word) -- and to the statistical properties every
later pin relies on.
"""
import ctypes
import ctypes.util

import numpy as np
import pytest
from scipy import stats

import oracle


def _curand():
    names = ["/usr/local/cuda/lib64/libcurand.so"]
    found = ctypes.util.find_library("curand")
    if found:
        names.append(found)
    for name in names:
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    return None


CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


@pytest.mark.parametrize("seed", [0, 1, 0x0123456789ABCDEF, 0xFFFFFFFFFFFFFFFF, 0xDEADBEEF00000000])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("cuRAND is not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 256
        out = np.zeros(4 * n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(4 * n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(n):
        assert list(oracle.philox4x32_10([0, 0, i, 0], key)) == [int(x) for x in out[4 * i:4 * i + 4]], (seed, i)


def test_philox_counter_words_all_matter():
    # every counter and key word changes every output word (a dropped or swapped
    # word in the rounds would leave some output unchanged)
    base_c, base_k = [5, 6, 7, 8], [9, 10]
    ref = oracle.philox4x32_10(base_c, base_k)
    for w in range(4):
        c = list(base_c)
        c[w] ^= 1
        assert all(a != b for a, b in zip(oracle.philox4x32_10(c, base_k), ref)), w
    for w in range(2):
        k = list(base_k)
        k[w] ^= 1
        assert all(a != b for a, b in zip(oracle.philox4x32_10(base_c, k), ref)), w


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


# ------------------------------------------------- Philox-4x32-7 (the opt-in Metropolis stream)
def test_round_generic_philox_is_the_pinned_generator_at_ten_rounds():
    # the round-generic function at 10 rounds is the generator pinned to cuRAND
    # above, so the seven-round stream is the same round function stopped earlier
    rng = np.random.default_rng(1)
    for _ in range(200):
        c = [int(x) for x in rng.integers(0, 1 << 32, 4, dtype=np.uint64)]
        k = [int(x) for x in rng.integers(0, 1 << 32, 2, dtype=np.uint64)]
        assert list(oracle.philox4x32(c, k, 10)) == list(oracle.philox4x32_10(c, k))
        assert list(oracle.philox4x32(c, k, 7)) != list(oracle.philox4x32_10(c, k))
        assert list(oracle.philox4x32(c, k, 0)) == c  # no round: the counter itself


def test_seven_rounds_every_word_matters_and_output_is_uniform():
    base_c, base_k = [5, 6, 7, 8], [9, 10]
    ref = oracle.philox4x32(base_c, base_k, 7)
    for w in range(4):
        c = list(base_c)
        c[w] ^= 1
        assert all(a != b for a, b in zip(oracle.philox4x32(c, base_k, 7), ref)), w
    for w in range(2):
        k = list(base_k)
        k[w] ^= 1
        assert all(a != b for a, b in zip(oracle.philox4x32(base_c, k, 7), ref)), w
    # consecutive counters: every output word uniform, and its bits balanced
    words = np.array([oracle.philox4x32([q, 0, 3, oracle.TAG_METRO], [77, 0], 7) for q in range(8192)],
                     dtype=np.uint64)
    for s in range(4):
        counts = np.bincount((words[:, s] >> np.uint64(26)).astype(np.int64), minlength=64)
        assert stats.chisquare(counts).pvalue > 1e-4, s
        bits = ((words[:, s][:, None] >> np.arange(32, dtype=np.uint64)) & np.uint64(1)).mean(0)
        assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / np.sqrt(words.shape[0])), s


def test_seven_round_metropolis_draw_layout():
    seed, f, P, i, B = 99, 3, 1000, 17, 5
    prop, unif = oracle.metropolis_draws(seed, f, P, i, B, rounds=7)
    key = [seed, 0]
    for b in range(B):
        r = oracle.philox4x32([i, b // 2, f, oracle.TAG_METRO], key, 7)
        x_j, x_u = (r[0], r[1]) if b % 2 == 0 else (r[2], r[3])
        assert prop[b] == (int(x_j) * P) >> 32
        assert unif[b] == oracle.u23(int(x_u))
