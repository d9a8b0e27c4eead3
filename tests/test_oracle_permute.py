"""Pins of the oracle's in-place ancestor form (Section 2: offspring and
ancestors are interchangeable).  A hand-worked example, the defining
invariants on random and resampler-made ancestor vectors, and every ancestor
vector of P = 4 by brute force."""
import itertools

import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import workloads


def test_worked_example():
    # o = (3, 0, 1, 2, 0, 0): particles 0, 2, 3 keep their slots; the extra
    # copies 0, 0, 3 fill the empty slots 1, 4, 5 in order
    assert oracle.permute([0, 0, 0, 2, 3, 3]).tolist() == [0, 0, 2, 3, 0, 3]
    assert oracle.permute([5, 5, 5, 5, 5, 5]).tolist() == [5, 5, 5, 5, 5, 5]
    assert oracle.permute([1, 0, 3, 2]).tolist() == [0, 1, 2, 3]


def check_invariants(anc):
    out = oracle.permute(anc)
    P = len(anc)
    o = np.bincount(anc, minlength=P)
    assert np.array_equal(np.bincount(out, minlength=P), o)  # same offspring counts
    surv = np.nonzero(o > 0)[0]
    assert np.array_equal(out[surv], surv)  # survivors keep their slots
    assert np.array_equal(out[out], out)  # sources are fixed points: movable in place
    dead = np.nonzero(o == 0)[0]
    extras = np.repeat(np.arange(P), np.maximum(o - 1, 0))
    assert np.array_equal(out[dead], extras)  # extras fill the empty slots in order
    return out


@pytest.mark.parametrize("seed", range(5))
def test_invariants_random_and_resampled(seed):
    rng = np.random.default_rng(seed)
    for P in (1, 2, 7, 100, 5000):
        check_invariants(rng.integers(0, P, size=P).astype(np.int32))
        check_invariants(np.sort(rng.integers(0, P, size=P)).astype(np.int32))
    lw = workloads.gaussian_logw(3000, 2.0, seed=seed)
    for fn in (oracle.systematic, oracle.multinomial):
        check_invariants(fn(lw, seed))


def test_all_ancestor_vectors_of_four():
    rows = np.arange(4) * 10.0
    for anc in itertools.product(range(4), repeat=4):
        anc = np.array(anc, np.int32)
        out = check_invariants(anc)
        # moving rows in place by `out` gives the same multiset as the gather by anc
        x = rows.copy()
        for j in range(4):
            if out[j] != j:
                x[j] = x[out[j]]
        assert sorted(x) == sorted(rows[anc])


def test_invalid_ancestor():
    with pytest.raises(oracle.OracleError):
        oracle.permute([0, 4, 1, 1])
