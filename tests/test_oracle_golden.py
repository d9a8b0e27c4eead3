"""The oracle's effective sample size against the values Section 3 states for
the paper's Dirichlet weight sets (tests/golden/dirichlet_ess_section3.txt).

The paper gives them as approximations ("approximately .5P", "about .1P",
"about .01P"); the exact expectation for symmetric Dirichlet(alpha) weights is
alpha / (1 + alpha) (0.5, 0.0909, 0.0099), so the mean over eight weight sets
of 2^16 particles must lie within 12% of the stated value, and within 5% of the
exact expectation."""
import os

import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "dirichlet_ess_section3.txt")


def _rows():
    rows = []
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                a, r = line.split()
                rows.append((float(a), float(r)))
    return rows


@pytest.mark.parametrize("alpha,stated", _rows())
def test_dirichlet_ess_fraction_matches_section3(alpha, stated):
    P = 1 << 16
    frac = np.mean([oracle.ess(workloads.dirichlet_logw(P, alpha, seed=s))[0] / P for s in range(8)])
    assert abs(frac - stated) <= 0.12 * stated, (alpha, frac)
    assert abs(frac - alpha / (1 + alpha)) <= 0.05 * alpha / (1 + alpha), (alpha, frac)
