"""Randomised parity sweep: many seeded random shapes against the oracle.

Each case draws a size, a log-weight law (Gaussian of a random spread, a
heavy tail, runs of zero weights, near-ties of equal values, one dominant
weight), a buffer offset of 0-3 floats for the log-weights and for the
ancestors, and a seed; every resampler runs on it through the C ABI and is
checked with the near-tie rule, and the guard words around the ancestors must
be untouched.  Batched cases draw random filter layouts (including empty and
one-particle filters) and a random mask.  The cases are fixed by the seed of
the sweep, so a failure reproduces."""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf
from parity import check_cumulative, check_metropolis

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CUM = {"systematic": (pf.pf_resample_systematic, oracle.systematic),
       "stratified": (pf.pf_resample_stratified, oracle.stratified),
       "multinomial": (pf.pf_resample_multinomial, oracle.multinomial)}
GUARD = -5


def random_logw(rng, P):
    law = rng.integers(0, 5)
    if law == 0:
        lw = rng.normal(0.0, rng.uniform(0.05, 6.0), P)
    elif law == 1:  # heavy tail: a few weights e^8 above the rest
        lw = rng.normal(0.0, 1.0, P)
        lw[rng.random(P) < 0.002] += 8.0
    elif law == 2:  # runs of zero weights
        lw = rng.normal(0.0, 1.0, P)
        z = rng.random(P) < rng.uniform(0.0, 0.9)
        lw[z] = -np.inf
        if not np.isfinite(lw).any():
            lw[rng.integers(0, P)] = 0.0
    elif law == 3:  # few distinct values: many exact ties
        lw = rng.choice(np.array([-1.0, 0.0, 0.5, 2.0]), P)
    else:  # one dominant weight
        lw = rng.normal(-30.0, 1.0, P)
        lw[rng.integers(0, P)] = 0.0
    return lw.astype(np.float32), int(law)


def run_single(fn, lw, seed, B, off_w, off_a):
    P = lw.size
    buf = torch.zeros(P + 8, device="cuda")
    buf[off_w:off_w + P] = torch.from_numpy(lw).cuda()
    abuf = torch.full((P + 8,), GUARD, dtype=torch.int32, device="cuda")
    fn(buf.data_ptr() + 4 * off_w, P, B, seed, abuf.data_ptr() + 4 * off_a)
    st = pf.pf_get_device_status()
    out = abuf.cpu().numpy()
    assert np.all(out[:off_a] == GUARD) and np.all(out[off_a + P:] == GUARD), "write outside the ancestors"
    return out[off_a:off_a + P], st


@pytest.mark.parametrize("block", range(4))
def test_single_calls_random_shapes(block):
    rng = np.random.default_rng(1000 + block)
    for case in range(60):
        P = int(np.exp(rng.uniform(0.0, np.log(400000))))
        lw, law = random_logw(rng, P)
        seed = int(rng.integers(0, 2**63 - 1))
        off_w, off_a = int(rng.integers(0, 4)), int(rng.integers(0, 4))
        for name, (fn, orc) in CUM.items():
            a, st = run_single(fn, lw, seed, 0, off_w, off_a)
            assert st == pf.PF_OK, (case, P, law, name, pf.pf_status_string(st))
            rep = check_cumulative(name, lw, a, orc(lw, seed), seed)
            assert rep.ok, (case, P, law, name, rep.summary(), rep.failures[:3])
            if name != "multinomial":
                assert np.all(np.diff(a) >= 0)
        B = int(rng.integers(0, 40))
        a, st = run_single(pf.pf_resample_metropolis, lw, seed, B, off_w, off_a)
        assert st == pf.PF_OK
        idx = np.unique(rng.integers(0, P, size=min(P, 3000)))
        rep = check_metropolis(lw, B, a[idx], oracle.metropolis(lw, B, seed, chains=idx), seed, chains=idx)
        assert rep.ok, (case, P, law, "metropolis", B, rep.summary())


@pytest.mark.parametrize("block", range(3))
def test_batched_random_layouts(block):
    rng = np.random.default_rng(2000 + block)
    for case in range(12):
        F = int(rng.integers(1, 150))
        sizes = np.where(rng.random(F) < 0.05, rng.integers(0, 2, F),
                         np.exp(rng.uniform(0.0, np.log(70000), F)).astype(np.int64))
        off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        lw = np.concatenate([random_logw(rng, int(n))[0] if n > 0 else np.zeros(0, np.float32) for n in sizes])
        seeds = rng.integers(0, 2**63 - 1, F).astype(np.uint64)
        mask = (rng.random(F) < 0.8).astype(np.int32)
        d_lw = torch.from_numpy(lw).cuda() if lw.size else torch.zeros(1, device="cuda")
        d_off = torch.from_numpy(off).cuda()
        d_seeds = torch.from_numpy(seeds.view(np.int64)).cuda()
        d_mask = torch.from_numpy(mask).cuda()
        for kind, orc in ((pf.PF_SYSTEMATIC, oracle.systematic), (pf.PF_STRATIFIED, oracle.stratified),
                          (pf.PF_MULTINOMIAL, oracle.multinomial), (pf.PF_METROPOLIS, None)):
            B = int(rng.integers(1, 30)) if kind == pf.PF_METROPOLIS else 0
            anc = torch.full((max(lw.size, 1),), GUARD, dtype=torch.int32, device="cuda")
            pf.pf_resample_batched_masked(kind, d_lw, d_off, F, B, d_seeds, d_mask, anc)
            assert pf.pf_get_device_status() == pf.PF_OK
            a = anc.cpu().numpy()
            for f in range(F):
                lo, hi = int(off[f]), int(off[f + 1])
                if hi == lo:
                    continue
                if not mask[f]:
                    assert np.all(a[lo:hi] == GUARD), "a masked filter was written"
                    continue
                l = lw[lo:hi]
                if kind == pf.PF_METROPOLIS:
                    rep = check_metropolis(l, B, a[lo:hi], oracle.metropolis(l, B, int(seeds[f]), f), int(seeds[f]),
                                           filter_id=f)
                else:
                    rep = check_cumulative({pf.PF_SYSTEMATIC: "systematic", pf.PF_STRATIFIED: "stratified",
                                            pf.PF_MULTINOMIAL: "multinomial"}[kind], l, a[lo:hi],
                                           orc(l, int(seeds[f]), f), int(seeds[f]), filter_id=f)
                assert rep.ok, (case, f, hi - lo, kind, rep.summary())
