"""GPU parity on the paper's own weight law (Section 3, Experiments): symmetric
Dirichlet(alpha) weights, alpha in {10, 1, .1, .01}, P in {2^8, 2^12, 2^16}.
Small alpha spreads the log-weights over hundreds to thousands (log U / alpha),
the regime where most weights underflow relative to the largest and the
zero-weight handling decides.  Every resampler, single call and batched, is
compared element by element with the FP64 oracle under the near-tie rule."""
import numpy as np
import pytest

import oracle
from paper_1202_6163_gb300 import pf, workloads
from parity import check_cumulative, check_metropolis

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ALPHAS = (10.0, 1.0, 0.1, 0.01)
SIZES = (1 << 8, 1 << 12, 1 << 16)
CUMULATIVE = {"systematic": (pf.PF_SYSTEMATIC, pf.pf_resample_systematic, oracle.systematic),
              "stratified": (pf.PF_STRATIFIED, pf.pf_resample_stratified, oracle.stratified),
              "multinomial": (pf.PF_MULTINOMIAL, pf.pf_resample_multinomial, oracle.multinomial)}


def weight_sets():
    return [(a, P, workloads.dirichlet_logw(P, a, seed=17 * ai + P)) for ai, a in enumerate(ALPHAS) for P in SIZES]


def metropolis_steps(lw):
    w = np.exp(lw.astype(np.float64) - lw.max())
    return min(pf.pf_metropolis_B(lw.size, w.max() / w.sum(), 0.01), 200)


@pytest.mark.parametrize("name", list(CUMULATIVE))
@pytest.mark.parametrize("alpha", ALPHAS)
def test_dirichlet_single_calls(name, alpha):
    kind, fn, orc = CUMULATIVE[name]
    for a, P, lw in weight_sets():
        if a != alpha:
            continue
        d = torch.from_numpy(lw).cuda()
        anc = torch.full((P,), -3, dtype=torch.int32, device="cuda")
        seed = 11 + P
        fn(d, P, 0, seed, anc)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative(name, lw, anc.cpu().numpy(), orc(lw, seed), seed)
        assert rep.ok, (alpha, P, rep.summary(), rep.failures[:3])


@pytest.mark.parametrize("alpha", ALPHAS)
def test_dirichlet_metropolis(alpha):
    for a, P, lw in weight_sets():
        if a != alpha:
            continue
        B = metropolis_steps(lw)
        d = torch.from_numpy(lw).cuda()
        anc = torch.full((P,), -3, dtype=torch.int32, device="cuda")
        pf.pf_resample_metropolis(d, P, B, 5, anc)
        assert pf.pf_get_device_status() == pf.PF_OK
        idx = np.unique(np.random.default_rng(P).integers(0, P, size=min(P, 3000)))
        rep = check_metropolis(lw, B, anc.cpu().numpy()[idx], oracle.metropolis(lw, B, 5, chains=idx), 5, chains=idx)
        assert rep.ok, (alpha, P, B, rep.summary())


@pytest.mark.parametrize("kind", [pf.PF_SYSTEMATIC, pf.PF_STRATIFIED, pf.PF_MULTINOMIAL, pf.PF_METROPOLIS])
def test_dirichlet_batched(kind):
    # the twelve weight sets as twelve filters of one batched call (filter id f, key seeds[f])
    sets = weight_sets()
    sizes = [P for _, P, _ in sets]
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lw = np.concatenate([l for _, _, l in sets]).astype(np.float32)
    seeds = np.arange(100, 100 + len(sets), dtype=np.uint64)
    B = 64 if kind == pf.PF_METROPOLIS else 0
    anc = torch.full((lw.size,), -3, dtype=torch.int32, device="cuda")
    pf.pf_resample_batched(kind, torch.from_numpy(lw).cuda(), torch.from_numpy(off).cuda(), len(sets), B,
                           torch.from_numpy(seeds.view(np.int64)).cuda(), anc)
    assert pf.pf_get_device_status() == pf.PF_OK
    a = anc.cpu().numpy()
    names = {pf.PF_SYSTEMATIC: "systematic", pf.PF_STRATIFIED: "stratified", pf.PF_MULTINOMIAL: "multinomial"}
    for f, (alpha, P, l) in enumerate(sets):
        lo, hi = off[f], off[f + 1]
        sd = int(seeds[f])
        if kind == pf.PF_METROPOLIS:
            rep = check_metropolis(l, B, a[lo:hi], oracle.metropolis(l, B, sd, f), sd, filter_id=f)
        else:
            name = names[kind]
            rep = check_cumulative(name, l, a[lo:hi], CUMULATIVE[name][2](l, sd, f), sd, filter_id=f)
        assert rep.ok, (alpha, P, rep.summary())
