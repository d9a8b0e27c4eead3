"""The tile-size autotuner of the single-launch resamplers, and the bias bound
on the Metropolis step count B (Section 2, Eqs. 1-5) checked on the GPU's own
chains against the exact transition matrix."""
import numpy as np
import pytest
from scipy import stats

import oracle
from paper_1202_6163_gb300 import pf, tuning, workloads
from parity import check_cumulative

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

KINDS = {"multinomial": (pf.PF_MULTINOMIAL, pf.pf_resample_multinomial, oracle.multinomial),
         "stratified": (pf.PF_STRATIFIED, pf.pf_resample_stratified, oracle.stratified),
         "systematic": (pf.PF_SYSTEMATIC, pf.pf_resample_systematic, oracle.systematic)}
CANDIDATES = {1024, 1536, 2048, 3072, 4096, 6144, 8192}


@pytest.mark.parametrize("name", list(KINDS))
@pytest.mark.parametrize("P", [5000, 1 << 20])
def test_autotune_then_parity(name, P):
    kind, fn, orc = KINDS[name]
    lw = workloads.gaussian_logw(P, 1.0, seed=P + kind)
    d = torch.from_numpy(lw).cuda()
    a = torch.empty(P, dtype=torch.int32, device="cuda")
    try:
        tile, us = pf.pf_autotune(kind, d, P, a, reps=5)
        assert tile in CANDIDATES and us > 0
        assert pf.pf_get_min_tile(kind, P) == tile
        print(f"\n{name} P={P}: min_tile {tile}, {us:.1f} us")
        fn(d, P, 0, 31, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative(name, lw, a.cpu().numpy(), orc(lw, 31), 31)
        assert rep.ok, rep.summary()
    finally:
        pf.pf_set_min_tile(kind, P, 0)


def test_min_tile_table():
    P = 300000
    assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, P) == 2048
    pf.pf_set_min_tile(pf.PF_SYSTEMATIC, P, 6144)
    try:
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, P) == 6144
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, P + 1000) == 6144  # same size class
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, 2 * P) == 2048
        assert pf.pf_get_min_tile(pf.PF_STRATIFIED, P) == 2048
        lw = workloads.gaussian_logw(P, 2.0, seed=9)
        d = torch.from_numpy(lw).cuda()
        a = torch.empty(P, dtype=torch.int32, device="cuda")
        pf.pf_resample_systematic(d, P, 0, 4, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative("systematic", lw, a.cpu().numpy(), oracle.systematic(lw, 4), 4)
        assert rep.ok, rep.summary()
    finally:
        pf.pf_set_min_tile(pf.PF_SYSTEMATIC, P, 0)
    assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, P) == 2048
    for bad in [(7, P, 0), (pf.PF_METROPOLIS, P, 0), (pf.PF_SYSTEMATIC, 0, 0), (pf.PF_SYSTEMATIC, P, 9000),
                (pf.PF_SYSTEMATIC, P, -1)]:
        with pytest.raises(pf.PFError):
            pf.pf_set_min_tile(*bad)
    with pytest.raises(pf.PFError):
        pf.pf_autotune(pf.PF_METROPOLIS, torch.zeros(16, device="cuda"), 16,
                       torch.zeros(16, dtype=torch.int32, device="cuda"))


def test_tuned_tiles_saved_and_loaded_in_a_later_call(tmp_path):
    # a pick stored in the JSON file is set again by tuning.load, at the library's
    # own size classes (pf_get_min_tile reads the table the calls use)
    path = str(tmp_path / "tiles.json")
    P = 300000
    lw = workloads.gaussian_logw(P, 1.0, seed=77)
    d = torch.from_numpy(lw).cuda()
    a = torch.empty(P, dtype=torch.int32, device="cuda")
    try:
        tile, us = tuning.tune_and_record(path, pf.PF_SYSTEMATIC, d, P, a, reps=5)
        assert tile in CANDIDATES and us > 0
        tuning.record(path, tuning.device_key(), pf.PF_MULTINOMIAL, 5000, 6144)
        for kind, Pk in ((pf.PF_SYSTEMATIC, P), (pf.PF_MULTINOMIAL, 5000)):
            pf.pf_set_min_tile(kind, Pk, 0)  # as in a fresh process
        assert pf.pf_get_min_tile(pf.PF_MULTINOMIAL, 5000) == 2048
        assert tuning.load(path) == 2
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, P) == tile
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, 1 << 19) == tile  # the top of P's class
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, (1 << 18) + 1) == tile  # its bottom
        assert pf.pf_get_min_tile(pf.PF_SYSTEMATIC, (1 << 19) + 1) == 2048
        assert pf.pf_get_min_tile(pf.PF_MULTINOMIAL, 4097) == 6144
        assert pf.pf_get_min_tile(pf.PF_MULTINOMIAL, 4096) == 2048
        assert tuning.load(path, key="another GPU|1 SMs|sm_00") == 0
        pf.pf_resample_multinomial(d[:5000], 5000, 0, 8, a)
        assert pf.pf_get_device_status() == pf.PF_OK
        rep = check_cumulative("multinomial", lw[:5000], a[:5000].cpu().numpy(), oracle.multinomial(lw[:5000], 8), 8)
        assert rep.ok, rep.summary()
    finally:
        pf.pf_set_min_tile(pf.PF_SYSTEMATIC, P, 0)
        pf.pf_set_min_tile(pf.PF_MULTINOMIAL, 5000, 0)


@pytest.mark.parametrize("lw,eps", [([0.0, -0.5, 1.2, -2.0, 0.3], 0.01), ([0.0, 0.0, 0.0, 1.5], 0.02),
                                    ([2.0, -1.0, -1.0, -1.0, -1.0, 0.5], 0.05)])
def test_metropolis_bias_bound_on_gpu_chains(lw, eps):
    # F identical filters (distinct streams through the filter id): chain i of
    # every filter ends at k with probability (M^B)[i, k]; Eq. 5's B keeps the
    # probability of ending at the heaviest particle within eps of w_max
    lw = np.array(lw, np.float32)
    P = lw.size
    w = np.exp(lw.astype(np.float64) - lw.max())
    w_max = w.max() / w.sum()
    B = pf.pf_metropolis_B(P, w_max, eps)
    assert B == oracle.metropolis_B(P, w_max, eps) and B >= 1
    MB = np.linalg.matrix_power(oracle.metropolis_matrix(lw), B)
    F = 60000
    off = np.arange(F + 1, dtype=np.int64) * P
    d_lw = torch.from_numpy(np.tile(lw, F)).cuda()
    anc = torch.empty(F * P, dtype=torch.int32, device="cuda")
    seeds = torch.full((F,), 12345, dtype=torch.int64, device="cuda")
    pf.pf_resample_batched(pf.PF_METROPOLIS, d_lw, torch.from_numpy(off).cuda(), F, B, seeds, anc)
    assert pf.pf_get_device_status() == pf.PF_OK
    a = anc.cpu().numpy().reshape(F, P)
    pmax = int(np.argmax(lw))
    for i in range(P):
        counts = np.bincount(a[:, i], minlength=P)
        # the GPU chain's law is the exact B-step row
        chi2 = ((counts - F * MB[i]) ** 2 / (F * MB[i])).sum()
        assert stats.chi2.sf(chi2, P - 1) > 1e-4, (i, counts, F * MB[i])
        # and the bound holds on it: |P(end at p_max) - w_max| <= eps (+ sampling error)
        freq = counts[pmax] / F
        se = np.sqrt(MB[i, pmax] * (1 - MB[i, pmax]) / F)
        assert abs(freq - w_max) <= eps + 5 * se
    # the bound is tight: one step fewer leaves some start further than eps away
    MB1 = np.linalg.matrix_power(oracle.metropolis_matrix(lw), B - 1)
    assert np.abs(MB1[:, pmax] - w_max).max() > eps
