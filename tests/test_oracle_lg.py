"""Pins of the oracle's bootstrap filter on the linear-Gaussian test model
(Section 1, steps 1-4: initialise, propagate, weight, resample).

What fixes it, independently of its own code:
  * the Box-Muller draws are N(0,1) (Kolmogorov-Smirnov, moments, independence);
  * with q = 0 a step is a closed form: x_next = a x_prev[src] exactly, and the
    weight, log-sum-exp and ESS follow from scipy's normal log-density and
    logsumexp;
  * the bootstrap filter's likelihood estimate is unbiased: E[Z_hat] equals the
    exact Kalman-filter likelihood for every resampling schedule and scheme
    (many independent filters on one data set);
  * with many particles log Z_hat is close to the Kalman value.
"""
import math

import numpy as np
import pytest
from scipy import special, stats

import oracle
from paper_1202_6163_gb300 import workloads as wl


def test_normals_are_standard():
    st = oracle.lg_init(2, 30000, 8, 0.0, 1.0, seed=11)
    x = st["x"].reshape(-1, 8)
    assert stats.kstest(x.ravel(), "norm").pvalue > 1e-4
    assert np.abs(x.mean(0)).max() < 0.02
    assert np.abs(x.var(0) - 1).max() < 0.03
    c = np.corrcoef(x.T) - np.eye(8)
    assert np.abs(c).max() < 0.02
    # the initial draw is m0 + sqrt(p0) z with the same z
    st2 = oracle.lg_init(2, 30000, 8, 1.5, 4.0, seed=11)
    np.testing.assert_allclose(st2["x"], 1.5 + 2.0 * st["x"], rtol=1e-14, atol=1e-14)
    assert np.all(st["logw"] == 0) and np.all(st["resample"] == 0)
    np.testing.assert_allclose(st["log_sum"], math.log(30000))
    np.testing.assert_allclose(st["ess"], 30000)


def _inputs(F, P, D, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal((F, P, D)).astype(np.float32)
    lw = (rng.standard_normal((F, P)) - 3).astype(np.float32)
    anc = np.sort(rng.integers(0, P, size=(F, P)), axis=1).astype(np.int32)
    y = rng.standard_normal((F, D)).astype(np.float32)
    a = rng.uniform(0.8, 0.99, F).astype(np.float32)
    resample = (np.arange(F) % 2).astype(np.int32)
    log_sum = special.logsumexp(lw.astype(np.float64), axis=1)
    loglik = rng.standard_normal(F)
    return x, lw, anc, y, a, resample, log_sum, loglik


def test_step_closed_form_without_noise():
    F, P, D, r = 3, 50, 8, 0.5
    x, lw, anc, y, a, resample, log_sum, loglik = _inputs(F, P, D, 1)
    out = oracle.lg_step(a, 0.0, r, 0.5, y, 3, 9, anc, x, lw, resample, log_sum, loglik)
    for f in range(F):
        src = anc[f] if resample[f] else np.arange(P)
        xn = a[f].astype(np.float64) * x[f][src].astype(np.float64)
        np.testing.assert_array_equal(out["x"][f], xn)
        prev = 0.0 if resample[f] else lw[f].astype(np.float64)
        logg = stats.norm.logpdf(y[f].astype(np.float64)[None, :], xn, math.sqrt(r)).sum(axis=1)
        np.testing.assert_allclose(out["logw"][f], prev + logg, rtol=1e-13, atol=1e-12)
        L = special.logsumexp(out["logw"][f])
        L_prev = math.log(P) if resample[f] else log_sum[f]
        np.testing.assert_allclose(out["loglik"][f], loglik[f] + L - L_prev, rtol=1e-13, atol=1e-12)
        np.testing.assert_allclose(out["log_sum"][f], L, rtol=1e-14)
        w = np.exp(out["logw"][f] - out["logw"][f].max())
        ess = w.sum() ** 2 / (w ** 2).sum()
        np.testing.assert_allclose(out["ess"][f], ess, rtol=1e-12)
        assert out["resample"][f] == int(ess < 0.5 * P)


def test_step_noise_is_scaled_normal():
    F, P, D, q = 2, 20000, 4, 0.3
    x, lw, anc, y, a, resample, log_sum, loglik = _inputs(F, P, D, 2)
    out = oracle.lg_step(np.zeros(F, np.float32), q, 0.5, 0.5, y, 5, 4, anc, x, lw, resample, log_sum, loglik)
    z = out["x"].ravel() / math.sqrt(q)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # the noise of time t is not that of time t + 1
    out2 = oracle.lg_step(np.zeros(F, np.float32), q, 0.5, 0.5, y, 6, 4, anc, x, lw, resample, log_sum, loglik)
    assert abs(np.corrcoef(out["x"].ravel(), out2["x"].ravel())[0, 1]) < 0.02


def test_thresholds_zero_and_above_one():
    F, P, D = 4, 300, 4
    x, lw, anc, y, a, resample, log_sum, loglik = _inputs(F, P, D, 3)
    never = oracle.lg_step(a, 0.1, 0.5, 0.0, y, 1, 1, anc, x, lw, resample, log_sum, loglik)
    always = oracle.lg_step(a, 0.1, 0.5, 1.01, y, 1, 1, anc, x, lw, resample, log_sum, loglik)
    assert not never["resample"].any() and always["resample"].all()


@pytest.mark.parametrize("kind,threshold", [(oracle.KIND_SYSTEMATIC, 0.5), (oracle.KIND_SYSTEMATIC, 1.01),
                                            (oracle.KIND_SYSTEMATIC, 0.0), (oracle.KIND_STRATIFIED, 0.5),
                                            (oracle.KIND_MULTINOMIAL, 0.5)])
def test_likelihood_estimate_is_unbiased(kind, threshold):
    # 6000 independent filters (filter ids separate their streams) on one data
    # set; r = 2 keeps the weights flat enough for a tight standard error
    F, P, T, D, r = 6000, 32, 6, 4, 2.0
    a1 = wl.lg_params(1, seed=5)
    y1 = wl.lg_observations(a1, T=T, D=D, r=r, seed=6)
    a = np.repeat(a1, F)
    y = np.repeat(y1, F, axis=1)
    ll = oracle.lg_filter(a, wl.LG_Q, r, y, 21, wl.lg_step_seeds(T, F), P, threshold=threshold, kind=kind)
    kf = oracle.kalman_loglik(float(a1[0]), wl.LG_Q, r, y1[:, 0, :].astype(np.float64), wl.LG_M0, wl.LG_P0)
    ratio = np.exp(ll - kf)
    se = ratio.std() / math.sqrt(F)
    assert abs(ratio.mean() - 1.0) < 4 * se, (ratio.mean(), se)
    assert se < 0.05


def test_many_particles_approach_kalman():
    F, P, T = 4, 8192, 20
    a = wl.lg_params(F, seed=8)
    y = wl.lg_observations(a, T=T, seed=9)
    ll = oracle.lg_filter(a, wl.LG_Q, wl.LG_R, y, 3, wl.lg_step_seeds(T, F), P)
    kf = np.array([oracle.kalman_loglik(float(a[f]), wl.LG_Q, wl.LG_R, y[:, f, :].astype(np.float64),
                                        wl.LG_M0, wl.LG_P0) for f in range(F)])
    assert np.abs(ll - kf).max() < 0.5, ll - kf
