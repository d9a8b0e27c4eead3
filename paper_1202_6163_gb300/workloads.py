"""Seeded synthetic inputs shaped like the paper's resampling workloads.

This module holds no resampling arithmetic: it only draws log-weights, particle
states and filter layouts with numpy's seeded PCG64 generator, so that the GPU
library and the CPU oracle can be fed identical arrays.  The paper simulates
weight sets rather than using a dataset (Section 3: Dirichlet weights over
P = 256 ... 65536); the Gaussian log-weight sets below stand in for those, with
the log-weight spread s playing the role of the Dirichlet concentration
(ESS/P is about exp(-s^2) for Gaussian log-weights and about alpha/(1+alpha)
for symmetric Dirichlet weights).
"""
from __future__ import annotations

import math

import numpy as np


def gaussian_logw(P: int, s: float = 1.0, seed: int = 0) -> np.ndarray:
    """P i.i.d. N(0, s^2) log-weights drawn in float64 and rounded once to float32."""
    rng = np.random.default_rng(seed)
    return (s * rng.standard_normal(P)).astype(np.float32)


def heavy_tail_logw(P: int, shift: float = 10.0, frac: float = 0.01, seed: int = 0) -> np.ndarray:
    """N(0,1) log-weights with exactly floor(P*frac) seeded positions shifted by +shift."""
    rng = np.random.default_rng(seed)
    lw = rng.standard_normal(P)
    k = int(math.floor(P * frac))
    if k:
        idx = rng.choice(P, size=k, replace=False)
        lw[idx] += shift
    return lw.astype(np.float32)


def dirichlet_logw(P: int, alpha: float, seed: int = 0) -> np.ndarray:
    """Log of unnormalised symmetric Dirichlet(alpha) weights (the paper's Section 3
    weight model): log G with G ~ Gamma(alpha), drawn as log Gamma(alpha+1) + log(U)/alpha
    so that small alpha does not underflow."""
    rng = np.random.default_rng(seed)
    g = rng.gamma(alpha + 1.0, 1.0, size=P)
    u = rng.random(P)
    return (np.log(g) + np.log(u) / alpha).astype(np.float32)


def states(P: int, D: int, seed: int = 1) -> np.ndarray:
    """P x D float32 particle states, N(0,1)."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal((P, D)).astype(np.float32)


def batched_layout(F: int = 4096, p_lo: int = 256, p_hi: int = 65536, s_lo: float = 0.5,
                   s_hi: float = 3.0, seed: int = 0):
    """F filters with P_f = floor(exp(U(ln p_lo, ln p_hi))) particles and spread
    s_f ~ U[s_lo, s_hi].  Returns (offsets int64[F+1], spreads float64[F])."""
    rng = np.random.default_rng(seed)
    Pf = np.floor(np.exp(rng.uniform(math.log(p_lo), math.log(p_hi), size=F))).astype(np.int64)
    Pf = np.clip(Pf, p_lo, p_hi)
    sf = rng.uniform(s_lo, s_hi, size=F)
    off = np.zeros(F + 1, dtype=np.int64)
    np.cumsum(Pf, out=off[1:])
    return off, sf


def batched_logw(offsets: np.ndarray, spreads: np.ndarray, seed: int = 0) -> np.ndarray:
    """Concatenated per-filter N(0, s_f^2) log-weights (float32)."""
    rng = np.random.default_rng(seed + 1)
    total = int(offsets[-1])
    z = rng.standard_normal(total)
    scale = np.repeat(spreads, np.diff(offsets))
    return (z * scale).astype(np.float32)


def batched_seeds(F: int, base: int = 0) -> np.ndarray:
    """Per-filter Philox seeds base + f."""
    return (np.uint64(base) + np.arange(F, dtype=np.uint64)).astype(np.uint64)


# ---------------------------------------------------------------------------
# Linear-Gaussian test model for whole bootstrap-filter runs: 256 filters (one
# per parameter set, as in particle MCMC), x_t = a_f x_{t-1} + N(0, q I),
# y_t = x_t + N(0, r I) in D = 4 dimensions, a_f ~ U[0.8, 0.99].
# ---------------------------------------------------------------------------
LG_Q, LG_R, LG_M0, LG_P0 = 0.1, 0.5, 0.0, 1.0


def lg_params(F: int = 256, lo: float = 0.8, hi: float = 0.99, seed: int = 0) -> np.ndarray:
    """Per-filter autoregression coefficients a_f ~ U[lo, hi], float32."""
    return np.random.default_rng(seed).uniform(lo, hi, size=F).astype(np.float32)


def lg_observations(a: np.ndarray, T: int = 200, D: int = 4, q: float = LG_Q, r: float = LG_R,
                    m0: float = LG_M0, p0: float = LG_P0, seed: int = 1) -> np.ndarray:
    """Simulate one state path per filter from the model (float64) and return the
    observations y[t-1, f, :] of times t = 1..T as float32 [T, F, D]."""
    rng = np.random.default_rng(seed)
    F = a.size
    af = a.astype(np.float64)[:, None]
    x = m0 + math.sqrt(p0) * rng.standard_normal((F, D))
    y = np.empty((T, F, D))
    for t in range(T):
        x = af * x + math.sqrt(q) * rng.standard_normal((F, D))
        y[t] = x + math.sqrt(r) * rng.standard_normal((F, D))
    return y.astype(np.float32)


def lg_step_seeds(T: int, F: int, base: int = 1000) -> np.ndarray:
    """Resampling keys: step t (1-based) of filter f uses base + t (the filter id
    separates the filters' streams), as a uint64 [T, F] array."""
    return np.repeat((base + np.arange(1, T + 1, dtype=np.uint64))[:, None], F, axis=1)
