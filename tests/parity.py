"""Comparison of GPU ancestors with the FP64 oracle under the near-tie rule.

The rule: GPU ancestors must equal the oracle's, except at decisions whose
uniform lies within TAU = 1e-6 (relative) of a cumulative-weight or
weight-ratio threshold.  Read concretely:

* cumulative schemes -- decision j compares its normalised position
  x_j ((j+u)/P systematic, (j+u_j)/P stratified, u_j multinomial) with the
  normalised cumulative weights theta_b = c_b / W.  A mismatch a_gpu != a_orc
  is excused only if EVERY threshold theta_b the two picks disagree on
  (b in [min, max) of the two picks) satisfies |x_j - theta_b| <= TAU theta_b,
  and the GPU pick has positive weight.
* Metropolis -- step b of chain i compares u_b with r = exp(lw_j - lw_k).  A
  chain whose final state differs is excused only if flipping some of its
  near-tie decisions (|u_b - r| <= TAU r) in the oracle's replay reaches the
  GPU's final state.

Every excused mismatch is listed; anything else fails.  A listed cumulative
mismatch carries its size: the index gap |a_gpu - a_orc|, the number of
positive-weight particles strictly between the two picks (0 when the picks are
adjacent non-empty intervals), and its relative distance max |x_j - theta_b| /
theta_b.  A listed Metropolis mismatch carries the first step whose decision
the replay flipped and the number of flips.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import NamedTuple

import numpy as np

import oracle

TAU = 1e-6


class Excused(NamedTuple):
    """One cumulative decision the two sides took differently, at a near tie."""
    j: int          # decision (offset or draw)
    gpu: int        # GPU pick
    orc: int        # oracle pick
    x: float        # normalised position x_j
    theta: float    # smallest threshold the picks disagree on
    rel: float      # max |x_j - theta_b| / theta_b over those thresholds
    gap: int        # |gpu - orc|
    between: int    # positive-weight particles strictly between the picks


class ExcusedChain(NamedTuple):
    """One Metropolis chain whose final state differs, reached by flipping near ties."""
    chain: int
    gpu: int
    orc: int
    first_step: int  # first step whose decision the replay flipped
    flips: int       # near-tie decisions flipped


@dataclass
class ParityReport:
    n: int
    mismatches: int = 0
    excused: list = field(default_factory=list)
    failures: list = field(default_factory=list)
    in_band: int = 0

    @property
    def ok(self):
        return not self.failures

    @property
    def worst_rel(self):
        """Largest relative distance of an excused cumulative mismatch (0 if none)."""
        return max((e.rel for e in self.excused if isinstance(e, Excused)), default=0.0)

    @property
    def worst_gap(self):
        return max((e.gap for e in self.excused if isinstance(e, Excused)), default=0)

    @property
    def worst_between(self):
        return max((e.between for e in self.excused if isinstance(e, Excused)), default=0)

    @property
    def non_adjacent(self):
        """Excused cumulative mismatches with a positive-weight particle between the picks."""
        return sum(1 for e in self.excused if isinstance(e, Excused) and e.between > 0)

    def summary(self):
        return (f"n={self.n} mismatches={self.mismatches} excused={len(self.excused)} "
                f"failures={len(self.failures)} in_band_decisions={self.in_band} "
                f"worst_rel={self.worst_rel:.2e} worst_gap={self.worst_gap} worst_between={self.worst_between}")


def positions(kind: str, lw: np.ndarray, seed: int, filter_id: int = 0) -> np.ndarray:
    """Normalised positions x_j the oracle's cumulative decisions use."""
    P = lw.size
    j = np.arange(P, dtype=np.float64)
    if kind == "systematic":
        u = oracle.stream_uniforms(seed, filter_id, oracle.TAG_SYS, 1)[0]
        return (j + u) / P
    if kind == "stratified":
        u = oracle.stream_uniforms(seed, filter_id, oracle.TAG_STRAT, P)
        return (j + u) / P
    if kind == "multinomial":
        return oracle.stream_uniforms(seed, filter_id, oracle.TAG_MULTI, P, kind=1)
    raise ValueError(kind)


def check_cumulative(kind: str, lw, a_gpu, a_orc, seed: int = 0, filter_id: int = 0,
                     tau: float = TAU, x=None) -> ParityReport:
    """x: the normalised positions, if not those of the library's streams for `seed`."""
    lw = np.asarray(lw, dtype=np.float32)
    a_gpu = np.asarray(a_gpu).astype(np.int64)
    a_orc = np.asarray(a_orc).astype(np.int64)
    P = lw.size
    rep = ParityReport(n=P)
    if a_gpu.shape != a_orc.shape:
        rep.failures.append(("shape", a_gpu.shape, a_orc.shape))
        return rep
    if np.any((a_gpu < 0) | (a_gpu >= P)):
        bad = np.nonzero((a_gpu < 0) | (a_gpu >= P))[0][:10]
        rep.failures.append(("out_of_range", bad.tolist(), a_gpu[bad].tolist()))
        return rep
    theta = oracle.normalised_cumsum(lw)
    if x is None:
        x = positions(kind, lw, seed, filter_id)
    # decisions inside the band around the thresholds that bracket the oracle pick
    hi_t = theta[a_orc]
    lo_t = np.where(a_orc > 0, theta[np.maximum(a_orc - 1, 0)], 0.0)
    near = (np.abs(x - hi_t) <= tau * hi_t) | ((a_orc > 0) & (np.abs(x - lo_t) <= tau * lo_t))
    rep.in_band = int(near.sum())
    mism = np.nonzero(a_gpu != a_orc)[0]
    rep.mismatches = int(mism.size)
    for j in mism:
        g, o = int(a_gpu[j]), int(a_orc[j])
        lo, hi = min(g, o), max(g, o)
        th = theta[lo:hi]
        tie = bool(np.all(np.abs(x[j] - th) <= tau * th)) and lw[g] > -np.inf
        rec = Excused(int(j), g, o, float(x[j]), float(th.min()) if th.size else float("nan"),
                      float(np.max(np.abs(x[j] - th) / th)) if th.size else float("nan"),
                      hi - lo, int(np.count_nonzero(lw[lo + 1:hi] > -np.inf)))
        (rep.excused if tie else rep.failures).append(rec)
    return rep


def _replay(lw64, P, k, props, unifs, b0, flips_left, target, tau):
    """Depth-first replay of a chain from step b0 in state k.  Returns the list of
    steps whose near-tie decisions were flipped to reach target (empty if none were
    needed), or None if target is not reachable by flipping at most flips_left of them.
    The threshold of every step is r = exp(lw_j - lw_k), including r >= 1 (a move the
    exact rule always takes is a near tie when u lies within tau r of r, i.e. when
    r < 1 / (1 - tau))."""
    for b in range(b0, len(props)):
        j = int(props[b])
        u = float(unifs[b])
        d = lw64[j] - lw64[k]  # +inf (state of zero weight), -inf (proposal of zero weight) or nan (both)
        acc = bool(lw64[j] >= lw64[k]) or u < math.exp(d)
        if flips_left > 0 and math.isfinite(d) and d < 1e-3:
            r = math.exp(d)
            if abs(u - r) <= tau * r:
                alt = k if acc else j
                rest = _replay(lw64, P, alt, props, unifs, b + 1, flips_left - 1, target, tau)
                if rest is not None:
                    return [b] + rest
        if acc:
            k = j
    return [] if k == target else None


def check_metropolis(lw, B, a_gpu, a_orc, seed, chains=None, filter_id=0, tau=TAU, max_flips=3,
                     draws=None, rounds=10) -> ParityReport:
    """a_gpu, a_orc: ancestors of the chains listed in `chains` (all chains if None).
    draws: (proposals, uniforms), each of shape (P, B), in place of the library's streams;
    rounds: the Philox rounds of those streams (10, or 7 for the opt-in stream)."""
    lw = np.asarray(lw, dtype=np.float32)
    lw64 = lw.astype(np.float64)
    P = lw.size
    idx = np.arange(P) if chains is None else np.asarray(chains)
    a_gpu = np.asarray(a_gpu).astype(np.int64)
    a_orc = np.asarray(a_orc).astype(np.int64)
    rep = ParityReport(n=idx.size)
    if np.any((a_gpu < 0) | (a_gpu >= P)):
        rep.failures.append(("out_of_range",))
        return rep
    mism = np.nonzero(a_gpu != a_orc)[0]
    rep.mismatches = int(mism.size)
    for q in mism:
        i = int(idx[q])
        if draws is None:
            props, unifs = oracle.metropolis_draws(seed, filter_id, P, i, B, rounds=rounds)
        else:
            props, unifs = draws[0][i], draws[1][i]
        flips = _replay(lw64, P, i, props, unifs, 0, max_flips, int(a_gpu[q]), tau)
        if flips:
            rep.excused.append(ExcusedChain(i, int(a_gpu[q]), int(a_orc[q]), flips[0], len(flips)))
        else:
            rep.failures.append((i, int(a_gpu[q]), int(a_orc[q])))
    return rep
