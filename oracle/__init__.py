"""FP64 CPU oracle for the particle-filter resampling stage (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The GPU library never calls it and has
no fallback to it.  The numerical work is in ``pf_oracle.c`` (plain C, FP64,
single-threaded); this module only marshals numpy arrays through ctypes.

Each function cites the part of Murray, "GPU acceleration of the particle
filter: the Metropolis resampler" that it follows:
  * resampling contract ............ Section 1, step 4
  * multinomial / stratified /
    systematic / Metropolis ........ Figure 1 (a)-(d), Section 2
  * bound on Metropolis steps B .... Section 2, Eqs. 1-5
  * effective sample size .......... Section 3 (standard (sum w)^2 / sum w^2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pf_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TAG_SYS, TAG_STRAT, TAG_MULTI, TAG_METRO = 1, 2, 3, 4
KIND_MULTINOMIAL, KIND_STRATIFIED, KIND_SYSTEMATIC, KIND_METROPOLIS = 0, 1, 2, 3

OK, ERR_INVALID, ERR_DOMAIN = 0, 1, 2


class OracleError(RuntimeError):
    pass


def build(force: bool = False) -> str:
    """Compile pf_oracle.c into liboracle.so beside it (gcc, no FP contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
             "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        c_f = ctypes.POINTER(ctypes.c_float)
        c_d = ctypes.POINTER(ctypes.c_double)
        c_i32 = ctypes.POINTER(ctypes.c_int32)
        c_i64 = ctypes.POINTER(ctypes.c_int64)
        c_u32 = ctypes.POINTER(ctypes.c_uint32)
        c_u64 = ctypes.POINTER(ctypes.c_uint64)
        i64, u64, u32, i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int
        sig = {
            "orc_philox4x32_10": (None, [c_u32, c_u32, c_u32]),
            "orc_philox4x32_r": (None, [c_u32, c_u32, c_u32, i32]),
            "orc_metropolis_draws_r": (None, [u64, u32, i64, i64, i32, i32, c_i32, c_d]),
            "orc_metropolis_chains_r": (i32, [c_f, i64, i32, u64, u32, c_i64, i64, i32, c_i32]),
            "orc_u23": (ctypes.c_double, [u32]),
            "orc_u32": (ctypes.c_double, [u32]),
            "orc_index": (u32, [u32, u32]),
            "orc_stream_words": (None, [u64, u32, u32, i64, c_u32]),
            "orc_stream_uniforms": (None, [u64, u32, u32, i64, i32, c_d]),
            "orc_metropolis_draws": (None, [u64, u32, i64, i64, i32, c_i32, c_d]),
            "orc_normalised_cumsum": (i32, [c_f, i64, c_d]),
            "orc_ess": (i32, [c_f, i64, c_d, c_d]),
            "orc_systematic_u": (i32, [c_f, i64, ctypes.c_double, c_i32]),
            "orc_stratified_u": (i32, [c_f, i64, c_d, c_i32]),
            "orc_multinomial_u": (i32, [c_f, i64, c_d, c_i32]),
            "orc_metropolis_u": (i32, [c_f, i64, i32, c_i32, c_d, c_i32]),
            "orc_systematic": (i32, [c_f, i64, u64, u32, c_i32]),
            "orc_stratified": (i32, [c_f, i64, u64, u32, c_i32]),
            "orc_multinomial": (i32, [c_f, i64, u64, u32, c_i32]),
            "orc_metropolis": (i32, [c_f, i64, i32, u64, u32, c_i32]),
            "orc_metropolis_chains": (i32, [c_f, i64, i32, u64, u32, c_i64, i64, c_i32]),
            "orc_gather": (i32, [ctypes.c_void_p, i64, i64, c_i32, i64, ctypes.c_void_p]),
            "orc_offspring": (None, [c_i32, i64, i64, c_i64]),
            "orc_metropolis_matrix": (i32, [c_f, i64, c_d]),
            "orc_metropolis_B": (i64, [i64, ctypes.c_double, ctypes.c_double]),
            "orc_batched": (i32, [i32, c_f, c_i64, i32, i32, c_u64, c_i32]),
            "orc_kalman_loglik": (ctypes.c_double, [ctypes.c_double] * 5 + [c_d, i32, i32]),
            "orc_permute": (i32, [c_i32, i64, c_i32]),
            "orc_lg_normals": (None, [u64, u32, u32, u32, c_d]),
            "orc_lg_init": (i32, [i32, i64, i32, ctypes.c_double, ctypes.c_double, u64, c_d, c_d, c_d, c_d, c_d,
                                  c_i32]),
            "orc_lg_step": (i32, [i32, i64, i32, c_f, ctypes.c_double, ctypes.c_double, ctypes.c_double, c_f, i32,
                                  u64, c_i32, c_f, c_f, c_i32, c_d, c_d, c_d, c_d, c_d, c_d, c_d, c_i32]),
            "orc_lg_filter": (i32, [i32, i32, i64, i32, c_f, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                    ctypes.c_double, ctypes.c_double, c_f, i32, u64, c_u64, c_d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f32(lw):
    return np.ascontiguousarray(lw, dtype=np.float32)


def _check(st):
    if st == ERR_DOMAIN:
        raise OracleError("domain error: NaN or +inf log-weight, or every weight zero")
    if st != OK:
        raise OracleError(f"oracle status {st}")


# --------------------------------------------------------------------------
# Philox-4x32-10 streams (Salmon et al., SC'11) in the library's layout.
# --------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32),
                              _p(out, ctypes.c_uint32))
    return out


def philox4x32(ctr, key, rounds):
    """Philox-4x32 with `rounds` rounds (the same round function)."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_r(_p(c, ctypes.c_uint32), _p(k, ctypes.c_uint32), _p(out, ctypes.c_uint32), int(rounds))
    return out


def u23(x: int) -> float:
    return _load().orc_u23(int(x))


def u32(x: int) -> float:
    return _load().orc_u32(int(x))


def index(x: int, P: int) -> int:
    return int(_load().orc_index(int(x), int(P)))


def stream_words(seed, filter_id, tag, n):
    out = np.zeros(n, dtype=np.uint32)
    _load().orc_stream_words(seed, filter_id, tag, n, _p(out, ctypes.c_uint32))
    return out


def stream_uniforms(seed, filter_id, tag, n, kind=0):
    """kind 0: u23 (systematic, stratified); kind 1: u32 (multinomial)."""
    out = np.zeros(n, dtype=np.float64)
    _load().orc_stream_uniforms(seed, filter_id, tag, n, kind, _p(out, ctypes.c_double))
    return out


def metropolis_draws(seed, filter_id, P, i, B, rounds=10):
    """Proposals and uniforms of chain i, steps 0..B-1 (Philox-4x32 with `rounds` rounds)."""
    prop = np.zeros(max(B, 1), dtype=np.int32)
    unif = np.zeros(max(B, 1), dtype=np.float64)
    _load().orc_metropolis_draws_r(seed, filter_id, P, i, B, int(rounds), _p(prop, ctypes.c_int32),
                                   _p(unif, ctypes.c_double))
    return prop[:B], unif[:B]


# --------------------------------------------------------------------------
# Weights and normalisation (Section 1 step 4; ESS as quoted in Section 3).
# --------------------------------------------------------------------------
def normalised_cumsum(lw):
    lw = _f32(lw)
    out = np.zeros(lw.size, dtype=np.float64)
    _check(_load().orc_normalised_cumsum(_p(lw, ctypes.c_float), lw.size, _p(out, ctypes.c_double)))
    return out


def ess(lw):
    """Returns (ESS, log sum_i exp(lw_i))."""
    lw = _f32(lw)
    e = ctypes.c_double()
    ls = ctypes.c_double()
    _check(_load().orc_ess(_p(lw, ctypes.c_float), lw.size, ctypes.byref(e), ctypes.byref(ls)))
    return e.value, ls.value


# --------------------------------------------------------------------------
# Resamplers (Figure 1, Section 2).
# --------------------------------------------------------------------------
def systematic_u(lw, u):
    lw = _f32(lw)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_systematic_u(_p(lw, ctypes.c_float), lw.size, float(u), _p(a, ctypes.c_int32)))
    return a


def stratified_u(lw, u):
    lw = _f32(lw)
    u = np.ascontiguousarray(u, dtype=np.float64)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_stratified_u(_p(lw, ctypes.c_float), lw.size, _p(u, ctypes.c_double),
                                    _p(a, ctypes.c_int32)))
    return a


def multinomial_u(lw, u):
    lw = _f32(lw)
    u = np.ascontiguousarray(u, dtype=np.float64)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_multinomial_u(_p(lw, ctypes.c_float), lw.size, _p(u, ctypes.c_double),
                                     _p(a, ctypes.c_int32)))
    return a


def metropolis_u(lw, B, prop, unif):
    """prop, unif: arrays of shape (P, B)."""
    lw = _f32(lw)
    prop = np.ascontiguousarray(prop, dtype=np.int32)
    unif = np.ascontiguousarray(unif, dtype=np.float64)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_metropolis_u(_p(lw, ctypes.c_float), lw.size, int(B), _p(prop, ctypes.c_int32),
                                    _p(unif, ctypes.c_double), _p(a, ctypes.c_int32)))
    return a


def systematic(lw, seed, filter_id=0):
    lw = _f32(lw)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_systematic(_p(lw, ctypes.c_float), lw.size, seed, filter_id, _p(a, ctypes.c_int32)))
    return a


def stratified(lw, seed, filter_id=0):
    lw = _f32(lw)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_stratified(_p(lw, ctypes.c_float), lw.size, seed, filter_id, _p(a, ctypes.c_int32)))
    return a


def multinomial(lw, seed, filter_id=0):
    lw = _f32(lw)
    a = np.zeros(lw.size, dtype=np.int32)
    _check(_load().orc_multinomial(_p(lw, ctypes.c_float), lw.size, seed, filter_id, _p(a, ctypes.c_int32)))
    return a


def metropolis(lw, B, seed, filter_id=0, chains=None, rounds=10):
    """All chains, or only the chain indices in ``chains``; draws from Philox-4x32 with
    `rounds` rounds (10: the default stream; 7: the opt-in cheaper stream)."""
    lw = _f32(lw)
    if chains is None and rounds == 10:
        a = np.zeros(lw.size, dtype=np.int32)
        _check(_load().orc_metropolis(_p(lw, ctypes.c_float), lw.size, int(B), seed, filter_id,
                                      _p(a, ctypes.c_int32)))
        return a
    idx = np.arange(lw.size, dtype=np.int64) if chains is None else np.ascontiguousarray(chains, dtype=np.int64)
    a = np.zeros(idx.size, dtype=np.int32)
    _check(_load().orc_metropolis_chains_r(_p(lw, ctypes.c_float), lw.size, int(B), seed, filter_id,
                                           _p(idx, ctypes.c_int64), idx.size, int(rounds), _p(a, ctypes.c_int32)))
    return a


def gather(src, anc):
    """dst[j] = src[anc[j]] row by row (src: 2-D array, C-contiguous)."""
    src = np.ascontiguousarray(src)
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    dst = np.empty((anc.size,) + src.shape[1:], dtype=src.dtype)
    row_bytes = src.strides[0] if src.ndim > 1 else src.itemsize
    _check(_load().orc_gather(src.ctypes.data, src.shape[0], row_bytes, _p(anc, ctypes.c_int32),
                              anc.size, dst.ctypes.data))
    return dst


def offspring(anc, P):
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    o = np.zeros(P, dtype=np.int64)
    _load().orc_offspring(_p(anc, ctypes.c_int32), anc.size, P, _p(o, ctypes.c_int64))
    return o


def metropolis_matrix(lw):
    lw = _f32(lw)
    P = lw.size
    M = np.zeros((P, P), dtype=np.float64)
    _check(_load().orc_metropolis_matrix(_p(lw, ctypes.c_float), P, _p(M, ctypes.c_double)))
    return M


def metropolis_B(P, w_max, eps=0.01):
    return int(_load().orc_metropolis_B(int(P), float(w_max), float(eps)))


def batched(kind, lw, offsets, B, seeds):
    lw = _f32(lw)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    sd = np.ascontiguousarray(seeds, dtype=np.uint64)
    a = np.zeros(lw.size, dtype=np.int32)
    F = off.size - 1
    _check(_load().orc_batched(int(kind), _p(lw, ctypes.c_float), _p(off, ctypes.c_int64), F, int(B),
                               _p(sd, ctypes.c_uint64), _p(a, ctypes.c_int32)))
    return a


# --------------------------------------------------------------------------
# Exact log-likelihood of the linear-Gaussian test model (Kalman filter).
# --------------------------------------------------------------------------
def kalman_loglik(a, q, r, y, m0=0.0, p0=1.0):
    """log p(y_{1:T}) for D independent AR(1) dimensions; y has shape (T, D)."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    T, D = y.shape
    return float(_load().orc_kalman_loglik(float(a), float(q), float(r), float(m0), float(p0),
                                           _p(y, ctypes.c_double), T, D))


# --------------------------------------------------------------------------
# Bootstrap filter on the linear-Gaussian test model (Section 1, steps 1-4):
# x_0 ~ N(m0, p0 I), x_t = a_f x_{t-1} + N(0, q I), y_t = x_t + N(0, r I).
# --------------------------------------------------------------------------
TAG_PROPAGATE = 6


def lg_normals(seed, f, j, c1):
    """The four N(0,1) draws of Philox counter (j, c1, f, 6) (Box-Muller)."""
    z = np.zeros(4)
    _load().orc_lg_normals(seed, f, j, c1, _p(z, ctypes.c_double))
    return z


def lg_init(F, P, D, m0, p0, seed):
    """Initial particles x [F, P, D] and filter scalars (FP64)."""
    x = np.zeros((F, P, D))
    lw = np.zeros((F, P))
    ll, ls, es = np.zeros(F), np.zeros(F), np.zeros(F)
    rs = np.zeros(F, dtype=np.int32)
    _check(_load().orc_lg_init(F, P, D, float(m0), float(p0), seed, _p(x, ctypes.c_double),
                               _p(lw, ctypes.c_double), _p(ll, ctypes.c_double), _p(ls, ctypes.c_double),
                               _p(es, ctypes.c_double), _p(rs, ctypes.c_int32)))
    return dict(x=x, logw=lw, loglik=ll, log_sum=ls, ess=es, resample=rs)


def lg_step(a, q, r, threshold, y, t, seed, anc, x_prev, lw, resample, log_sum, loglik):
    """One step (propagate from the ancestors where resample[f], weight,
    log-likelihood increment, ESS and the next decision), FP64 throughout;
    array inputs are taken as the FP32 (int32) values the caller holds."""
    x_prev = np.ascontiguousarray(x_prev, dtype=np.float32)
    F, P, D = x_prev.shape
    a = np.ascontiguousarray(a, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32).reshape(F, D)
    anc = np.ascontiguousarray(anc, dtype=np.int32).reshape(F, P)
    lw = np.ascontiguousarray(lw, dtype=np.float32).reshape(F, P)
    resample = np.ascontiguousarray(resample, dtype=np.int32)
    log_sum = np.ascontiguousarray(log_sum, dtype=np.float64)
    loglik = np.ascontiguousarray(loglik, dtype=np.float64)
    xn = np.zeros((F, P, D))
    lo = np.zeros((F, P))
    ll, ls, es = np.zeros(F), np.zeros(F), np.zeros(F)
    rs = np.zeros(F, dtype=np.int32)
    _check(_load().orc_lg_step(F, P, D, _p(a, ctypes.c_float), float(q), float(r), float(threshold),
                               _p(y, ctypes.c_float), int(t), seed, _p(anc, ctypes.c_int32),
                               _p(x_prev, ctypes.c_float), _p(lw, ctypes.c_float), _p(resample, ctypes.c_int32),
                               _p(log_sum, ctypes.c_double), _p(loglik, ctypes.c_double), _p(xn, ctypes.c_double),
                               _p(lo, ctypes.c_double), _p(ll, ctypes.c_double), _p(ls, ctypes.c_double),
                               _p(es, ctypes.c_double), _p(rs, ctypes.c_int32)))
    return dict(x=xn, logw=lo, loglik=ll, log_sum=ls, ess=es, resample=rs)


def lg_filter(a, q, r, y, seed, step_seeds, P, m0=0.0, p0=1.0, threshold=0.5, kind=KIND_SYSTEMATIC):
    """A whole bootstrap-filter run in FP64; y is [T, F, D], step_seeds [T, F].
    Returns the log-likelihood estimates [F]."""
    y = np.ascontiguousarray(y, dtype=np.float32)
    T, F, D = y.shape
    a = np.ascontiguousarray(a, dtype=np.float32)
    ss = np.ascontiguousarray(step_seeds, dtype=np.uint64).reshape(-1)
    assert ss.size >= T * F
    ll = np.zeros(F)
    _check(_load().orc_lg_filter(int(kind), F, P, D, _p(a, ctypes.c_float), float(q), float(r), float(m0),
                                 float(p0), float(threshold), _p(y, ctypes.c_float), T, seed,
                                 _p(ss, ctypes.c_uint64), _p(ll, ctypes.c_double)))
    return ll


# --------------------------------------------------------------------------
# Offspring/ancestor conversion for in-place moves (Section 2).
# --------------------------------------------------------------------------
def permute(anc):
    """Ancestors with the same offspring counts, every particle with offspring
    keeping one in its own slot, the other copies filling the empty slots in order."""
    anc = np.ascontiguousarray(anc, dtype=np.int32)
    out = np.zeros(anc.size, dtype=np.int32)
    _check(_load().orc_permute(_p(anc, ctypes.c_int32), anc.size, _p(out, ctypes.c_int32)))
    return out
