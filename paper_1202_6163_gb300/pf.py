"""Thin ctypes binding of libpf.so (declared in include/pf.h).

Argument marshalling only: every function forwards to the C entry point of the
same name.  Array arguments may be torch CUDA tensors (their data pointers are
passed) or raw integer device addresses.  ``stream`` defaults to torch's
current CUDA stream.  A non-zero status raises :class:`PFError`.  The library
must have been built (``python -m paper_1202_6163_gb300.build``); there is no
fallback of any kind when it is missing.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpf.so")

PF_OK, PF_ERR_INVALID, PF_ERR_DOMAIN, PF_ERR_TIMEOUT, PF_ERR_CUDA, PF_ERR_NOMEM = range(6)
PF_MULTINOMIAL, PF_STRATIFIED, PF_SYSTEMATIC, PF_METROPOLIS = range(4)
STATUS_NAMES = {0: "PF_OK", 1: "PF_ERR_INVALID", 2: "PF_ERR_DOMAIN", 3: "PF_ERR_TIMEOUT", 4: "PF_ERR_CUDA",
                5: "PF_ERR_NOMEM"}

# name -> (restype, argtypes); the full set of symbols include/pf.h declares
_VP, _I64, _U64, _INT = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int
SIGNATURES = {
    "pf_resample_systematic": (_INT, [_VP, _I64, _INT, _U64, _VP, _VP]),
    "pf_resample_stratified": (_INT, [_VP, _I64, _INT, _U64, _VP, _VP]),
    "pf_resample_multinomial": (_INT, [_VP, _I64, _INT, _U64, _VP, _VP]),
    "pf_resample_metropolis": (_INT, [_VP, _I64, _INT, _U64, _VP, _VP]),
    "pf_gather": (_INT, [_VP, _I64, _I64, _VP, _I64, _VP, _VP]),
    "pf_ess": (_INT, [_VP, _I64, _VP, _VP, _VP]),
    "pf_resample_batched": (_INT, [_INT, _VP, _VP, _INT, _INT, _VP, _VP, _VP]),
    "pf_reserve": (_INT, [_I64, _I64, _INT, _VP]),
    "pf_get_device_status": (_INT, [_VP, ctypes.POINTER(ctypes.c_int)]),
    "pf_metropolis_B": (_I64, [_I64, ctypes.c_double, ctypes.c_double]),
    "pf_status_string": (ctypes.c_char_p, [_INT]),
    "pf_is_device_accessible": (_INT, [_VP]),
    "pf_permute": (_INT, [_VP, _I64, _VP, _VP]),
    "pf_gather_inplace": (_INT, [_VP, _I64, _I64, _VP, _VP]),
    "pf_metropolis_bias": (ctypes.c_double, [_I64, ctypes.c_double, _I64]),
    "pf_set_wait_limit_ns": (_INT, [_U64]),
    "pf_debug_skip_publish": (_INT, [_I64]),
    "pf_set_trace_buffer": (_INT, [_VP, _I64]),
    "pf_version": (_INT, []),
    "pf_resample_multinomial_static": (_INT, [_VP, _I64, _U64, _VP, _VP, _VP]),
    "pf_probe_l2_random_reads": (_INT, [_VP, _I64, _INT, ctypes.POINTER(ctypes.c_double)]),
    "pf_autotune": (_INT, [_INT, _VP, _I64, _VP, _INT, _VP, ctypes.POINTER(ctypes.c_int),
                           ctypes.POINTER(ctypes.c_float)]),
    "pf_set_min_tile": (_INT, [_INT, _I64, _INT]),
    "pf_get_min_tile": (_INT, [_INT, _I64]),
    "pf_resample_batched_masked": (_INT, [_INT, _VP, _VP, _INT, _INT, _VP, _VP, _VP, _VP]),
    "pf_resample_batched_metropolis_bound": (_INT, [_VP, _VP, _INT, ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
    "pf_set_metropolis_philox_rounds": (_INT, [_INT]),
    "pf_debug_tile_weights": (_INT, [_VP, _I64, _INT, _VP, _VP]),
    "pf_get_metropolis_philox_rounds": (_INT, []),
    "pf_lg_init": (_INT, [_INT, _I64, _INT, ctypes.c_float, ctypes.c_float, _U64, _VP, _VP, _VP, _VP, _VP, _VP,
                          _VP]),
    "pf_lg_step": (_INT, [_INT, _I64, _INT, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP, _INT, _U64,
                          _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP]),
}


class PFError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}")


_lib = None


def load(path: str = LIB_PATH):
    """Load libpf.so (once).  Raises OSError if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise OSError(f"libpf.so not built at {path}; run python -m paper_1202_6163_gb300.build")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(st: int, where: str):
    if st != PF_OK:
        raise PFError(st, where)


def pf_resample_systematic(logw, P, B, seed, ancestors, stream=None):
    _check(load().pf_resample_systematic(_ptr(logw), P, B, seed, _ptr(ancestors), _stream(stream)),
           "pf_resample_systematic")


def pf_resample_stratified(logw, P, B, seed, ancestors, stream=None):
    _check(load().pf_resample_stratified(_ptr(logw), P, B, seed, _ptr(ancestors), _stream(stream)),
           "pf_resample_stratified")


def pf_resample_multinomial(logw, P, B, seed, ancestors, stream=None):
    _check(load().pf_resample_multinomial(_ptr(logw), P, B, seed, _ptr(ancestors), _stream(stream)),
           "pf_resample_multinomial")


def pf_resample_metropolis(logw, P, B, seed, ancestors, stream=None):
    _check(load().pf_resample_metropolis(_ptr(logw), P, B, seed, _ptr(ancestors), _stream(stream)),
           "pf_resample_metropolis")


def pf_gather(src, P_src, row_bytes, ancestors, P_dst, dst, stream=None):
    _check(load().pf_gather(_ptr(src), P_src, row_bytes, _ptr(ancestors), P_dst, _ptr(dst), _stream(stream)),
           "pf_gather")


def pf_ess(logw, P, ess_out, log_sum_out=None, stream=None):
    _check(load().pf_ess(_ptr(logw), P, _ptr(ess_out), _ptr(log_sum_out), _stream(stream)), "pf_ess")


def pf_resample_batched(kind, logw, offsets, F, B, seeds, ancestors, stream=None):
    _check(load().pf_resample_batched(kind, _ptr(logw), _ptr(offsets), F, B, _ptr(seeds), _ptr(ancestors),
                                      _stream(stream)), "pf_resample_batched")


def pf_resample_batched_metropolis_bound(logw, offsets, F, eps, seeds, ancestors, B_out=None, mask=None,
                                         stream=None):
    _check(load().pf_resample_batched_metropolis_bound(_ptr(logw), _ptr(offsets), F, float(eps), _ptr(seeds),
                                                       _ptr(mask), _ptr(ancestors), _ptr(B_out), _stream(stream)),
           "pf_resample_batched_metropolis_bound")


def pf_debug_tile_weights(logw, n, k, weights, stream=None):
    _check(load().pf_debug_tile_weights(_ptr(logw), n, int(k), _ptr(weights), _stream(stream)),
           "pf_debug_tile_weights")


def pf_set_metropolis_philox_rounds(rounds):
    _check(load().pf_set_metropolis_philox_rounds(int(rounds)), "pf_set_metropolis_philox_rounds")


def pf_get_metropolis_philox_rounds():
    return int(load().pf_get_metropolis_philox_rounds())


def pf_resample_batched_masked(kind, logw, offsets, F, B, seeds, mask, ancestors, stream=None):
    _check(load().pf_resample_batched_masked(kind, _ptr(logw), _ptr(offsets), F, B, _ptr(seeds), _ptr(mask),
                                             _ptr(ancestors), _stream(stream)), "pf_resample_batched_masked")


def pf_lg_init(F, P, D, m0, p0, seed, x, logw, loglik, log_sum, ess, resample, stream=None):
    _check(load().pf_lg_init(F, P, D, m0, p0, seed, _ptr(x), _ptr(logw), _ptr(loglik), _ptr(log_sum), _ptr(ess),
                             _ptr(resample), _stream(stream)), "pf_lg_init")


def pf_lg_step(F, P, D, a, q, r, threshold, y, t, seed, ancestors, x_prev, x_next, logw, loglik, log_sum, ess,
               resample, stream=None):
    _check(load().pf_lg_step(F, P, D, _ptr(a), q, r, threshold, _ptr(y), t, seed, _ptr(ancestors), _ptr(x_prev),
                             _ptr(x_next), _ptr(logw), _ptr(loglik), _ptr(log_sum), _ptr(ess), _ptr(resample),
                             _stream(stream)), "pf_lg_step")


def pf_autotune(kind, logw, P, ancestors, reps=20, stream=None):
    """Returns (min_tile, median microseconds) of the fastest candidate."""
    t = ctypes.c_int(0)
    us = ctypes.c_float(0)
    _check(load().pf_autotune(kind, _ptr(logw), P, _ptr(ancestors), reps, _stream(stream), ctypes.byref(t),
                              ctypes.byref(us)), "pf_autotune")
    return t.value, us.value


def pf_set_min_tile(kind, P, min_tile):
    _check(load().pf_set_min_tile(kind, P, min_tile), "pf_set_min_tile")


def pf_get_min_tile(kind, P) -> int:
    return load().pf_get_min_tile(kind, P)


def pf_reserve(P_max, total_max=0, F_max=0, stream=None):
    _check(load().pf_reserve(P_max, total_max, F_max, _stream(stream)), "pf_reserve")


def pf_get_device_status(stream=None) -> int:
    out = ctypes.c_int(0)
    _check(load().pf_get_device_status(_stream(stream), ctypes.byref(out)), "pf_get_device_status")
    return out.value


def pf_metropolis_B(P, w_max, eps=0.01) -> int:
    return int(load().pf_metropolis_B(P, w_max, eps))


def pf_metropolis_bias(P, w_max, B) -> float:
    return load().pf_metropolis_bias(P, w_max, B)


def pf_permute(ancestors, P, permuted, stream=None):
    _check(load().pf_permute(_ptr(ancestors), P, _ptr(permuted), _stream(stream)), "pf_permute")


def pf_gather_inplace(x, P, row_bytes, permuted, stream=None):
    _check(load().pf_gather_inplace(_ptr(x), P, row_bytes, _ptr(permuted), _stream(stream)), "pf_gather_inplace")


def pf_is_device_accessible(ptr) -> bool:
    return bool(load().pf_is_device_accessible(_ptr(ptr)))


def pf_status_string(status: int) -> str:
    return load().pf_status_string(status).decode()


def pf_set_wait_limit_ns(ns: int):
    _check(load().pf_set_wait_limit_ns(ns), "pf_set_wait_limit_ns")


def pf_debug_skip_publish(tile: int):
    _check(load().pf_debug_skip_publish(tile), "pf_debug_skip_publish")


PF_TRACE_WORDS = 8


def pf_set_trace_buffer(buf, capacity: int = 0):
    """Phase trace of the tile kernels into buf (device, capacity x PF_TRACE_WORDS
    64-bit words); None turns tracing off."""
    _check(load().pf_set_trace_buffer(_ptr(buf), capacity if buf is not None else 0), "pf_set_trace_buffer")


def pf_resample_multinomial_static(logw, P, seed, ancestors, device_status=None, stream=None):
    """Multinomial resampling with the library's fixed scratch array (no allocation)."""
    _check(load().pf_resample_multinomial_static(_ptr(logw), P, seed, _ptr(ancestors), _ptr(device_status),
                                                 _stream(stream)), "pf_resample_multinomial_static")


def pf_probe_l2_random_reads(buf, n, reads_per_thread=256) -> float:
    """Random 4-byte L2 reads per second from the device buffer buf[0..n)."""
    out = ctypes.c_double(0.0)
    _check(load().pf_probe_l2_random_reads(_ptr(buf), n, reads_per_thread, ctypes.byref(out)),
           "pf_probe_l2_random_reads")
    return out.value


def pf_version() -> int:
    return int(load().pf_version())


# The four resamplers by kind, as the batched call numbers them.
RESAMPLERS = {
    PF_MULTINOMIAL: pf_resample_multinomial,
    PF_STRATIFIED: pf_resample_stratified,
    PF_SYSTEMATIC: pf_resample_systematic,
    PF_METROPOLIS: pf_resample_metropolis,
}
