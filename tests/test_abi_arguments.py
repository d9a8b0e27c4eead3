"""Argument errors of the C ABI are caught on the host, before any CUDA call.

Each call below breaks one documented precondition of include/pf.h or
include/pf_lg.h and must return PF_ERR_INVALID.  The calls run in a child
process with no CUDA device visible, so no fake address is ever handed to a
kernel: a check that is missing shows up as PF_ERR_CUDA (the device query
failing), never as a launch.  The last calls are well-formed and, with no
device, must get PF_ERR_CUDA, which shows that the INVALID results above come
from the argument checks and not from the missing device.
"""
import os
import subprocess
import sys
import textwrap

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent(r"""
    import ctypes, json, math
    from paper_1202_6163_gb300 import pf
    lib = pf.load()
    A = 1 << 20            # a 16-byte aligned address that is never dereferenced
    B_ = A + (1 << 16)     # a second one, far enough from A not to overlap small buffers
    MAXC = 1 << 25         # PF_MAX_CUMULATIVE
    calls = []

    def add(name, *args):
        calls.append((name, args))

    for fn in ("pf_resample_systematic", "pf_resample_stratified", "pf_resample_multinomial",
               "pf_resample_metropolis"):
        add(fn, None, 1024, 0, 1, B_, None)          # null logw
        add(fn, A, 1024, 0, 1, None, None)           # null ancestors
        add(fn, A, 0, 0, 1, B_, None)                # P = 0
        add(fn, A, -5, 0, 1, B_, None)               # P < 0
        add(fn, A, (1 << 31), 0, 1, B_, None)        # P > PF_MAX_PARTICLES
        add(fn, A + 2, 1024, 0, 1, B_, None)         # logw not 4-byte aligned
        add(fn, A, 1024, 0, 1, B_ + 1, None)         # ancestors not 4-byte aligned
    add("pf_resample_metropolis", A + 4, 1024, -1, 1, B_, None)   # B < 0 needs 16-byte logw

    add("pf_gather", None, 16, 4, A, 16, B_, None)    # null src
    add("pf_gather", A, 16, 4, None, 16, B_, None)    # null ancestors
    add("pf_gather", A, 0, 4, A, 16, B_, None)        # P_src = 0
    add("pf_gather", A, 16, 4, A, -1, B_, None)       # P_dst < 0
    add("pf_gather", A, 16, 0, A, 16, B_, None)       # row_bytes = 0
    add("pf_gather", A, 16, 6, A, 16, B_, None)       # row_bytes not a multiple of 4
    add("pf_gather", A, 16, 4, B_, 16, A + 32, None)  # dst overlaps src
    add("pf_gather", A + 2, 16, 4, B_, 16, B_ + 4096, None)   # src misaligned

    add("pf_ess", A + 4, 1024, B_, None, None)        # logw not 16-byte aligned
    add("pf_ess", A, 1024, None, None, None)          # null ess_out
    add("pf_ess", A, 0, B_, None, None)               # P = 0

    K = (pf.PF_MULTINOMIAL, pf.PF_STRATIFIED, pf.PF_SYSTEMATIC, pf.PF_METROPOLIS)
    for k in K:
        add("pf_resample_batched", k, A, B_, 0, 0, B_ + 4096, B_ + 8192, None)          # F = 0
        add("pf_resample_batched", k, A, B_, (1 << 24) + 1, 0, B_ + 4096, B_ + 8192, None)
        add("pf_resample_batched", k, A, None, 4, 0, B_ + 4096, B_ + 8192, None)       # null offsets
        add("pf_resample_batched", k, A, B_ + 4, 4, 0, B_ + 4096, B_ + 8192, None)     # offsets misaligned
        add("pf_resample_batched", k, A, B_, 4, 0, B_ + 4100, B_ + 8192, None)         # seeds misaligned
        add("pf_resample_batched", k, A + 2, B_, 4, 0, B_ + 4096, B_ + 8192, None)     # logw misaligned
        add("pf_resample_batched_masked", k, A, B_, 4, 0, B_ + 4096, None, B_ + 8192, None)   # null mask
        add("pf_resample_batched_masked", k, A, B_, 4, 0, B_ + 4096, B_ + 2, B_ + 8192, None)  # mask misaligned
    add("pf_resample_batched", -1, A, B_, 4, 0, B_ + 4096, B_ + 8192, None)            # bad kind
    add("pf_resample_batched", 4, A, B_, 4, 0, B_ + 4096, B_ + 8192, None)
    add("pf_resample_batched_metropolis_bound", A, B_, 4, 0.0, B_ + 4096, None, B_ + 8192, None, None)  # eps = 0
    add("pf_resample_batched_metropolis_bound", A, B_, 4, 1.0, B_ + 4096, None, B_ + 8192, None, None)  # eps = 1
    add("pf_resample_batched_metropolis_bound", A, B_, 4, 0.01, B_ + 4096, None, B_ + 8192, B_ + 2, None)  # B_out
    add("pf_resample_batched_metropolis_bound", A, B_, 0, 0.01, B_ + 4096, None, B_ + 8192, None, None)  # F = 0

    add("pf_reserve", -1, 0, 0, None)
    add("pf_reserve", 0, -1, 0, None)
    add("pf_reserve", 0, 0, -1, None)
    add("pf_get_device_status", None, None)           # null out
    add("pf_set_wait_limit_ns", 0)
    add("pf_debug_tile_weights", A, 0, 0, B_, None)
    add("pf_debug_tile_weights", A, 16, (1 << 24) + 1, B_, None)
    add("pf_set_metropolis_philox_rounds", 8)
    add("pf_set_metropolis_philox_rounds", 0)
    add("pf_set_trace_buffer", A + 4, 64)             # not 8-byte aligned
    add("pf_set_trace_buffer", A, 0)                  # buffer without capacity
    add("pf_set_trace_buffer", None, -1)
    add("pf_permute", None, 16, B_, None)
    add("pf_permute", A, 0, B_, None)
    add("pf_permute", A, 16, A + 8, None)             # overlapping
    add("pf_permute", A, 16, B_ + 2, None)            # misaligned
    add("pf_gather_inplace", A, 16, 2, B_, None)      # row_bytes < 4
    add("pf_gather_inplace", A, 0, 4, B_, None)
    add("pf_gather_inplace", A, 16, 4, None, None)
    add("pf_autotune", pf.PF_METROPOLIS, A, 1024, B_, 5, None, None, None)   # not tunable
    add("pf_autotune", pf.PF_SYSTEMATIC, A, 1024, B_, 0, None, None, None)  # reps < 1
    add("pf_autotune", pf.PF_SYSTEMATIC, A, 1024, B_, 1001, None, None, None)
    add("pf_set_min_tile", pf.PF_METROPOLIS, 1024, 2048)
    add("pf_set_min_tile", pf.PF_SYSTEMATIC, 0, 2048)
    add("pf_set_min_tile", pf.PF_SYSTEMATIC, 1024, 8193)
    add("pf_set_min_tile", pf.PF_SYSTEMATIC, 1024, -1)
    add("pf_probe_l2_random_reads", A, 0, 256, ctypes.byref(ctypes.c_double()))
    add("pf_probe_l2_random_reads", A, 1024, 4, ctypes.byref(ctypes.c_double()))
    add("pf_resample_multinomial_static", A + 4, 1024, 1, B_, None, None)   # 16-byte alignment
    add("pf_resample_multinomial_static", A, 0, 1, B_, None, None)

    X, LW, LL, LS, ES, RS = A, B_, B_ + 4096, B_ + 8192, B_ + 12288, B_ + 16384
    add("pf_lg_init", 2, 64, 6, 0.0, 1.0, 1, X, LW, LL, LS, ES, RS, None)      # D not a multiple of 4
    add("pf_lg_init", 2, 64, 68, 0.0, 1.0, 1, X, LW, LL, LS, ES, RS, None)     # D > 64
    add("pf_lg_init", 0, 64, 4, 0.0, 1.0, 1, X, LW, LL, LS, ES, RS, None)      # F = 0
    add("pf_lg_init", 2, 0, 4, 0.0, 1.0, 1, X, LW, LL, LS, ES, RS, None)       # P = 0
    add("pf_lg_init", 2, 64, 4, 0.0, -1.0, 1, X, LW, LL, LS, ES, RS, None)     # p0 < 0
    add("pf_lg_init", 2, 64, 4, math.nan, 1.0, 1, X, LW, LL, LS, ES, RS, None) # m0 not finite
    add("pf_lg_init", 2, 64, 4, 0.0, 1.0, 1, X + 4, LW, LL, LS, ES, RS, None)  # x not 16-byte aligned
    add("pf_lg_init", 2, 64, 4, 0.0, 1.0, 1, X, None, LL, LS, ES, RS, None)    # null logw
    add("pf_lg_init", 2, 64, 4, 0.0, 1.0, 1, X, LW, LL + 4, LS, ES, RS, None)  # loglik not 8-byte aligned
    XN, AY, AN = A + (1 << 14), B_ + 20480, B_ + 24576
    def step(**kw):
        a = dict(F=2, P=64, D=4, a=AY, q=0.5, r=1.0, th=0.5, y=AY + 64, t=1, seed=1, anc=AN, xp=X, xn=XN,
                 lw=LW, ll=LL, ls=LS, es=ES, rs=RS)
        a.update(kw)
        add("pf_lg_step", a["F"], a["P"], a["D"], a["a"], a["q"], a["r"], a["th"], a["y"], a["t"], a["seed"],
            a["anc"], a["xp"], a["xn"], a["lw"], a["ll"], a["ls"], a["es"], a["rs"], None)
    step(t=0)
    step(q=-1.0)
    step(r=0.0)
    step(q=math.inf)
    step(th=math.nan)
    step(xn=X)                 # x_prev == x_next
    step(xn=X + 16)            # the two state buffers overlap
    step(y=AY + 68)            # y not 16-byte aligned
    step(anc=None)
    step(D=5)

    out = []
    for name, args in calls:
        out.append([name, repr(args), int(getattr(lib, name)(*args))])
    # well-formed calls: with no device they fail in the device query
    wf = [int(lib.pf_resample_systematic(A, 1024, 0, 1, B_, None)),
          int(lib.pf_ess(A, 1024, B_, None, None)),
          int(lib.pf_get_min_tile(pf.PF_METROPOLIS, 1024))]
    # beyond one cooperative launch's tiles the cumulative calls are well formed too
    wf_large = [int(getattr(lib, fn)(A + 4, MAXC, 0, 1, B_ + (1 << 28), None))
                for fn in ("pf_resample_systematic", "pf_resample_stratified", "pf_resample_multinomial")]
    print(json.dumps({"invalid": out, "well_formed": wf, "well_formed_large": wf_large}))
""")


@pytest.fixture(scope="module")
def child_result():
    import shutil
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1202_6163_gb300 import build
    build.build()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", CHILD], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    import json
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_every_broken_precondition_is_rejected_on_the_host(child_result):
    bad = [(name, args, st) for name, args, st in child_result["invalid"] if st != 1]
    assert len(child_result["invalid"]) > 100
    assert not bad, bad


def test_well_formed_calls_reach_the_device_query(child_result):
    st_sys, st_ess, min_tile = child_result["well_formed"]
    assert st_sys == 4 and st_ess == 4      # PF_ERR_CUDA: no device visible
    assert min_tile == -1                   # Metropolis has no tile setting
    assert child_result["well_formed_large"] == [4, 4, 4]  # P + lead beyond PF_MAX_CUMULATIVE: accepted
