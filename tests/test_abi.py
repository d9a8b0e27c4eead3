"""The C-ABI library builds for sm_103a, loads, and exports every entry point
the headers under include/ declare (no GPU needed; no compute calls are made
here)."""
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", h) for h in sorted(os.listdir(os.path.join(ROOT, "include")))
           if h.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        src = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names.update(re.findall(r"\b(pf_[A-Za-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if not shutil.which("nvcc") and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_1202_6163_gb300 import build, pf
    build.build()
    return pf.load()


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pf_resample_multinomial", "pf_resample_stratified", "pf_resample_systematic",
                     "pf_resample_metropolis", "pf_gather", "pf_ess", "pf_resample_batched",
                     "pf_get_device_status", "pf_metropolis_B", "pf_status_string",
                     "pf_resample_batched_masked", "pf_lg_init", "pf_lg_step"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (pf_\w+)", out))
    missing = [n for n in declared_symbols() if n not in exported]
    assert not missing, missing


def test_binding_covers_the_header(lib):
    from paper_1202_6163_gb300 import pf
    assert sorted(pf.SIGNATURES) == declared_symbols()
    for name in declared_symbols():
        assert hasattr(pf, name)


def test_host_only_entry_points(lib):
    from paper_1202_6163_gb300 import pf
    assert pf.pf_version() >= 100
    assert "domain" in pf.pf_status_string(pf.PF_ERR_DOMAIN)
    # Eq. 5 bound: the library's host copy agrees with the oracle's independent copy
    rng = np.random.default_rng(0)
    for _ in range(500):
        P = int(rng.integers(1, 1 << 24))
        w = float(min(1.0, max(1.0 / P, 10 ** rng.uniform(-7, 0))))
        eps = float(10 ** rng.uniform(-4, -0.5))
        assert pf.pf_metropolis_B(P, w, eps) == oracle.metropolis_B(P, w, eps)
    assert pf.pf_metropolis_B(0, 0.5, 0.01) == -1
    assert pf.pf_metropolis_B(10, 0.0, 0.01) == -1


def test_metropolis_bias_is_the_exact_chain_deviation(lib):
    # host-only: the deviation max_i |(M^B)[i, p_max] - w_max| of the exact
    # transition matrix equals the closed form for every B, and the bound's B
    # is the first with deviation <= eps
    from paper_1202_6163_gb300 import pf
    for lw in ([0.0, -0.5, 1.2, -2.0, 0.3], [0.0, 0.0, 0.0, 1.5], [2.0, -1.0, -1.0, -1.0, -1.0, 0.5]):
        lw = np.array(lw, np.float32)
        P = lw.size
        w = np.exp(lw.astype(np.float64) - lw.max())
        w_max = w.max() / w.sum()
        M = oracle.metropolis_matrix(lw)
        pmax = int(np.argmax(lw))
        MB = np.eye(P)
        for B in range(40):
            dev = np.abs(MB[:, pmax] - w_max).max()
            assert pf.pf_metropolis_bias(P, w_max, B) == pytest.approx(dev, rel=1e-9, abs=1e-15)
            MB = MB @ M
        for eps in (0.1, 0.01, 0.001):
            B = pf.pf_metropolis_B(P, w_max, eps)
            assert pf.pf_metropolis_bias(P, w_max, B) <= eps * (1 + 1e-12)
            assert B == 0 or pf.pf_metropolis_bias(P, w_max, B - 1) > eps
    assert pf.pf_metropolis_bias(0, 0.5, 3) == -1 and pf.pf_metropolis_bias(10, 0.5, -1) == -1
