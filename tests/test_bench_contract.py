"""The benchmark's reference arm (the FP64 oracle on the host) prints one JSON
line with the contract's keys; no GPU is needed for it."""
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    t0 = time.perf_counter()
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "3", "--P", "65536"], capture_output=True, text=True, timeout=600,
                       env=dict(os.environ, RANK="0", WORLD_SIZE="1"))
    wall = time.perf_counter() - t0
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert "workload" in d["config"]
    # the step time is measured on the sample that ran, so the timed steps fit inside the run
    assert d["ms_per_step"] * d["steps"] / 1e3 <= d["cpu_baseline"]["seconds_measured"] * 1.01 + 1e-3
    assert d["cpu_baseline"]["seconds_measured"] <= wall
    assert d["ms_per_step_full_P_estimate"] >= d["ms_per_step"]


def test_profiled_counters_follow_their_sources(tmp_path, monkeypatch):
    """The roofline's committed counters (profiles/traffic.json) are used only while
    the hash of the kernel's sources matches the captured build."""
    sys.path.insert(0, ROOT)
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        d = json.load(fh)
    e = d["metropolis"]
    for k in ("sources", "source_hash", "dram_bytes_per_launch", "l1tex_pct_of_peak", "lts_pct_of_peak",
              "l2_hit_pct"):
        assert k in e, k
    if bench.source_hash(e["sources"]) == e["source_hash"]:
        assert bench.profiled_entry("metropolis")["l1tex_pct_of_peak"] == e["l1tex_pct_of_peak"]
        assert bench.profiled_traffic("metropolis") == float(e["dram_bytes_per_launch"])
    # a copy whose hash no longer matches its sources gives nothing
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    for s in e["sources"]:
        dst = root / s
        dst.parent.mkdir(parents=True, exist_ok=True)
        with open(os.path.join(ROOT, s), "rb") as fh:
            dst.write_bytes(fh.read() + b"\n// changed\n")
    (root / "profiles" / "traffic.json").write_text(json.dumps({"metropolis": e}))
    monkeypatch.setattr(bench, "ROOT", str(root))
    assert bench.profiled_entry("metropolis") is None
    assert bench.profiled_traffic("metropolis") is None
