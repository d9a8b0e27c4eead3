"""Benchmark of the resampling stage on GB300 (one JSON line on rank 0).

Workload: one filter of P = 2^20 particles, log-weights N(0, 1) (float32),
states P x 16 float32.  One step runs the whole single-filter hot path on that
input through the C ABI: ESS, systematic, stratified, multinomial and
Metropolis (B = 32) resampling, and the ancestor gather of the states (by the
systematic ancestors).  value = ancestors produced per second (4 P per step).

Timing: W untimed warm-up steps, then K steps timed on the device with CUDA
events on the launching stream; before each step a short device-side sleep
lets the host queue the step's launches, and L2 is flushed (a 256 MiB write,
outside the timed interval) between steps.  Per-kernel durations come from
events around each launch.  N > 1 (torchrun): independent replicas, one per
GPU, max time over ranks.

--impl reference times the FP64 CPU oracle (the project's reference
implementation of the same method) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

P_DEFAULT = 1 << 20
D_STATE = 16
METRO_B = 32
REF_BUDGET_S = 90.0  # wall time of the reference arm's timed oracle work
N_GRAPHS = 4  # graph captures of the timed step (different seeds, replayed in turn)
SPREAD = 1.0
SEED = 0
METRIC = "ancestors/s at P=2^20 (%HBM peak); batched filters/s vs per-filter launches"
UNIT = "ancestors/s"
L2_FLUSH_BYTES = 256 << 20


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def dist_env():
    from paper_1202_6163_gb300.replicas import dist_env as _d
    return _d()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower() in ("active", "1", "yes"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def source_hash(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_entry(kernel: str):
    """The kernel's counters recorded by the committed ncu summary, if its sources
    have not changed since (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            e = json.load(fh)[kernel]
        return e if source_hash(e["sources"]) == e["source_hash"] else None
    except Exception:
        return None


def profiled_traffic(kernel: str):
    """dram bytes per launch recorded by the committed ncu summary, if the kernel's
    sources have not changed since."""
    e = profiled_entry(kernel)
    try:
        return None if e is None else float(e["dram_bytes_per_launch"]) * float(e.get("scale_to_bench", 1.0))
    except Exception:
        return None


# ----------------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import numpy as np
    import torch

    from paper_1202_6163_gb300 import pf, workloads

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pf.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    if args.only:
        # one secondary leg alone (used for profiling); prints that leg's JSON only
        hbm_peak, _ = load_peaks()
        leg = {"batched": lambda: run_batched_compare(args, pf, torch, dev, stream, hbm_peak),
               "bootstrap": lambda: run_bootstrap(args, pf, torch, dev, hbm_peak),
               "figure2": lambda: run_figure2(args, pf, torch, dev),
               "metropolis": lambda: run_metropolis_sweep(args, pf, torch, dev),
               "inplace": lambda: run_inplace(args, pf, torch, dev),
               "sweep": lambda: run_size_sweep(args, pf, torch, dev, hbm_peak),
               "sorted": lambda: run_sorted_ablation(args, pf, torch, dev),
               "phases": lambda: run_phases(args, pf, torch, dev, stream),
               "single": lambda: run_single(args, pf, torch, dev),
               "config3": lambda: run_config3(args, pf, torch, dev, hbm_peak)}[args.only]()
        if rank == 0:
            print(json.dumps({"leg": args.only, **leg}))
        return
    P = args.P
    lw_h = workloads.gaussian_logw(P, SPREAD, seed=SEED + rank)
    st_h = workloads.states(P, D_STATE, seed=SEED + 1 + rank)
    lw = torch.from_numpy(lw_h).to(dev)
    src = torch.from_numpy(st_h).to(dev)
    dst = torch.empty_like(src)
    anc = {k: torch.empty(P, dtype=torch.int32, device=dev) for k in ("sys", "strat", "multi", "metro")}
    ess = torch.zeros(1, device=dev)
    log_sum = torch.zeros(1, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pf.pf_reserve(P, 0, 0, stream)
    row_bytes = D_STATE * 4
    seed_box = [SEED]

    kernels = ["ess", "systematic", "stratified", "multinomial", "metropolis", "gather"]

    # tile sizes of the single-launch resamplers from the library's autotuner (untimed)
    tuned = {}
    if not args.no_autotune:
        for name, kind in (("systematic", pf.PF_SYSTEMATIC), ("stratified", pf.PF_STRATIFIED),
                           ("multinomial", pf.PF_MULTINOMIAL)):
            tile, us = pf.pf_autotune(kind, lw, P, anc["sys"], 20, stream)
            tuned[name] = {"min_tile": tile, "tuning_median_us": round(us, 2)}

    def step(evs=None, st=None):
        st = stream if st is None else st
        s = seed_box[0]
        seed_box[0] += 1

        def mark(i):
            if evs is not None:
                evs[i].record(st)

        mark(0)
        pf.pf_ess(lw, P, ess, log_sum, st)
        mark(1)
        pf.pf_resample_systematic(lw, P, 0, s, anc["sys"], st)
        mark(2)
        pf.pf_resample_stratified(lw, P, 0, s, anc["strat"], st)
        mark(3)
        pf.pf_resample_multinomial(lw, P, 0, s, anc["multi"], st)
        mark(4)
        pf.pf_resample_metropolis(lw, P, METRO_B, s, anc["metro"], st)
        mark(5)
        pf.pf_gather(src, P, row_bytes, anc["sys"], P, dst, st)
        mark(6)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    if pf.pf_get_device_status(stream) != pf.PF_OK:
        raise RuntimeError("device status not OK after warm-up")

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    per_kernel = {k: 0.0 for k in kernels}
    per_kernel_steps = {k: [] for k in kernels}
    step_ms = []
    total_ms = 0.0
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    ev_sets = []
    for _ in range(args.steps):
        flush.zero_()  # evict L2 (outside the timed interval)
        torch.cuda._sleep(20000)  # let the host queue the step's launches
        evs = [torch.cuda.Event(enable_timing=True) for _ in range(7)]
        step(evs)
        ev_sets.append(evs)
        if len(ev_sets) >= 64:
            torch.cuda.synchronize(dev)
            for e in ev_sets:
                step_ms.append(e[0].elapsed_time(e[6]))
                total_ms += step_ms[-1]
                for i, k in enumerate(kernels):
                    per_kernel[k] += e[i].elapsed_time(e[i + 1])
                    per_kernel_steps[k].append(e[i].elapsed_time(e[i + 1]))
            ev_sets = []
    torch.cuda.synchronize(dev)
    for e in ev_sets:
        step_ms.append(e[0].elapsed_time(e[6]))
        total_ms += step_ms[-1]
        for i, k in enumerate(kernels):
            per_kernel[k] += e[i].elapsed_time(e[i + 1])
            per_kernel_steps[k].append(e[i].elapsed_time(e[i + 1]))
    eager_step_ms, eager_total_ms = step_ms, total_ms
    # the same step as a CUDA graph (the six calls captured on a stream whose
    # workspace is reserved, four captures with different seeds used in turn),
    # replayed with the L2 flushed before each replay: the launch cost of six
    # separate calls goes, the work does not (every replay recomputes all six)
    gs = torch.cuda.Stream(dev)
    pf.pf_reserve(P, 0, 0, gs)
    graphs = []
    with torch.cuda.stream(gs):
        for _ in range(N_GRAPHS):
            step(st=gs)
        gs.synchronize()
        for _ in range(N_GRAPHS):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=gs):
                step(st=gs)
            graphs.append(g)
        for g in graphs:
            g.replay()
        gs.synchronize()
        if world > 1:
            torch.distributed.barrier()
        gs.synchronize()
        pairs = []
        for i in range(args.steps):
            flush.zero_()  # evict L2 (outside the timed interval)
            torch.cuda._sleep(20000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(gs)
            graphs[i % N_GRAPHS].replay()
            e1.record(gs)
            pairs.append((e0, e1))
        gs.synchronize()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in pairs]
    total_ms = sum(step_ms)
    wall = time.perf_counter() - wall0
    time.sleep(0.2)
    clocks = sampler.stop()
    for st in (stream, gs):
        status = pf.pf_get_device_status(st)
        if status != pf.PF_OK:
            raise RuntimeError(f"device status {status} after the timed steps")
    from paper_1202_6163_gb300.replicas import job_rate, max_over_ranks
    ancestors_per_step = 4 * P
    value = job_rate(ancestors_per_step * args.steps, total_ms / 1e3, dev)  # all ranks' units / slowest rank
    total_ms = max_over_ranks(total_ms, dev)
    ms_per_step = total_ms / args.steps
    ms_per_step_eager = max_over_ranks(eager_total_ms, dev) / args.steps

    hbm_peak, peak_kind = load_peaks()
    # algorithmic bytes per launch
    alg = {
        "ess": 4 * P,
        "systematic": 8 * P,
        "stratified": 8 * P,
        "multinomial": 8 * P,
        "metropolis": 8 * P,
        "gather": (2 * row_bytes + 4) * P,
    }
    breakdown = {}
    for k in kernels:
        us = per_kernel[k] / args.steps * 1e3
        gbs = alg[k] / (us * 1e-6) / 1e9
        q = sorted(per_kernel_steps[k])
        breakdown[k] = {"us": round(us, 3), "algorithmic_bytes": alg[k], "achieved_gbs": round(gbs, 1),
                        "hbm_frac": round(gbs / hbm_peak, 4), "share": round(per_kernel[k] / eager_total_ms, 4),
                        "us_p10_p50_p90": [round(1e3 * q[int(f * (len(q) - 1))], 2) for f in (0.1, 0.5, 0.9)]}
    dominant = max(kernels, key=lambda k: per_kernel[k])
    sources = {"systematic": "pf_persistent.cu", "stratified": "pf_persistent.cu",
               "multinomial": "pf_persistent.cu", "metropolis": "pf_metropolis.cu", "gather": "pf_misc.cu",
               "ess": "pf_misc.cu"}
    dk = breakdown[dominant]
    roofline = {"kernel": dominant, "bound": "hbm", "achieved": dk["achieved_gbs"], "peak": hbm_peak,
                "unit": "GB/s", "frac": dk["hbm_frac"], "traffic": profiled_traffic(dominant),
                "peak_source": f"{peak_kind} hbm_gbs (copy)"}
    # Metropolis reads one random log-weight per chain step from L2: its ceiling is
    # the random 4-byte L2 read rate, measured live on this GPU
    l2_rate = pf.pf_probe_l2_random_reads(lw, P, 256)
    steps_per_s = P * METRO_B / (breakdown["metropolis"]["us"] * 1e-6)
    breakdown["metropolis"].update({"steps_per_s": round(steps_per_s, 1),
                                    "l2_random_reads_per_s_peak": round(l2_rate, 1),
                                    "l2_frac": round(steps_per_s / l2_rate, 4)})
    if dominant == "metropolis":
        roofline.update({"bound": "l2", "achieved": round(steps_per_s * 32 / 1e9, 1), "unit": "GB/s",
                         "peak": round(l2_rate * 32 / 1e9, 1), "frac": round(steps_per_s / l2_rate, 4),
                         "peak_source": "measured random 4-byte L2 read rate x 32-byte sectors "
                                        "(pf_probe_l2_random_reads, same run)",
                         "note": "one random 4-byte log-weight read (a 32-byte L2 sector) per chain step; the "
                                 "array is L2-resident, so neither HBM bandwidth nor ALU throughput bounds the "
                                 "chains: the SMs issue about one such sector request per cycle"})
        # the probe's rate against figures that do not come from the probe: one
        # sector request per SM per cycle at this run's SM clock, and ncu's own
        # L1TEX and L2 throughput for the kernel (committed capture)
        n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
        sm_mhz = (clocks or {}).get("sm_mhz")
        ent = profiled_entry("metropolis") or {}
        check = {"sm_count": n_sm, "sm_mhz": sm_mhz,
                 "ncu_l1tex_pct_of_peak": ent.get("l1tex_pct_of_peak"),
                 "ncu_lts_pct_of_peak": ent.get("lts_pct_of_peak"),
                 "ncu_l2_hit_pct": ent.get("l2_hit_pct")}
        if sm_mhz:
            unit_rate = n_sm * sm_mhz * 1e6
            check.update({"one_request_per_sm_cycle_per_s": round(unit_rate, 1),
                          "probe_over_that_rate": round(l2_rate / unit_rate, 4),
                          "kernel_over_that_rate": round(steps_per_s / unit_rate, 4)})
        roofline["peak_check"] = check
    headline = breakdown["systematic"]

    e2e = run_e2e(args, pf, torch, dev, stream, lw_h, st_h, P, row_bytes) if not args.no_e2e else None
    figure2 = None
    if not args.no_figure2:  # the paper's experiment at P = 2^16, compact
        f2 = run_figure2(args, pf, torch, dev, Ps=[1 << 16], R=200)
        figure2 = {"workload": f2["workload"],
                   "by_alpha": {str(r["alpha"]): {"ess_over_P": r["ess_over_P"], "metropolis_B": r["metropolis_B"],
                                                  **{k: {"us": r[k]["us"], "error": r[k]["error"]}
                                                     for k in ("multinomial", "stratified", "systematic",
                                                               "metropolis")}}
                                for r in f2["rows"]}}
    batched = run_batched_compare(args, pf, torch, dev, stream, hbm_peak) if not args.no_batched else None
    bootstrap = run_bootstrap(args, pf, torch, dev, hbm_peak) if not args.no_bootstrap else None
    config3 = run_config3(args, pf, torch, dev, hbm_peak) if not args.no_config3 else None

    launches_per_step = 6 + 0  # one kernel per entry point (the autotuned-B reduction is not used here)
    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5),
        "ms_per_step_p10_p50_p90": [round(sorted(step_ms)[int(f * (len(step_ms) - 1))], 5) for f in (0.1, 0.5, 0.9)],
        "ms_per_step_eager": round(ms_per_step_eager, 5),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "single filter P=2^20, log-weights N(0,1) f32, states Px16 f32; "
                               "ess + systematic + stratified + multinomial + metropolis(B=32) + gather",
                   "P": P, "state_dim": D_STATE, "metropolis_B": METRO_B, "spread": SPREAD,
                   "l2": "flushed between steps (256 MiB write, outside the timed interval)",
                   "autotuned_tiles": tuned,
                   "launch": f"the step's six calls as a CUDA graph ({N_GRAPHS} captures with different seeds, "
                             "replayed in turn); per-kernel times from the same steps run eagerly with CUDA "
                             "events between the calls (ms_per_step_eager)",
                   "parallelism": f"replicas x{world}"},
        "roofline": roofline,
        "headline_systematic": {"ancestors_per_s": round(P / (headline["us"] * 1e-6), 1),
                                "us": headline["us"], "hbm_frac": headline["hbm_frac"],
                                "achieved_gbs": headline["achieved_gbs"]},
        "per_kernel": breakdown,
        "gpu_launches": launches_per_step * args.steps,
        "e2e": e2e,
        "batched": batched,
        "bootstrap": bootstrap,
        "figure2": figure2,
        "config3": config3,
        "clocks": clocks,
        "wall_s": round(wall, 3),
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args)
        if batched is not None:
            out["cpu_baseline"]["batched"] = cpu_baseline_batched()
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(args, pf, torch, dev, stream, lw_h, st_h, P, row_bytes):
    """Same step through the C ABI with host buffers: every step copies its
    inputs from pinned host memory to the device, runs the six calls, and copies
    all of its outputs back, inside the timed interval.  Steps are pipelined
    over three streams with two device buffer sets -- the copy engines move
    step k+1's inputs and step k-1's outputs while the SMs compute step k --
    so the time per step is set by the slowest of the three."""
    lw_p = torch.from_numpy(lw_h).pin_memory()
    st_p = torch.from_numpy(st_h).pin_memory()
    out_anc = torch.empty((4, P), dtype=torch.int32).pin_memory()
    out_st = torch.empty_like(st_p).pin_memory()
    out_ess = torch.empty(1).pin_memory()
    NB = 2
    lw = [torch.empty(P, device=dev) for _ in range(NB)]
    src = [torch.empty((P, D_STATE), device=dev) for _ in range(NB)]
    dst = [torch.empty_like(src[0]) for _ in range(NB)]
    anc = [torch.empty((4, P), dtype=torch.int32, device=dev) for _ in range(NB)]
    ess = [torch.zeros(1, device=dev) for _ in range(NB)]
    s_in, s_cmp, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    pf.pf_reserve(P, 0, 0, s_cmp)
    cmp = s_cmp.cuda_stream
    ev = {k: [torch.cuda.Event() for _ in range(NB)] for k in ("in", "cmp", "out")}
    used = [False] * NB

    def one(k, seed):
        b = k % NB
        with torch.cuda.stream(s_in):
            if used[b]:
                s_in.wait_event(ev["cmp"][b])  # step k - NB has finished reading buffer set b
            lw[b].copy_(lw_p, non_blocking=True)
            src[b].copy_(st_p, non_blocking=True)
            ev["in"][b].record(s_in)
        s_cmp.wait_event(ev["in"][b])
        if used[b]:
            s_cmp.wait_event(ev["out"][b])  # step k - NB's outputs have left the device
        pf.pf_ess(lw[b], P, ess[b], None, cmp)
        pf.pf_resample_systematic(lw[b], P, 0, seed, anc[b][0], cmp)
        pf.pf_resample_stratified(lw[b], P, 0, seed, anc[b][1], cmp)
        pf.pf_resample_multinomial(lw[b], P, 0, seed, anc[b][2], cmp)
        pf.pf_resample_metropolis(lw[b], P, METRO_B, seed, anc[b][3], cmp)
        pf.pf_gather(src[b], P, row_bytes, anc[b][0], P, dst[b], cmp)
        ev["cmp"][b].record(s_cmp)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev["cmp"][b])
            out_anc.copy_(anc[b], non_blocking=True)
            out_st.copy_(dst[b], non_blocking=True)
            out_ess.copy_(ess[b], non_blocking=True)
            ev["out"][b].record(s_out)
        used[b] = True

    steps = max(3, min(args.steps, 50))
    for i in range(4):
        one(i, 1000 + i)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s_in)
    s_in.wait_event(ev["out"][(4 - 1) % NB])  # start from an idle pipeline
    for i in range(steps):
        one(i, 2000 + i)
    e1.record(s_out)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    if pf.pf_get_device_status(s_cmp) != pf.PF_OK:
        raise RuntimeError("device status not OK in the end-to-end run")
    # copy rates alone, for the record (one pinned copy each way)
    t = {}
    for name, (dst_t, src_t, st) in {"h2d": (src[0], st_p, s_in), "d2h": (out_st, dst[0], s_out)}.items():
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(st):
            a.record(st)
            for _ in range(5):
                dst_t.copy_(src_t, non_blocking=True)
            z.record(st)
        torch.cuda.synchronize(dev)
        t[name] = round(5 * src_t.numel() * 4 / (a.elapsed_time(z) * 1e-3) / 1e9, 1)
    h2d = lw_p.numel() * 4 + st_p.numel() * 4
    d2h = out_anc.numel() * 4 + out_st.numel() * 4 + 4
    return {"value": round(4 * P / (ms * 1e-3), 1), "unit": UNIT, "ms_per_step": round(ms, 4),
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "pipeline": "3 streams (copy in, compute, copy out), 2 device buffer sets",
            "pinned_copy_gbs": t}


def run_batched_compare(args, pf, torch, dev, stream, hbm_peak):
    """Batched filters/s (one launch for F filters) against one launch per filter,
    on F = 4096 filters with P_f log-uniform in [256, 65536] and s_f ~ U[0.5, 3].

    The per-filter baseline is timed twice: as F eager calls from Python (host
    submission included, as a caller looping over filters would see it) and as
    one CUDA graph holding the same F launches, replayed (launch count only, no
    host cost); the ratio is reported against both.  Under torchrun the filters
    are sharded: rank r resamples its contiguous range of filters (no collective
    on the data path), filter ids within a call being local, and the whole-job
    rate is all filters over the slowest rank's time."""
    import numpy as np

    from paper_1202_6163_gb300 import replicas, workloads
    rank, world, _ = dist_env()
    F_all = 4096
    off_all, sf = workloads.batched_layout(F=F_all, seed=0)
    lw_all = workloads.batched_logw(off_all, sf, seed=0)
    seeds_all = workloads.batched_seeds(F_all, base=0)
    f_lo, f_hi = replicas.shard(F_all, rank, world)
    F = f_hi - f_lo
    off = (off_all[f_lo:f_hi + 1] - off_all[f_lo]).astype(np.int64)
    lw = torch.from_numpy(np.ascontiguousarray(lw_all[off_all[f_lo]:off_all[f_hi]])).to(dev)
    total = int(off[-1])
    d_off = torch.from_numpy(off).to(dev)
    seeds = torch.from_numpy(np.ascontiguousarray(seeds_all[f_lo:f_hi]).view(np.int64)).to(dev)
    anc = torch.empty(total, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    kinds = {"systematic": pf.PF_SYSTEMATIC, "stratified": pf.PF_STRATIFIED, "multinomial": pf.PF_MULTINOMIAL,
             "metropolis": pf.PF_METROPOLIS}
    singles = {"systematic": pf.pf_resample_systematic, "stratified": pf.pf_resample_stratified,
               "multinomial": pf.pf_resample_multinomial, "metropolis": pf.pf_resample_metropolis}
    # workspace for the largest single filter and the batch, so graph capture allocates nothing
    pf.pf_reserve(int(np.max(np.diff(off))) + 4, total, F, stream)
    by_kind = {}
    reps = 10
    for name, kind in kinds.items():
        B = METRO_B if kind == pf.PF_METROPOLIS else 0
        for _ in range(2):
            pf.pf_resample_batched(kind, lw, d_off, F, B, seeds, anc, stream)
        torch.cuda.synchronize(dev)
        ms = 0.0
        for r in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pf.pf_resample_batched(kind, lw, d_off, F, B, seeds, anc, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms += e0.elapsed_time(e1)
        ms /= reps
        # one launch per filter (each filter's slice of the same buffers; same work, F launches)
        base_lw, base_anc = lw.data_ptr(), anc.data_ptr()
        fn = singles[name]

        def per_filter(st):
            for f in range(F):
                fn(base_lw + 4 * int(off[f]), int(off[f + 1] - off[f]), B, f, base_anc + 4 * int(off[f]), st)

        per_filter(stream)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        per_filter(stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_pf = e0.elapsed_time(e1)
        # the same F launches captured once in a CUDA graph and replayed
        cap = torch.cuda.Stream(dev)
        cap.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(cap):
            per_filter(cap)  # the capture stream's workspace, sized before capture
            pf.pf_reserve(int(np.max(np.diff(off))) + 4, total, F, cap)
            cap.synchronize()
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=cap):
                per_filter(cap)
        g.replay()
        torch.cuda.synchronize(dev)
        ms_g = []
        cur = torch.cuda.current_stream(dev)  # replay() launches on the current stream
        for r in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(cur)
            g.replay()
            e1.record(cur)
            torch.cuda.synchronize(dev)
            ms_g.append(e0.elapsed_time(e1))
        ms_graph = statistics.median(ms_g)
        del g
        if pf.pf_get_device_status(stream) != pf.PF_OK or pf.pf_get_device_status(cap) != pf.PF_OK:
            raise RuntimeError(f"device status not OK after batched {name}")
        ms_job = replicas.max_over_ranks(ms, dev) if world > 1 else ms
        by_kind[name] = {"batched_ms": round(ms, 4), "per_filter_ms": round(ms_pf, 3),
                         "per_filter_graph_ms": round(ms_graph, 3),
                         "batched_filters_per_s": round(F_all / (ms_job * 1e-3), 1),
                         "per_filter_launch_filters_per_s": round(F / (ms_pf * 1e-3), 1),
                         "per_filter_graph_filters_per_s": round(F / (ms_graph * 1e-3), 1),
                         "ratio": round(ms_pf / ms, 2), "ratio_vs_graph": round(ms_graph / ms, 2),
                         "achieved_gbs": round(8 * total / (ms * 1e-3) / 1e9, 1),
                         "hbm_frac": round(8 * total / (ms * 1e-3) / 1e9 / hbm_peak, 4)}
    # Metropolis B = 32 on the opt-in seven-round Philox stream (same work, fewer rounds per step)
    pf.pf_set_metropolis_philox_rounds(7)
    try:
        pf.pf_resample_batched(pf.PF_METROPOLIS, lw, d_off, F, METRO_B, seeds, anc, stream)
        torch.cuda.synchronize(dev)
        ms7 = 0.0
        for r in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            pf.pf_resample_batched(pf.PF_METROPOLIS, lw, d_off, F, METRO_B, seeds, anc, stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms7 += e0.elapsed_time(e1)
        ms7 /= reps
    finally:
        pf.pf_set_metropolis_philox_rounds(10)
    steps_total = total * METRO_B
    by_kind["metropolis_philox7"] = {"batched_ms": round(ms7, 4), "chain_steps_per_s": round(steps_total / (ms7 * 1e-3), 1),
                                     "philox10_chain_steps_per_s":
                                         round(steps_total / (by_kind["metropolis"]["batched_ms"] * 1e-3), 1),
                                     "speedup_vs_philox10": round(by_kind["metropolis"]["batched_ms"] / ms7, 3)}
    # Metropolis with each filter's own B from Eq. 5 (eps = 0.01): the B range and the rate
    B_out = torch.zeros(F, dtype=torch.int32, device=dev)
    pf.pf_resample_batched_metropolis_bound(lw, d_off, F, 0.01, seeds, anc, B_out, None, stream)
    torch.cuda.synchronize(dev)
    ms_b = []
    for r in range(1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pf.pf_resample_batched_metropolis_bound(lw, d_off, F, 0.01, seeds, anc, B_out, None, stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms_b.append(e0.elapsed_time(e1))
    if pf.pf_get_device_status(stream) != pf.PF_OK:
        raise RuntimeError("device status not OK after the bound-driven batched Metropolis")
    Bv = B_out.cpu().numpy().astype(np.int64)
    chain_steps = int(np.sum(np.diff(off) * Bv))
    ms_bound = statistics.median(ms_b)
    by_kind["metropolis_bound"] = {"eps": 0.01, "batched_ms": round(ms_bound, 3),
                                   "batched_filters_per_s": round(F / (ms_bound * 1e-3), 1),
                                   "B_min": int(Bv.min()), "B_median": int(np.median(Bv)), "B_max": int(Bv.max()),
                                   "chain_steps": chain_steps,
                                   "chain_steps_per_s": round(chain_steps / (ms_bound * 1e-3), 1)}
    head = by_kind["systematic"]
    return {"workload": "4096 filters, P_f log-uniform in [256, 65536], log-weights N(0, s_f^2), s_f ~ U[0.5, 3]",
            "F": F_all, "filters_this_rank": F, "ranks": world, "total_particles_this_rank": total,
            "kind": "systematic",
            "batched_filters_per_s": head["batched_filters_per_s"],
            "per_filter_launch_filters_per_s": head["per_filter_launch_filters_per_s"],
            "per_filter_graph_filters_per_s": head["per_filter_graph_filters_per_s"],
            "ratio": head["ratio"], "ratio_vs_graph": head["ratio_vs_graph"], "metropolis_B": METRO_B,
            "by_kind": by_kind,
            "per_filter_baselines": "per_filter_ms: F eager calls from Python (host submission included); "
                                    "per_filter_graph_ms: the same F launches as one CUDA graph, replayed",
            "sharding": "filters split over ranks in contiguous ranges; whole-job rate = all filters / slowest "
                        "rank" if world > 1 else "one rank",
            "l2": "flushed before each timed launch (batched) / pass (per-filter)"}


def run_bootstrap(args, pf, torch, dev, hbm_peak):
    """A whole batched bootstrap filter on the linear-Gaussian test model: 256
    filters of P = 2^16 particles, D = 4, T = 200 steps, resampling (systematic)
    when ESS < P/2.  Each step is two launches -- the masked batched resampler
    and the fused propagate/weight/ESS step -- and the whole run (initial draw
    plus T steps) is one CUDA graph, replayed."""
    import numpy as np

    from paper_1202_6163_gb300 import workloads
    F, P, T, D = 256, 1 << 16, 200, 4
    s = torch.cuda.Stream(dev)
    a = torch.from_numpy(workloads.lg_params(F, seed=0)).to(dev)
    y = torch.from_numpy(workloads.lg_observations(workloads.lg_params(F, seed=0), T=T, D=D, seed=1)).to(dev)
    ss = torch.from_numpy(workloads.lg_step_seeds(T, F, base=1000).view(np.int64)).to(dev)
    off = torch.arange(F + 1, dtype=torch.int64, device=dev) * P
    x = [torch.empty((F, P, D), device=dev) for _ in range(2)]
    lw = torch.empty((F, P), device=dev)
    anc = torch.empty(F * P, dtype=torch.int32, device=dev)
    ll = torch.empty(F, dtype=torch.float64, device=dev)
    ls = torch.empty(F, dtype=torch.float64, device=dev)
    es = torch.empty(F, device=dev)
    rs = torch.empty(F, dtype=torch.int32, device=dev)
    pf.pf_reserve(P, F * P, F, s)
    stream = s.cuda_stream

    def run():
        pf.pf_lg_init(F, P, D, workloads.LG_M0, workloads.LG_P0, 0, x[0], lw, ll, ls, es, rs, stream)
        for t in range(1, T + 1):
            pf.pf_resample_batched_masked(pf.PF_SYSTEMATIC, lw, off, F, 0, ss[t - 1], rs, anc, stream)
            pf.pf_lg_step(F, P, D, a, workloads.LG_Q, workloads.LG_R, 0.5, y[t - 1], t, 0, anc, x[(t - 1) % 2],
                          x[t % 2], lw, ll, ls, es, rs, stream)

    # eager pass with events around every launch: per-kernel times and the resampling rate
    with torch.cuda.stream(s):
        run()
        s.synchronize()
        evs = [None] + [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(T)]
        flags = []
        pf.pf_lg_init(F, P, D, workloads.LG_M0, workloads.LG_P0, 0, x[0], lw, ll, ls, es, rs, stream)
        for t in range(1, T + 1):
            flags.append(rs.clone())
            evs[t][0].record(s)
            pf.pf_resample_batched_masked(pf.PF_SYSTEMATIC, lw, off, F, 0, ss[t - 1], rs, anc, stream)
            evs[t][1].record(s)
            pf.pf_lg_step(F, P, D, a, workloads.LG_Q, workloads.LG_R, 0.5, y[t - 1], t, 0, anc, x[(t - 1) % 2],
                          x[t % 2], lw, ll, ls, es, rs, stream)
            evs[t][2].record(s)
        s.synchronize()
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK after the bootstrap filter")
    res_us = [evs[t][0].elapsed_time(evs[t][1]) * 1e3 for t in range(1, T + 1)]
    step_us = [evs[t][1].elapsed_time(evs[t][2]) * 1e3 for t in range(1, T + 1)]
    frac_resampled = float(torch.stack(flags).float().mean().item())

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        run()
    reps = 5
    with torch.cuda.stream(s):  # replay launches on the current stream
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize(dev)
    run_ms = e0.elapsed_time(e1) / reps
    eager_ms = sum(evs[t][0].elapsed_time(evs[t][2]) for t in range(1, T + 1))
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK after the graph replays")
    # algorithmic bytes of one step launch: read x (16 B), write x (16 B), write
    # logw (4 B), and either read logw (no resampling) or read the ancestor (4 B)
    step_bytes = F * P * (4 * D + 4 * D + 4 + 4)
    st_us = statistics.median(step_us)
    return {"workload": "256 bootstrap filters, linear-Gaussian model D=4, a_f ~ U[0.8,0.99], q=0.1, r=0.5, "
                        "P=2^16 per filter, T=200, systematic resampling when ESS < P/2",
            "F": F, "P": P, "T": T, "graph_nodes": 1 + 2 * T,
            "run_ms": round(run_ms, 3), "ms_per_step": round(run_ms / T, 4),
            "eager_steps_ms": round(eager_ms, 3),
            "particle_steps_per_s": round(F * P * T / (run_ms * 1e-3), 1),
            "fraction_of_filter_steps_resampled": round(frac_resampled, 4),
            "step_kernel_us_median": round(st_us, 2),
            "step_kernel_gbs": round(step_bytes / (st_us * 1e-6) / 1e9, 1),
            "step_kernel_hbm_frac": round(step_bytes / (st_us * 1e-6) / 1e9 / hbm_peak, 4),
            "step_kernel_algorithmic_bytes": step_bytes,
            "masked_resample_us_median": round(statistics.median(res_us), 2),
            "l2": "inputs (256 MiB of states per buffer) larger than L2"}


def run_figure2(args, pf, torch, dev, Ps=None, R=1000):
    """The paper's experiment (Section 3, Figure 2) on this GPU: symmetric
    Dirichlet(alpha) weights, alpha in {10, 1, .1, .01}, P = 256 ... 65536;
    for each resampler the mean error sum_i (o_i/P - w_i/W)^2 over 1000
    resamplings and the runtime of one call.  Metropolis uses B from the Eq. 5
    bound (eps = 0.01).  The 1000 resamplings run as one batched launch of 1000
    copies of the weight set (filter ids give independent streams); the error
    is evaluated with torch ops on the device."""
    import numpy as np

    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    kinds = {"multinomial": (pf.PF_MULTINOMIAL, pf.pf_resample_multinomial),
             "stratified": (pf.PF_STRATIFIED, pf.pf_resample_stratified),
             "systematic": (pf.PF_SYSTEMATIC, pf.pf_resample_systematic),
             "metropolis": (pf.PF_METROPOLIS, pf.pf_resample_metropolis)}
    rows = []
    alphas = [10.0, 1.0, 0.1, 0.01]
    Ps = Ps or [1 << k for k in range(8, 17)]
    for ai, alpha in enumerate(alphas):
        for P in Ps:
            lw_h = workloads.dirichlet_logw(P, alpha, seed=1000 * ai + P)
            lw = torch.from_numpy(lw_h).to(dev)
            p64 = torch.softmax(lw.double(), 0)
            w_max = float(p64.max())
            B = pf.pf_metropolis_B(P, w_max, 0.01)
            row = {"alpha": alpha, "P": P, "ess_over_P": round(float(1.0 / (p64 * p64).sum()) / P, 4),
                   "metropolis_B": B}
            anc1 = torch.empty(P, dtype=torch.int32, device=dev)
            for name, (kind, fn) in kinds.items():
                b = B if kind == pf.PF_METROPOLIS else 0
                # runtime of one call (median of 30, back to back after 3 warm-up calls)
                for i in range(3):
                    fn(lw, P, b, i, anc1, stream)
                evs = [torch.cuda.Event(enable_timing=True) for _ in range(31)]
                for i in range(30):
                    evs[i].record(s)
                    fn(lw, P, b, 100 + i, anc1, stream)
                evs[30].record(s)
                torch.cuda.synchronize(dev)
                us = statistics.median(evs[i].elapsed_time(evs[i + 1]) * 1e3 for i in range(30))
                # error over resamplings: one batched launch of r copies
                r = R
                if kind == pf.PF_METROPOLIS:
                    r = int(max(50, min(R, 2e11 // max(1, P * B))))  # bounded chain steps
                lw_r = lw.repeat(r)
                off = torch.arange(r + 1, dtype=torch.int64, device=dev) * P
                seeds = torch.full((r,), 7 + ai, dtype=torch.int64, device=dev)
                anc = torch.empty(r * P, dtype=torch.int32, device=dev)
                pf.pf_resample_batched(kind, lw_r, off, r, b, seeds, anc, stream)
                fil = torch.arange(r, device=dev, dtype=torch.int64).repeat_interleave(P)
                o = torch.bincount(anc.long() + fil * P, minlength=r * P).view(r, P).double()
                err = ((o / P - p64[None, :]) ** 2).sum(1)
                torch.cuda.synchronize(dev)
                if pf.pf_get_device_status(s) != pf.PF_OK:
                    raise RuntimeError(f"device status not OK in figure-2 {name} P={P} alpha={alpha}")
                row[name] = {"us": round(us, 2), "error": float(err.mean()), "resamplings": r}
                del lw_r, anc, fil, o, err
            rows.append(row)
    return {"workload": "symmetric Dirichlet(alpha) weights, alpha in {10,1,.1,.01}, P = "
                        + ", ".join(f"2^{P.bit_length() - 1}" for P in Ps)
                        + f"; error = mean over {R} resamplings of sum_i (o_i/P - w_i/W)^2; runtime = median single call",
            "rows": rows}


def run_metropolis_sweep(args, pf, torch, dev):
    """Metropolis at P = 2^20 over log-weight spreads s in {0.25, 1, 2, 4} and
    B in {8, 32, 128, 512}: time per call, chain steps/s, and the bias each B
    leaves (pf_metropolis_bias: the exact deviation of the probability of
    ending on the heaviest particle) beside the B that Eq. 5 asks for eps = 0.01."""
    import numpy as np

    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    P = 1 << 20
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    anc = torch.empty(P, dtype=torch.int32, device=dev)
    rows = []
    for sp in (0.25, 1.0, 2.0, 4.0):
        lw_h = workloads.gaussian_logw(P, sp, seed=int(100 * sp))
        lw = torch.from_numpy(lw_h).to(dev)
        w_max = float(torch.softmax(lw.double(), 0).max())
        row = {"s": sp, "w_max": w_max, "B_bound_eps_0.01": pf.pf_metropolis_B(P, w_max, 0.01), "by_B": {}}
        for B in (8, 32, 128, 512):
            for i in range(3):
                pf.pf_resample_metropolis(lw, P, B, i, anc, stream)
            ts = []
            for i in range(10):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(s)
                pf.pf_resample_metropolis(lw, P, B, 10 + i, anc, stream)
                e1.record(s)
                torch.cuda.synchronize(dev)
                ts.append(e0.elapsed_time(e1) * 1e3)
            us = statistics.median(ts)
            row["by_B"][B] = {"us": round(us, 2), "steps_per_s": round(P * B / (us * 1e-6), 1),
                              "bias": pf.pf_metropolis_bias(P, w_max, B)}
        rows.append(row)
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK in the Metropolis sweep")
    return {"workload": "P=2^20, log-weights N(0, s^2), Metropolis B in {8,32,128,512}; L2 flushed before each call",
            "rows": rows}


def run_inplace(args, pf, torch, dev):
    """Out-of-place gather against the in-place form (pf_permute, then
    pf_gather_inplace) at P = 2^20, states P x 16 float32, systematic ancestors
    of N(0, s^2) log-weights (L2 flushed before each timed call)."""
    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    P, D = 1 << 20, 16
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    src = torch.from_numpy(workloads.states(P, D, seed=3)).to(dev)
    dst = torch.empty_like(src)
    anc = torch.empty(P, dtype=torch.int32, device=dev)
    perm = torch.empty_like(anc)
    pf.pf_reserve(P, 0, 0, stream)
    rows = []

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            z.record(s)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(z) * 1e3)
        return statistics.median(ts)

    for sp in (1.0, 2.0):
        lw = torch.from_numpy(workloads.gaussian_logw(P, sp, seed=7)).to(dev)
        pf.pf_resample_systematic(lw, P, 0, 1, anc, stream)
        survivors = int(torch.unique(anc).numel())
        t_gather = timed(lambda: pf.pf_gather(src, P, 4 * D, anc, P, dst, stream))
        t_perm = timed(lambda: pf.pf_permute(anc, P, perm, stream))
        pf.pf_permute(anc, P, perm, stream)
        t_inplace = timed(lambda: pf.pf_gather_inplace(src, P, 4 * D, perm, stream))
        rows.append({"s": sp, "distinct_ancestors": survivors, "gather_us": round(t_gather, 2),
                     "permute_us": round(t_perm, 2), "gather_inplace_us": round(t_inplace, 2),
                     "rows_moved_in_place": P - survivors})
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK in the in-place leg")
    return {"workload": "P=2^20, states Px16 f32, systematic ancestors of N(0,s^2) log-weights", "rows": rows}


def run_single(args, pf, torch, dev):
    """One call kind at one size, `--reps` times (the first three untimed), L2
    flushed before each: the command line the single-kernel ncu captures in
    profiles/ use.  N(0,1) log-weights, states P x 16 f32 for the gather,
    Metropolis B = 32."""
    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    P = args.P
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pf.pf_reserve(P, 0, 0, stream)
    lw = torch.from_numpy(workloads.gaussian_logw(P, SPREAD, seed=5)).to(dev)
    anc = torch.empty(P, dtype=torch.int32, device=dev)
    ess = torch.zeros(1, device=dev)
    if args.kind == "gather":
        st = torch.from_numpy(workloads.states(P, D_STATE, seed=6)).to(dev)
        dst = torch.empty_like(st)
        pf.pf_resample_systematic(lw, P, 0, 1, anc, stream)
    calls = {"ess": lambda: pf.pf_ess(lw, P, ess, None, stream),
             "systematic": lambda: pf.pf_resample_systematic(lw, P, 0, 1, anc, stream),
             "stratified": lambda: pf.pf_resample_stratified(lw, P, 0, 1, anc, stream),
             "multinomial": lambda: pf.pf_resample_multinomial(lw, P, 0, 1, anc, stream),
             "metropolis": lambda: pf.pf_resample_metropolis(lw, P, METRO_B, 1, anc, stream),
             "gather": lambda: pf.pf_gather(st, P, D_STATE * 4, anc, P, dst, stream)}
    fn = calls[args.kind]
    ts = []
    for r in range(max(args.reps, 4)):
        flush.zero_()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        z.record(s)
        torch.cuda.synchronize(dev)
        if r >= 3:
            ts.append(a.elapsed_time(z) * 1e3)
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK")
    return {"kind": args.kind, "P": P, "calls": len(ts) + 3, "median_us": round(statistics.median(ts), 2),
            "l2": "flushed before each call"}


def run_config3(args, pf, torch, dev, hbm_peak):
    """The large single filter: P = 2^24 log-weights N(0,1) with exactly 1% of
    them shifted by +10 (heavy upper tail), states P x 8 f32.  Systematic (20
    calls), Metropolis with B chosen on the device from the Eq. 5 bound (B < 0,
    eps = 0.01; two timed calls of ~1e12 chain steps each) and the gather; L2
    flushed before each call.  The Metropolis rate is set against the random
    4-byte read rate measured on the same 64 MiB vector."""
    import numpy as np

    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    P = 1 << 24
    D = 8
    lw_h = workloads.heavy_tail_logw(P, shift=10.0, frac=0.01, seed=3)
    w64 = np.exp(lw_h.astype(np.float64) - float(lw_h.max()))
    B_host = pf.pf_metropolis_B(P, float(w64.max() / w64.sum()), 0.01)
    lw = torch.from_numpy(lw_h).to(dev)
    st = torch.from_numpy(workloads.states(P, D, seed=4)).to(dev)
    dst = torch.empty_like(st)
    anc = torch.empty(P, dtype=torch.int32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    pf.pf_reserve(P, 0, 0, stream)

    def timed(fn, reps, warm=3):
        for _ in range(warm):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            z.record(s)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(z) * 1e3)
        return statistics.median(ts)

    us_sys = timed(lambda: pf.pf_resample_systematic(lw, P, 0, 1, anc, stream), 20)
    distinct = int(torch.unique(anc).numel())
    us_gather = timed(lambda: pf.pf_gather(st, P, D * 4, anc, P, dst, stream), 20)
    us_met = timed(lambda: pf.pf_resample_metropolis(lw, P, -1, 2, anc, stream), 2, warm=1)
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK in the config-3 leg")
    l2_rate = pf.pf_probe_l2_random_reads(lw, P, 256)
    steps = float(P) * B_host
    return {"workload": "P=2^24 log-weights N(0,1), exactly 1% shifted by +10, f32; states Px8 f32",
            "systematic": {"us": round(us_sys, 2), "ancestors_per_s": round(P / (us_sys * 1e-6), 1),
                           "hbm_frac": round(8 * P / (us_sys * 1e-6) / 1e9 / hbm_peak, 4)},
            "metropolis_bound": {"eps": 0.01, "B_host_bound": int(B_host),
                                 "note": "B chosen on the device from its own FP32 w_max (may differ by one step)",
                                 "ms": round(us_met / 1e3, 2), "chain_steps_per_s": round(steps / (us_met * 1e-6), 1),
                                 "l2_random_reads_per_s": round(l2_rate, 1),
                                 "l2_frac": round(steps / (us_met * 1e-6) / l2_rate, 4)},
            "gather_8f": {"us": round(us_gather, 2),
                          "achieved_gbs": round((2 * D * 4 + 4) * P / (us_gather * 1e-6) / 1e9, 1),
                          "distinct_ancestors": distinct,
                          "note": "by the systematic ancestors: the heavy 1% of particles hold nearly all the "
                                  "weight, so the row reads repeat a few distinct rows and mostly hit L2 (no HBM "
                                  "fraction is given)"},
            "l2": "flushed before each call"}


def run_size_sweep(args, pf, torch, dev, hbm_peak):
    """Every single-filter call over P = 2^10 ... 2^24 (N(0,1) log-weights,
    states P x 16 for the gather): median time of 20 calls with L2 flushed
    before each, ancestors/s, and the fraction of the measured HBM copy rate
    (of the measured random-L2-read rate for Metropolis, B = 32; past 2^22
    the log-weights no longer fit in L2 and the chains read HBM)."""
    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    Pmax = 1 << 24
    pf.pf_reserve(Pmax, 0, 0, stream)
    lw_all = torch.from_numpy(workloads.gaussian_logw(Pmax, 1.0, seed=5)).to(dev)
    anc = torch.empty(Pmax, dtype=torch.int32, device=dev)
    st = torch.empty((Pmax, 16), device=dev)
    dst = torch.empty_like(st)
    ess = torch.zeros(1, device=dev)
    l2_rate = pf.pf_probe_l2_random_reads(lw_all, 1 << 20, 256)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            z.record(s)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(z) * 1e3)
        return statistics.median(ts)

    rows = []
    for k in range(10, 25, 2):
        P = 1 << k
        lw = lw_all[:P]
        row = {"P": P}
        for name, fn in (("systematic", pf.pf_resample_systematic), ("stratified", pf.pf_resample_stratified),
                         ("multinomial", pf.pf_resample_multinomial)):
            us = timed(lambda: fn(lw, P, 0, 1, anc, stream))
            row[name] = {"us": round(us, 2), "ancestors_per_s": round(P / (us * 1e-6), 1),
                         "hbm_frac": round(8 * P / (us * 1e-6) / 1e9 / hbm_peak, 4)}
        us = timed(lambda: pf.pf_resample_metropolis(lw, P, METRO_B, 1, anc, stream))
        row["metropolis_B32"] = {"us": round(us, 2), "ancestors_per_s": round(P / (us * 1e-6), 1),
                                 "l2_frac": round(P * METRO_B / (us * 1e-6) / l2_rate, 4)}
        us = timed(lambda: pf.pf_ess(lw, P, ess, None, stream))
        row["ess"] = {"us": round(us, 2), "hbm_frac": round(4 * P / (us * 1e-6) / 1e9 / hbm_peak, 4)}
        pf.pf_resample_systematic(lw, P, 0, 1, anc, stream)
        us = timed(lambda: pf.pf_gather(st, P, 64, anc, P, dst, stream))
        row["gather_16f"] = {"us": round(us, 2), "hbm_frac": round(132 * P / (us * 1e-6) / 1e9 / hbm_peak, 4)}
        rows.append(row)
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK in the size sweep")
    return {"workload": "single filter, P = 2^10..2^24, log-weights N(0,1) f32, states Px16 f32",
            "l2_random_reads_per_s": round(l2_rate, 1), "hbm_peak_gbs": hbm_peak, "rows": rows}


def run_sorted_ablation(args, pf, torch, dev):
    """The paper's remark on pre-sorting (Section 3: the binary search is faster
    on sorted weights, but the sort costs more than it saves), re-tested here:
    multinomial resampling of N(0, s^2) log-weights as given, against a
    descending sort (torch.sort, a library sort: this is an ablation, not the
    library's path) followed by multinomial resampling of the sorted weights
    (ancestors then map back through the sort's index), with systematic
    resampling for scale.  L2 flushed before each timed call."""
    from paper_1202_6163_gb300 import workloads
    s = torch.cuda.current_stream(dev)
    stream = s.cuda_stream
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(s)
            fn()
            z.record(s)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(z) * 1e3)
        return statistics.median(ts)

    for k in (16, 20, 24):
        P = 1 << k
        pf.pf_reserve(P, 0, 0, stream)
        for sp in (1.0, 3.0):
            lw = torch.from_numpy(workloads.gaussian_logw(P, sp, seed=k)).to(dev)
            anc = torch.empty(P, dtype=torch.int32, device=dev)
            t_multi = timed(lambda: pf.pf_resample_multinomial(lw, P, 0, 1, anc, stream))
            t_sys = timed(lambda: pf.pf_resample_systematic(lw, P, 0, 1, anc, stream))
            with torch.cuda.stream(s):
                srt, idx = torch.sort(lw, descending=True)
                t_sort = timed(lambda: torch.sort(lw, descending=True))
            t_multi_sorted = timed(lambda: pf.pf_resample_multinomial(srt, P, 0, 1, anc, stream))
            with torch.cuda.stream(s):
                t_map = timed(lambda: idx[anc.long()])
            rows.append({"P": P, "s": sp, "multinomial_us": round(t_multi, 2), "systematic_us": round(t_sys, 2),
                         "sort_us": round(t_sort, 2), "multinomial_sorted_us": round(t_multi_sorted, 2),
                         "map_back_us": round(t_map, 2),
                         "sorted_total_us": round(t_sort + t_multi_sorted + t_map, 2)})
    if pf.pf_get_device_status(s) != pf.PF_OK:
        raise RuntimeError("device status not OK in the sorting ablation")
    return {"workload": "single filter, P = 2^16, 2^20, 2^24, log-weights N(0, s^2), s in {1, 3}", "rows": rows}


# ----------------------------------------------------------------------------- oracle arm
def oracle_step_time(Ps, seed, lw=None, st=None):
    """Seconds of one oracle step over a bounded sample: every part of the step -- ESS,
    systematic, stratified, multinomial, Metropolis (B = METRO_B) on all Ps chains, and
    the gather -- on the first Ps log-weights and state rows of the workload.  Nothing
    is sampled within the step or scaled.  lw / st: the workload's arrays (generated
    when not given); only the oracle calls are timed."""
    import oracle
    from paper_1202_6163_gb300 import workloads
    lw = workloads.gaussian_logw(Ps, SPREAD, seed=SEED) if lw is None else lw[:Ps]
    st = workloads.states(Ps, D_STATE, seed=SEED + 1) if st is None else st[:Ps]
    t0 = time.perf_counter()
    oracle.ess(lw)
    a = oracle.systematic(lw, seed)
    oracle.stratified(lw, seed)
    oracle.multinomial(lw, seed)
    oracle.metropolis(lw, METRO_B, seed)
    oracle.gather(st, a)
    return time.perf_counter() - t0


ORACLE_SAMPLE = 1 << 16  # particles of one oracle step (both oracle legs)


def oracle_sample_size(P, steps, budget_s, lw, st):
    """Particles per oracle step: ORACLE_SAMPLE, or fewer (down to 2^12, halving) when
    `steps` steps of it would take longer than budget_s (from one probe step)."""
    Ps = min(P, ORACLE_SAMPLE)
    t = oracle_step_time(Ps, 1, lw, st)
    while Ps > (1 << 12) and steps * t > budget_s:
        Ps //= 2
        t /= 2
    return Ps


def cpu_baseline(args, budget_s=None):
    """The oracle timed on one host core: oracle steps over the first ORACLE_SAMPLE
    particles of the workload, repeated for about budget_s seconds; value = ancestors
    per second of those steps (4 Ps per step), s_per_step = the measured seconds of
    one such step.  A full-P time is only an estimate and has its own key."""
    import oracle
    from paper_1202_6163_gb300 import workloads
    oracle.build()
    budget_s = budget_s if budget_s is not None else args.cpu_budget
    P = args.P
    lw = workloads.gaussian_logw(P, SPREAD, seed=SEED)
    st = workloads.states(P, D_STATE, seed=SEED + 1)
    Ps = min(P, ORACLE_SAMPLE)
    times = []
    wall0 = time.perf_counter()
    while time.perf_counter() - wall0 < budget_s or not times:
        times.append(oracle_step_time(Ps, 100 + len(times), lw, st))
    per_step = sum(times) / len(times)
    return {"value": round(4 * Ps / per_step, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{len(times)} oracle steps, each over the first {Ps} of the P=2^20 log-weights and state rows: "
                      f"ess, systematic, stratified, multinomial, Metropolis (B={METRO_B}) on all {Ps} chains and "
                      f"the gather, all in full; ancestors/s of those steps",
            "particles_per_step": Ps, "steps": len(times), "s_per_step": round(per_step, 5),
            "seconds_measured": round(sum(times), 3),
            "s_per_step_full_P_estimate": round(per_step * P / Ps, 4)}


def run_phases(args, pf, torch, dev, stream):
    """Where the time of one call goes, from the library's phase trace
    (pf_set_trace_buffer): for the single-launch systematic, stratified and
    multinomial calls at P = 2^20, per CTA, the median time of each phase
    (scan, grid-wide wait, carries, assignment or draws) and when the last CTA
    had passed it, in us after the first CTA started, beside the CUDA-event time
    of the call; for the batched systematic call over the 4096 filters, per work
    item, the median phase times and how busy the CTAs were.  Medians over 20
    calls, L2 flushed before each."""
    import numpy as np

    from paper_1202_6163_gb300 import workloads
    W = pf.PF_TRACE_WORDS
    cap = 1 << 14
    buf = torch.zeros(cap * W, dtype=torch.int64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    reps = 20

    def traced(call):
        out = []
        for r in range(reps + 3):
            buf.zero_()
            flush.zero_()
            torch.cuda._sleep(20000)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(r)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            rec = buf.view(cap, W).cpu().numpy()
            rec = rec[rec[:, 0] != 0]
            if r >= 3:
                out.append((e0.elapsed_time(e1) * 1e3, rec))
        if pf.pf_get_device_status(stream) != pf.PF_OK:
            raise RuntimeError("device status not OK in the phase trace")
        return out

    def med(x):
        return round(float(np.median(x)), 2)

    P = args.P
    lw = torch.from_numpy(workloads.gaussian_logw(P, SPREAD, seed=SEED)).to(dev)
    anc = torch.empty(P, dtype=torch.int32, device=dev)
    pf.pf_set_trace_buffer(buf, cap)
    try:
        single = {}
        for name, fn in (("systematic", pf.pf_resample_systematic), ("stratified", pf.pf_resample_stratified),
                         ("multinomial", pf.pf_resample_multinomial)):
            runs = traced(lambda r, fn=fn: fn(lw, P, 0, SEED + r, anc, stream))
            rows = []
            for ev, rec in runs:
                t = (rec[:, :5] - rec[:, 0].min()) / 1e3  # us after the first CTA started
                rows.append([ev, len(rec), t[:, 0].max(), np.median(t[:, 1] - t[:, 0]), t[:, 1].max(),
                             np.median(t[:, 2] - t[:, 1]), t[:, 2].max(), np.median(t[:, 3] - t[:, 2]), t[:, 3].max(),
                             np.median(t[:, 4] - t[:, 3]), t[:, 4].max()])
            m = np.median(np.array(rows), axis=0)
            single[name] = {"event_us": round(m[0], 2), "ctas": int(m[1]), "last_cta_start_us": round(m[2], 2),
                            "scan_us": round(m[3], 2), "all_scanned_us": round(m[4], 2),
                            "wait_us": round(m[5], 2), "all_released_us": round(m[6], 2),
                            "carries_us": round(m[7], 2), "all_carried_us": round(m[8], 2),
                            "assign_us": round(m[9], 2), "last_cta_end_us": round(m[10], 2),
                            "outside_kernel_us": round(m[0] - m[10], 2)}
        F = 4096
        off, sf = workloads.batched_layout(F=F, seed=0)
        blw = torch.from_numpy(workloads.batched_logw(off, sf, seed=0)).to(dev)
        d_off = torch.from_numpy(off).to(dev)
        seeds = torch.from_numpy(workloads.batched_seeds(F, base=0).view(np.int64)).to(dev)
        banc = torch.empty(blw.numel(), dtype=torch.int32, device=dev)
        runs = traced(lambda r: pf.pf_resample_batched(pf.PF_SYSTEMATIC, blw, d_off, F, 0, seeds, banc, stream))
        rows = []
        for ev, rec in runs:
            t = (rec[:, :5] - rec[:, 0].min()) / 1e3
            span = t[:, 4].max()
            ctas = np.unique(rec[:, 5])
            busy = float(np.sum(t[:, 4] - t[:, 0]))
            split = rec[:, 7] != 31
            rows.append([ev, len(rec), len(ctas), span, np.median(t[:, 1] - t[:, 0]),
                         np.median((t[:, 2] - t[:, 1])[split]) if split.any() else 0.0,
                         np.median(t[:, 3] - t[:, 2]), np.median(t[:, 4] - t[:, 3]), busy / (len(ctas) * span)])
        m = np.median(np.array(rows), axis=0)
        batched = {"event_us": round(m[0], 2), "items": int(m[1]), "ctas": int(m[2]), "kernel_span_us": round(m[3], 2),
                   "item_scan_us": round(m[4], 2), "split_item_wait_us": round(m[5], 2),
                   "item_carries_us": round(m[6], 2), "item_assign_us": round(m[7], 2),
                   "cta_busy_fraction": round(m[8], 3)}
    finally:
        pf.pf_set_trace_buffer(None)
    return {"workload": f"single filter P={P}, log-weights N(0,1); batched: 4096 filters, P_f log-uniform in "
                        f"[256, 65536]", "reps": reps, "single": single, "batched_systematic": batched,
            "time_base": "GPU global timer, us after the first CTA started"}


def cpu_baseline_batched():
    """The oracle on the whole 4096-filter workload of the batched leg (every
    filter, each resampler), filters spread over all host cores by threads:
    the oracle's C calls release the interpreter lock, so the threads run in
    parallel.  Filter f uses key seeds[f] and Philox filter id f, as the
    batched call does."""
    import concurrent.futures as cf

    import oracle
    from paper_1202_6163_gb300 import workloads
    oracle.build()
    F = 4096
    off, sf = workloads.batched_layout(F=F, seed=0)
    lw = workloads.batched_logw(off, sf, seed=0)
    seeds = workloads.batched_seeds(F, base=0)
    cores = os.cpu_count() or 1
    calls = {"systematic": lambda x, sd, f: oracle.systematic(x, sd, f),
             "stratified": lambda x, sd, f: oracle.stratified(x, sd, f),
             "multinomial": lambda x, sd, f: oracle.multinomial(x, sd, f),
             "metropolis": lambda x, sd, f: oracle.metropolis(x, METRO_B, sd, f)}
    order = sorted(range(F), key=lambda f: -(off[f + 1] - off[f]))  # largest first, as the GPU plan
    by_kind = {}
    with cf.ThreadPoolExecutor(cores) as ex:
        for name, fn in calls.items():
            def one(f, fn=fn):
                fn(lw[off[f]:off[f + 1]], int(seeds[f]), f)
            t0 = time.perf_counter()
            list(ex.map(one, order))
            dt = time.perf_counter() - t0
            by_kind[name] = {"s": round(dt, 3), "filters_per_s": round(F / dt, 1)}
    return {"value": by_kind["systematic"]["filters_per_s"], "unit": "filters/s", "cores": cores, "kind": "oracle",
            "sample": f"all {F} filters of the batched leg ({int(off[-1])} particles), largest first over "
                      f"{cores} threads; Metropolis B={METRO_B}",
            "by_kind": by_kind}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1202_6163_gb300 import workloads
    oracle.build()
    P = args.P
    lw = workloads.gaussian_logw(P, SPREAD, seed=SEED)
    st = workloads.states(P, D_STATE, seed=SEED + 1)
    # each step runs the oracle over the first Ps particles of the workload (the same
    # sample as the main arm's cpu_baseline unless K + W steps of it would exceed
    # REF_BUDGET_S seconds); the step's time is measured, never scaled
    Ps = oracle_sample_size(P, args.steps + args.warmup, REF_BUDGET_S, lw, st)
    for i in range(args.warmup):
        oracle_step_time(Ps, 10 + i, lw, st)
    times = [oracle_step_time(Ps, 100 + i, lw, st) for i in range(args.steps)]
    per_step = sum(times) / len(times)
    value = 4 * Ps / per_step
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(per_step * 1e3, 3),  # measured: one step over the Ps-particle sample
        "ms_per_step_full_P_estimate": round(per_step * 1e3 * P / Ps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": "single filter P=2^20, log-weights N(0,1) f32, states Px16 f32; "
                               "ess + systematic + stratified + multinomial + metropolis(B=32) + gather",
                   "P": P, "sample_particles_per_step": Ps, "state_dim": D_STATE, "metropolis_B": METRO_B,
                   "spread": SPREAD, "parallelism": "single host thread"},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"each step: the oracle over the first {Ps} of the P=2^20 log-weights and state "
                                   f"rows (ess, systematic, stratified, multinomial, Metropolis on all {Ps} chains, "
                                   f"gather), all in full; ancestors/s of that sample",
                         "seconds_measured": round(sum(times), 3)},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--P", type=int, default=P_DEFAULT)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-bootstrap", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-figure2", action="store_true")
    ap.add_argument("--no-config3", action="store_true")
    ap.add_argument("--only", choices=["batched", "bootstrap", "figure2", "metropolis", "inplace", "sweep", "sorted",
                                       "phases", "single", "config3"],
                    default=None,
                    help="run one secondary leg alone and print its JSON (for profiling)")
    ap.add_argument("--kind", choices=["ess", "systematic", "stratified", "multinomial", "metropolis", "gather"],
                    default="systematic", help="with --only single")
    ap.add_argument("--reps", type=int, default=6, help="with --only single: calls, the first three untimed")
    ap.add_argument("--cpu-budget", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
