"""Multi-process replica logic on CPU (gloo, world size 2): the unit sharding,
the max/sum over ranks behind the whole-job rate, and the reference arm's
rank-0-only rule."""
import os
import socket
import subprocess
import sys

import pytest

from paper_1202_6163_gb300 import replicas

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_shard_partitions():
    for n in (0, 1, 7, 4096, 4097):
        for world in (1, 2, 3, 8):
            ranges = [replicas.shard(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [hi - lo for lo, hi in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        replicas.shard(10, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = replicas.shard(4096, rank, world)
        units = float(hi - lo)
        seconds = 1.0 + rank  # rank 1 is the slow one
        q.put((rank, replicas.max_over_ranks(seconds), replicas.sum_over_ranks(units),
               replicas.job_rate(units, seconds)))
    finally:
        dist.destroy_process_group()


def test_gloo_world_two():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, total, rate in res:
        assert mx == 2.0 and total == 4096.0 and rate == pytest.approx(2048.0)


def test_reference_arm_runs_on_rank_zero_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
