"""Replicas across GPUs (one process per GPU, launched by torchrun).

The resampling path does not shard one filter without an exchange step, so a
multi-GPU run is independent replicas: every rank resamples its own filters
(or its own single-filter workload) and the ranks meet only to time the job.
These helpers are backend-agnostic (gloo on CPU tensors, nccl on CUDA
tensors) and hold no resampling arithmetic.
"""
from __future__ import annotations

import os


def dist_env():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(n_units: int, rank: int, world: int):
    """The contiguous range [lo, hi) of n_units work units owned by `rank`;
    the ranges of all ranks partition [0, n_units) and differ in size by at most one."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard arguments")
    lo = n_units * rank // world
    hi = n_units * (rank + 1) // world
    return lo, hi


def max_over_ranks(x: float, device=None) -> float:
    """Maximum of x over all ranks of the default process group (x itself
    without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_rate(units_local: float, seconds_local: float, device=None) -> float:
    """Whole-job throughput of a weak-scaling run: all ranks' units divided by
    the slowest rank's time."""
    return sum_over_ranks(units_local, device) / max_over_ranks(seconds_local, device)
