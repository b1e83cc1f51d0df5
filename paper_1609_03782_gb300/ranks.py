"""Multi-process timing helpers for weak scaling over independent cubes.

Cubes are independent problems, so ranks share nothing on the data path:
every rank filters its own cube(s).  The only collective is the one that
turns per-rank timings into a job-wide figure: the slowest rank's time, and
the sum of the work all ranks did.  Works with any torch.distributed backend
(NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os

import torch
import torch.distributed as dist


def world_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def barrier():
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def _reduce(x: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """The largest value over all ranks (the job's time is the slowest rank's)."""
    return _reduce(x, dist.ReduceOp.MAX, device or "cpu")


def sum_over_ranks(x: float, device=None) -> float:
    return _reduce(x, dist.ReduceOp.SUM, device or "cpu")


def job_rate(units_this_rank: float, seconds_this_rank: float, device=None) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    units = sum_over_ranks(units_this_rank, device)
    secs = max_over_ranks(seconds_this_rank, device)
    return units / secs if secs > 0 else float("inf")
