"""Replica bookkeeping for multi-GPU runs (one process per GPU).

The product has no exchange step on one GPU per replica, so N GPUs run N
independent replicas of a workload (each with its own seed); a run's time is
the slowest rank's, and its rate counts the work of all ranks.
"""
from __future__ import annotations

import os


def world() -> tuple:
    """(world_size, rank, local_rank) from the torchrun environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_seed(base: int, rank: int) -> int:
    """Seed of rank `rank`'s replica: distinct per rank, base for rank 0."""
    return base + 1000 * rank


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest `value` over all ranks (value itself without a process group)."""
    if dist is None or not dist.is_initialized():
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world_size: int, seconds: float) -> float:
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return float(units_per_rank) * world_size / seconds
