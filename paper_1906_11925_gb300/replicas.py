"""Replica bookkeeping for multi-GPU benchmark runs.

The sparse lattice-Boltzmann path runs on one GPU; ``bench.py --gpus N``
(launched with torchrun) runs N independent replicas of the same workload,
one per GPU, with no data exchange between them.  This module holds the
only cross-rank logic: rank discovery from the environment, a barrier, the
maximum of a per-rank time, and the whole-job throughput (the units all
ranks processed over the slowest rank's time).
"""
from __future__ import annotations

import os
from typing import Tuple


def rank_env() -> Tuple[int, int, int]:
    """(rank, local_rank, world_size) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0")),
            int(os.environ.get("WORLD_SIZE", "1")))


def barrier(world: int) -> None:
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The maximum of value over all ranks (value itself for one rank)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Whole-job throughput of N replicas: N * units / slowest time."""
    return world * float(units_per_rank) / float(seconds_max)
