"""Replica-parallel host logic for several GPUs (one process per GPU).

The hot path has no exchange step between instances: each rank evolves its own
instances (weak scaling) and only scalars cross ranks.  These helpers are the
whole multi-rank surface: which instances a rank owns, the max over ranks of a
rank's time, and the sum over ranks of a count.  They work with any
torch.distributed backend (nccl on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(count: int, rank: int, world: int) -> list[int]:
    """Instance indices owned by `rank`: a round-robin split of range(count)."""
    if not (0 <= rank < world):
        raise ValueError(f"rank {rank} outside world {world}")
    return list(range(rank, count, world))


def _reduce(x: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device="cpu") -> float:
    """The slowest rank's value (the job's time is the slowest rank's)."""
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device="cpu") -> float:
    """Whole-job total of a per-rank count (e.g. amplitude-layer updates)."""
    return _reduce(x, dist.ReduceOp.SUM, device)


def job_throughput(units_local: float, seconds_local: float, device="cpu") -> float:
    """Units processed by all ranks divided by the slowest rank's time."""
    return sum_over_ranks(units_local, device) / max_over_ranks(seconds_local, device)
