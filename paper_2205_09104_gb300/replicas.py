"""Replica-parallel execution (one process per GPU, independent solves per rank).

The coarsest-level solves shard without any data-path exchange: each rank owns whole
solves (its own right-hand sides, or its share of a batch of operators), so the only
collectives are the timing barrier and the max-over-ranks reduction of the timed region.
"""
from __future__ import annotations

import os


def dist_env() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def rhs_key(key: tuple, rank: int, stream_base: int = 100) -> tuple:
    """Seed key of rank `rank`'s right-hand sides: disjoint streams per rank."""
    return (*key, stream_base + rank)


def shard(count: int, world: int, rank: int) -> range:
    """Contiguous share of `count` independent items (operators of a batch) for `rank`:
    every item on exactly one rank, shares differing by at most one."""
    lo = count * rank // world
    hi = count * (rank + 1) // world
    return range(lo, hi)


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over the ranks of the default process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time (weak scaling)."""
    return world * units_per_rank / (ms_max / 1e3)
