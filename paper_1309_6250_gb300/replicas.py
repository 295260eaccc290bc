"""Replica (weak-scaling) runs over several processes, one GPU each.

Positions (walkers) are independent, so N processes each evaluate their own walkers
against their own copy of the tables: no data moves between ranks.  The only
collectives are the ones a measurement needs: a barrier before the timed region and the
maximum of the per-rank elapsed times after it.  Works with any torch.distributed
backend (NCCL on GPUs, gloo on CPUs).
"""
from __future__ import annotations

import os
from typing import Optional, Tuple

POSITION_SEED_STRIDE = 7919   # rank r draws its walkers from seed base + 7919 r


def env_rank_world() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment (defaults: one process)."""
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, ws, local


def position_seed(base_seed: int, rank: int) -> int:
    """Seed of rank `rank`'s walkers: rank 0 keeps the workload's own positions."""
    return base_seed + POSITION_SEED_STRIDE * rank


def rank_positions(lattice, n_pos: int, base_seed: int, rank: int):
    """The walkers a rank evaluates (uniform in the cell, rank-specific seed)."""
    from .inputs import positions
    return positions(lattice, n_pos, position_seed(base_seed, rank))


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """Largest `value` over all ranks (the job's wall time is the slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world / seconds
