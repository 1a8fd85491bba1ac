"""Host-side helpers for running the solver as independent replicas on
several GPUs (one process per GPU, launched by torchrun).

The magnitude path does not shard a single solve: one n = 1e5 problem fits
one GB300.  What spreads over GPUs is independent work -- replicas of a
workload, the (cloud, t) problems of a batch, the t values of a grid -- so
there is no collective on the data path.  The only communication is the
barrier and the max-over-ranks of the measured time.
"""
from __future__ import annotations

import os

import torch


def rank_world():
    """(rank, world size, local rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(items, rank: int, world: int):
    """Round-robin share of `items` for `rank` (disjoint, covering all)."""
    return list(items)[rank::world]


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a scalar over all ranks (identity without a process group)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
