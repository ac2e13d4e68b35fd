"""Host-side helpers for running on several GPUs of one node (one process per
GPU, torchrun-style environment).

The sweep does not exchange data between lattices, so nothing on the data
path communicates: a single lattice runs as independent replicas (one seed per
rank), and a parameter scan is split so that each rank sweeps its own subset
of lattices.  Only timing is reduced across ranks.
"""
from __future__ import annotations

import os


def world() -> tuple[int, int, int]:
    """(world_size, rank, local_rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def shard(weights, world_size: int, rank: int) -> list[int]:
    """Indices of the items this rank takes: longest-processing-time-first
    assignment (heaviest item to the least loaded rank, ties to the lower
    rank), so every rank's total weight is within one item of the mean.
    Deterministic: every rank computes the same partition."""
    if world_size < 1 or not 0 <= rank < world_size:
        raise ValueError("bad world_size / rank")
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    load = [0.0] * world_size
    owner = [0] * len(weights)
    for i in order:
        r = min(range(world_size), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += weights[i]
    return [i for i in range(len(weights)) if owner[i] == rank]


def replica_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s independent replica."""
    return seed + 1000 * rank


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of `value` over all ranks (the slowest rank's time); the value
    itself when no process group is running."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, device=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())
