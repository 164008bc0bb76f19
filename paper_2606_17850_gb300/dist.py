"""Multi-process helpers (one process per GPU).

The solve path shards by independent problems: every rank runs its own
trajectories (replicas) or its own share of a batch of stacks, with no data-path
collective.  Only the timing is combined: the job time is the maximum over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of n_items for this rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the process group (the value itself on one rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
