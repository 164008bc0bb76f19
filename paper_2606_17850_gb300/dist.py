"""Multi-process helpers (one process per GPU).

The solve path shards by independent problems: every rank runs its own
trajectories (replicas) or its own share of a batch of stacks, with no data-path
collective.  Only the timing and the per-instance results are combined: the job
time is the maximum over ranks, and each rank's results are gathered on the host.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional

import torch
import torch.distributed as dist


def shard(n_items: int, rank: int, world: int) -> range:
    """Contiguous, balanced share of n_items for this rank (sizes differ by at most 1)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def rank_world() -> tuple:
    """(rank, world size) of the default process group, (0, 1) without one."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def max_over_ranks(value: float, device=None) -> float:
    """Maximum of a per-rank scalar over the process group (the value itself on one rank)."""
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def solve_sharded(n_items: int, solve_shard: Callable[[List[int]], Dict[int, object]],
                  rank: Optional[int] = None, world: Optional[int] = None) -> Dict[int, object]:
    """Solves a batch of n_items independent instances across the ranks.

    This rank calls ``solve_shard(indices)`` on its contiguous share (``shard``) and
    returns {index: result} for it; the results (small, picklable: statistics,
    checksums) are then gathered from every rank, so each rank returns all n_items
    entries.  Instances never exchange data: the only collective is the host-side
    gather after the solves.
    """
    if rank is None or world is None:
        rank, world = rank_world()
    mine = list(shard(n_items, rank, world))
    local = dict(solve_shard(mine)) if mine else {}
    if set(local) != set(mine):
        raise RuntimeError(f"rank {rank}: solve_shard returned indices {sorted(local)} for its share {mine}")
    if world == 1:
        return local
    parts: List[Optional[Dict[int, object]]] = [None] * world
    dist.all_gather_object(parts, local)
    out: Dict[int, object] = {}
    for p in parts:
        out.update(p or {})
    return out
