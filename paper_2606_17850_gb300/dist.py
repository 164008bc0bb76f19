"""Multi-process helpers (one process per GPU).

The solve path shards by independent problems: every rank runs its own
trajectories (replicas) or its own share of a batch of stacks, with no data-path
collective.  Only the timing and the per-instance results are combined: the job
time is the maximum over ranks, and each rank's results are gathered on the host.

One grid over several ranks is partitioned into y-slabs (all layers of a range of
rows per rank; the few layers of a stack are never split).  The 7-point product is
point-wise (Sec. 4.1), so a slab needs only the boundary rows of its two
y-neighbours: one row per product, and S rows before a chunk of S Chebyshev steps,
which need no reductions (Sec. 4.3) and so no exchange inside the chunk.  The slab
helpers below give the rows, halos and exchange plan of that partition.
"""
from __future__ import annotations

from typing import Callable, Dict, List, Optional, Tuple

import numpy as np
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


# ---------------------------------------------------------------- y-slab partition


def slab_rows(ny: int, rank: int, world: int) -> Tuple[int, int]:
    """Rows [y0, y1) of this rank's slab (contiguous, balanced; every layer)."""
    r = shard(ny, rank, world)
    return r.start, r.stop


def slab_halo(ny: int, rank: int, world: int, width: int) -> Tuple[int, int]:
    """Rows [h0, h1) a slab reads for `width` stencil applications with no exchange
    in between: its own rows and `width` rows of each y-neighbour (1 for a product,
    S for a chunk of S Chebyshev steps).  Every slab must be at least `width` rows
    high, so that a halo comes from the adjacent slab only."""
    if width < 0:
        raise ValueError("width >= 0")
    if world > 1 and min(len(shard(ny, q, world)) for q in range(world)) < width:
        raise ValueError(f"slabs of {ny} rows over {world} ranks are thinner than a {width}-row halo")
    y0, y1 = slab_rows(ny, rank, world)
    return max(0, y0 - width), min(ny, y1 + width)


def halo_exchange_plan(ny: int, rank: int, world: int, width: int) -> List[Tuple[int, Tuple[int, int], Tuple[int, int]]]:
    """This rank's halo exchange before `width` stencil applications: one entry per
    y-neighbour, (peer, rows sent to it [a, b), rows received from it [c, d)).  What
    a rank sends to a peer is what that peer receives from it."""
    h0, h1 = slab_halo(ny, rank, world, width)
    y0, y1 = slab_rows(ny, rank, world)
    plan = []
    if width > 0 and rank > 0:
        plan.append((rank - 1, (y0, min(y1, y0 + width)), (h0, y0)))
    if width > 0 and rank + 1 < world:
        plan.append((rank + 1, (max(y0, y1 - width), y1), (y1, h1)))
    return plan


def slab_cells(nx: int, ny: int, layers: int, a: int, b: int) -> np.ndarray:
    """Indices i = x + nx (y + ny z) of rows [a, b) in every layer, in the order of
    the global vector (layer, then row, then column)."""
    z = np.arange(layers, dtype=np.int64)[:, None, None]
    y = np.arange(a, b, dtype=np.int64)[None, :, None]
    x = np.arange(nx, dtype=np.int64)[None, None, :]
    return (x + nx * (y + ny * z)).reshape(-1)
