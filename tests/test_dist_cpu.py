"""The multi-process path on CPU ranks (gloo, world size 2): balanced disjoint
shards of a batch, the max-over-ranks job time that bench.py reports, and the
sharded batch solve (dist.solve_sharded) with per-rank results gathered and
compared with the single-rank run.  On CPU ranks the oracle stands in for the
GPU batch solve that bench.py passes as the per-shard solver."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_17850_gb300.dist import max_over_ranks, shard, solve_sharded


def test_shard_is_a_balanced_partition():
    for n in (0, 1, 5, 64, 67):
        for world in (1, 2, 3, 8):
            parts = [shard(n, r, world) for r in range(world)]
            items = [i for p in parts for i in p]
            assert items == list(range(n))
            assert max(len(p) for p in parts) - min(len(p) for p in parts) <= 1
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = max_over_ranks(10.0 + 5.0 * rank)        # per-rank trajectory times
        mine = list(shard(64, rank, world))           # this rank's stacks of a 64-stack batch
        got = [None] * world
        dist.all_gather_object(got, mine)
        out.put((rank, t, got))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_time_and_shards():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, got in res:
        assert t == 15.0                                  # the job time is the slowest rank's
        assert sorted(i for part in got for i in part) == list(range(64))
        assert set(got[0]).isdisjoint(got[1])


def _oracle_shard(idx, insts, who):
    """Per-shard solver for CPU ranks: the oracle's exact steady solve of each instance,
    reduced to a few numbers (and the rank that solved it)."""
    import numpy as np
    from oracle import discretisation as disc, solve as osolve
    out = {}
    for i in idx:
        it = insts[i]
        p = it.power.astype(np.float64)
        T = osolve.steady(it.nx, it.ny, it.stack, p)
        A = disc.assemble(it.nx, it.ny, it.stack)
        rel = osolve.rel_residual(A, T, disc.rhs_steady(it.nx, it.ny, it.stack, p), it.stack.t_amb)
        out[i] = {"sum": float(T.sum()), "max": float(T.max()), "rel_res": rel, "rank": who}
    return out


def _sharded_main(rank, world, port, out):
    import thermal_inputs as ti
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        insts = ti.c4_instances(n=7, scale=16)
        res = solve_sharded(len(insts), lambda idx: _oracle_shard(idx, insts, rank))
        out.put((rank, res))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sharded_batch_equals_single_rank():
    import thermal_inputs as ti
    insts = ti.c4_instances(n=7, scale=16)
    single = solve_sharded(len(insts), lambda idx: _oracle_shard(idx, insts, 0), rank=0, world=1)
    assert sorted(single) == list(range(7)) and all(v["rel_res"] < 1e-10 for v in single.values())
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_sharded_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got in res:
        assert sorted(got) == list(range(7))
        for i in range(7):
            # each instance was solved once, by the rank whose share holds it, with the
            # single-rank result
            assert got[i]["rank"] == (0 if i in shard(7, 0, world) else 1)
            for k in ("sum", "max", "rel_res"):
                assert got[i][k] == single[i][k]


def test_solve_sharded_rejects_a_wrong_shard():
    with pytest.raises(RuntimeError):
        solve_sharded(4, lambda idx: {i + 1: None for i in idx}, rank=0, world=1)
