"""The multi-process path on CPU ranks (gloo, world size 2): balanced disjoint
shards of a batch and the max-over-ranks job time that bench.py reports."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_17850_gb300.dist import max_over_ranks, shard


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
