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


# ----------------------------------------------------------------- one grid in y-slabs

def test_slab_partition_halo_and_exchange_plan():
    """y-slabs cover the rows once; a slab's halo is its rows plus `width` rows of each
    neighbour, received from the adjacent slab only; what a rank sends a peer is what
    the peer receives from it."""
    from paper_2606_17850_gb300.dist import halo_exchange_plan, slab_halo, slab_rows
    for ny in (7, 24, 33):
        for world in (1, 2, 3):
            rows = [slab_rows(ny, r, world) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == ny
            assert all(rows[r][1] == rows[r + 1][0] for r in range(world - 1))
            for width in (0, 1, 2):
                for r in range(world):
                    h0, h1 = slab_halo(ny, r, world, width)
                    y0, y1 = rows[r]
                    assert h0 == max(0, y0 - width) and h1 == min(ny, y1 + width)
                    got = set(range(y0, y1))
                    for peer, (a, b), (c, d) in halo_exchange_plan(ny, r, world, width):
                        assert abs(peer - r) == 1
                        assert set(range(a, b)) <= set(range(y0, y1))      # sends own rows
                        assert set(range(c, d)) <= set(range(*rows[peer]))  # receives the peer's rows
                        back = [e for e in halo_exchange_plan(ny, peer, world, width) if e[0] == r]
                        assert back and back[0][1] == (c, d) and back[0][2] == (a, b)
                        got |= set(range(c, d))
                    assert got == set(range(h0, h1))
    with pytest.raises(ValueError):
        slab_halo(6, 0, 3, 3)  # 2-row slabs cannot supply a 3-row halo


def _slab_main(rank, world, port, out):
    import numpy as np
    import scipy.sparse.linalg as spla
    import thermal_inputs as ti
    from oracle import discretisation as disc
    from paper_2606_17850_gb300.dist import halo_exchange_plan, slab_cells, slab_halo, slab_rows
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        st = ti.stack_c1()
        nx, ny, L, dt = 20, 24, st.L, 1e-4
        A = disc.assemble(nx, ny, st, dt=dt).tocsr()
        D = A.diagonal()
        b = ti.random_vector(A.shape[0], 41)
        y0, y1 = slab_rows(ny, rank, world)
        own = slab_cells(nx, ny, L, y0, y1)
        A_own = A[own, :]

        def exchange(buf, width):
            """Fills buf's halo rows from the y-neighbours (send/recv, neighbours only)."""
            reqs, recvs = [], []
            for peer, (a, bb), (c, d) in halo_exchange_plan(ny, rank, world, width):
                reqs.append(dist.isend(torch.from_numpy(buf[slab_cells(nx, ny, L, a, bb)].copy()), peer))
                t = torch.empty(len(slab_cells(nx, ny, L, c, d)), dtype=torch.float64)
                recvs.append((t, slab_cells(nx, ny, L, c, d), dist.irecv(t, peer)))
            for t, idx, rq in recvs:
                rq.wait()
                buf[idx] = t.numpy()
            for rq in reqs:
                rq.wait()

        n_reduce = [0]

        def allreduce(v):
            n_reduce[0] += 1
            t = torch.tensor(v, dtype=torch.float64)
            dist.all_reduce(t)
            return t.numpy()

        # Jacobi-PCG (Algorithm 1) on the slab: one 1-row exchange per product, the
        # scalars reduced over the ranks
        buf = np.zeros(A.shape[0])
        x = np.zeros(len(own))
        r = b[own].copy()
        z = r / D[own]
        rz, bb2 = allreduce([r @ z, r @ r])
        p = z.copy()
        it, reduces_per_it = 0, set()
        while True:
            before = n_reduce[0]
            buf[own] = p
            exchange(buf, 1)
            q = A_own @ buf
            (pq,) = allreduce([p @ q])
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            z = r / D[own]
            rz_new, rr = allreduce([r @ z, r @ r])
            reduces_per_it.add(n_reduce[0] - before)
            it += 1
            if rr <= 1e-26 * bb2 or it >= 500:
                break
            p = z + (rz_new / rz) * p
            rz = rz_new
        parts = [None] * world
        dist.all_gather_object(parts, (own, x))
        xg = np.zeros(A.shape[0])
        for idx, v in parts:
            xg[idx] = v
        x_ref = spla.spsolve(A.tocsc(), b)
        err = float(np.abs(xg - x_ref).max() / np.abs(x_ref).max())

        # one chunk of S Chebyshev steps: the S-row halos of z_m, z_{m-1}, r exchanged
        # once before it, none during it; the slab's own rows must equal the steps on
        # the whole grid
        S = 4
        c1 = [0.3, 0.5, 0.7, 0.9]
        c2 = [0.8, 0.6, 0.9, 0.7]
        zm, zp, rc = (ti.random_vector(A.shape[0], s) for s in (42, 43, 44))
        gm, gp = zm.copy(), zp.copy()
        for j in range(S):
            gn = gm + c1[j] * (gm - gp) + c2[j] * (rc - A @ gm) / D
            gp, gm = gm, gn
        h0, h1 = slab_halo(ny, rank, world, S)
        ext = slab_cells(nx, ny, L, h0, h1)
        A_ext = A[ext, :][:, ext]
        bufs = []
        for v in (zm, zp, rc):
            bv = np.zeros(A.shape[0])
            bv[own] = v[own]
            exchange(bv, S)
            bufs.append(bv[ext])
        em, ep, er = bufs
        for j in range(S):
            en = em + c1[j] * (em - ep) + c2[j] * (er - A_ext @ em) / D[ext]
            ep, em = em, en
        pos = np.searchsorted(ext, own)
        chunk_equal = bool(np.array_equal(em[pos], gm[own]))
        out.put((rank, err, it, sorted(reduces_per_it), chunk_equal))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_slab_pcg_and_chebyshev_chunk():
    """The one-grid partition run on CPU ranks with the oracle's matrix: PCG on two
    y-slabs (a 1-row exchange per product, two reductions per iteration) reaches the
    single-domain solution, and a chunk of four Chebyshev steps on a slab with its
    4-row halo (exchanged once) gives the whole grid's values on the slab's rows."""
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_slab_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, err, it, per_it, chunk_equal in res:
        assert err <= 1e-10, (rank, err)
        assert it < 500
        assert per_it == [2]          # p^T A p, then (r^T z, r^T r) as one reduction
        assert chunk_equal, rank
    assert res[0][2] == res[1][2]     # both ranks took the same iterations
