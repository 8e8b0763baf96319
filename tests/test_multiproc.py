"""Host logic of the multi-rank bench path on CPU: world_size 2 over gloo.

Each rank counts its own independent graph (the weak-scaling layout: units are
whole problems, no data-path collective); the only exchange is the final gather of
the per-rank 128-bit counts and the max of the step times.  Here the GPU work is
replaced by the oracle so the exchange itself is exercised on CPU.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist

    import bench
    import oracle as O
    from synth import graphs as G

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = G.gnp(60, 0.4, seed=rank)
    mine = O.count(g, 4)["count"] + (1 << 70) * rank  # exercise limbs above 64 bits
    got = bench.allgather_ints([mine, 7], world)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, [x[0] for x in got], [x[1] for x in got], float(t.item())))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_gather_of_128bit_counts_world2():
    import oracle as O
    from synth import graphs as G
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=240) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want = [O.count(G.gnp(60, 0.4, seed=r), 4)["count"] + (1 << 70) * r for r in range(world)]
    for rank, firsts, seconds, tmax in res:
        assert firsts == want
        assert seconds == [7, 7]
        assert tmax == 2.0
    import bench
    assert bench.combine_counts(want) == sum(want)


def _shard_worker(rank, world, port, q):
    import numpy as np
    import torch.distributed as dist

    import oracle as O
    from paper_2311_13798_gb300 import shard
    from synth import graphs as G

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    g = G.chung_lu(n=3000, w_max=300.0, i0=30.0, planted=5, planted_min=10, planted_max=20, seed=3)
    cg = O.CleanGraph.of(g)
    _, rnd, _ = O.truss_peel(cg)
    vs = O.vset_sizes(cg, rnd)
    out = []
    for k in (4, 6):
        # this rank's shard: the edges whose |VSet| falls in its size range (the GPU runs
        # the same set as the ticket range partition_by_size gives); the oracle's
        # per-edge sub-branch counts stand in for the GPU's shard count
        mine = np.nonzero(np.isin(vs, shard.shard_sizes(vs, k, world, rank)))[0]
        cnt, cs = O.edge_counts(cg, k, rnd, mine) if mine.size else ([], [])
        big = sum(cnt) + (1 << 100) * rank    # exercise limbs above 64 bits
        total, csum = shard.allreduce_result(big, sum(cs) & shard.MASK64)
        out.append((k, int(mine.size), total, csum))
    q.put((rank, out))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_one_graph_split_over_two_ranks():
    """Two ranks split one graph's sub-branches by |VSet| size ranges, count their shares
    and all-reduce (128-bit count as 32-bit limbs, 64-bit checksum): the reduced result
    is the whole graph's."""
    import numpy as np

    import oracle as O
    from paper_2311_13798_gb300 import shard
    from synth import graphs as G
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    g = G.chung_lu(n=3000, w_max=300.0, i0=30.0, planted=5, planted_min=10, planted_max=20, seed=3)
    cg = O.CleanGraph.of(g)
    _, rnd, _ = O.truss_peel(cg)
    vs = O.vset_sizes(cg, rnd)
    for i, k in enumerate((4, 6)):
        want = O.count(g, k)
        for r in range(world):
            kk, n_edges, total, csum = res[r][i]
            assert kk == k and total == want["count"] + (1 << 100) and csum == want["checksum"]
        assert res[0][i][1] > 0 and res[1][i][1] > 0          # both ranks had work
        assert res[0][i][1] + res[1][i][1] == int((vs >= k - 2).sum())
        # the ticket ranges cover the live tickets once, in order
        rng = shard.partition_by_size(vs, k, world)
        assert rng[0][0] == 0 and rng[0][1] == rng[1][0] == res[0][i][1]
        assert rng[1][1] == int((vs >= k - 2).sum())


def test_partition_properties():
    import numpy as np

    from paper_2311_13798_gb300 import shard
    rng = np.random.default_rng(1)
    vs = np.concatenate([rng.integers(0, 30, 5000), rng.integers(100, 250, 40)])
    for k in (3, 5, 7):
        for n in (1, 2, 3, 8):
            parts = shard.partition_by_size(vs, k, n)
            assert len(parts) == n and parts[0][0] == 0 and parts[-1][1] == int((vs >= k - 2).sum())
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [shard.shard_sizes(vs, k, n, r) for r in range(n)]
            assert sum(int(np.isin(vs, s).sum()) for s in sizes) == int((vs >= k - 2).sum())
    assert shard.from_limbs([a + b for a, b in zip(shard.to_limbs(2**127 + 5, 2**64 - 1),
                                                   shard.to_limbs(2**126, 3))]) == (2**127 + 2**126 + 5, 2)
