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
