"""The N > 1 path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank traces its own independent instance of the workload (weak
scaling, no data-path collective); the timing is the max over ranks and the
work the sum.  Here the per-rank work is a small oracle run, so the test
needs no GPU.
"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import workloads as W
        from oracle import oracle as O
        prob = W.silicon_film(n_particles=4000, precision="fp64")
        mine = bench.rank_problem(prob, rank, world)
        r = O.run(mine, n_threads=1)
        segs = bench.sum_over_ranks(r["segments"], dist)
        tmax = bench.max_over_ranks(float(rank + 1), dist)
        ids = [None] * world
        dist.all_gather_object(ids, mine["run"]["instance_id"])
        out[rank] = (mine["run"]["instance_id"], r["segments"], segs, tmax, ids)
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_by_instance():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    (i0, s0, tot0, m0, ids0), (i1, s1, tot1, m1, ids1) = out[0], out[1]
    assert i0 != i1 and sorted(ids0) == sorted([i0, i1])
    assert tot0 == tot1 == s0 + s1
    assert m0 == m1 == 2.0
    # the same shards traced serially give the same work
    import bench
    import workloads as W
    from oracle import oracle as O
    prob = W.silicon_film(n_particles=4000, precision="fp64")
    serial = sum(O.run(bench.rank_problem(prob, r, world), n_threads=1)["segments"] for r in range(world))
    assert serial == s0 + s1
