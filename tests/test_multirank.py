"""Multi-rank path of the benchmark on CPU (gloo, world size 2): each rank
solves its own shard of scenarios (disjoint scenario ids, weak scaling) and the
whole-job figures are the max of the ranks' times and the sum of their solves.
No GPU and no collective on the solver's data."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = bench.workload_batch(3, rank)
    t_local = 1.0 + rank           # rank 1 is the slower one
    solves_local = 2 + 3 * rank
    t, s = bench.aggregate(t_local, solves_local, dist, "cpu")
    out[rank] = (t, s, float(b.x_init.sum()), int(b.N.sum()))
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregation():
    port = _free_port()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    (t0, s0, x0, n0), (t1, s1, x1, n1) = out[0], out[1]
    assert t0 == t1 == 2.0
    assert s0 == s1 == 7.0
    assert x0 != x1                      # disjoint shards of the workload


def test_shards_are_the_single_rank_batch_split():
    import bench
    from instances import make_workload
    full = make_workload("mixed", n_scen=6)
    r0, r1 = bench.workload_batch(3, 0), bench.workload_batch(3, 1)
    assert np.array_equal(np.concatenate([r0.N, r1.N]), full.N)
    assert np.array_equal(np.concatenate([r0.a, r1.a]), full.a)
