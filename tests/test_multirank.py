"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2): every rank
advances its own instance (distinct seed, no data-path collective) and the
whole-job figures are the slowest rank's time and the summed updates."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = 10.0 + 5.0 * rank
    upd = 1.0e6 * (rank + 1)
    t, u = bench.reduce_timing(ms, upd, dist, "cpu")
    q.put((rank, t, u, bench.rank_seed(rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_time_and_updates():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, seed in res:
        assert t == 15.0 and u == 3.0e6
    assert res[0][3] != res[1][3]


def test_rank_workloads_are_independent():
    import bench
    from paper_2506_23917_gb300 import workloads as W

    a = bench.make_workload(W, "cylinder", 0.05, bench.rank_seed(0))
    b = bench.make_workload(W, "cylinder", 0.05, bench.rank_seed(1))
    assert a[0]["seed"] != b[0]["seed"]
    assert not np.array_equal(a[2][:, :100], b[2][:, :100])
