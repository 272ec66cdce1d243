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


class _OracleEngine:
    """The CPU oracle advancing a list of instances one after another."""

    def __init__(self, cfgs, parts):
        import oracle

        self.o = []
        for c, (p, v) in zip(cfgs, parts):
            o = oracle.Oracle(c)
            o.set_particles(p, v)
            self.o.append(o)

    def step(self, n):
        for o in self.o:
            o.step(n)


def _ensemble_instances():
    from paper_2506_23917_gb300 import workloads as W

    return W.batch(n_inst=7, seed=3, Nmin=200, Nmax=1500, Kn_min=1e-3, Kn_max=1e-1, n_steady=2)


def _averages(engine, k):
    return engine.o[k].moments(1)


def _ensemble_rank(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2506_23917_gb300 import ensemble

    res = ensemble.run_partition(_ensemble_instances(), 6, _OracleEngine, _averages, dist)
    q.put((rank, res, ensemble.owned(7, world, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_ensemble_partition_gathers_the_single_process_result():
    """Two gloo ranks each advance their share of a 7-instance ensemble
    (rank r: instances i = r mod 2) with the oracle; the averaged fields
    gathered on rank 0 equal those of one process advancing all seven,
    bit for bit."""
    from paper_2506_23917_gb300 import ensemble

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 31000 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_ensemble_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {r: (res, mine) for r, res, mine in (q.get(timeout=300) for _ in procs)}
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0][1] == [0, 2, 4, 6] and out[1][1] == [1, 3, 5]
    assert out[1][0] is None
    gathered = out[0][0]
    single = ensemble.run_partition(_ensemble_instances(), 6, _OracleEngine, _averages, None)
    assert len(gathered) == len(single) == 7
    for g, s in zip(gathered, single):
        assert g.shape == s.shape
        np.testing.assert_array_equal(g, s)


def test_ensemble_partition_covers_every_instance_once():
    from paper_2506_23917_gb300 import ensemble

    for world in (1, 2, 3, 8):
        seen = sorted(i for r in range(world) for i in ensemble.owned(21, world, r))
        assert seen == list(range(21))
    with pytest.raises(ValueError):
        ensemble.gather_fields({0: np.zeros(2)}, 2)
