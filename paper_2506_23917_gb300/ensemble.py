"""Independent flow instances of a batched ensemble spread over ranks.

The instances of an ensemble (the 1-D Sod tubes and homogeneous-relaxation
boxes of the batched workload) never exchange particles, so the per-step
path needs no collective: rank r of N advances the instances i = r, r + N,
r + 2N, ... (round robin keeps ranks balanced when instance sizes are drawn
at random), each rank in one context of its own, and only the results are
gathered at the end.

``owned`` gives the partition, ``gather_fields`` collects per-instance
arrays (e.g. the time-averaged moments of ``Sim.moments(i, 1)``) on one rank
in global instance order, and ``run_partition`` is the whole cycle for any
engine that steps a list of instances (the GPU context here; the tests use
the CPU oracle on gloo ranks).
"""
from __future__ import annotations

import numpy as np


def owned(n_inst: int, world: int, rank: int) -> list[int]:
    """Instances of rank `rank` out of `world`: i = rank (mod world)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    return list(range(rank, n_inst, world))


def gather_fields(local: dict, n_inst: int, dist=None, dst: int = 0):
    """Collect {instance: ndarray} of every rank on rank `dst`.

    Returns the list of n_inst arrays in instance order on `dst` (None on the
    other ranks).  The arrays travel as pickled objects, so the gathered
    values are the ranks' values bit for bit.  Without a process group
    (dist None or not initialised) the local dict must hold every instance.
    """
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        parts = [local]
        rank = dst
    else:
        rank = dist.get_rank()
        parts = [None] * dist.get_world_size() if rank == dst else None
        dist.gather_object(local, parts, dst=dst)
    if rank != dst:
        return None
    merged = {}
    for p in parts:
        for i, a in p.items():
            if i in merged:
                raise ValueError(f"instance {i} was advanced by two ranks")
            merged[i] = np.asarray(a)
    missing = [i for i in range(n_inst) if i not in merged]
    if missing:
        raise ValueError(f"instances {missing[:8]} were advanced by no rank")
    return [merged[i] for i in range(n_inst)]


def run_partition(instances, steps: int, make_engine, fields, dist=None, dst: int = 0):
    """Advance this rank's share of `instances` (a list of (cfg, pos, vel))
    by `steps` steps and gather one result array per instance on `dst`.

    make_engine(cfgs, parts) -> engine with .step(n); fields(engine, k)
    returns the result of the engine's k-th instance.  Returns the gathered
    list on `dst`, None elsewhere.
    """
    world = dist.get_world_size() if (dist is not None and dist.is_initialized()) else 1
    rank = dist.get_rank() if world > 1 else dst
    mine = owned(len(instances), world, rank)
    local = {}
    if mine:
        eng = make_engine([instances[i][0] for i in mine], [instances[i][1:] for i in mine])
        eng.step(steps)
        for k, i in enumerate(mine):
            local[i] = fields(eng, k)
    return gather_fields(local, len(instances), dist, dst)
