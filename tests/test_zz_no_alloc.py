"""sp_sort_cells_static: the allocation-free stable sort of cell keys.

For callers that cannot allocate device memory the library offers one entry
point whose scratch is a file-scope device array.  Here it is called
through the C ABI on caller-owned device buffers, twice in a row with
different inputs (the shared scratch must be cleared by each call), and
its cell offsets and order are checked against the regular indexing path
(sp_set_particles, then sp_get_cell_start / sp_get_particles) on the same
particles.  Integer outputs, so the bar is bit-exact.
"""
import ctypes

import numpy as np
import pytest

from paper_2506_23917_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _keys(cfg, pos):
    """Cell of each particle: floor((x - lo) n / (hi - lo)) per axis, clamped."""
    idx = np.zeros(pos.shape[1], dtype=np.int64)
    mul = 1
    for d in range(cfg["dim"]):
        n = cfg["n"][d]
        inv = float(n) / (cfg["hi"][d] - cfg["lo"][d])
        i = np.floor((pos[d] - cfg["lo"][d]) * inv).astype(np.int64)
        i = np.clip(i, 0, n - 1)
        idx += mul * i
        mul *= n
    return idx.astype(np.uint32)


def _reference(sp, cfg, pos, vel):
    s = sp.Sim(cfg, sp.FP64, capacity=pos.shape[1] + 16)
    s.set_particles(0, pos, vel)
    start = s.cell_start(0)
    p, v, _ = s.particles(0)
    s.close()
    return start, p, v


def _call(sp, torch, keys, ncells):
    dk = torch.from_numpy(keys.astype(np.int32)).cuda()
    dstart = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
    dperm = torch.full((len(keys),), -1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    rc = sp.lib().sp_sort_cells_static(ctypes.c_void_p(dk.data_ptr()), len(keys), ncells,
                                       ctypes.c_void_p(dstart.data_ptr()), ctypes.c_void_p(dperm.data_ptr()),
                                       ctypes.c_void_p(stream.cuda_stream))
    assert rc == 0
    torch.cuda.synchronize()
    return dstart.cpu().numpy().view(np.uint32), dperm.cpu().numpy().view(np.uint32)


@pytest.fixture(scope="module")
def sp():
    import torch

    assert torch.cuda.is_available()
    from paper_2506_23917_gb300 import build

    build.build()
    import paper_2506_23917_gb300 as sp

    return sp


def test_static_sort_matches_indexing_path_twice(sp):
    import torch

    cases = []
    cfg, regions = W.box2d(nx=40, ny=20, ppc=25.0, seed=11)
    pos, vel = W.fill_regions(cfg, regions, 11)
    cases.append((cfg, pos, vel))
    cfg2, regions2 = W.sod(ncell=300, ppc_left=60.0)
    pos2, vel2 = W.fill_regions(cfg2, regions2, 12)
    cases.append((cfg2, pos2, vel2))
    for cfg, pos, vel in cases:  # two calls in a row on the shared scratch
        ncells = int(np.prod(cfg["n"][: cfg["dim"]]))
        keys = _keys(cfg, pos)
        start, perm = _call(sp, torch, keys, ncells)
        ref_start, ref_pos, ref_vel = _reference(sp, cfg, pos, vel)
        np.testing.assert_array_equal(start, ref_start)
        assert start[-1] == pos.shape[1]
        np.testing.assert_array_equal(pos[:, perm], ref_pos)
        np.testing.assert_array_equal(vel[:, perm], ref_vel)


def _stable_reference(keys, ncells):
    """Cell offsets and the stable order of the kept keys (numpy's stable
    argsort: equal keys keep their index order)."""
    k = keys.astype(np.int64)
    keep = k < ncells
    counts = np.bincount(k[keep], minlength=ncells)
    start = np.concatenate([[0], np.cumsum(counts)]).astype(np.uint32)
    idx = np.nonzero(keep)[0]
    order = idx[np.argsort(k[keep], kind="stable")].astype(np.uint32)
    return start, order


def test_static_sort_edge_cases_match_stable_argsort(sp):
    """Removed particles (0xFFFFFFFF), keys past the last cell, empty cells
    and two heavily loaded cells: one of 6000 entries (sorted by a block in
    shared memory) and one of 20000 (sorted by a block in global memory),
    each mixed with a few thousand lightly loaded ones, twice in a row."""
    import torch

    rng = np.random.default_rng(5)
    ncells = 3000
    light = rng.integers(0, ncells, 30000)
    heavy_a = np.full(6000, 17)
    heavy_b = np.full(20000, 2999)
    gone = np.full(500, 0xFFFFFFFF)
    past = rng.integers(ncells, ncells + 50, 300)
    keys = np.concatenate([light, heavy_a, heavy_b, gone, past]).astype(np.uint64)
    for rep in range(2):
        k = keys[rng.permutation(len(keys))].astype(np.uint32)
        start, perm = _call(sp, torch, k, ncells)
        ref_start, ref_order = _stable_reference(k, ncells)
        np.testing.assert_array_equal(start, ref_start)
        np.testing.assert_array_equal(perm[: start[-1]], ref_order)
        assert np.diff(start.astype(np.int64)).max() == 20000 + np.sum(light == 2999)


def test_static_sort_rejects_too_many_cells(sp):
    import torch

    keys = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = sp.lib().sp_sort_cells_static(ctypes.c_void_p(keys.data_ptr()), 4, (1 << 20) + 1,
                                       ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -3
