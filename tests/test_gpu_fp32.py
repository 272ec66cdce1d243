"""FP32 particle mode on the GPU, checked statistically against the FP64 mode
(which matches the oracle particle for particle, see test_gpu_parity.py).

Bar: time-averaged n, u_x and T within relative L2 1e-2 of the FP64 fields,
and per cell within 3 combined standard errors (batch means over 20
batches) for at least 95 % of the cells.  The two runs use different
random streams (FP32 draws one word per uniform), so only statistics can
agree.
"""
import math

import numpy as np
import pytest

from paper_2506_23917_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    import torch

    assert torch.cuda.is_available()
    from paper_2506_23917_gb300 import build

    build.build()
    import paper_2506_23917_gb300 as sp

    return sp


def _batch_fields(sim, cfg, nbatch, per, R):
    """Run nbatch x per steps, return per-batch mean fields (n, ux, T)."""
    out = []
    prev = None
    for b in range(nbatch):
        sim.step(per)
        m = sim.moments(0, 1)
        _, nsamp = None, None
        N_avg, n, ux, uy, uz, T = m[0], m[1], m[2], m[3], m[4], m[5]
        steps_done = (b + 1) * per
        sN = N_avg * steps_done
        sc = np.stack([ux, uy, uz]) * sN
        sc2 = (3.0 * R * T + ux ** 2 + uy ** 2 + uz ** 2) * sN
        cur = (sN, sc, sc2, n / np.where(N_avg > 0, N_avg, 1))
        if prev is not None:
            dN = cur[0] - prev[0]
            dc = cur[1] - prev[1]
            dc2 = cur[2] - prev[2]
            with np.errstate(invalid="ignore", divide="ignore"):
                bux = dc[0] / dN
                bT = (dc2 / dN - (dc ** 2).sum(axis=0) / dN ** 2) / (3 * R)
            bn = dN / per * cur[3]
            out.append((bn, bux, bT))
        prev = cur
    return out


def _compare(sp, cfg, pos, vel, warm, nbatch, per, min_frac=0.95, reproducible=True, min_n=0.0, prec32=None):
    res = {}
    prec32 = sp.FP32 if prec32 is None else prec32
    for prec in (sp.FP64, prec32):
        c = dict(cfg, n_steady=warm)
        s = sp.Sim(c, prec, capacity=4 * vel.shape[1] + 10000)
        if prec != sp.FP64 and not reproducible:
            s.set_reproducible(False)
        s.set_particles(0, pos, vel)
        s.step(warm)
        b = _batch_fields(s, c, nbatch + 1, per, cfg["R"])
        s.sync()
        assert s.errors()["capacity"] == 0 and s.errors()["cell_cap"] == 0
        res[prec] = b
    stats = {}
    # cells compared: finite in every batch of both runs and, if asked, at a
    # mean density of at least min_n (sparse cells have ill-defined T)
    dense = np.array([x[0] for x in res[sp.FP64]]).mean(axis=0) >= min_n
    for fi, name in enumerate(("n", "ux", "T")):
        a = np.array([x[fi] for x in res[sp.FP64]])
        b = np.array([x[fi] for x in res[prec32]])
        ok = np.all(np.isfinite(a), axis=0) & np.all(np.isfinite(b), axis=0) & dense
        ma, mb = a[:, ok].mean(axis=0), b[:, ok].mean(axis=0)
        se = np.sqrt(a[:, ok].var(axis=0, ddof=1) / len(a) + b[:, ok].var(axis=0, ddof=1) / len(b))
        l2 = np.linalg.norm(mb - ma) / np.linalg.norm(ma)
        noise = np.linalg.norm(se) / np.linalg.norm(ma)  # the L2 the sampling noise alone gives
        within = np.mean(np.abs(mb - ma) <= 3 * se + 1e-300)
        stats[name] = (l2, within, noise)
        assert l2 < 1e-2, (name, l2, "noise", noise)
        assert within >= min_frac, (name, within)
    return stats


@pytest.mark.parametrize("mode", ["FP32", "FP32_CELL32"])
@pytest.mark.parametrize("reproducible", [True, False])
def test_fp32_channel_time_averages_match_fp64(sp, reproducible, mode):
    """Both FP32-state modes (FP64 per-cell arithmetic, and the opt-in
    all-FP32 variant), also with the scatter's arrival order kept inside
    cells: the statistics must not change."""
    cfg, regions = W.box2d(nx=24, ny=12, ppc=200.0, Kn=0.02)
    pos, vel = W.fill_regions(cfg, regions, 3)
    _compare(sp, cfg, pos, vel, warm=300, nbatch=20, per=100, reproducible=reproducible,
             prec32=getattr(sp, mode))


def test_fp32_sod_ensemble_profile_matches_fp64(sp):
    """Unsteady flow: 64 Sod tubes with different seeds run as one batched
    context to t = 0.15 (fixed step), in FP64 and in FP32; the ensemble mean
    density, velocity and temperature profiles must agree (relative L2 1e-2,
    3 standard errors of the ensemble means for >= 95 % of the cells)."""
    R = 64
    cfgs, parts = [], []
    for r in range(R):
        cfg, regions = W.sod(ncell=100, ppc_left=1000.0, lam_left=1e-3, seed=100 + r)
        cfg["dt_fixed"] = 1e-3
        pos, vel = W.fill_regions(cfg, regions, 100 + r)
        cfgs.append(cfg)
        parts.append((pos, vel))
    M = sum(v.shape[1] for _, v in parts)
    prof = {}
    for prec in (sp.FP64, sp.FP32):
        s = sp.Sim(cfgs, prec, capacity=M + 1000)
        for i, (p, v) in enumerate(parts):
            s.set_particles(i, p, v)
        s.step(150)
        s.sync()
        assert s.errors()["capacity"] == 0 and s.errors()["cell_cap"] == 0
        prof[prec] = np.array([s.moments(i, 0)[[1, 2, 5]] for i in range(R)])  # (R, 3, cells)
        s.close()
    for fi, name in enumerate(("n", "ux", "T")):
        a = prof[sp.FP64][:, fi]
        b = prof[sp.FP32][:, fi]
        ma, mb = a.mean(axis=0), b.mean(axis=0)
        se = np.sqrt(a.var(axis=0, ddof=1) / R + b.var(axis=0, ddof=1) / R)
        scale = np.linalg.norm(ma) if name != "ux" else np.linalg.norm(np.abs(ma) + np.sqrt(prof[sp.FP64][:, 2].mean(axis=0)))
        l2 = np.linalg.norm(mb - ma) / scale
        within = np.mean(np.abs(mb - ma) <= 3 * se)
        assert l2 < 1e-2, (name, l2)
        assert within >= 0.95, (name, within)


@pytest.mark.parametrize("mode", ["FP32", "FP32_CELL32"])
def test_fp32_closed_box_conserves_energy(sp, mode):
    """Energy of the FP32 state over 50 steps of a closed homogeneous cell
    (the FP32 store of every collided velocity rounds it: drift at the FP32
    level only)."""
    N = 3000
    cfg = W.homogeneous(N=N, Kn=0.05, omega=0.81)
    pos, vel = W.homogeneous_particles(cfg, N, Tx=2.0, skew=0.1, seed=3)
    s = sp.Sim(cfg, getattr(sp, mode), capacity=2 * N)
    s.set_particles(0, pos, vel)
    e0 = (vel.astype(np.float32).astype(np.float64) ** 2).sum()
    for _ in range(10):
        s.step(5)
        _, v, _ = s.particles(0)
        assert abs((v ** 2).sum() / e0 - 1.0) < 5e-5
    assert s.count(0) == N


@pytest.mark.parametrize("prec_name", ["FP32", "FP64"])
def test_fp32_host_input_gives_the_same_state(prec_name):
    """sp_set_particles_f32 (FP32 host arrays) leaves the same state as
    sp_set_particles given the same values as FP64 arrays, and the same
    state after a few steps."""
    import paper_2506_23917_gb300 as sp
    from paper_2506_23917_gb300 import build

    build.build()
    prec = getattr(sp, prec_name)
    cfg, regions = W.box2d(nx=24, ny=12, ppc=30.0)
    pos, vel = W.fill_regions(cfg, regions, 3)
    pos32, vel32 = pos.astype(np.float32), vel.astype(np.float32)
    a = sp.Sim(cfg, prec, capacity=4 * vel.shape[1])
    b = sp.Sim(cfg, prec, capacity=4 * vel.shape[1])
    a.set_particles(0, pos32.astype(np.float64), vel32.astype(np.float64))
    b.set_particles_f32(0, pos32, vel32)
    for sim in (a, b):
        sim.step(5)
        sim.sync()
    pa, va, ca = a.particles(0)
    pb, vb, cb = b.particles(0)
    np.testing.assert_array_equal(ca, cb)
    np.testing.assert_array_equal(pa, pb)
    np.testing.assert_array_equal(va, vb)
    assert a.dt(0) == b.dt(0)
    a.close()
    b.close()


def test_fp32_o_grid_time_averages_match_fp64(sp):
    """Body-fitted O-grid about a diffuse body (24 x 48 quadrilaterals,
    freestream at speed ratio 2 through the outer polygon): FP32 (FP64
    per-cell arithmetic, scatter order kept) and FP64 give the same
    time-averaged n, u_x and T (relative L2 1e-2, 3 combined standard
    errors for >= 95 % of the cells; 600 particles per mean cell so that the
    sampling noise stays well below the bar)."""
    cfg, regions = W.ogrid_box(nr=24, nt=48, r_out=3.0, growth=1.05, ppc=600.0, Kn=0.05)
    pos, vel = W.fill_regions(cfg, regions, 3)
    _compare(sp, cfg, pos, vel, warm=300, nbatch=20, per=200, reproducible=False)


def _fp32_states():
    """(name, cfg, pos, vel, steps): a channel with a cut-cell body, the same
    channel at ~3 particles per cell (cells of 0, 1, 2, 3 particles), and a
    tube whose cells hold 20000 / 6000 / 1500 / 300 particles (counts past
    the 1/k table)."""
    cfg, regions = W.box2d(nx=24, ny=12, ppc=40.0)
    pos, vel = W.fill_regions(cfg, regions, 3)
    yield "channel", cfg, pos, vel, 20
    cfg, regions = W.box2d(nx=24, ny=12, ppc=3.0)
    pos, vel = W.fill_regions(cfg, regions, 4)
    yield "sparse", cfg, pos, vel, 5
    cfg, pos, vel = W.huge_cells()
    yield "huge", cfg, pos, vel, 2


@pytest.mark.parametrize("case", ["channel", "sparse", "huge"])
def test_fp32_instantaneous_moments_match_oracle_on_the_same_state(sp, case):
    """sp_moments of an FP32 state (FP32-pair sums, FP64 fields from
    reciprocal products, tau from tau_k exp((omega-1) ln T) / n) against the
    oracle's FP64 moments of the same particles widened to FP64.  n and U
    carry only the rounding of the pair sums (relative 1e-10 of the thermal
    speed at 20000 particles a cell); T, q, tau, dt_c and the ratio the FP32
    rounding of the thermal velocities (relative 1e-6).  The write into
    mapped page-locked memory gives the bits of the device-buffer copy."""
    import torch
    import oracle

    name, cfg, pos, vel, steps = next(c for c in _fp32_states() if c[0] == case)
    s = sp.Sim(cfg, sp.FP32, capacity=4 * vel.shape[1] + 1000)
    s.set_particles(0, pos, vel)
    s.step(steps)
    s.sync()
    p, v, _ = s.particles(0)
    m = s.moments(0, 0)
    pinned = torch.zeros((len(sp.FIELDS), s.ncells[0]), dtype=torch.float64).pin_memory()
    s.moments_into(0, 0, pinned.data_ptr())
    np.testing.assert_array_equal(pinned.numpy(), m)
    s.close()
    o = oracle.Oracle(cfg)
    o.set_particles(p, v)
    mo = o.moments(0)
    np.testing.assert_array_equal(m[0], mo[0])  # N
    if case == "sparse":
        assert {0, 1, 2, 3} <= set(np.unique(mo[0]).astype(int))
    if case == "huge":
        assert mo[0].max() > 1024
    vs = np.sqrt(np.max(mo[5][np.isfinite(mo[5])]) * cfg["R"])  # thermal speed scale

    def near(f, rtol, atol=0.0, what=""):
        a, b = m[f], mo[f]
        fin = np.isfinite(b)
        np.testing.assert_array_equal(np.isfinite(a), fin, err_msg=what)
        bad = np.abs(a[fin] - b[fin]) > rtol * np.abs(b[fin]) + atol
        assert not bad.any(), (what, np.flatnonzero(bad)[:5], a[fin][bad][:5], b[fin][bad][:5])

    near(1, 1e-13, what="n")
    for d in range(3):
        near(2 + d, 1e-10, 1e-10 * vs, what=f"U{d}")
    near(5, 1e-6, what="T")
    qs = max(np.max(np.abs(mo[6:9])), 1e-300)
    for d in range(3):
        near(6 + d, 1e-5, 1e-6 * qs, what=f"q{d}")
    near(9, 1e-6, what="tau")
    near(10, 1e-6, what="dt_c")
    # the ratio: tau / dt_c below 1, else 1 (a cell at the switch may flip)
    fin = np.isfinite(mo[9]) & np.isfinite(mo[10])
    edge = fin & (np.abs(mo[9] / np.where(fin, mo[10], 1.0) - 1) < 1e-5)
    ok = ~edge
    np.testing.assert_allclose(m[11][ok], mo[11][ok], rtol=1e-6, atol=0)


def test_fp32_sampled_energy_is_the_post_collision_energy(sp):
    """Step 5 in the FP32 mode keeps sum |c|^2 of each cell from what the
    collision sub-steps conserve (a rescaled cell: the rescale's FP64 sums;
    a cell with DSMC collisions alone: its Step 3 energy).  In a closed tube
    the free flight that follows keeps every speed (specular walls), so
    after one sampled step the sum over cells of N (3 R T + |U|^2) from the
    averaged fields equals sum |c|^2 of the particles then, to the FP32
    rounding of the collided velocities.  Sod tube: continuum cells on the
    left resample, rarefied cells on the right collide only."""
    cfg, regions = W.sod(ncell=100, ppc_left=200.0, lam_left=1e-3, n_steady=0)
    pos, vel = W.fill_regions(cfg, regions, 11)
    s = sp.Sim(cfg, sp.FP32, capacity=2 * vel.shape[1])
    s.set_particles(0, pos, vel)
    s.set_record(True)
    s.step(1)
    s.sync()
    cell4, _, _ = s.record(0)
    assert (cell4[2] > 0).sum() > 10  # rescaled cells
    assert ((cell4[2] == 0) & (cell4[1] > 0)).sum() > 10  # DSMC-only cells with collisions
    m = s.moments(0, 1)
    _, v, _ = s.particles(0)
    s.close()
    N, U, T = m[0], m[2:5], m[5]
    sampled = float(np.sum(N * (3.0 * cfg["R"] * T + np.sum(U ** 2, axis=0))))
    state = float(np.sum(v.astype(np.float64) ** 2))
    assert abs(sampled / state - 1) < 1e-5, (sampled, state)
