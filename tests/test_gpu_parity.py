"""GPU FP64 mode against the oracle, through the C ABI.

The bar (FP64 mode): bit-exact cell offsets, stable-sort permutations,
per-cell candidate / accepted / resampled / acceptance-rejection counts and
resampled-particle sets after every step; positions and velocities within
1e-12 relative element by element (with a floor of 1e-2 of the largest
magnitude for components near zero); Delta t, (sigma c)_max and moment
fields within 1e-12 of their largest magnitude.  Both sides draw the same Philox4x32-10 streams; they
differ only in the order of floating-point sums and in the last bits of
the transcendental functions (CUDA vs the C library), which is what the
1e-12 tolerance absorbs.
"""
import numpy as np
import pytest

import oracle
from paper_2506_23917_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-12


@pytest.fixture(scope="module")
def sp():
    import torch

    assert torch.cuda.is_available(), "GPU test needs CUDA"
    from paper_2506_23917_gb300 import build

    build.build()
    import paper_2506_23917_gb300 as sp

    return sp


def _close(a, b, rtol=RTOL, what=""):
    """Largest difference within rtol of the largest magnitude (fields whose
    entries may cancel to near zero, e.g. heat fluxes)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if a.size == 0:
        return
    scale = max(np.max(np.abs(b)), 1e-300)
    err = np.max(np.abs(a - b))
    assert err <= rtol * scale, f"{what}: max abs err {err:.3e} vs scale {scale:.3e}"


def _close_each(a, b, rtol=RTOL, floor=1e-2, what=""):
    """Element by element: |a_i - b_i| <= rtol (|b_i| + floor max|b|), the
    floor standing for components near zero (a velocity component of a fast
    particle, a coordinate next to an origin)."""
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    assert a.shape == b.shape, (what, a.shape, b.shape)
    if a.size == 0:
        return
    tol = rtol * (np.abs(b) + floor * max(np.max(np.abs(b)), 1e-300))
    bad = np.abs(a - b) > tol
    if bad.any():
        i = np.unravel_index(np.argmax(np.abs(a - b) / tol), a.shape)
        raise AssertionError(f"{what}: {int(bad.sum())} of {a.size} elements off; worst at {i}: "
                             f"{a[i]!r} vs {b[i]!r}")


def compare_state(o, s, inst=0, what=""):
    assert s.count(inst) == o.M, (what, s.count(inst), o.M)
    np.testing.assert_array_equal(s.cell_start(inst), o.cell_start(), err_msg=what + " cell offsets")
    po, vo, co = o.particles()
    ps, vs, cs = s.particles(inst)
    np.testing.assert_array_equal(cs, co, err_msg=what + " cells")
    _close_each(vs, vo, what=what + " velocities")
    _close_each(ps, po, what=what + " positions")
    _close([s.dt(inst)], [o.dt], what=what + " dt")
    _close(s.sigc_max(inst), o.sigc_max(), what=what + " sigc_max")


def compare_record(o, s, inst=0, what=""):
    c_o, r_o, p_o = o.record()
    c_s, r_s, p_s = s.record(inst)
    names = ["candidates", "accepted", "resampled", "AR attempts"]
    for i in range(4):
        np.testing.assert_array_equal(c_s[i], c_o[i], err_msg=f"{what} {names[i]}")
    np.testing.assert_array_equal(r_s, r_o, err_msg=what + " resampled set")
    if s.cfgs[inst] is s.cfgs[0] and len(s.cfgs) == 1:
        np.testing.assert_array_equal(p_s, p_o, err_msg=what + " permutation")
    return c_o


def compare_surface(o, s, inst=0, what=""):
    """Body wall tallies: hit counts exact, momentum and energy given to the
    wall within the tolerance (the device adds them with atomics, in any
    order), and the sampled time."""
    to, t_o = o.surface()
    ts, t_s = s.surface(inst)
    assert to.shape == ts.shape and to.shape[1] > 0
    np.testing.assert_array_equal(ts[0], to[0], err_msg=what + " surface hits")
    for k in range(1, 5):
        _close(ts[k], to[k], what=f"{what} surface tally {k}")
    _close([t_s], [t_o], what=what + " surface time")
    return to


def run_pair(sp, cfg, pos, vel, steps, capacity=None):
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    s = sp.Sim(cfg, sp.FP64, capacity=capacity or max(4 * vel.shape[1], 4096))
    s.set_particles(0, pos, vel)
    s.set_record(True)
    compare_state(o, s, what="initial")
    totals = np.zeros(4, dtype=np.int64)
    for n in range(steps):
        o.step(1)
        s.step(1)
        c = compare_record(o, s, what=f"step {n}")
        totals += c.sum(axis=1)
        compare_state(o, s, what=f"step {n}")
    assert s.errors()["capacity"] == 0 and s.errors()["cell_cap"] == 0
    return o, s, totals


def test_sod_fp64_matches_oracle(sp):
    cfg, regions = W.sod(ncell=200, ppc_left=100.0, lam_left=1e-3, n_steady=10)
    pos, vel = W.fill_regions(cfg, regions, 1)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=25)
    assert tot[0] > 0 and tot[1] > 0 and tot[2] > 0  # both sub-steps ran
    # Step 5/6 time averages and the instantaneous moments
    _close(s.moments(0, 1), o.moments(1), what="averaged moments")
    mi_s, mi_o = s.moments(0, 0), o.moments(0)
    for f in range(mi_o.shape[0]):
        fin = np.isfinite(mi_o[f])
        np.testing.assert_array_equal(np.isfinite(mi_s[f]), fin)
        _close(mi_s[f][fin], mi_o[f][fin], what=f"instant field {f}")


def test_big_cell_hybrid_matches_oracle(sp):
    """One cell above the per-warp staging capacity (big-cell launch), with
    both the DSMC and the Shakhov sub-steps active."""
    N = 1500
    cfg = W.homogeneous(N=N, Kn=0.05, omega=0.81)
    pos, vel = W.homogeneous_particles(cfg, N, Tx=2.0, skew=0.1, seed=3)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=6)
    assert tot[0] > 0 and tot[2] > 0


def test_channel_with_body_inflow_outflow_matches_oracle(sp):
    cfg, regions = W.box2d(nx=24, ny=12, ppc=30.0)
    cfg.update(n_surf=24, n_steady=4)
    pos, vel = W.fill_regions(cfg, regions, 3)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=12)
    t = o.totals()
    assert t["injected"] > 0 and t["removed"] > 0
    tal = compare_surface(o, s, what="channel")
    assert tal[0].sum() > 100


def test_sphere_box_matches_oracle(sp):
    cfg, regions = W.box3d(n=(12, 8, 8), ppc=12.0)
    cfg.update(n_surf=12, n_steady=1)
    pos, vel = W.fill_regions(cfg, regions, 5)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=6)
    assert o.totals()["injected"] > 0
    tal = compare_surface(o, s, what="sphere")
    assert tal[0].sum() > 50


def test_jet_orifice_matches_oracle(sp):
    """Sonic jet: inflow only through an orifice window of the left face
    (diffuse lips elsewhere), vacuum outflow, and a dense plenum block whose
    cells exceed the per-warp staging capacity (big-cell launch)."""
    cfg, regions = W.jet(scale=1.0 / 16, ppc=200.0, n_steady=2)
    pos, vel = W.fill_regions(cfg, regions, 7)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=6)
    t = o.totals()
    assert t["injected"] > 0 and t["removed"] > 0
    assert np.diff(o.cell_start().astype(np.int64)).max() > 512


def test_carried_remainder_ntc_matches_oracle(sp):
    """Bird's carried NTC remainder (per-cell state across steps) in place
    of stochastic rounding: candidate counts bit-exact every step."""
    cfg, regions = W.sod(ncell=60, ppc_left=60.0, lam_left=1e-3)
    cfg["ntc_carry"] = 1
    pos, vel = W.fill_regions(cfg, regions, 4)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=10)
    assert tot[0] > 0


@pytest.mark.parametrize("mode", [W.MODE_DSMC, W.MODE_SHAKHOV])
def test_forced_modes_match_oracle(sp, mode):
    cfg, regions = W.sod(ncell=60, ppc_left=60.0, lam_left=1e-3, mode=mode)
    pos, vel = W.fill_regions(cfg, regions, 2)
    run_pair(sp, cfg, pos, vel, steps=8)


def test_tiny_cells_edge_cases(sp):
    """Cells with 0, 1, 2 (DSMC only) and 3 (Shakhov allowed) particles and
    an empty tail of the domain."""
    cfg = W.base_config(1, [12], [0.0], [1.2])
    cfg.update(d_ref=0.3, mu_ref=0.02, Fn=0.05, dt_fixed=0.02, sigc_T0=1.0)
    counts = [0, 1, 2, 3, 0, 5, 2, 1, 3, 0, 0, 0]
    rng = np.random.default_rng(9)
    xs, vs = [], []
    for k, n in enumerate(counts):
        xs.append(0.1 * k + 0.1 * rng.random(n))
        vs.append(rng.normal(0, 1, (3, n)))
    pos = np.concatenate(xs)[None, :]
    vel = np.concatenate(vs, axis=1)
    run_pair(sp, cfg, pos, vel, steps=10)


def test_batch_instances_match_separate_oracles(sp):
    insts = W.batch(n_inst=4, Nmin=300, Nmax=3000, Kn_min=1e-3, Kn_max=1e-1, n_steady=3)
    cfgs = [c for c, _, _ in insts]
    s = sp.Sim(cfgs, sp.FP64, capacity=40000)
    s.set_record(True)
    os_ = []
    for i, (c, p, v) in enumerate(insts):
        s.set_particles(i, p, v)
        o = oracle.Oracle(c)
        o.set_particles(p, v)
        os_.append(o)
    for n in range(6):
        s.step(1)
        for i, o in enumerate(os_):
            o.step(1)
            compare_record(o, s, inst=i, what=f"inst {i} step {n}")
            compare_state(o, s, inst=i, what=f"inst {i} step {n}")
    for i, o in enumerate(os_):
        _close(s.moments(i, 1), o.moments(1), what=f"inst {i} averages")


def test_empty_instance_with_fixed_step(sp):
    cfg = W.base_config(1, [8], [0.0], [1.0])
    cfg.update(dt_fixed=0.01)
    s = sp.Sim(cfg, sp.FP64, capacity=64)
    s.set_particles(0, np.zeros((1, 0)), np.zeros((3, 0)))
    s.step(3)
    s.sync()
    assert s.count(0) == 0


def test_capacity_overflow_is_reported(sp):
    cfg, regions = W.box2d(nx=16, ny=8, ppc=20.0)
    pos, vel = W.fill_regions(cfg, regions, 3)
    s = sp.Sim(cfg, sp.FP64, capacity=vel.shape[1] + 5)
    s.set_particles(0, pos, vel)
    s.step(4)
    with pytest.raises(sp.SpError) as e:
        s.sync()
    assert e.value.code == -3
    assert s.errors()["capacity"] > 0
    small = sp.Sim(cfg, sp.FP64, capacity=10)
    with pytest.raises(sp.SpError) as e:
        small.set_particles(0, pos, vel)
    assert e.value.code == -3


def test_moments_and_first_step_do_not_depend_on_scatter_order(sp):
    """The scatter's atomics leave each cell in an arbitrary order.  The
    upload puts the cells back in source order before the moments that set
    the first Delta t, and sp_moments does so in FP64 mode: two contexts on
    the same particles give bit-identical Delta t and instantaneous fields,
    at upload and after steps with different batch plans."""
    cfg, regions = W.box2d(nx=24, ny=12, ppc=40.0)
    pos, vel = W.fill_regions(cfg, regions, 7)
    out = []
    for sched in ((512, 4), (128, 2), (1024, 2)):
        s = sp.Sim(cfg, sp.FP64, capacity=4 * vel.shape[1])
        s.set_particles(0, pos, vel)
        s.set_schedule(*sched)
        dt0, m0 = s.dt(0), s.moments(0, 0)
        s.step(7)
        s.sync()
        out.append((dt0, m0, s.dt(0), s.moments(0, 0)))
        s.close()
    for r in out[1:]:
        assert r[0] == out[0][0] and r[2] == out[0][2]
        np.testing.assert_array_equal(r[1], out[0][1])
        np.testing.assert_array_equal(r[3], out[0][3])


def test_schedule_and_autotune_do_not_change_results(sp):
    """Batch composition (staging capacity, warps per block) and the
    autotuner's choice must not change any result."""
    cfg, regions = W.box2d(nx=24, ny=12, ppc=40.0)
    pos, vel = W.fill_regions(cfg, regions, 7)
    runs = []
    for sched in ((512, 4), (128, 2), (1024, 2), None):
        s = sp.Sim(cfg, sp.FP64, capacity=4 * vel.shape[1])
        s.set_particles(0, pos, vel)
        if sched is None:
            s.step(2)
            cap, w = s.autotune(steps_per_trial=1)
            assert cap >= 128 and w in (2, 4, 8)
        else:
            s.set_schedule(*sched)
        s.step(60 - s.step_index())
        s.sync()
        runs.append((s.particles(0), s.sigc_max(0)))
        s.close()
    for r in runs[1:]:
        for x, y in zip(r[0], runs[0][0]):
            np.testing.assert_array_equal(x, y)
        np.testing.assert_array_equal(r[1], runs[0][1])


def test_huge_cells_match_oracle(sp):
    """Cells of 20 000 and 6000 particles (above kHugeCell: one block per
    cell, staged in the cell's output slots in global memory), one of 1500
    (one block, staged in shared memory) and a small one, with the DSMC and
    the Shakhov sub-steps active: bit-exact integer outputs and 1e-12
    velocities, and no capacity error (no cell is too large to collide)."""
    cfg, pos, vel = W.huge_cells()
    assert np.histogram(pos[0], bins=4, range=(0.0, 4.0))[0].max() == 20000
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=5)
    assert tot[0] > 1000 and tot[1] > 0 and tot[2] > 1000
    assert np.diff(o.cell_start().astype(np.int64)).max() > 4096  # still above every staging area
    _close(s.moments(0, 1), o.moments(1), what="averaged moments")


@pytest.mark.parametrize("case", ["channel2d", "sphere3d", "huge1d"])
def test_subcells_match_oracle(sp, case):
    """Bird's sub-cells (option; 2 x 2 in 2-D, 2 x 2 x 2 in 3-D, 4 in the 1-D
    tube with cells of 20 000 / 6000 / 1500 / 300 particles): the cells'
    slots ordered by sub-cell and each candidate's partner drawn from the
    first particle's sub-cell -- bit-exact integers, 1e-12 floats."""
    if case == "channel2d":
        cfg, regions = W.box2d(nx=24, ny=12, ppc=40.0)
        cfg["subcells"] = 2
        pos, vel = W.fill_regions(cfg, regions, 3)
        steps = 8
    elif case == "sphere3d":
        cfg, regions = W.box3d(n=(12, 8, 8), ppc=16.0)
        cfg["subcells"] = 2
        pos, vel = W.fill_regions(cfg, regions, 5)
        steps = 5
    else:
        cfg, pos, vel = W.huge_cells()
        cfg["subcells"] = 4
        steps = 4
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=steps)
    assert tot[0] > 0 and tot[1] > 0


@pytest.mark.parametrize("outer", ["inflow", "diffuse", "specular"])
def test_o_grid_matches_oracle(sp, outer):
    """Body-fitted O-grid (12 x 24 quadrilaterals about a diffuse body,
    radial spacing growing by 8 % a layer): point location by face crossing
    at upload, the face-crossing flight with the body polygon and the outer
    polygon (a freestream reservoir, a diffuse or a specular wall), per-cell
    sizes in Delta t_c, surface tallies -- bit-exact integers and 1e-12
    floats against the oracle."""
    bc = {"inflow": W.BC_INFLOW, "diffuse": W.BC_DIFFUSE, "specular": W.BC_SPECULAR}[outer]
    cfg, regions = W.ogrid_box(nr=12, nt=24, r_out=3.0, growth=1.08, ppc=30.0, outer=bc)
    cfg.update(n_surf=24, n_steady=3)
    pos, vel = W.fill_regions(cfg, regions, 3)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=10)
    assert tot[0] > 0 and tot[1] > 0
    if bc == W.BC_INFLOW:
        t = o.totals()
        assert t["injected"] > 0 and t["removed"] > 0
    tal = compare_surface(o, s, what="o-grid")
    assert tal[0].sum() > 50


def test_o_grid_dense_cells_match_oracle(sp):
    """An O-grid whose inner cells hold more than 1024 particles (the
    one-block-per-cell launch with the face-crossing flight)."""
    cfg, regions = W.ogrid_box(nr=3, nt=4, r_out=2.0, growth=1.0, ppc=1500.0, outer=W.BC_SPECULAR, Kn=0.02)
    pos, vel = W.fill_regions(cfg, regions, 5)
    o, s, tot = run_pair(sp, cfg, pos, vel, steps=4)
    assert np.diff(o.cell_start().astype(np.int64)).max() > 1024
    assert tot[0] > 0


def test_batched_o_grids_match_separate_oracles(sp):
    """Three O-grid instances of different shape (sizes, growth, outer
    boundary, body radius) in one context: each equals its own oracle run
    bit for bit (node, face and radius offsets per instance)."""
    specs = [dict(nr=8, nt=16, r_out=2.5, growth=1.1, outer=W.BC_INFLOW, seed=3),
             dict(nr=5, nt=9, r_out=3.0, growth=1.0, outer=W.BC_DIFFUSE, seed=4, body_r=0.5),
             dict(nr=12, nt=20, r_out=2.0, growth=1.05, outer=W.BC_SPECULAR, seed=5)]
    insts = []
    for sp_ in specs:
        cfg, regions = W.ogrid_box(ppc=25.0, n_steady=2, **sp_)
        pos, vel = W.fill_regions(cfg, regions, sp_["seed"])
        insts.append((cfg, pos, vel))
    s = sp.Sim([c for c, _, _ in insts], sp.FP64, capacity=60000)
    s.set_record(True)
    os_ = []
    for i, (c, p, v) in enumerate(insts):
        s.set_particles(i, p, v)
        o = oracle.Oracle(c)
        o.set_particles(p, v)
        os_.append(o)
    for n in range(6):
        s.step(1)
        for i, o in enumerate(os_):
            o.step(1)
            compare_record(o, s, inst=i, what=f"o-grid {i} step {n}")
            compare_state(o, s, inst=i, what=f"o-grid {i} step {n}")
    for i, o in enumerate(os_):
        _close(s.moments(i, 1), o.moments(1), what=f"o-grid {i} averages")
