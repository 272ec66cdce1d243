"""Pins of the oracle's free-flight, wall, reservoir and sorting steps
(Step 2 and the indexing of Step 3, Sec. III.B) against closed forms.

* specular walls: the position is the triangle-wave reflection of x0 + c t;
* diffuse walls: re-emitted normal speed follows the flux-weighted
  (Rayleigh) law P(|c_n| > a) = exp(-a^2 / (2 R T_w)), tangential speeds are
  Gaussian with variance R T_w;
* open faces remove particles; particle count bookkeeping is exact;
* the circle hit point lies on the circle and the re-emitted velocity points
  away from it;
* the reservoir (ghost-cell) inflow injects, per unit area and time, the
  one-way flux of a drifting Maxwellian (Bird's textbook closed form);
* a face open only on a window (an orifice) removes particles that cross it
  inside the window and reflects the others diffusely, and a windowed
  inflow face injects the one-way flux through the window's area only;
* the sort is a stable counting sort by cell;
* the analytic cut-cell volumes add up to the domain minus the body.
"""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2506_23917_gb300 import workloads as W


def _free_cfg(nc=1000, L=1.0, dt=0.37):
    cfg = W.base_config(1, [nc], [0.0], [L])
    cfg.update(d_ref=1e-12, dt_fixed=dt, Fn=1.0)  # no collisions: <=1 particle per cell
    return cfg


def _reflect(x, L):
    y = np.mod(x, 2 * L)
    return np.where(y > L, 2 * L - y, y)


def test_specular_walls_triangle_wave():
    nc, L, dt = 1000, 1.0, 0.37
    cfg = _free_cfg(nc, L, dt)
    rng = np.random.default_rng(1)
    cells = rng.choice(nc, 400, replace=False)
    x0 = (cells + rng.random(400)) / nc * L
    v = rng.normal(0, 3.0, (3, 400))
    o = oracle.Oracle(cfg)
    o.set_particles(x0[None, :], v)
    # initial order is by cell; map back
    order = np.argsort(cells, kind="stable")
    o.step(1)
    pos, vel, _ = o.particles()
    _, _, perm = o.record()
    xi, vi = x0[order][perm], v[:, order][:, perm]
    expect = _reflect(xi + vi[0] * dt, L)
    assert np.max(np.abs(pos[0] - expect)) < 1e-12
    nref = np.floor((xi + vi[0] * dt) / L)
    sign = np.where(np.mod(nref, 2) == 0, 1.0, -1.0)
    assert np.allclose(vel[0], sign * vi[0], rtol=0, atol=0)
    assert np.array_equal(vel[1:], vi[1:])
    assert o.M == 400


def test_diffuse_walls_rayleigh_and_gaussian():
    # each particle hits x = 1 once and cannot reach x = 0 in the rest of
    # the step (a second hit would bias the last sample toward slow speeds);
    # d_ref ~ 0 switches collisions off
    nc, Tw = 20000, 1.7
    cfg = _free_cfg(1000, 1.0, dt=0.03)
    cfg["face_bc"][0] = cfg["face_bc"][1] = W.BC_DIFFUSE
    cfg["face_T"][0] = cfg["face_T"][1] = Tw
    x0 = 0.9 + 0.1 * (np.arange(nc) + 0.5) / nc
    v = np.zeros((3, nc))
    v[0] = 5.0
    o = oracle.Oracle(cfg)
    o.set_particles(x0[None, :], v)
    o.step(1)
    _, vel, _ = o.particles()
    s = math.sqrt(Tw)  # R = 1
    cn = np.abs(vel[0])
    p = stats.kstest(cn, lambda a: 1 - np.exp(-a * a / (2 * s * s))).pvalue
    assert p > 1e-3
    for d in (1, 2):
        assert stats.kstest(vel[d] / s, "norm").pvalue > 1e-3
    assert o.M == nc


def test_outflow_removes_and_counts():
    nc = 500
    cfg = _free_cfg(nc, 1.0, dt=0.1)
    cfg["face_bc"][1] = W.BC_OUTFLOW
    rng = np.random.default_rng(2)
    x0 = (np.arange(nc) + 0.5) / nc
    v = rng.normal(0, 2.0, (3, nc))
    o = oracle.Oracle(cfg)
    o.set_particles(x0[None, :], v)
    o.step(1)
    out = np.sum(x0 + v[0] * 0.1 > 1.0)
    assert o.totals()["removed"] == out
    assert o.M == nc - out


def test_circle_hit_point_and_reemission():
    cfg, _ = W.box2d(nx=40, ny=20, ppc=1, inflow=False)
    cfg.update(dt_fixed=0.11, d_ref=1e-12)
    cfg["face_bc"] = [W.BC_SPECULAR] * 6
    c, r = cfg["body_c"], cfg["body_r"]
    # particles heading right, each reaching the circle at t = 0.1; the rest
    # of the step (0.01) is too short to reach any other boundary
    ys = np.linspace(0.1, 0.28, 12)
    xh = c[0] - np.sqrt(r * r - ys * ys)
    pos = np.stack([xh - 0.1, ys])
    vel = np.zeros((3, len(ys)))
    vel[0] = 1.0
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    p0, _, _ = o.particles()
    o.step(1)
    p1, v1, _ = o.particles()
    _, _, perm = o.record()
    for k in range(len(ys)):
        y0 = p0[1, perm[k]]
        i = int(np.argmin(np.abs(ys - y0)))
        back = p1[:, k] - v1[:2, k] * 0.01
        assert abs(back[0] - xh[i]) < 1e-12 and abs(back[1] - ys[i]) < 1e-12
        assert abs(math.hypot(back[0] - c[0], back[1] - c[1]) - r) < 1e-12
        nrm = np.array([xh[i] - c[0], ys[i] - c[1]]) / r
        assert float(nrm @ v1[:2, k]) > 0


@pytest.mark.parametrize("Un_over_a", [0.0, 0.7, 2.5])
def test_inflow_reservoir_flux_matches_drifting_maxwellian(Un_over_a):
    nc, T, n = 50, 1.0, 1.0
    cfg = W.base_config(1, [nc], [0.0], [1.0])
    cfg.update(d_ref=1e-12, Fn=2e-5, dt_fixed=0.004, ghost_layers=3)
    cfg["face_bc"][0] = W.BC_INFLOW
    cfg["face_bc"][1] = W.BC_OUTFLOW
    cfg["face_T"][0] = T
    cfg["face_n"][0] = n
    s2 = math.sqrt(2 * T)
    Un = Un_over_a * s2
    cfg["face_u"][0] = [Un, 0.0, 0.0]
    o = oracle.Oracle(cfg)
    o.set_particles(np.array([[0.5, 0.51]]), np.zeros((3, 2)))
    steps = 40
    o.step(steps)
    got = o.totals()["injected"]
    s = Un / s2
    flux = n * (math.sqrt(T / (2 * math.pi)) * math.exp(-s * s) + 0.5 * Un * (1 + math.erf(s)))
    expect = flux * 1.0 * cfg["dt_fixed"] * steps / cfg["Fn"]
    assert abs(got - expect) < 4 * math.sqrt(expect) + 2


def test_windowed_outflow_face_removes_inside_reflects_outside():
    nc = 20
    cfg = W.base_config(2, [nc, nc], [0.0, 0.0], [1.0, 1.0])
    cfg.update(d_ref=1e-12, Fn=1.0, dt_fixed=0.1)
    cfg["face_bc"] = [W.BC_OUTFLOW, W.BC_SPECULAR, W.BC_SPECULAR, W.BC_SPECULAR, 0, 0]
    cfg["face_T"][0] = 1e-3  # slow re-emission: no second wall within the step
    cfg["win_lo"][0] = [0.4, 0.0]
    cfg["win_hi"][0] = [0.6, 0.0]
    y = (np.arange(nc) + 0.5) / nc
    pos = np.stack([np.full(nc, 0.02), y])
    vel = np.zeros((3, nc))
    vel[0] = -1.0
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    o.step(1)
    inside = (y >= 0.4) & (y <= 0.6)
    assert o.totals()["removed"] == int(inside.sum())
    assert o.M == nc - int(inside.sum())
    p, v, _ = o.particles()
    # survivors were re-emitted from the wall part of the face (hit at
    # t = 0.02, then 0.08 of free flight): moving away from it, hit point
    # outside the window
    assert np.all(v[0] > 0)
    assert np.allclose(p[0], v[0] * 0.08, rtol=1e-9, atol=1e-12)
    y_hit = p[1] - v[1] * 0.08
    assert np.all((y_hit < 0.4) | (y_hit > 0.6))
    assert np.allclose(np.sort(y_hit), np.sort(y[~inside]), atol=1e-12)


@pytest.mark.parametrize("Un_over_a", [0.0, 1.0])
def test_windowed_inflow_injects_through_window_only(Un_over_a):
    nc, T, n = 40, 1.0, 1.0
    cfg = W.base_config(2, [nc, nc], [0.0, 0.0], [1.0, 1.0])
    cfg.update(d_ref=1e-12, Fn=1e-5, dt_fixed=0.002, ghost_layers=3)
    cfg["face_bc"] = [W.BC_INFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_OUTFLOW, 0, 0]
    cfg["face_T"][0] = T
    cfg["face_n"][0] = n
    s2 = math.sqrt(2 * T)
    Un = Un_over_a * s2
    cfg["face_u"][0] = [Un, 0.0, 0.0]
    cfg["win_lo"][0] = [0.25, 0.0]
    cfg["win_hi"][0] = [0.5, 0.0]
    o = oracle.Oracle(cfg)
    o.set_particles(np.array([[0.9], [0.9]]), np.zeros((3, 1)))
    steps = 30
    o.step(steps)
    got = o.totals()["injected"]
    s = Un / s2
    flux = n * (math.sqrt(T / (2 * math.pi)) * math.exp(-s * s) + 0.5 * Un * (1 + math.erf(s)))
    expect = flux * 0.25 * cfg["dt_fixed"] * steps / cfg["Fn"]
    assert abs(got - expect) < 4 * math.sqrt(expect) + 2
    # every injected particle entered through the window
    p, v, _ = o.particles()
    fresh = p[0] < 0.9 - 1e-9
    y0 = p[1][fresh] - v[1][fresh] * (p[0][fresh] / v[0][fresh])
    assert np.all((y0 >= 0.25 - 1e-9) & (y0 <= 0.5 + 1e-9))


def test_sort_is_stable_counting_sort():
    cfg, regions = W.box2d(nx=16, ny=8, ppc=12)
    pos, vel = W.fill_regions(cfg, regions, 4)
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    M0 = o.M
    o.step(2)
    st = o.cell_start()
    _, _, cell = o.particles()
    assert np.all(np.diff(cell.astype(np.int64)) >= 0)
    _, _, perm = o.record()
    for k in range(len(st) - 1):
        seg = perm[st[k]:st[k + 1]].astype(np.int64)
        assert np.all(np.diff(seg) > 0)
    assert len(np.unique(perm)) == len(perm)
    t = o.totals()
    assert t["injected"] > 0 and t["removed"] > 0
    o2 = oracle.Oracle(cfg)
    o2.set_particles(pos, vel)
    o2.step(2)
    assert o2.M == o.M
    assert np.array_equal(o2.particles()[1], o.particles()[1])


def test_cut_cell_volumes_close():
    """Sum of fluid volumes = domain - half disk, up to the cells raised to
    the minimum fraction (each adds at most MIN_CUT_FRACTION V0)."""
    cfg, _ = W.box2d(nx=60, ny=30, ppc=1)
    vol = cfg["cell_volume"]
    dl = W.cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    r = cfg["body_r"]
    clamped = int(np.sum(vol == W.MIN_CUT_FRACTION * V0))
    exact = 2.0 * 1.0 - 0.5 * math.pi * r * r
    excess = vol.sum() - exact
    assert -1e-9 <= excess <= clamped * W.MIN_CUT_FRACTION * V0 + 1e-9
    cut = np.sum((vol < V0) & (vol > W.MIN_CUT_FRACTION * V0))
    assert cut > 10


def test_sphere_cut_cell_volumes_close():
    cfg, _ = W.box3d(n=(24, 16, 16))
    vol = cfg["cell_volume"]
    dl = W.cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    r = cfg["body_r"]
    exact = 1.5 * 1.0 * 1.0 - 0.5 * (4.0 / 3.0) * math.pi * r ** 3
    clamped = int(np.sum(vol == W.MIN_CUT_FRACTION * V0))
    # midpoint sub-sampling: a few parts in 1e3 of the body volume
    assert abs(vol.sum() - exact) < 5e-3 * (2.0 / 3.0) * math.pi * r ** 3 + clamped * W.MIN_CUT_FRACTION * V0
