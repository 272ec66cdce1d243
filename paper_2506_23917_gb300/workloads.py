"""Seeded synthetic inputs: flow configurations and initial particle sets.

This module holds no arithmetic of the particle method itself.  It builds
the inputs a user of the library would supply -- a gas model, a uniform
Cartesian mesh with cut-cell volumes, boundary states, and the Step-1
initial particles of the paper (uniform positions, drifting Maxwellian
velocities; arXiv:2506.23917 Sec. III.B Step 1) -- from numpy's seeded
PCG64 generator.  The same dicts and arrays feed both the CUDA library and
the CPU oracle.

The workloads are shaped like the paper's test cases (Sec. IV): the Sod
shock tube (Sec. IV.A, Table I), hypersonic flow past a cylinder
(Sec. IV.B), jet expansion into vacuum (Sec. IV.C), hypersonic flow past a
sphere (Sec. IV.D), plus a batched ensemble of small independent flows.
The paper's meshes and reference data are not public, so uniform Cartesian
grids with analytic cut cells stand in for its body-fitted meshes.

Gas-model relations used to derive a config from (Kn, L, T):
  * mean free path of VHS molecules (Sec. IV, equation after the Kn
    definition):  lambda = 1 / (sqrt(2) pi d_ref^2 n (T_ref/T)^(omega-1/2))
  * Bird's VHS viscosity from the reference diameter:
        mu_ref = 15 sqrt(m k T_ref / pi) / (2 (5-2w)(7-2w) d_ref^2)
    which reproduces the paper's argon mu_ref = 2.117e-5 Pa s (Sec. IV)
    from d_ref = 4.17e-10 m, T_ref = 273 K.
"""
from __future__ import annotations

import math
import warnings

import numpy as np

KB = 1.380649e-23
# Argon as quoted in Sec. IV of the paper (VHS, d_ref, T_ref, omega, mu_ref).
ARGON = dict(m=6.63e-26, d_ref=4.17e-10, T_ref=273.0, omega=0.81, mu_ref_paper=2.117e-5)

BC_SPECULAR, BC_DIFFUSE, BC_OUTFLOW, BC_INFLOW = 0, 1, 2, 3
BODY_NONE, BODY_CIRCLE, BODY_SPHERE = 0, 1, 2
MODE_HYBRID, MODE_DSMC, MODE_SHAKHOV = 0, 1, 2
MIN_CUT_FRACTION = 0.05


def vhs_mu_ref(m, d_ref, T_ref, omega, kB=KB):
    """Bird's VHS relation between reference diameter and viscosity."""
    return 15.0 * math.sqrt(m * kB * T_ref / math.pi) / (
        2.0 * (5.0 - 2.0 * omega) * (7.0 - 2.0 * omega) * d_ref ** 2)


def vhs_mfp(n, d_ref, T_ref, T, omega):
    """VHS mean free path, Sec. IV (definition of Kn)."""
    return 1.0 / (math.sqrt(2.0) * math.pi * d_ref ** 2 * n * (T_ref / T) ** (omega - 0.5))


def n_for_kn(Kn, L, d_ref, T_ref, T, omega):
    """Number density giving Kn = lambda / L."""
    return 1.0 / (math.sqrt(2.0) * math.pi * d_ref ** 2 * (Kn * L) * (T_ref / T) ** (omega - 0.5))


def d_for_mfp(lam, n, T_ref, T, omega):
    """Reference diameter giving mean free path lam at (n, T)."""
    return math.sqrt(1.0 / (math.sqrt(2.0) * math.pi * lam * n * (T_ref / T) ** (omega - 0.5)))


def base_config(dim, n, lo, hi):
    n = list(n) + [1] * (3 - len(n))
    lo = list(lo) + [0.0] * (3 - len(lo))
    hi = list(hi) + [1.0] * (3 - len(hi))
    return dict(
        dim=dim, n=n, lo=lo, hi=hi,
        m=1.0, R=1.0, gamma=5.0 / 3.0, Pr=2.0 / 3.0, omega=0.5, T_ref=1.0, mu_ref=1.0,
        d_ref=1.0, Fn=1.0, cfl=0.5, dt_fixed=0.0,
        face_bc=[BC_SPECULAR] * 6, face_T=[1.0] * 6, face_n=[0.0] * 6,
        face_u=[[0.0, 0.0, 0.0] for _ in range(6)], ghost_layers=1,
        body=BODY_NONE, body_c=[0.0, 0.0, 0.0], body_r=0.0, body_Tw=1.0,
        cell_volume=None, sigc_T0=1.0, n_steady=0, seed=1, mode=MODE_HYBRID, ar_max=64,
        n_surf=0, win_lo=[[0.0, 0.0] for _ in range(6)], win_hi=[[0.0, 0.0] for _ in range(6)],
        ntc_carry=0, subcells=0, mesh=0, mesh_r_out=0.0, mesh_growth=1.0,
    )


def ncells(cfg):
    return int(cfg["n"][0] * cfg["n"][1] * cfg["n"][2])


def cell_size(cfg):
    return [(cfg["hi"][d] - cfg["lo"][d]) / cfg["n"][d] for d in range(3)]


# ---------------------------------------------------------------------------
# Cut-cell volumes (mesh generation)
# ---------------------------------------------------------------------------

def _chord_area(x0, x1, y0, y1, cx, cy, r):
    """Area of [x0,x1]x[y0,y1] outside nothing, inside the disk (exact quadrature)."""
    from scipy.integrate import quad

    a, b = max(x0, cx - r), min(x1, cx + r)
    if a >= b:
        return 0.0

    def L(x):
        h2 = r * r - (x - cx) ** 2
        if h2 <= 0:
            return 0.0
        h = math.sqrt(h2)
        return max(0.0, min(y1, cy + h) - max(y0, cy - h))

    pts = [a, b]
    for yb in (y0, y1):
        dy = yb - cy
        if abs(dy) < r:
            w = math.sqrt(r * r - dy * dy)
            for xb in (cx - w, cx + w):
                if a < xb < b:
                    pts.append(xb)
    pts = sorted(set(pts))
    tot = 0.0
    with warnings.catch_warnings():
        warnings.simplefilter("ignore")
        for p, q in zip(pts[:-1], pts[1:]):
            tot += quad(L, p, q, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
    return tot


def circle_cut_volumes(cfg):
    """Fluid volume of each cell of a 2-D grid outside a circle (unit depth)."""
    nx, ny = cfg["n"][0], cfg["n"][1]
    dx, dy, dz = cell_size(cfg)
    cx, cy, _ = cfg["body_c"]
    r = cfg["body_r"]
    V0 = dx * dy * dz
    vol = np.full(nx * ny, V0)
    xs = cfg["lo"][0] + dx * np.arange(nx + 1)
    ys = cfg["lo"][1] + dy * np.arange(ny + 1)
    ix0 = max(0, int((cx - r - cfg["lo"][0]) / dx) - 1)
    ix1 = min(nx, int((cx + r - cfg["lo"][0]) / dx) + 2)
    iy0 = max(0, int((cy - r - cfg["lo"][1]) / dy) - 1)
    iy1 = min(ny, int((cy + r - cfg["lo"][1]) / dy) + 2)
    for j in range(iy0, iy1):
        for i in range(ix0, ix1):
            x0, x1, y0, y1 = xs[i], xs[i + 1], ys[j], ys[j + 1]
            # farthest / nearest corner distance decide full / empty / cut
            fx = max(abs(x0 - cx), abs(x1 - cx))
            fy = max(abs(y0 - cy), abs(y1 - cy))
            if fx * fx + fy * fy <= r * r:
                frac = 0.0
            else:
                nx_ = min(max(cx, x0), x1) - cx
                ny_ = min(max(cy, y0), y1) - cy
                if nx_ * nx_ + ny_ * ny_ >= r * r:
                    continue
                inside = _chord_area(x0, x1, y0, y1, cx, cy, r)
                frac = 1.0 - inside / (dx * dy)
            vol[i + nx * j] = max(frac, MIN_CUT_FRACTION) * V0
    return vol


def sphere_cut_volumes(cfg, sub=8):
    """Fluid volume of each cell of a 3-D grid outside a sphere (midpoint sub-sampling)."""
    n0, n1, n2 = cfg["n"]
    d = cell_size(cfg)
    c = cfg["body_c"]
    r = cfg["body_r"]
    V0 = d[0] * d[1] * d[2]
    vol = np.full(n0 * n1 * n2, V0)
    lo = cfg["lo"]
    rng = [(max(0, int((c[a] - r - lo[a]) / d[a]) - 1), min(cfg["n"][a], int((c[a] + r - lo[a]) / d[a]) + 2))
           for a in range(3)]
    off = (np.arange(sub) + 0.5) / sub
    ox, oy, oz = np.meshgrid(off, off, off, indexing="ij")
    for k in range(*rng[2]):
        for j in range(*rng[1]):
            for i in range(*rng[0]):
                x0 = lo[0] + i * d[0]
                y0 = lo[1] + j * d[1]
                z0 = lo[2] + k * d[2]
                near = [min(max(c[0], x0), x0 + d[0]) - c[0], min(max(c[1], y0), y0 + d[1]) - c[1],
                        min(max(c[2], z0), z0 + d[2]) - c[2]]
                if near[0] ** 2 + near[1] ** 2 + near[2] ** 2 >= r * r:
                    continue
                px = x0 + ox * d[0] - c[0]
                py = y0 + oy * d[1] - c[1]
                pz = z0 + oz * d[2] - c[2]
                frac = float(np.mean(px * px + py * py + pz * pz > r * r))
                vol[i + n0 * (j + n1 * k)] = max(frac, MIN_CUT_FRACTION) * V0
    return vol


# ---------------------------------------------------------------------------
# Initial particles (Step 1 of the paper)
# ---------------------------------------------------------------------------

def _inside_body(cfg, pos):
    if cfg["body"] == BODY_NONE:
        return np.zeros(pos.shape[1], dtype=bool)
    D = 2 if cfg["body"] == BODY_CIRCLE else 3
    r2 = np.zeros(pos.shape[1])
    for a in range(D):
        r2 += (pos[a] - cfg["body_c"][a]) ** 2
    return r2 < cfg["body_r"] ** 2


def fill_regions(cfg, regions, seed):
    """Particles for a list of regions.

    Each region: dict(lo=[...], hi=[...], n=number density, T=temperature,
    u=[3 drift], count=number of particles) -- or ``ppc`` (particles per full
    cell) instead of count.  Positions are uniform in the region minus the
    body; velocities are Maxwellian at T plus the drift.
    Returns pos (dim, M) and vel (3, M) float64.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    dim = cfg["dim"]
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    P, Vv = [], []
    for reg in regions:
        lo = list(reg["lo"]) + [cfg["lo"][d] for d in range(len(reg["lo"]), 3)]
        hi = list(reg["hi"]) + [cfg["hi"][d] for d in range(len(reg["hi"]), 3)]
        box = 1.0
        for d in range(3):
            box *= hi[d] - lo[d]
        if "count" in reg:
            count = int(reg["count"])
            pos = np.empty((dim, 0))
            need = count
            while need > 0:
                m = int(need * 1.2) + 16
                cand = np.stack([lo[d] + (hi[d] - lo[d]) * rng.random(m) for d in range(dim)])
                cand = cand[:, ~_inside_body(cfg, cand)][:, :need]
                pos = np.concatenate([pos, cand], axis=1)
                need = count - pos.shape[1]
        else:
            # uniform in the box at density n; those inside the body are dropped
            m = int(round(reg["n"] * box / cfg["Fn"]))
            cand = np.stack([lo[d] + (hi[d] - lo[d]) * rng.random(m) for d in range(dim)])
            pos = cand[:, ~_inside_body(cfg, cand)]
            count = pos.shape[1]
        s = math.sqrt(cfg["R"] * reg["T"])
        vel = rng.normal(0.0, s, size=(3, count)) + np.asarray(reg["u"], dtype=np.float64)[:, None]
        P.append(pos)
        Vv.append(vel)
    pos = np.concatenate(P, axis=1) if P else np.zeros((dim, 0))
    vel = np.concatenate(Vv, axis=1) if Vv else np.zeros((3, 0))
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)


# ---------------------------------------------------------------------------
# Workloads
# ---------------------------------------------------------------------------

def sod(ncell=200, ppc_left=100.0, lam_left=1e-3, seed=1, n_steady=10**9, mode=MODE_HYBRID,
        omega=0.5):
    """1-D Sod shock tube (Sec. IV.A shape): x in [0,1], diaphragm at 0.5,
    rho_L=1, p_L=1 / rho_R=0.125, p_R=0.1, u=0; hard sphere (omega=1/2) by
    default, Pr=2/3; nondimensional with m = R = k = 1 so n = rho and
    T = p/rho; specular end walls; CFL 0.5 on the local time step."""
    cfg = base_config(1, [ncell], [0.0], [1.0])
    nL, TL, nR, TR = 1.0, 1.0, 0.125, 0.8
    d = d_for_mfp(lam_left, nL, 1.0, TL, omega)
    cfg.update(omega=omega, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, omega, kB=1.0),
               Fn=nL * (1.0 / ncell) / ppc_left, cfl=0.5, sigc_T0=TL, seed=seed,
               n_steady=n_steady, mode=mode)
    regions = [dict(lo=[0.0], hi=[0.5], n=nL, T=TL, u=[0, 0, 0]),
               dict(lo=[0.5], hi=[1.0], n=nR, T=TR, u=[0, 0, 0])]
    return cfg, regions


def homogeneous(N=20000, Kn=1e-2, omega=0.5, Tx=2.0, Tyz=1.0, skew=0.0, seed=1,
                mode=MODE_HYBRID, dt=None):
    """A single cell with specular walls (space-homogeneous relaxation).

    The initial sample is a bi-Maxwellian with T_x != T_y = T_z; ``skew`` > 0
    adds a heat flux along x by mixing in a shifted population (drift
    removed afterwards).  Velocities returned separately by
    :func:`homogeneous_particles`.
    """
    cfg = base_config(1, [1], [0.0], [1.0])
    n = 1.0
    T = (Tx + 2 * Tyz) / 3.0
    d = d_for_mfp(Kn, n, 1.0, T, omega)
    cfg.update(omega=omega, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, omega, kB=1.0),
               Fn=n * 1.0 / N, sigc_T0=T, seed=seed, mode=mode)
    if dt is not None:
        cfg["dt_fixed"] = dt
    return cfg


def homogeneous_particles(cfg, N, Tx=2.0, Tyz=1.0, skew=0.0, seed=1):
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.random((1, N))
    vel = np.stack([rng.normal(0, math.sqrt(Tx), N), rng.normal(0, math.sqrt(Tyz), N),
                    rng.normal(0, math.sqrt(Tyz), N)])
    if skew > 0:
        # an exponential tail along x carries a heat flux q_x > 0
        m = int(skew * N)
        vel[0, :m] = rng.exponential(math.sqrt(Tx), m) * 1.5
    vel -= vel.mean(axis=1, keepdims=True)
    return np.ascontiguousarray(pos), np.ascontiguousarray(vel)


def cylinder(scale=1.0, ppc=40.0, Kn=0.01, Ma=5.0, seed=1, n_steady=1000, T_inf=273.0,
             ghost_layers=1):
    """2-D hypersonic argon flow past a cylinder (Sec. IV.B shape).

    Radius R = 1 m is the reference length; Kn = lambda_inf / R; argon VHS
    (omega = 0.81, d_ref, T_ref, mu_ref of Sec. IV); freestream T = 273 K;
    diffuse wall at T_w = T_inf.  Domain [-3R, 3R] x [0, 3R] with the y = 0
    plane specular (half symmetry), inflow at x = -3R and y = 3R, outflow at
    x = 3R.  Grid 600 x 300 (cell 0.01 R) at scale 1; ``scale`` < 1 shrinks
    the cell count per axis for tests (same physical domain).
    """
    gas = ARGON
    m, d_ref, T_ref, omega = gas["m"], gas["d_ref"], gas["T_ref"], gas["omega"]
    R_gas = KB / m
    Rb = 1.0
    nx, ny = max(4, int(round(600 * scale))), max(2, int(round(300 * scale)))
    cfg = base_config(2, [nx, ny], [-3.0 * Rb, 0.0], [3.0 * Rb, 3.0 * Rb])
    n_inf = n_for_kn(Kn, Rb, d_ref, T_ref, T_inf, omega)
    a_inf = math.sqrt(5.0 / 3.0 * R_gas * T_inf)
    U = Ma * a_inf
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    cfg.update(m=m, R=R_gas, omega=omega, T_ref=T_ref, d_ref=d_ref,
               mu_ref=vhs_mu_ref(m, d_ref, T_ref, omega), Fn=n_inf * V0 / ppc, cfl=0.5,
               sigc_T0=T_inf, seed=seed, n_steady=n_steady, ghost_layers=ghost_layers,
               body=BODY_CIRCLE, body_c=[0.0, 0.0, 0.0], body_r=Rb, body_Tw=T_inf, n_surf=360)
    fb = [BC_INFLOW, BC_OUTFLOW, BC_SPECULAR, BC_INFLOW, BC_SPECULAR, BC_SPECULAR]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T_inf] * 6
    cfg["face_n"] = [n_inf if b == BC_INFLOW else 0.0 for b in fb]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    cfg["cell_volume"] = circle_cut_volumes(cfg)
    regions = [dict(lo=[-3.0 * Rb, 0.0], hi=[3.0 * Rb, 3.0 * Rb], n=n_inf, T=T_inf, u=[U, 0, 0])]
    return cfg, regions


def cylinder_ogrid(nr=96, nt=192, r_out=4.0, growth=1.03, ppc=40.0, Kn=0.05, Ma=5.0, seed=1,
                   n_steady=1000, T_inf=273.0, ghost_layers=2):
    """2-D hypersonic argon flow past a cylinder on a body-fitted O-grid.

    The cylinder case on a synthetic body-fitted mesh (the paper's own
    cylinder meshes are body-fitted and not available): nr radial layers x
    nt sectors of straight-edged quadrilaterals from the body (radius R = 1 m,
    diffuse at T_inf) to radius r_out R, radial spacing growing by ``growth``
    per layer.  The whole outer polygon is a freestream boundary (reservoir
    of ghost_layers rings at n_inf, T_inf, U): it feeds the upstream side and
    absorbs what leaves downstream.  Argon VHS as in ``cylinder``; Kn =
    lambda_inf / R; F_N sets ppc particles in a cell of the mean area.
    """
    gas = ARGON
    m, d_ref, T_ref, omega = gas["m"], gas["d_ref"], gas["T_ref"], gas["omega"]
    R_gas = KB / m
    Rb = 1.0
    cfg = base_config(2, [nr, nt], [-r_out * Rb, -r_out * Rb], [r_out * Rb, r_out * Rb])
    n_inf = n_for_kn(Kn, Rb, d_ref, T_ref, T_inf, omega)
    U = Ma * math.sqrt(5.0 / 3.0 * R_gas * T_inf)
    depth = cfg["hi"][2] - cfg["lo"][2]
    mean_area = math.pi * ((r_out * Rb) ** 2 - Rb ** 2) / (nr * nt)
    cfg.update(m=m, R=R_gas, omega=omega, T_ref=T_ref, d_ref=d_ref,
               mu_ref=vhs_mu_ref(m, d_ref, T_ref, omega), Fn=n_inf * mean_area * depth / ppc, cfl=0.5,
               sigc_T0=T_inf, seed=seed, n_steady=n_steady, ghost_layers=ghost_layers,
               body=BODY_CIRCLE, body_c=[0.0, 0.0, 0.0], body_r=Rb, body_Tw=T_inf,
               mesh=1, mesh_r_out=r_out * Rb, mesh_growth=growth)
    fb = [BC_OUTFLOW, BC_INFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_SPECULAR, BC_SPECULAR]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T_inf] * 6
    cfg["face_n"] = [0.0, n_inf, 0.0, 0.0, 0.0, 0.0]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    regions = [dict(lo=[-r_out * Rb, -r_out * Rb], hi=[r_out * Rb, r_out * Rb], n=n_inf, T=T_inf,
                    u=[U, 0, 0])]
    return cfg, regions


def ogrid_box(nr=12, nt=24, r_out=3.0, growth=1.08, ppc=30.0, seed=3, T=1.0, U=2.0, Kn=0.05,
              outer=BC_INFLOW, mode=MODE_HYBRID, body_r=1.0, n_steady=0):
    """Small nondimensional O-grid about a unit-radius body (parity and pin
    cases): freestream (T, U along x) at Kn = lambda / body_r through the
    outer polygon (``outer``: inflow, specular or diffuse at T), body
    diffuse at T."""
    cfg = base_config(2, [nr, nt], [-r_out, -r_out], [r_out, r_out])
    n = 1.0
    d = d_for_mfp(Kn * body_r, n, 1.0, T, 0.5)
    mean_area = math.pi * (r_out ** 2 - body_r ** 2) / (nr * nt)
    cfg.update(omega=0.5, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, 0.5, kB=1.0),
               Fn=n * mean_area / ppc, sigc_T0=T, seed=seed, n_steady=n_steady, ghost_layers=2,
               body=BODY_CIRCLE, body_c=[0.0, 0.0, 0.0], body_r=body_r, body_Tw=T, mode=mode,
               mesh=1, mesh_r_out=r_out, mesh_growth=growth)
    cfg["face_bc"] = [BC_OUTFLOW, outer, BC_OUTFLOW, BC_OUTFLOW, BC_SPECULAR, BC_SPECULAR]
    cfg["face_T"] = [T] * 6
    cfg["face_n"] = [0.0, n if outer == BC_INFLOW else 0.0, 0.0, 0.0, 0.0, 0.0]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    regions = [dict(lo=[-r_out, -r_out], hi=[r_out, r_out], n=n, T=T, u=[U, 0, 0])]
    return cfg, regions


# A nitrogen-like monatomic VHS model: N2's mass, reference diameter and
# viscosity exponent (Bird's tables) with a monatomic gamma of 5/3.
NITROGEN_LIKE = dict(m=4.65e-26, d_ref=4.17e-10, T_ref=273.0, omega=0.74)


def jet(scale=1.0, ppc=500.0, Kn=0.02, Ma=1.0, plenum=4.0, seed=1, n_steady=500, T0=300.0,
        ghost_layers=3):
    """2-D sonic jet expanding into vacuum (Sec. IV.C shape).

    Orifice width w = 1 mm is the reference length; Kn = lambda_0 / w at the
    orifice state n_0.  Domain [0, 8w] x [-4w, 4w] on a 512 x 512 grid at
    scale 1 (cell w/64).  The left face is an inflow only on the orifice
    |y| <= w/2 (Ma = 1 at n_0, T_0); the rest of it is a diffuse wall at T_0
    (the lips).  The other faces are outflow to vacuum.  A plenum block
    [0, w] x [-w, w] starts at plenum * n_0 and rest, and drains into the
    vacuum, so per-cell occupancy spans 0 to ~plenum * ppc.
    """
    gas = NITROGEN_LIKE
    m, d_ref, T_ref, omega = gas["m"], gas["d_ref"], gas["T_ref"], gas["omega"]
    R_gas = KB / m
    w = 1e-3
    nc = max(8, int(round(512 * scale)))
    cfg = base_config(2, [nc, nc], [0.0, -4.0 * w], [8.0 * w, 4.0 * w])
    n0 = n_for_kn(Kn, w, d_ref, T_ref, T0, omega)
    U = Ma * math.sqrt(5.0 / 3.0 * R_gas * T0)
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    cfg.update(m=m, R=R_gas, omega=omega, T_ref=T_ref, d_ref=d_ref,
               mu_ref=vhs_mu_ref(m, d_ref, T_ref, omega), Fn=n0 * V0 / ppc, cfl=0.5,
               sigc_T0=T0, seed=seed, n_steady=n_steady, ghost_layers=ghost_layers)
    fb = [BC_INFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_OUTFLOW, BC_SPECULAR, BC_SPECULAR]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T0] * 6
    cfg["face_n"] = [n0, 0.0, 0.0, 0.0, 0.0, 0.0]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    cfg["win_lo"][0] = [-0.5 * w, 0.0]
    cfg["win_hi"][0] = [0.5 * w, 0.0]
    regions = [dict(lo=[0.0, -w], hi=[w, w], n=plenum * n0, T=T0, u=[0.0, 0.0, 0.0])]
    return cfg, regions


def sphere(scale=1.0, ppc=30.0, Kn=0.005, Ma=10.0, seed=1, n_steady=750, T_inf=65.0,
           Tw_ratio=4.0):
    """3-D hypersonic argon flow past a sphere (Sec. IV.D shape), half symmetry
    in y; grid 256 x 128 x 128 over [-3R, 5R] x [0, 4R] x [-2R, 2R] at scale 1."""
    gas = ARGON
    m, d_ref, T_ref, omega = gas["m"], gas["d_ref"], gas["T_ref"], gas["omega"]
    R_gas = KB / m
    Rb = 1.0
    n0, n1, n2 = (max(4, int(round(v * scale))) for v in (256, 128, 128))
    cfg = base_config(3, [n0, n1, n2], [-3.0, 0.0, -2.0], [5.0, 4.0, 2.0])
    n_inf = n_for_kn(Kn, Rb, d_ref, T_ref, T_inf, omega)
    U = Ma * math.sqrt(5.0 / 3.0 * R_gas * T_inf)
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    cfg.update(m=m, R=R_gas, omega=omega, T_ref=T_ref, d_ref=d_ref,
               mu_ref=vhs_mu_ref(m, d_ref, T_ref, omega), Fn=n_inf * V0 / ppc, cfl=0.5,
               sigc_T0=T_inf, seed=seed, n_steady=n_steady, body=BODY_SPHERE,
               body_c=[0.0, 0.0, 0.0], body_r=Rb, body_Tw=Tw_ratio * T_inf, n_surf=90)
    fb = [BC_INFLOW, BC_OUTFLOW, BC_SPECULAR, BC_INFLOW, BC_INFLOW, BC_INFLOW]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T_inf] * 6
    cfg["face_n"] = [n_inf if b == BC_INFLOW else 0.0 for b in fb]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    cfg["cell_volume"] = sphere_cut_volumes(cfg)
    regions = [dict(lo=[-3.0, 0.0, -2.0], hi=[5.0, 4.0, 2.0], n=n_inf, T=T_inf, u=[U, 0, 0])]
    return cfg, regions


def box2d(nx=24, ny=12, ppc=30.0, seed=3, body=True, inflow=True, T=1.0, U=2.0, Kn=0.05,
          mode=MODE_HYBRID):
    """Small nondimensional 2-D channel with every boundary kind, for parity
    tests: inflow at -x, outflow at +x, specular y=0, diffuse wall at +y, and
    an optional diffuse circular body (cut cells)."""
    cfg = base_config(2, [nx, ny], [0.0, 0.0], [2.0, 1.0])
    n = 1.0
    d = d_for_mfp(Kn, n, 1.0, T, 0.81)
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    cfg.update(omega=0.81, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, 0.81, kB=1.0),
               Fn=n * V0 / ppc, sigc_T0=T, seed=seed, mode=mode, ghost_layers=2)
    fb = [BC_INFLOW if inflow else BC_SPECULAR, BC_OUTFLOW, BC_SPECULAR, BC_DIFFUSE,
          BC_SPECULAR, BC_SPECULAR]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T, T, T, 1.5 * T, T, T]
    cfg["face_n"] = [n if b == BC_INFLOW else 0.0 for b in fb]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    if body:
        cfg.update(body=BODY_CIRCLE, body_c=[0.8, 0.0, 0.0], body_r=0.3, body_Tw=2.0 * T)
        cfg["cell_volume"] = circle_cut_volumes(cfg)
    regions = [dict(lo=[0.0, 0.0], hi=[2.0, 1.0], n=n, T=T, u=[U, 0, 0])]
    return cfg, regions


def box3d(n=(12, 8, 8), ppc=20.0, seed=5, T=1.0, U=3.0, Kn=0.05):
    """Small nondimensional 3-D box with a diffuse sphere, inflow and outflow."""
    cfg = base_config(3, list(n), [0.0, 0.0, -0.5], [1.5, 1.0, 0.5])
    nd = 1.0
    d = d_for_mfp(Kn, nd, 1.0, T, 0.81)
    dl = cell_size(cfg)
    V0 = dl[0] * dl[1] * dl[2]
    cfg.update(omega=0.81, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, 0.81, kB=1.0),
               Fn=nd * V0 / ppc, sigc_T0=T, seed=seed, ghost_layers=2,
               body=BODY_SPHERE, body_c=[0.5, 0.0, 0.0], body_r=0.25, body_Tw=2.0 * T)
    fb = [BC_INFLOW, BC_OUTFLOW, BC_SPECULAR, BC_DIFFUSE, BC_INFLOW, BC_OUTFLOW]
    cfg["face_bc"] = fb
    cfg["face_T"] = [T] * 6
    cfg["face_n"] = [nd if b == BC_INFLOW else 0.0 for b in fb]
    cfg["face_u"] = [[U, 0.0, 0.0] for _ in range(6)]
    cfg["cell_volume"] = sphere_cut_volumes(cfg)
    regions = [dict(lo=[0.0, 0.0, -0.5], hi=[1.5, 1.0, 0.5], n=nd, T=T, u=[U, 0, 0])]
    return cfg, regions


def homogeneous_box(N, Kn, seed=1, Tx=2.0, Tyz=1.0, skew=0.05, ppc=56.25, n_steady=10**9):
    """Spatially homogeneous relaxation in a 1-D box of unit length with
    specular walls: nx = round(N/ppc) cells, uniform positions, a
    bi-Maxwellian (T_x != T_y = T_z) with a heat-flux-carrying skew."""
    nx = max(1, int(round(N / ppc)))
    cfg = base_config(1, [nx], [0.0], [1.0])
    T = (Tx + 2 * Tyz) / 3.0
    d = d_for_mfp(Kn, 1.0, 1.0, T, 0.5)
    cfg.update(omega=0.5, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, 0.5, kB=1.0),
               Fn=1.0 / N, sigc_T0=T, seed=seed, n_steady=n_steady)
    pos, vel = homogeneous_particles(cfg, N, Tx=Tx, Tyz=Tyz, skew=skew, seed=seed)
    return cfg, pos, vel


def huge_cells(counts=(20000, 6000, 1500, 300), seed=5):
    """A 1-D tube of len(counts) unit cells holding the given particle
    counts (each a bi-Maxwellian with a heat-flux skew), specular ends, the
    gas dense enough in the first cell that both collision sub-steps run.
    Returns (cfg, pos, vel)."""
    nc = len(counts)
    cfg = base_config(1, [nc], [0.0], [float(nc)])
    T = (2.0 + 2 * 1.0) / 3.0
    d = d_for_mfp(0.05, 1.0, 1.0, T, 0.5)
    cfg.update(omega=0.5, T_ref=1.0, d_ref=d, mu_ref=vhs_mu_ref(1.0, d, 1.0, 0.5, kB=1.0),
               Fn=1.0 / counts[0], sigc_T0=T, seed=seed, n_steady=1)
    ps, vs = [], []
    for k, N in enumerate(counts):
        p, v = homogeneous_particles(cfg, N, Tx=2.0, skew=0.1, seed=seed + k)
        ps.append(p + k)
        vs.append(v)
    return cfg, np.ascontiguousarray(np.concatenate(ps, axis=1)), np.ascontiguousarray(np.concatenate(vs, axis=1))


def batch(n_inst=256, seed=1, Nmin=1e3, Nmax=5e5, Kn_min=1e-4, Kn_max=1.0, n_steady=10**9):
    """Ensemble of independent 1-D instances: even i a Sod tube with
    nx = round(2 N_i / 112.5) cells, odd i a spatially homogeneous
    relaxation box (~56 particles per cell); N_i and Kn log-uniform.
    Returns a list of (cfg, pos, vel)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ns = np.exp(rng.uniform(math.log(Nmin), math.log(Nmax), n_inst))
    Kns = np.exp(rng.uniform(math.log(Kn_min), math.log(Kn_max), n_inst))
    out = []
    for i in range(n_inst):
        N = int(Ns[i])
        if i % 2 == 0:
            nx = max(2, int(round(2 * N / 112.5)))
            cfg, regions = sod(ncell=nx, ppc_left=100.0, lam_left=float(Kns[i]), seed=seed * 1000 + i,
                               n_steady=n_steady)
            pos, vel = fill_regions(cfg, regions, seed * 7919 + i)
        else:
            cfg, pos, vel = homogeneous_box(N, float(Kns[i]), seed=seed * 1000 + i, n_steady=n_steady)
        out.append((cfg, pos, vel))
    return out
