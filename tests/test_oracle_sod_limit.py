"""Whole-method pin: the hybrid solution of the Sod problem (Sec. IV.A)
approaches the exact Euler Riemann solution as Kn -> 0, and at Kn large
enough for dt_c <= tau everywhere the hybrid is pure DSMC (DSMC ratio 1,
as the paper reports for Kn = 1e-2 with cell size lambda)."""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23917_gb300 import workloads as W
from tests import riemann

G = 5.0 / 3.0
LEFT, RIGHT = (1.0, 0.0, 1.0), (0.125, 0.0, 0.1)


def test_riemann_star_state_satisfies_jump_conditions():
    ps, us = riemann.star(LEFT, RIGHT, G)
    # right-moving shock: Rankine-Hugoniot mass and momentum balance
    rr, ur, pr = RIGHT
    q = riemann.sample(LEFT, RIGHT, G, [us + 1e-9])[:, 0]
    rs = q[0]
    S = (rs * us - rr * ur) / (rs - rr)
    assert abs((rs * (us - S)) - (rr * (ur - S))) < 1e-12
    assert abs((rs * (us - S) ** 2 + ps) - (rr * (ur - S) ** 2 + pr)) < 1e-10
    # left rarefaction is isentropic: p / rho^g equal on both sides
    ql = riemann.sample(LEFT, RIGHT, G, [us - 1e-9])[:, 0]
    assert abs(ql[2] / ql[0] ** G - LEFT[2] / LEFT[0] ** G) < 1e-12
    assert abs(ql[2] - ps) < 1e-12 and abs(q[2] - ps) < 1e-12


def _run(lam, ppc=600, t_end=0.15, seed=1):
    cfg, regions = W.sod(ncell=200, ppc_left=ppc, lam_left=lam, seed=seed)
    pos, vel = W.fill_regions(cfg, regions, seed)
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    t = 0.0
    while t + 0.5 * o.dt < t_end:
        t += o.dt
        o.step(1)
    return o, t, cfg


def _l1(o, t):
    m = o.moments(0)
    rho = m[oracle.FIELDS.index("n")]  # m = 1: n = rho
    x = (np.arange(200) + 0.5) / 200
    ex = riemann.sample(LEFT, RIGHT, G, (x - 0.5) / t)[0]
    k = np.ones(5) / 5.0  # 5-cell running mean damps the particle noise
    sm = np.convolve(rho, k, mode="same")
    inner = slice(3, 197)
    return float(np.mean(np.abs(sm[inner] - ex[inner]))), m


@pytest.mark.slow
def test_sod_approaches_riemann_as_kn_goes_to_zero():
    errs = {}
    ratios = {}
    for lam in (1e-2, 1e-4):
        o, t, cfg = _run(lam)
        assert abs(t - 0.15) < 0.01
        errs[lam], m = _l1(o, t)
        ratios[lam] = m[oracle.FIELDS.index("ratio")]
        assert o.M == 60000 + 7500  # closed tube: count is exact
    assert errs[1e-4] < 0.03
    assert errs[1e-4] < 0.7 * errs[1e-2]
    # Kn = 1e-2, cell 0.5 lambda: pure DSMC everywhere
    assert np.all(ratios[1e-2] == 1.0)
    # Kn = 1e-4, cell 50 lambda: the Shakhov part carries most of the step
    assert np.median(ratios[1e-4]) < 0.2
