"""Bird's sub-cells in the oracle (an option: Sec. II.A selects a pair
anywhere in the cell).  Pinned by

* the exact selection probabilities of a candidate's pair, from a
  quadrature of the two uniforms fine enough that every pool size divides
  it (so the frequencies are exact rationals): i uniform over the cell, j
  uniform over the other particles of i's sub-cell, or of the cell when i
  is alone in its sub-cell;
* the sub-cell order of particles placed at known sub-cell centres;
* the pseudo-Maxwell (omega = 1) anisotropy decay per step of full oracle
  steps in a homogeneous box with four sub-cells, which must equal the one
  without sub-cells (each particle still takes part in a candidate with
  probability 2/N, independently of its velocity).
"""
import math
from fractions import Fraction

import numpy as np

import oracle
from paper_2506_23917_gb300 import workloads as W


def _exact_pair_probabilities(sizes):
    """P(i, j) for sub-cells of the given sizes (slots in sub-cell order)."""
    N = sum(sizes)
    P = {}
    off = np.concatenate([[0], np.cumsum(sizes)])
    for t, m in enumerate(sizes):
        for i in range(off[t], off[t + 1]):
            pool = [j for j in range(off[t], off[t + 1]) if j != i] if m >= 2 else [j for j in range(N) if j != i]
            for j in pool:
                P[(i, j)] = Fraction(1, N) * Fraction(1, len(pool))
    return P, off


def test_pair_selection_probabilities_are_exact():
    sizes = [3, 0, 2, 1, 4]  # a sub-cell empty, one alone (falls back to the cell)
    P, off = _exact_pair_probabilities(sizes)
    N = sum(sizes)
    pools = {m - 1 for m in sizes if m >= 2} | {N - 1}
    L2 = math.lcm(*pools) * 3
    L1 = N * 5
    counts = {}
    for a in range(L1):
        u1 = (a + 0.5) / L1
        for b in range(L2):
            u2 = (b + 0.5) / L2
            ij = oracle.select_pair(N, u1, u2, soff=off)
            counts[ij] = counts.get(ij, 0) + 1
    total = L1 * L2
    assert set(counts) == set(P)
    for ij, c in counts.items():
        assert Fraction(c, total) == P[ij], (ij, Fraction(c, total), P[ij])
    # without sub-cells: j uniform over the other N - 1
    counts = {}
    for a in range(L1):
        for b in range(L2):
            ij = oracle.select_pair(N, (a + 0.5) / L1, (b + 0.5) / L2)
            counts[ij] = counts.get(ij, 0) + 1
    for (i, j), c in counts.items():
        assert i != j and Fraction(c, total) == Fraction(1, N * (N - 1))


def test_subcell_order_of_particles_at_known_subcells():
    cfg = W.base_config(2, [5, 4], [0.0, -1.0], [2.5, 1.0])
    cfg["subcells"] = 2
    cell = 2 + 5 * 3  # ix = 2, iy = 3
    dx, dy = 0.5, 0.5
    x0, y0 = 0.0 + 2 * dx, -1.0 + 3 * dy
    rng = np.random.default_rng(4)
    lab = rng.integers(0, 4, 25)  # sub-cell = sx + 2 sy
    sx, sy = lab % 2, lab // 2
    pos = np.stack([x0 + (sx + rng.uniform(0.1, 0.9, lab.size)) * dx / 2,
                    y0 + (sy + rng.uniform(0.1, 0.9, lab.size)) * dy / 2])
    order, soff = oracle.subcell_order(cfg, cell, pos)
    np.testing.assert_array_equal(order, np.argsort(lab, kind="stable"))
    np.testing.assert_array_equal(soff[:5], np.concatenate([[0], np.cumsum(np.bincount(lab, minlength=4))]))


def _aniso(v):
    C = v - v.mean(axis=1, keepdims=True)
    return np.sum(C[0] ** 2 - (C ** 2).sum(axis=0) / 3.0)


def test_subcells_keep_the_pseudo_maxwell_rate():
    N, steps, seeds = 4000, 6, 8
    cfg0 = W.homogeneous(N=N, Kn=0.02, omega=1.0, mode=W.MODE_DSMC)
    K = oracle.sigc(cfg0, 1.0)
    n = N * cfg0["Fn"]
    p_over_mu = n * cfg0["m"] * cfg0["R"] * cfg0["T_ref"] / cfg0["mu_ref"]
    dt = 0.2 / p_over_mu
    smax = 2.0 * K  # (sigma c)_max = 2 sigma(cbar) cbar (sigc_T0 = pi/16: cbar = 1); P_c = 1/2
    ncr = 0.5 * N * (N - 1) * cfg0["Fn"] * smax * dt / 1.0
    a = 1.0 - 0.5 / (N - 1)
    n0, f = math.floor(ncr), ncr - math.floor(ncr)
    expect = ((1 - f) * a ** n0 + f * a ** (n0 + 1)) ** steps
    assert abs(expect / math.exp(-0.2 * steps) - 1.0) < 3e-3
    res = {}
    for sub in (0, 4):
        r = []
        for seed in range(seeds):
            cfg = dict(cfg0, dt_fixed=dt, subcells=sub, sigc_T0=math.pi / 16.0, seed=100 + seed)
            pos, vel = W.homogeneous_particles(cfg, N, Tx=2.5, seed=11 + seed)
            o = oracle.Oracle(cfg)
            o.set_particles(pos, vel)
            B0 = _aniso(o.particles()[1])
            o.step(steps)
            r.append(_aniso(o.particles()[1]) / B0)
            assert np.allclose(o.sigc_max(), smax)
        res[sub] = (np.mean(r), np.std(r, ddof=1) / math.sqrt(seeds))
    for sub in (0, 4):
        m, se = res[sub]
        assert se < 0.02, res
        assert abs(m - expect) < 4 * se + 2e-3, (sub, m, expect, res)


def test_subcell_steps_keep_every_particle():
    """With sub-cells on, a step whose free flight is negligible (dt 1e-9)
    leaves the set of particle positions unchanged: the per-cell reordering
    neither loses nor duplicates a particle (the channel with a body has
    empty cells inside the body next to full ones)."""
    cfg, regions = W.box2d(nx=24, ny=12, ppc=40.0, body=True, inflow=False)
    pos, vel = W.fill_regions(cfg, regions, 3)
    cfg.update(subcells=2, dt_fixed=1e-9)
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    assert (np.diff(o.cell_start().astype(np.int64)) == 0).any()
    p0 = o.particles()[0]
    o.step(1)
    p1 = o.particles()[0]
    assert p1.shape == p0.shape
    key = lambda p: np.lexsort(np.round(p, 6))
    np.testing.assert_allclose(p1[:, key(p1)], p0[:, key(p0)], atol=1e-7)
