"""Pins of the oracle's collision step (Step 4 of Sec. III.B) against
invariants, closed forms and brute force.

DSMC part (Sec. II.A, NTC + VHS isotropic scattering):
  * momentum and energy conserved to 1e-12 relative by every step;
  * on a 4-particle cell, pair choice and acceptance match brute-force
    enumeration of all pairs (frequency of each pair proportional to
    sigma_T c_r / (sigma_T c_r)_max, candidate count equal to N_col);
  * for omega = 1 (constant sigma_T c_r) the stress anisotropy decays by
    exactly E[(1 - P_c/(N-1))^N_col] per step, which equals exp(-dt p/mu)
    with mu from Bird's VHS viscosity: this ties the cross-section to the
    viscosity that sets tau.
Shakhov part (Sec. II.B):
  * resampled fraction 1 - exp(-dt/tau);
  * stress anisotropy decays by exp(-dt/tau) and heat flux by
    1 - Pr (1 - exp(-dt/tau)) (Pr = 2/3), the rates that the Shakhov target
    g^S fixes;
  * a Maxwellian stays Maxwellian; conservation after the rescale.
Hybrid split (Eqs. tDSMC, tShakhov):
  * when dt_c <= tau the hybrid step is bitwise the pure-DSMC step;
  * otherwise the candidate count and the resampled fraction follow
    dt_DSMC = (tau/dt_c) dt_G and dt_SBGK = (1 - tau/dt_c) dt_G.
Moments (Step 3): the T and Q estimators are unbiased.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2506_23917_gb300 import workloads as W

FIELD = {n: i for i, n in enumerate(oracle.FIELDS)}


def _maxwell(N, T=1.0, seed=0, Tx=None):
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, math.sqrt(T), (3, N))
    if Tx is not None:
        v[0] *= math.sqrt(Tx / T)
    v -= v.mean(axis=1, keepdims=True)
    return v


def _tau_dtc(cfg, vel):
    """tau and dt_c of a one-cell context holding these velocities (from the
    oracle's own moment output)."""
    o = oracle.Oracle(cfg)
    N = vel.shape[1]
    pos = np.full((cfg["dim"], N), 0.5)
    o.set_particles(pos, vel)
    m = o.moments(0)
    return m[FIELD["tau"], 0], m[FIELD["dtc"], 0], m[FIELD["T"], 0]


def _aniso(v):
    C = v - v.mean(axis=1, keepdims=True)
    return np.sum(C[0] ** 2 - (C ** 2).sum(axis=0) / 3.0)


def _heat(v):
    C = v - v.mean(axis=1, keepdims=True)
    return np.sum((C ** 2).sum(axis=0) * C[0])


def _cons(v0, v1):
    p0, p1 = v0.sum(axis=1), v1.sum(axis=1)
    e0, e1 = (v0 ** 2).sum(), (v1 ** 2).sum()
    scale = np.abs(v0).sum()
    return np.max(np.abs(p1 - p0)) / scale, abs(e1 - e0) / e0


@pytest.mark.parametrize("mode", [W.MODE_DSMC, W.MODE_SHAKHOV, W.MODE_HYBRID])
def test_collision_conserves_momentum_and_energy(mode):
    N = 600
    cfg = W.homogeneous(N=N, Kn=0.05, omega=0.81, mode=mode)
    v = _maxwell(N, Tx=2.0, seed=1) + np.array([[0.3], [-0.2], [0.1]])
    tau, dtc, _ = _tau_dtc(cfg, v)
    dt = 2.0 * tau
    smax = 2.0 * oracle.sigc(cfg, 4.0 * math.sqrt(1.0 / math.pi))
    for step in range(5):
        v1, smax, rec, res = oracle.collide_cell(cfg, step, 0, 1.0, dt, smax, v)
        dp, de = _cons(v, v1)
        assert dp < 1e-12 and de < 1e-12
        if mode != W.MODE_SHAKHOV:
            assert rec[0] > 0
        if mode != W.MODE_DSMC:
            assert rec[2] > 0
        v = v1


def test_ntc_pair_statistics_match_brute_force_enumeration():
    """N = 4, N_col in {0, 1}: each accepted pair is chosen with probability
    (1/#pairs) * sigma c_r/(sigma c_r)_max (enumerated over all 6 pairs)."""
    N = 4
    cfg = W.homogeneous(N=N, Kn=0.05, omega=0.81, mode=W.MODE_DSMC)
    rng = np.random.default_rng(7)
    v = rng.normal(0.0, 1.0, (3, N))
    pairs = [(i, j) for i in range(N) for j in range(i + 1, N)]
    sc = np.array([oracle.sigc(cfg, float(np.linalg.norm(v[:, i] - v[:, j]))) for i, j in pairs])
    smax = 1.05 * sc.max()
    ncr = 0.8
    # dt giving N_col_real = ncr with V = 1: 0.5 N (N-1) Fn smax dt / V = ncr
    dt = ncr / (0.5 * N * (N - 1) * cfg["Fn"] * smax)
    trials = 12000
    counts = np.zeros(len(pairs))
    ncand = 0
    for t in range(trials):
        v1, s1, rec, _ = oracle.collide_cell(cfg, t, 3, 1.0, dt, smax, v)
        assert s1 == smax
        ncand += rec[0]
        if rec[1]:
            changed = tuple(np.nonzero(np.any(v1 != v, axis=0))[0])
            assert len(changed) == 2
            counts[pairs.index(changed)] += 1
    # candidate count: Bernoulli(ncr) per trial
    assert abs(ncand / trials - ncr) < 4 * math.sqrt(ncr * (1 - ncr) / trials)
    p = ncr * (sc / smax) / len(pairs)
    expected = trials * p
    chi2 = np.sum((counts - expected) ** 2 / expected)
    assert chi2 < 25.0  # 6 cells, p ~ 1e-4
    tot = counts.sum()
    assert abs(tot - expected.sum()) < 4 * math.sqrt(expected.sum())


def test_pseudo_maxwell_anisotropy_relaxes_at_p_over_mu():
    N = 2000
    cfg = W.homogeneous(N=N, Kn=0.02, omega=1.0, mode=W.MODE_DSMC)
    K = oracle.sigc(cfg, 1.0)
    assert abs(oracle.sigc(cfg, 7.3) / K - 1.0) < 1e-14  # omega = 1: sigma c_r constant
    smax = 2.0 * K  # P_c = 1/2 for every pair
    # p/mu for omega = 1: n m R T / (mu_ref T/T_ref) = n m R T_ref / mu_ref, n = N Fn / V
    n = N * cfg["Fn"] / 1.0
    p_over_mu = n * cfg["m"] * cfg["R"] * cfg["T_ref"] / cfg["mu_ref"]
    dt = 0.25 / p_over_mu
    ncr = 0.5 * N * (N - 1) * cfg["Fn"] * smax * dt / 1.0
    a = 1.0 - 0.5 / (N - 1)
    n0, f = math.floor(ncr), ncr - math.floor(ncr)
    expect = (1 - f) * a ** n0 + f * a ** (n0 + 1)
    # the finite-N factor is the continuum decay exp(-dt p/mu)
    assert abs(expect / math.exp(-0.25) - 1.0) < 1e-3
    v = _maxwell(N, Tx=2.5, seed=3)
    B0 = _aniso(v)
    ratios = []
    for t in range(160):
        v1, _, rec, _ = oracle.collide_cell(cfg, 1000 + t, 0, 1.0, dt, smax, v)
        ratios.append(_aniso(v1) / B0)
    ratios = np.array(ratios)
    se = ratios.std(ddof=1) / math.sqrt(len(ratios))
    assert abs(ratios.mean() - expect) < 4 * se + 1e-3
    # a cross-section off by the reduced-mass factor 2^(w-1/2) would miss by >5 %
    assert se < 0.01


def test_shakhov_maxwellian_stays_maxwellian():
    N = 40000
    cfg = W.homogeneous(N=N, Kn=0.01, omega=0.81, mode=W.MODE_SHAKHOV)
    v = _maxwell(N, seed=5)
    tau, _, T = _tau_dtc(cfg, v)
    x = 0.7
    dt = x * tau
    smax = 1.0
    v1, _, rec, res = oracle.collide_cell(cfg, 0, 0, 1.0, dt, smax, v)
    P = 1 - math.exp(-x)
    assert abs(rec[2] / N - P) < 4 * math.sqrt(P * (1 - P) / N)
    assert int(res.sum()) == rec[2]
    dp, de = _cons(v, v1)
    assert dp < 1e-12 and de < 1e-12
    C = v1 - v1.mean(axis=1, keepdims=True)
    RT = (C ** 2).sum() / (3 * (N - 1))
    kurt = np.mean(C ** 4) / (3 * RT ** 2)
    assert abs(kurt - 1.0) < 0.04
    for d in range(3):
        assert abs(np.mean(C[d] ** 2) / RT - 1.0) < 0.03


def test_shakhov_stress_relaxes_at_one_over_tau():
    N = 60000
    cfg = W.homogeneous(N=N, Kn=0.01, omega=0.81, mode=W.MODE_SHAKHOV)
    v = _maxwell(N, seed=9, Tx=2.0)
    tau, _, _ = _tau_dtc(cfg, v)
    x = 0.5
    B0 = _aniso(v)
    r = []
    for t in range(8):
        v1, _, _, _ = oracle.collide_cell(cfg, 50 + t, 0, 1.0, x * tau, 1.0, v)
        r.append(_aniso(v1) / B0)
    assert abs(np.mean(r) / math.exp(-x) - 1.0) < 0.02


def test_shakhov_heat_flux_relaxes_at_pr_over_tau():
    N = 100000
    cfg = W.homogeneous(N=N, Kn=0.01, omega=0.81, mode=W.MODE_SHAKHOV)
    _, v = W.homogeneous_particles(cfg, N, Tx=1.0, Tyz=1.0, skew=0.25, seed=11)
    tau, _, T = _tau_dtc(cfg, v)
    x = 0.5
    Q0 = _heat(v)
    r = []
    for t in range(12):
        v1, _, rec, _ = oracle.collide_cell(cfg, 70 + t, 0, 1.0, x * tau, 1.0, v)
        r.append(_heat(v1) / Q0)
    expect = math.exp(-x) + (1 - math.exp(-x)) * (1 - cfg["Pr"])
    bgk = math.exp(-x)
    se = np.std(r, ddof=1) / math.sqrt(len(r))
    assert abs(np.mean(r) - expect) < 4 * se + 0.01
    assert abs(np.mean(r) - bgk) > 0.08  # the Shakhov target carries (1-Pr) Q


def test_hybrid_equals_dsmc_when_observation_time_below_tau():
    N = 300
    cfg_h = W.homogeneous(N=N, Kn=5.0, omega=0.81, mode=W.MODE_HYBRID)
    cfg_d = dict(cfg_h, mode=W.MODE_DSMC)
    v = _maxwell(N, seed=2, Tx=1.5)
    tau, dtc, _ = _tau_dtc(cfg_h, v)
    assert dtc <= tau
    smax = 2.0 * oracle.sigc(cfg_h, 4.0 / math.sqrt(math.pi))
    for step in range(3):
        a = oracle.collide_cell(cfg_h, step, 5, 1.0, 0.9 * dtc, smax, v)
        b = oracle.collide_cell(cfg_d, step, 5, 1.0, 0.9 * dtc, smax, v)
        assert np.array_equal(a[0], b[0]) and a[1] == b[1] and np.array_equal(a[2], b[2])
        assert a[2][2] == 0  # nothing resampled
    # and with tau < dt_c the two differ
    cfg_h2 = W.homogeneous(N=N, Kn=1e-3, omega=0.81, mode=W.MODE_HYBRID)
    tau2, dtc2, _ = _tau_dtc(cfg_h2, v)
    assert tau2 < dtc2
    a = oracle.collide_cell(cfg_h2, 0, 5, 1.0, 0.9 * dtc2, smax, v)
    b = oracle.collide_cell(dict(cfg_h2, mode=W.MODE_DSMC), 0, 5, 1.0, 0.9 * dtc2, smax, v)
    assert not np.array_equal(a[0], b[0])


def test_hybrid_split_fractions():
    """tau/dt_c = r in (0,1): candidates follow dt_DSMC = r dt_G and the
    resampled fraction follows 1 - exp(-(1-r) dt_G / tau)."""
    N = 4000
    cfg = W.homogeneous(N=N, Kn=0.15, omega=0.81, mode=W.MODE_HYBRID)
    v = _maxwell(N, seed=4)
    tau, dtc, _ = _tau_dtc(cfg, v)
    r = tau / dtc
    assert 0.05 < r < 0.95
    dtG = 0.9 * dtc
    smax = 2.0 * oracle.sigc(cfg, 4.0 / math.sqrt(math.pi))
    ncr = 0.5 * N * (N - 1) * cfg["Fn"] * smax * (r * dtG) / 1.0
    Pres = 1 - math.exp(-(1 - r) * dtG / tau)
    ncand, nres = [], []
    for t in range(20):
        _, _, rec, _ = oracle.collide_cell(cfg, t, 2, 1.0, dtG, smax, v)
        ncand.append(rec[0])
        nres.append(rec[2])
    assert all(c in (math.floor(ncr), math.floor(ncr) + 1) for c in ncand)
    mres = np.mean(nres) / N
    assert abs(mres - Pres) < 4 * math.sqrt(Pres * (1 - Pres) / (N * 20))
    # DSMC ratio field reports min(1, tau/dt_c)
    o = oracle.Oracle(cfg)
    o.set_particles(np.full((1, N), 0.5), v)
    assert abs(o.moments(0)[FIELD["ratio"], 0] - r) < 1e-15


def test_moment_estimators_are_unbiased():
    """5 particles per cell: E[T] = T and E[q] = q of the parent distribution
    (T from 1/(N-1), Q from N/((N-1)(N-2)) of Step 3)."""
    nc, N = 40000, 5
    cfg = W.base_config(1, [nc], [0.0], [1.0])
    cfg["Fn"] = 1.0 / (N * nc)
    rng = np.random.default_rng(13)
    M = nc * N
    pos = ((np.repeat(np.arange(nc), N) + 0.5) / nc)[None, :]
    vel = np.stack([rng.exponential(1.0, M) - 1.0, rng.normal(0, 1, M), rng.normal(0, 1, M)])
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    m = o.moments(0)
    T = m[FIELD["T"]]
    qx = m[FIELD["qx"]]
    # parent: Var = 1 per component -> T = 1 (R = 1); q_x = E[|C|^2 C_x]/2 = mu3/2 = 1
    assert abs(T.mean() - 1.0) < 4 * T.std() / math.sqrt(nc)
    assert abs(qx.mean() - 1.0) < 4 * qx.std() / math.sqrt(nc)
    assert abs(m[FIELD["qy"]].mean()) < 4 * m[FIELD["qy"]].std() / math.sqrt(nc)


def _closed_cell_candidates(carry, steps, seed=1):
    """A closed homogeneous cell in pure DSMC with a fixed step and a
    (sigma c)_max seed far above any pair's sigma c, so that the NTC count
    N(N-1) F_N (sigma c)_max dt / (2 V) is the same every step."""
    N = 200
    cfg = W.homogeneous(N=N, Kn=0.3, mode=W.MODE_DSMC, dt=0.01, seed=seed)
    cfg["sigc_T0"] = 50.0
    cfg["ntc_carry"] = carry
    pos, vel = W.homogeneous_particles(cfg, N, Tx=1.0, Tyz=1.0, seed=seed)
    o = oracle.Oracle(cfg)
    o.set_particles(pos, vel)
    smax0 = o.sigc_max()[0]
    ncr = 0.5 * N * (N - 1) * cfg["Fn"] * smax0 * cfg["dt_fixed"] / 1.0
    counts = []
    for _ in range(steps):
        o.step(1)
        counts.append(int(o.record()[0][0][0]))
    assert o.sigc_max()[0] == smax0  # never raised: the count per step is constant
    return np.array(counts), ncr


def test_carried_remainder_ntc_count_telescopes():
    """Bird's carried remainder: after K steps the candidates add up to
    floor(K * N_col_real) exactly, and every step takes floor or ceil of
    N_col_real; stochastic rounding only matches it on average."""
    K = 300
    c, ncr = _closed_cell_candidates(1, K)
    assert ncr % 1.0 > 0.05 and ncr % 1.0 < 0.95
    assert c.sum() == math.floor(K * ncr)
    assert set(np.unique(c)) <= {math.floor(ncr), math.ceil(ncr)}
    for k in range(1, K + 1):
        assert abs(c[:k].sum() - k * ncr) < 1.0
    r, _ = _closed_cell_candidates(0, K)
    assert abs(r.sum() - K * ncr) < 5 * math.sqrt(K * 0.25) + 1
    assert r.sum() != c.sum() or not np.array_equal(r, c)
