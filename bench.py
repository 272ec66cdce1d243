#!/usr/bin/env python3
"""Throughput of the hybrid SP-Shakhov / DSMC time step on GB300.

Workload (default): 2-D hypersonic argon flow past a cylinder -- Ma 5,
Kn = 0.01 on the radius, VHS omega = 0.81, diffuse wall at T_inf, 600 x 300
cells with analytic circular cut cells, 40 particles per freestream cell
(~6.6 M particles), FP32 particle state with FP64 per-cell sums and
per-cell arithmetic.  The
flow is developed for --develop untimed steps from a uniform freestream,
then --warmup steps, then exactly --steps timed steps (one CUDA graph per
step).  value = particle-updates/s = (mean particle count) x steps / time,
summed over ranks; under torchrun each rank advances its own independent
instance (seed = rank), so scaling is weak.

Extra keys: roofline of the dominant kernel (collision + free flight),
the same workload in plain FP64 mode, an end-to-end figure through the C
ABI with host buffers, and the CPU oracle timed on a bounded sample.
--impl reference times the CPU oracle itself as the reference arm.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s and % HBM roofline, FP32+batched vs plain FP64 on one GB300"
UNIT = "particle-updates/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=4000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--develop", type=int, default=600)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--scale", type=float, default=1.0)
    p.add_argument("--config", default="cylinder", choices=["cylinder", "sphere", "sod", "jet", "ogrid"])
    p.add_argument("--precision", default="fp32", choices=["fp32", "fp32c", "fp64"],
                   help="fp32: FP32 state, FP64 per-cell sums and arithmetic; fp32c: the opt-in "
                        "all-FP32 variant; fp64: FP64 everything")
    p.add_argument("--no-fp64", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--profile-steps", type=int, default=40)
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--no-modes", action="store_true",
                   help="skip the pure-DSMC / pure-Shakhov legs of the same workload")
    p.add_argument("--no-tune", action="store_true")
    p.add_argument("--schedule", default=None,
                   help="CAP,WARPS: fixed collision-kernel schedule instead of the autotuner")
    p.add_argument("--reproducible", action="store_true",
                   help="FP32: restore the source order inside cells in the timed run")
    p.add_argument("--batch-steps", type=int, default=200)
    p.add_argument("--no-sod", action="store_true", help="skip the FP64 Sod shock-tube leg")
    p.add_argument("--state-file", default=None,
                   help="developed particle state (.npz): loaded when the file exists, else written after "
                        "the development steps (lets a profiler start at the developed flow)")
    return p.parse_args()


def workload_name(scale, config="cylinder"):
    if config == "sphere":
        n = [max(4, int(round(v * scale))) for v in (256, 128, 128)]
        return f"sphere3d_{n[0]}x{n[1]}x{n[2]}_ppc30_Ma10_Kn0.005_Tw4_argon_vhs"
    if config == "sod":
        return "sod1d_200cells_ppc500_62.5_lam1e-3_hardsphere"
    if config == "jet":
        nc = max(8, int(round(512 * scale)))
        return f"jet2d_{nc}x{nc}_orifice_ppc500_plenum4x_Ma1_Kn0.02_n2like_vhs"
    if config == "ogrid":
        nr, nt = max(4, int(round(150 * scale))), max(8, int(round(600 * scale)))
        return f"cylinder2d_ogrid_{nr}x{nt}_rout4_growth1.01_ppc40_Ma5_Kn0.01_argon_vhs"
    nx, ny = max(4, int(round(600 * scale))), max(2, int(round(300 * scale)))
    return f"cylinder2d_{nx}x{ny}_ppc40_Ma5_Kn0.01_argon_vhs"


def make_workload(W, config, scale, seed):
    if config == "sphere":
        cfg, regions = W.sphere(scale=scale, seed=seed, n_steady=0)
    elif config == "jet":
        cfg, regions = W.jet(scale=scale, seed=seed, n_steady=0)
    elif config == "sod":
        cfg, regions = W.sod(ncell=200, ppc_left=500.0, lam_left=1e-3, seed=seed, n_steady=0)
    elif config == "ogrid":
        cfg, regions = W.cylinder_ogrid(nr=max(4, int(round(150 * scale))), nt=max(8, int(round(600 * scale))),
                                        r_out=4.0, growth=1.01, ppc=40.0, Kn=0.01, seed=seed, n_steady=0)
    else:
        cfg, regions = W.cylinder(scale=scale, seed=seed, n_steady=0)
    pos, vel = W.fill_regions(cfg, regions, seed)
    return cfg, pos, vel


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            P = json.load(f)
        return float(P["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def collide_profile(src_hash):
    """Per-particle figures of the collision kernel from the committed ncu
    summary (DRAM bytes, warp-instructions), if it was taken on the current
    kernel source; else {}."""
    path = os.path.join(ROOT, "profiles", "collide_cylinder_traffic.txt")
    try:
        kv = {}
        for line in open(path):
            if "=" in line and not line.startswith("#"):
                k, v = line.strip().split("=", 1)
                kv[k.strip()] = v.strip()
        if kv.get("source_sha256") != src_hash:
            return {}
        return {k: float(v) for k, v in kv.items()
                if k in ("bytes_per_particle", "inst_per_particle", "threads_per_inst")}
    except Exception:
        return {}


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("sp_device.cuh", "sp_kern.cu", "sp_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_2506_23917_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def crop_config(cfg, x0, x1, y1):
    """A sub-window of the cylinder grid (same cells) with open faces, used to
    time the CPU oracle on a bounded sample of the workload."""
    from paper_2506_23917_gb300 import workloads as W

    dl = W.cell_size(cfg)
    i0 = int(round((x0 - cfg["lo"][0]) / dl[0]))
    i1 = int(round((x1 - cfg["lo"][0]) / dl[0]))
    j1 = int(round((y1 - cfg["lo"][1]) / dl[1]))
    c = dict(cfg)
    c["n"] = [i1 - i0, j1, 1]
    c["lo"] = [cfg["lo"][0] + i0 * dl[0], cfg["lo"][1], 0.0]
    c["hi"] = [cfg["lo"][0] + i1 * dl[0], cfg["lo"][1] + j1 * dl[1], 1.0]
    vol = np.asarray(cfg["cell_volume"]).reshape(cfg["n"][1], cfg["n"][0])
    c["cell_volume"] = np.ascontiguousarray(vol[:j1, i0:i1]).ravel()
    c["face_bc"] = [W.BC_OUTFLOW, W.BC_OUTFLOW, W.BC_SPECULAR, W.BC_OUTFLOW, W.BC_SPECULAR, W.BC_SPECULAR]
    c["face_n"] = [0.0] * 6
    return c


def time_oracle(cfg, pos, vel, budget_s, max_steps, min_steps=1, threads=1):
    """Step the oracle on (cfg, pos, vel) for up to budget_s seconds, its
    per-cell loop on `threads` threads (identical results for any count)."""
    import oracle

    o = oracle.Oracle(cfg)
    o.set_threads(threads)
    o.set_particles(pos, vel)
    upd, t, n = 0, 0.0, 0
    while n < max_steps and (n < min_steps or t < budget_s):
        m = o.M
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        upd += m
        n += 1
    return upd, t, n


def cpu_sample(cfg, pos, vel, budget_s=12.0):
    """The oracle on a window of the developed state, single-threaded and on
    every host core (the per-cell loop over threads)."""
    import oracle

    x0, x1, y1 = -1.8, 0.4, 1.5
    c = crop_config(cfg, x0, x1, y1)
    m = (pos[0] >= c["lo"][0]) & (pos[0] < c["hi"][0]) & (pos[1] < c["hi"][1])
    cores = os.cpu_count() or 1
    probe = oracle.Oracle(c)
    cores = probe.set_threads(cores)
    out = {}
    for nt in sorted({1, cores}):
        upd, t, n = time_oracle(c, pos[:, m], vel[:, m], budget_s, max_steps=10 ** 6, min_steps=2, threads=nt)
        out[nt] = (upd / t, n)
    sample = (f"oracle (FP64) on a {c['n'][0]}x{c['n'][1]}-cell window [{x0},{x1}]x[0,{y1}] R of the "
              f"developed state ({int(m.sum())} particles), {out[cores][1]} steps on {cores} threads "
              f"(per-cell loop over threads; the move, injection and sort stay sequential)")
    return out[cores][0], cores, sample, out[1][0]


def run_reference(args):
    """Reference arm: the CPU oracle as it stands, on a window of the same
    workload (uniform freestream start), sized so the run ends in minutes."""
    from paper_2506_23917_gb300 import workloads as W

    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cfg, regions = W.cylinder(scale=args.scale, n_steady=0)
    total = args.steps + args.warmup
    per_step_s = max(0.02, min(1.0, 120.0 / max(total, 1)))
    target = per_step_s * 3.0e6  # particles the oracle moves in per_step_s
    ppc = 40.0
    dl = W.cell_size(cfg)
    w = max(8, int(math.sqrt(target / ppc)))
    x1 = -1.0 + 0.3
    x0 = max(cfg["lo"][0], x1 - w * dl[0])
    y1 = min(cfg["hi"][1], w * dl[1])
    c = crop_config(cfg, x0, x1, y1)
    reg = [dict(lo=[c["lo"][0], 0.0], hi=[c["hi"][0], c["hi"][1]], n=cfg["face_n"][0], T=273.0,
                u=cfg["face_u"][0])]
    pos, vel = W.fill_regions(c, reg, 1)
    import oracle

    o = oracle.Oracle(c)
    cores = o.set_threads(os.cpu_count() or 1)
    o.set_particles(pos, vel)
    o.step(args.warmup)
    upd, t = 0, 0.0
    for _ in range(args.steps):
        m = o.M
        t0 = time.perf_counter()
        o.step(1)
        t += time.perf_counter() - t0
        upd += m
    value = upd / t if t > 0 else 0.0
    sample = (f"oracle (FP64, per-cell loop on {cores} threads) on a {c['n'][0]}x{c['n'][1]}-cell window of the "
              f"{workload_name(args.scale)} grid from a uniform freestream start, {len(vel[0])} particles")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload_name(args.scale), "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def reduce_timing(ms, updates, dist, device):
    """Whole-job figures: the slowest rank's time and the sum of the
    particle updates of all ranks (each rank advances its own instance)."""
    if dist is None:
        return ms, updates
    import torch

    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([updates], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def rank_seed(rank):
    """Each rank's instance gets its own Philox key and initial particles."""
    return 1 + rank


def bench_batch(sp, torch, stream, steps, dist=None, device="cuda"):
    """256 independent 1-D instances of uneven size.  Four legs: FP32 (FP64
    per-cell arithmetic) and plain FP64, each as one batched context
    (autotuned schedule; one set of launches per step) and as 256 separate
    contexts stepped one after another.  Under torchrun the instances are
    partitioned over the ranks (rank r: i = r mod N, no collective in the
    step); times are the slowest rank's, updates the sum over ranks."""
    from paper_2506_23917_gb300 import ensemble
    from paper_2506_23917_gb300 import workloads as W

    insts = W.batch(n_inst=256, seed=1, n_steady=0)
    world = dist.get_world_size() if dist else 1
    rank = dist.get_rank() if dist else 0
    mine = [insts[i] for i in ensemble.owned(len(insts), world, rank)]
    M = sum(v.shape[1] for _, _, v in mine)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn, k):
        torch.cuda.synchronize()
        e0.record(stream)
        fn(k)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def batched(prec, k):
        sim = sp.Sim([c for c, _, _ in mine], prec, capacity=int(1.3 * M) + 10000)
        if prec != sp.FP64:
            sim.set_reproducible(False)
        for i, (c, p, v) in enumerate(mine):
            sim.set_particles(i, p, v)
        sim.step(5)
        sched = sim.autotune(steps_per_trial=3)
        sim.step(3)
        sim.sync()
        t = timed(sim.step, k)
        sim.sync()
        launches = sim.launches_per_step()
        sim.close()
        return t, launches, sched

    def separate(prec, k):
        sims = []
        for c, p, v in mine:
            s = sp.Sim(c, prec, capacity=int(1.3 * v.shape[1]) + 1000)
            if prec != sp.FP64:
                s.set_reproducible(False)
            s.set_particles(0, p, v)
            s.step(5)
            sims.append(s)
        for s in sims:
            s.sync()

        def run(n):
            for _ in range(n):
                for s in sims:
                    s.step(1)

        t = timed(run, k)
        for s in sims:
            s.sync()
        launches = sum(s.launches_per_step() for s in sims)
        for s in sims:
            s.close()
        return t, launches

    ks = max(5, steps // 10)
    legs = {}
    for name, prec, k, fn in (("fp32_batched", sp.FP32, steps, batched), ("fp64_batched", sp.FP64, ks, batched),
                              ("fp32_separate", sp.FP32, ks, separate), ("fp64_separate", sp.FP64, ks, separate)):
        r = fn(prec, k)
        t, upd = reduce_timing(r[0], k * M, dist, device)
        legs[name] = {"value": upd / (t * 1e-3), "unit": UNIT, "ms_per_step": t / k, "steps": k,
                      "launches_per_step": r[1]}
        if fn is batched and r[2]:
            legs[name]["schedule"] = {"cap": r[2][0], "warps_per_block": r[2][1]}
    v = {k2: legs[k2]["value"] for k2 in legs}
    return {"workload": "256 x 1-D (even: Sod, nx = 2N/112.5; odd: homogeneous relaxation), "
                        "N log-uniform 1e3..5e5, Kn log-uniform 1e-4..1",
            "particles": int(sum(v_.shape[1] for _, _, v_ in insts)), "ranks": world,
            "partition": "rank r advances instances i = r mod N (strong scaling: fixed total work)",
            **legs,
            "batching_gain_fp32": v["fp32_batched"] / v["fp32_separate"],
            "batching_gain_fp64": v["fp64_batched"] / v["fp64_separate"],
            "precision_gain_batched": v["fp32_batched"] / v["fp64_batched"],
            "speedup": v["fp32_batched"] / v["fp64_separate"]}


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    import paper_2506_23917_gb300 as sp
    from paper_2506_23917_gb300 import build as spbuild
    from paper_2506_23917_gb300 import workloads as W

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        spbuild.build()
    if dist:
        dist.barrier()

    def barrier():
        if dist:
            dist.barrier()

    cfg, pos, vel = make_workload(W, args.config, args.scale, rank_seed(rank))
    M_init = vel.shape[1]
    cap = int(1.5 * M_init) + 200000
    stream = torch.cuda.current_stream()
    prec = {"fp32": sp.FP32, "fp32c": sp.FP32_CELL32, "fp64": sp.FP64}[args.precision]
    sim = sp.Sim(cfg, prec, capacity=cap)
    if prec != sp.FP64 and not args.reproducible:
        sim.set_reproducible(False)  # FP32 mode is checked statistically
    developed = args.develop
    if args.state_file and os.path.exists(args.state_file):
        z = np.load(args.state_file)
        sim.set_particles(0, z["pos"], z["vel"])
        developed = int(z["steps"])
    else:
        sim.set_particles(0, pos, vel)
        sim.step(args.develop)
        sim.sync()
        if args.state_file:
            ps, vs, _ = sim.particles(0)
            np.savez(args.state_file, pos=ps, vel=vs, steps=args.develop)
    if args.schedule:
        sched = tuple(int(x) for x in args.schedule.split(","))
        sim.set_schedule(*sched)
    else:
        sched = sim.autotune(steps_per_trial=20) if not args.no_tune else None
    sim.step(args.warmup)
    sim.sync()
    M0 = sim.count(0)
    launches = sim.launches_per_step()

    clocks = Clocks(local)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    sim.sync()
    ms = e0.elapsed_time(e1)
    M1 = sim.count(0)
    upd = args.steps * 0.5 * (M0 + M1)
    t_max, upd_sum = reduce_timing(ms, upd, dist, "cuda")
    value = upd_sum / (t_max * 1e-3)
    ms_per_step = t_max / args.steps

    # --- the same workload with the within-cell order restored every step
    # (bit-reproducible runs; FP64 mode always runs this way)
    repro = None
    if prec != sp.FP64 and not args.reproducible:
        sim.set_reproducible(True)
        sim.step(5)
        sim.sync()
        m0r = sim.count(0)
        kr = max(50, args.steps // 4)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.step(kr)
        e1.record(stream)
        torch.cuda.synchronize()
        sim.sync()
        tr = e0.elapsed_time(e1)
        repro = {"value": world * kr * 0.5 * (m0r + sim.count(0)) / (tr * 1e-3), "unit": UNIT,
                 "ms_per_step": tr / kr, "steps": kr,
                 "note": "source order restored inside every cell (bit-reproducible)"}
        sim.set_reproducible(False)

    # --- roofline of the dominant kernel (collision + free flight), measured
    # by CUDA event nodes around each kernel group of the step graph (the
    # graph the timed steps run), on the library's stream
    prof = sim.step_profiled(args.profile_steps)
    sim.sync()
    Mp = sim.count(0)
    S = 4 * (cfg["dim"] + 3) if prec != sp.FP64 else 8 * (cfg["dim"] + 3)
    collide_ms = prof[0] / args.profile_steps
    bytes_collide = (2 * S + 4) * Mp  # state read + state write + new key
    peak, peak_kind = load_peaks()
    achieved = bytes_collide / (collide_ms * 1e-3) / 1e9
    src_hash = kernel_source_hash()
    # the committed ncu figures cover the FP32 cylinder only
    prof_pp = collide_profile(src_hash) if (args.config == "cylinder" and prec == sp.FP32) else {}
    tpp = prof_pp.get("bytes_per_particle")
    step_ms = sum(prof) / args.profile_steps
    step_bytes = (2 * S + 8) * Mp
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": (tpp * Mp) if tpp is not None else None,
                "kernel": "k_collide (gather + moments + DSMC + Shakhov + rescale + sample + move + key)",
                "bytes_per_particle": 2 * S + 4, "peak_source": f"{peak_kind} hbm_gbs",
                "kernel_ms": collide_ms,
                "share_of_step": prof[0] / sum(prof),
                "group_ms_per_step": {k: v / args.profile_steps for k, v in
                                      zip(["collide", "inject", "scan", "scatter"], prof)},
                "step_frac": step_bytes / (step_ms * 1e-3) / 1e9 / peak,
                "step_bytes_per_particle": 2 * S + 8}
    # instruction-issue roof of the same kernel: warp-instructions per
    # particle (ncu) x particles / kernel time, against SMs x 4 schedulers x
    # the SM clock under load (one warp-instruction per scheduler per cycle)
    ipp = prof_pp.get("inst_per_particle")
    nsm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = clk.get("sm_mhz") or 2070.0
    issue_peak = nsm * 4 * clk_mhz * 1e6
    roofline["issue"] = {"inst_per_particle": ipp, "threads_per_inst": prof_pp.get("threads_per_inst"),
                         "unit": "warp-inst/s", "peak": issue_peak,
                         "achieved": (ipp * Mp / (collide_ms * 1e-3)) if ipp else None,
                         "frac": (ipp * Mp / (collide_ms * 1e-3) / issue_peak) if ipp else None,
                         "source": "ncu smsp__inst_executed.sum of the committed profile" if ipp else
                                   "no profile of the current kernel source"}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if prec != sp.FP64 else "f64", "data": "synthetic",
            "config": {"workload": workload_name(args.scale, args.config),
                       "cells": int(np.prod(cfg["n"][:cfg["dim"]])),
                       "particles_per_rank": int(0.5 * (M0 + M1)), "developed_steps": developed,
                       "state": {sp.FP32: "FP32 particles; per-cell sums accumulated to FP64 accuracy "
                                          "and all per-cell arithmetic in FP64",
                                 sp.FP32_CELL32: "FP32 particles, FP32 per-cell sums and arithmetic "
                                                 "(opt-in variant)",
                                 sp.FP64: "FP64"}[prec],
                       "l2": "inputs larger than L2 (state 2 x %.0f MB)" % (S * M0 / 1e6),
                       "graph": "one CUDA graph per step", "parallelism": f"replicas{world}",
                       "schedule": {"cap": sched[0], "warps_per_block": sched[1]} if sched else "default"},
            "clocks": clk, "gpu_launches": launches * args.steps, "roofline": roofline}
    line["config"]["within_cell_order"] = ("source order (bit-reproducible)" if (prec == sp.FP64 or args.reproducible)
                                           else "scatter order (statistically identical, not bit-reproducible)")
    if repro:
        line["fp32_reproducible_order"] = repro

    # --- plain FP64 form of the same workload
    if not args.no_fp64 and prec != sp.FP64:
        sim64 = sp.Sim(cfg, sp.FP64, capacity=cap)
        sim64.set_particles(0, pos, vel)
        sim64.step(args.develop)
        sim64.sync()
        sim64.step(args.warmup)
        sim64.sync()
        k64 = max(20, args.steps // 10)
        m0 = sim64.count(0)
        torch.cuda.synchronize()
        e0.record(stream)
        sim64.step(k64)
        e1.record(stream)
        torch.cuda.synchronize()
        sim64.sync()
        t64 = e0.elapsed_time(e1)
        m1 = sim64.count(0)
        v64 = k64 * 0.5 * (m0 + m1) / (t64 * 1e-3)
        p64 = sim64.step_profiled(10)
        line["fp64_plain"] = {"value": v64 * world, "unit": UNIT, "ms_per_step": t64 / k64, "steps": k64,
                              "collide_ms": p64[0] / 10, "fp32_over_fp64": value / (v64 * world)}
        sim64.close()

    # --- the opt-in all-FP32 per-cell variant on the same developed state
    if not args.no_modes and prec == sp.FP32 and rank == 0:
        po, vo, _ = sim.particles(0)
        sv = sp.Sim(cfg, sp.FP32_CELL32, capacity=cap)
        if not args.reproducible:
            sv.set_reproducible(False)
        sv.set_particles(0, po, vo)
        if sched:
            sv.set_schedule(*sched)
        sv.step(args.warmup + 20)
        sv.sync()
        kv = max(200, args.steps // 5)
        m0 = sv.count(0)
        torch.cuda.synchronize()
        e0.record(stream)
        sv.step(kv)
        e1.record(stream)
        torch.cuda.synchronize()
        sv.sync()
        tv = e0.elapsed_time(e1)
        line["precision_variants"] = {"fp32_cell32": {
            "value": kv * 0.5 * (m0 + sv.count(0)) / (tv * 1e-3), "unit": UNIT, "ms_per_step": tv / kv,
            "steps": kv, "note": "FP32 per-cell sums and arithmetic (opt-in), same state and schedule"}}
        sv.close()

    # --- Sod shock tube in FP64: 200 cells, 500 / 62.5 particles per cell
    # (56 250 particles), 400 steps at CFL 0.5 (L2-resident and latency bound)
    if not args.no_sod and rank == 0:
        cs, ps, vs = make_workload(W, "sod", 1.0, 1)
        s1 = sp.Sim(cs, sp.FP64, capacity=4 * vs.shape[1])
        s1.set_particles(0, ps, vs)
        s1.step(3)
        s1.sync()
        n_sod = 400
        m0 = s1.count(0)
        torch.cuda.synchronize()
        e0.record(stream)
        s1.step(n_sod)
        e1.record(stream)
        torch.cuda.synchronize()
        s1.sync()
        ts = e0.elapsed_time(e1)
        line["sod_fp64"] = {"workload": workload_name(1.0, "sod"), "value": n_sod * 0.5 * (m0 + s1.count(0)) / (ts * 1e-3),
                            "unit": UNIT, "ms_per_step": ts / n_sod, "steps": n_sod, "particles": m0}
        s1.close()

    # --- the same workload with one collision sub-step forced everywhere
    # (pure DSMC and pure stochastic-particle Shakhov), the method's two
    # limits, in the headline's precision and schedule
    if not args.no_modes and rank == 0:
        modes = {}
        for name, mode in (("dsmc", W.MODE_DSMC), ("shakhov", W.MODE_SHAKHOV)):
            cfg_m = dict(cfg, mode=mode)
            sm = sp.Sim(cfg_m, prec, capacity=cap)
            if prec != sp.FP64 and not args.reproducible:
                sm.set_reproducible(False)
            sm.set_particles(0, pos, vel)
            if sched:
                sm.set_schedule(*sched)
            sm.step(args.develop)
            sm.step(args.warmup)
            sm.sync()
            km = max(100, args.steps // 10)
            m0 = sm.count(0)
            torch.cuda.synchronize()
            e0.record(stream)
            sm.step(km)
            e1.record(stream)
            torch.cuda.synchronize()
            sm.sync()
            tm = e0.elapsed_time(e1)
            modes[name] = {"value": km * 0.5 * (m0 + sm.count(0)) / (tm * 1e-3), "unit": UNIT,
                           "ms_per_step": tm / km, "steps": km}
            sm.close()
        modes["note"] = "same workload, mode forced in every cell (hybrid = the headline)"
        line["pure_modes"] = modes

    # --- end to end through the C ABI with host buffers: per step, upload
    # the state from pinned host memory, advance one step, read the moments
    if not args.no_e2e:
        po, vo, _ = sim.particles(0)
        n_e2e = po.shape[1]
        # the context's own precision on the host side (FP32 state: FP32 input)
        hdt = np.float32 if prec != sp.FP64 else np.float64
        hp = torch.from_numpy(np.ascontiguousarray(po, dtype=hdt)).pin_memory()
        hv = torch.from_numpy(np.ascontiguousarray(vo, dtype=hdt)).pin_memory()
        upload = sim.set_particles_ptr_f32 if prec != sp.FP64 else sim.set_particles_ptr
        out = torch.empty((len(sp.FIELDS), sim.ncells[0]), dtype=torch.float64).pin_memory()
        K2 = 20
        for it in range(K2 + 2):
            if it == 2:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
            upload(0, hp.data_ptr(), hv.data_ptr(), n_e2e)
            sim.step(1)
            sim.moments_into(0, 0, out.data_ptr())
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        line["e2e"] = {"value": world * K2 * n_e2e / te, "unit": UNIT,
                       "h2d_bytes_per_step": hp.element_size() * (cfg["dim"] + 3) * n_e2e,
                       "d2h_bytes_per_step": 8 * len(sp.FIELDS) * sim.ncells[0],
                       "note": "per step: pinned host state -> device, one step, moments -> pinned host"}

    # --- batched ensemble: 256 independent 1-D Sod / relaxation instances of
    # uneven size, FP32 in one context (one set of launches per step) vs the
    # plain FP64 form as 256 separate contexts stepped one after another
    if not args.no_batch:
        line["batch256"] = bench_batch(sp, torch, stream, args.batch_steps, dist, "cuda")

    # --- CPU oracle on a bounded sample of the same (developed) state
    if rank == 0 and world >= 1 and not args.no_cpu and args.config == "cylinder":
        po, vo, _ = sim.particles(0)
        v_cpu, cores, sample, v_cpu1 = cpu_sample(cfg, po, vo)
        line["cpu_baseline"] = {"value": v_cpu, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                                "single_thread": v_cpu1}
    sim.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
