"""Python binding of libsp: the GB300 (sm_103a) hybrid stochastic-particle
Shakhov / DSMC time step of arXiv:2506.23917.

Argument marshalling only -- every step of the particle pipeline runs in the
CUDA kernels of ``libsp.so`` (see ``include/sp.h``).  There is no CPU
fallback: without the built library (``python -m paper_2506_23917_gb300.build``
or ``__graft_entry__.build()``) every call raises.

Configs are plain dicts, as produced by :mod:`paper_2506_23917_gb300.workloads`.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsp.so")

# precision modes (sp_precision): FP64 state and arithmetic; FP32 state with
# FP64 per-cell sums and arithmetic; FP32 state with FP32 per-cell sums and
# arithmetic (opt-in)
FP64, FP32, FP32_CELL32 = 0, 1, 2
FIELDS = ["N", "n", "ux", "uy", "uz", "T", "qx", "qy", "qz", "tau", "dtc", "ratio"]
ERRORS = ["capacity", "cell_cap", "bounce_cap", "ar_cap", "ncol_cap"]
STATUS = {0: "ok", -1: "invalid argument", -2: "CUDA runtime error", -3: "capacity exceeded",
          -4: "device error flag set", -5: "call out of order"}


class SpError(RuntimeError):
    def __init__(self, fn, code):
        super().__init__(f"{fn} failed: {STATUS.get(code, code)} ({code})")
        self.code = code


class SpConfig(C.Structure):
    _fields_ = [
        ("dim", C.c_int32), ("n", C.c_int32 * 3),
        ("lo", C.c_double * 3), ("hi", C.c_double * 3),
        ("m", C.c_double), ("R", C.c_double), ("gamma", C.c_double), ("Pr", C.c_double),
        ("omega", C.c_double), ("T_ref", C.c_double), ("mu_ref", C.c_double),
        ("d_ref", C.c_double), ("Fn", C.c_double), ("cfl", C.c_double), ("dt_fixed", C.c_double),
        ("face_bc", C.c_int32 * 6), ("face_T", C.c_double * 6), ("face_n", C.c_double * 6),
        ("face_u", (C.c_double * 3) * 6), ("ghost_layers", C.c_int32),
        ("body", C.c_int32), ("body_c", C.c_double * 3), ("body_r", C.c_double),
        ("body_Tw", C.c_double), ("cell_volume", C.POINTER(C.c_double)),
        ("sigc_T0", C.c_double), ("n_steady", C.c_int32), ("seed", C.c_uint64),
        ("mode", C.c_int32), ("ar_max", C.c_int32), ("n_surf", C.c_int32),
        ("win_lo", (C.c_double * 2) * 6), ("win_hi", (C.c_double * 2) * 6), ("ntc_carry", C.c_int32),
        ("subcells", C.c_int32), ("mesh", C.c_int32), ("mesh_r_out", C.c_double),
        ("mesh_growth", C.c_double),
    ]


SYMBOLS = ["sp_init", "sp_set_particles", "sp_step", "sp_moments", "sp_get_particles",
           "sp_set_record", "sp_get_step_record", "sp_get_cell_start", "sp_get_sigc_max",
           "sp_get_dt", "sp_get_surface", "sp_errors", "sp_sync", "sp_step_profiled", "sp_set_schedule", "sp_set_reproducible", "sp_autotune", "sp_launches_per_step", "sp_free",
           "sp_status_str", "sp_sort_cells_static", "sp_surface_coefficients",
           "sp_set_particles_f32", "sp_get_conservation"]

_lib = None


def lib():
    """Load libsp.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2506_23917_gb300.build")
        L = C.CDLL(LIB_PATH)
        P = C.c_void_p
        L.sp_init.argtypes = [C.POINTER(SpConfig), C.c_int, C.c_int, C.c_int64, P, C.POINTER(P)]
        L.sp_set_particles.argtypes = [P, C.c_int, P, P, C.c_int64]
        L.sp_set_particles_f32.argtypes = [P, C.c_int, P, P, C.c_int64]
        L.sp_step.argtypes = [P, C.c_int]
        L.sp_moments.argtypes = [P, C.c_int, C.c_int, P, C.c_int]
        L.sp_get_particles.argtypes = [P, C.c_int, P, P, P, P]
        L.sp_set_record.argtypes = [P, C.c_int]
        L.sp_get_step_record.argtypes = [P, C.c_int, P, P, P, P]
        L.sp_get_cell_start.argtypes = [P, C.c_int, P]
        L.sp_get_conservation.argtypes = [P, C.c_int, P]
        L.sp_get_sigc_max.argtypes = [P, C.c_int, P]
        L.sp_get_dt.argtypes = [P, C.c_int, P, P]
        L.sp_errors.argtypes = [P, P]
        L.sp_get_surface.argtypes = [P, C.c_int, P, P]
        L.sp_sync.argtypes = [P]
        L.sp_step_profiled.argtypes = [P, C.c_int, P, C.c_int]
        L.sp_set_schedule.argtypes = [P, C.c_int, C.c_int]
        L.sp_set_reproducible.argtypes = [P, C.c_int]
        L.sp_autotune.argtypes = [P, C.c_int, P, P]
        L.sp_launches_per_step.argtypes = [P]
        L.sp_free.argtypes = [P]
        L.sp_sort_cells_static.argtypes = [P, C.c_int64, C.c_int64, P, P, P]
        L.sp_surface_coefficients.argtypes = [C.POINTER(SpConfig), P, C.c_double, C.c_double,
                                              C.c_double, C.c_double, P, P]
        L.sp_status_str.argtypes = [C.c_int]
        L.sp_status_str.restype = C.c_char_p
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _chk(fn, rc):
    if rc != 0:
        raise SpError(fn, rc)


def make_config(cfg: dict):
    """Marshal a config dict into sp_config.  Returns (struct, keepalive)."""
    s = SpConfig()
    s.dim = cfg["dim"]
    for d in range(3):
        s.n[d] = cfg["n"][d]
        s.lo[d] = cfg["lo"][d]
        s.hi[d] = cfg["hi"][d]
    for k in ("m", "R", "gamma", "Pr", "omega", "T_ref", "mu_ref", "d_ref", "Fn", "cfl",
              "dt_fixed", "body_r", "body_Tw", "sigc_T0"):
        setattr(s, k, float(cfg[k]))
    for f in range(6):
        s.face_bc[f] = cfg["face_bc"][f]
        s.face_T[f] = cfg["face_T"][f]
        s.face_n[f] = cfg["face_n"][f]
        for d in range(3):
            s.face_u[f][d] = cfg["face_u"][f][d]
    s.ghost_layers = cfg["ghost_layers"]
    s.body = cfg["body"]
    for d in range(3):
        s.body_c[d] = cfg["body_c"][d]
    keep = None
    if cfg.get("cell_volume") is not None:
        keep = np.ascontiguousarray(cfg["cell_volume"], dtype=np.float64)
        s.cell_volume = keep.ctypes.data_as(C.POINTER(C.c_double))
    s.n_steady = cfg["n_steady"]
    s.seed = cfg["seed"]
    s.mode = cfg["mode"]
    s.ar_max = cfg["ar_max"]
    s.n_surf = int(cfg.get("n_surf", 0))
    for f in range(6):
        for i in range(2):
            s.win_lo[f][i] = cfg.get("win_lo", [[0.0, 0.0]] * 6)[f][i]
            s.win_hi[f][i] = cfg.get("win_hi", [[0.0, 0.0]] * 6)[f][i]
    s.ntc_carry = int(cfg.get("ntc_carry", 0))
    s.subcells = int(cfg.get("subcells", 0))
    s.mesh = int(cfg.get("mesh", 0))
    s.mesh_r_out = float(cfg.get("mesh_r_out", 0.0))
    s.mesh_growth = float(cfg.get("mesh_growth", 1.0))
    return s, keep


SURF_FIELDS = 7


def surface_coefficients(cfg: dict, tallies, time, rho_inf, u_inf, p_inf):
    """sp_surface_coefficients: per element (A, Cp, Cf, Ch) as [4][n_surf]
    and body dict(Cd, CL, Ch, A_ref)."""
    s, keep = make_config(cfg)
    ns = int(cfg.get("n_surf", 0))
    tal = np.ascontiguousarray(tallies, dtype=np.float64)
    if tal.shape != (SURF_FIELDS, ns):
        raise ValueError(f"tallies must be [{SURF_FIELDS}][{ns}]")
    elem = np.zeros((4, max(ns, 1)))
    body = np.zeros(4)
    _chk("sp_surface_coefficients",
         lib().sp_surface_coefficients(C.byref(s), _ptr(tal), float(time), float(rho_inf), float(u_inf),
                                       float(p_inf), _ptr(elem), _ptr(body)))
    return elem[:, :ns], dict(Cd=body[0], CL=body[1], Ch=body[2], A_ref=body[3])


def current_stream():
    """The current torch CUDA stream handle (or None for the default stream)."""
    try:
        import torch

        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover - torch absent
        pass
    return None


def sort_cells_static(keys_ptr, n, ncells, start_ptr, perm_ptr, stream=None):
    """sp_sort_cells_static on caller-owned device buffers (raw pointers):
    stable counting sort of cell keys with no device allocation."""
    st = stream if stream is not None else current_stream()
    _chk("sp_sort_cells_static", lib().sp_sort_cells_static(C.c_void_p(keys_ptr), n, ncells,
                                                             C.c_void_p(start_ptr), C.c_void_p(perm_ptr), st))


class Sim:
    """A libsp context: one or more flow instances advanced together."""

    def __init__(self, cfgs, precision=FP64, capacity=None, stream=None):
        if isinstance(cfgs, dict):
            cfgs = [cfgs]
        self.cfgs = list(cfgs)
        self.dim = self.cfgs[0]["dim"]
        self.precision = precision
        arr = (SpConfig * len(self.cfgs))()
        self._keep = []
        for i, c in enumerate(self.cfgs):
            s, keep = make_config(c)
            arr[i] = s
            self._keep.append(keep)
        self.ncells = [int(np.prod([c["n"][d] for d in range(c["dim"])])) for c in self.cfgs]
        if capacity is None:
            capacity = 1 << 20
        self.capacity = int(capacity)
        h = C.c_void_p()
        st = stream if stream is not None else current_stream()
        _chk("sp_init", lib().sp_init(arr, len(self.cfgs), precision, self.capacity, st, C.byref(h)))
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            lib().sp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_particles(self, inst, pos, vel):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        _chk("sp_set_particles", lib().sp_set_particles(self.h, inst, _ptr(pos), _ptr(vel), vel.shape[1]))

    def set_particles_ptr(self, inst, pos_ptr, vel_ptr, n):
        """Like set_particles with raw host pointers (e.g. pinned torch tensors)."""
        _chk("sp_set_particles", lib().sp_set_particles(self.h, inst, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr), n))

    def set_particles_f32(self, inst, pos, vel):
        """Like set_particles with FP32 host arrays (half the transfer)."""
        pos = np.ascontiguousarray(pos, dtype=np.float32)
        vel = np.ascontiguousarray(vel, dtype=np.float32)
        n = vel.shape[1]
        _chk("sp_set_particles_f32", lib().sp_set_particles_f32(self.h, inst, _ptr(pos), _ptr(vel), n))

    def set_particles_ptr_f32(self, inst, pos_ptr, vel_ptr, n):
        """set_particles_f32 with raw host pointers (e.g. pinned torch tensors)."""
        _chk("sp_set_particles_f32",
             lib().sp_set_particles_f32(self.h, inst, C.c_void_p(pos_ptr), C.c_void_p(vel_ptr), n))

    def step(self, n=1):
        _chk("sp_step", lib().sp_step(self.h, n))

    def step_profiled(self, n):
        """n steps with CUDA events around the kernel groups; returns summed
        ms of (collide, inject, scan + bookkeeping, scatter)."""
        ms = np.zeros(4)
        _chk("sp_step_profiled", lib().sp_step_profiled(self.h, n, _ptr(ms), 4))
        return [float(x) for x in ms]

    def sync(self):
        _chk("sp_sync", lib().sp_sync(self.h))

    def set_record(self, on=True):
        _chk("sp_set_record", lib().sp_set_record(self.h, 1 if on else 0))

    def moments(self, inst=0, kind=0):
        out = np.zeros((len(FIELDS), self.ncells[inst]))
        _chk("sp_moments", lib().sp_moments(self.h, inst, kind, _ptr(out), len(FIELDS)))
        return out

    def moments_into(self, inst, kind, out_ptr):
        """Moments into a caller-owned host buffer [12][ncells] (raw pointer)."""
        _chk("sp_moments", lib().sp_moments(self.h, inst, kind, C.c_void_p(out_ptr), len(FIELDS)))

    def count(self, inst=0):
        n = np.zeros(1, dtype=np.int64)
        _chk("sp_get_particles", lib().sp_get_particles(self.h, inst, None, None, None, _ptr(n)))
        return int(n[0])

    def particles(self, inst=0):
        M = self.count(inst)
        pos = np.zeros((self.dim, max(M, 1)))
        vel = np.zeros((3, max(M, 1)))
        cell = np.zeros(max(M, 1), dtype=np.uint32)
        n = np.zeros(1, dtype=np.int64)
        _chk("sp_get_particles", lib().sp_get_particles(self.h, inst, _ptr(pos), _ptr(vel), _ptr(cell), _ptr(n)))
        return pos[:, :M], vel[:, :M], cell[:M]

    def record(self, inst=0):
        nc = self.ncells[inst]
        cell4 = np.zeros((4, nc), dtype=np.int64)
        n_old = np.zeros(1, dtype=np.int64)
        _chk("sp_get_step_record", lib().sp_get_step_record(self.h, inst, _ptr(cell4), None, None, _ptr(n_old)))
        res = np.zeros(max(int(n_old[0]), 1), dtype=np.uint8)
        M = self.count(inst)
        perm = np.zeros(max(M, 1), dtype=np.uint32)
        _chk("sp_get_step_record", lib().sp_get_step_record(self.h, inst, None, _ptr(res), _ptr(perm), None))
        return cell4, res[: int(n_old[0])], perm[:M]

    def conservation(self, inst=0):
        """Rescale conservation record of the last recorded step, [6][ncells]:
        sum c'_d - N U_d (d = x, y, z), sum |c' - U|^2 - 3 R (N-1) T, the
        energy scale 3 R (N-1) T and the momentum scale N sqrt(|U|^2 + 3 R T),
        summed in FP64 before the store (zeros where nothing was rescaled)."""
        out = np.zeros((6, self.ncells[inst]))
        _chk("sp_get_conservation", lib().sp_get_conservation(self.h, inst, _ptr(out)))
        return out

    def cell_start(self, inst=0):
        st = np.zeros(self.ncells[inst] + 1, dtype=np.uint32)
        _chk("sp_get_cell_start", lib().sp_get_cell_start(self.h, inst, _ptr(st)))
        return st

    def sigc_max(self, inst=0):
        out = np.zeros(self.ncells[inst])
        _chk("sp_get_sigc_max", lib().sp_get_sigc_max(self.h, inst, _ptr(out)))
        return out

    def dt(self, inst=0):
        dt = np.zeros(1)
        step = np.zeros(1, dtype=np.int64)
        _chk("sp_get_dt", lib().sp_get_dt(self.h, inst, _ptr(dt), _ptr(step)))
        return float(dt[0])

    def step_index(self):
        """Global step counter (steps advanced since sp_init)."""
        dt = np.zeros(1)
        step = np.zeros(1, dtype=np.int64)
        _chk("sp_get_dt", lib().sp_get_dt(self.h, 0, _ptr(dt), _ptr(step)))
        return int(step[0])

    def surface(self, inst=0):
        """(tallies [7][n_surf]: hits, momentum to the wall x/y/z, energy to
        the wall, momentum along the inward normal, momentum along e_theta;
        sampled time)."""
        ns = int(self.cfgs[inst].get("n_surf", 0))
        out = np.zeros((SURF_FIELDS, max(ns, 1)))
        t = np.zeros(1)
        _chk("sp_get_surface", lib().sp_get_surface(self.h, inst, _ptr(out), _ptr(t)))
        return out[:, :ns], float(t[0])

    def errors(self):
        out = np.zeros(5, dtype=np.int64)
        _chk("sp_errors", lib().sp_errors(self.h, _ptr(out)))
        return dict(zip(ERRORS, (int(x) for x in out)))

    def set_reproducible(self, on=True):
        _chk("sp_set_reproducible", lib().sp_set_reproducible(self.h, 1 if on else 0))

    def set_schedule(self, cap, warps):
        _chk("sp_set_schedule", lib().sp_set_schedule(self.h, cap, warps))

    def autotune(self, steps_per_trial=3):
        """Time the candidate collision schedules on real steps; keep the fastest."""
        cap = np.zeros(1, dtype=np.int32)
        w = np.zeros(1, dtype=np.int32)
        _chk("sp_autotune", lib().sp_autotune(self.h, steps_per_trial, _ptr(cap), _ptr(w)))
        return int(cap[0]), int(w[0])

    def launches_per_step(self):
        return int(lib().sp_launches_per_step(self.h))
