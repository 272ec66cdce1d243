"""ctypes wrapper of the FP64 CPU oracle (test infrastructure only).

The oracle is the plain restatement of the hybrid SP-Shakhov / DSMC step of
arXiv:2506.23917 that the CUDA library is checked against.  Only tests, the
smoke check and the benchmark's CPU-baseline leg import this package; the
library itself never does.

Configs are plain dicts (the same dicts the input generators produce); see
``oracle.h`` for the meaning of each field.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

BC_SPECULAR, BC_DIFFUSE, BC_OUTFLOW, BC_INFLOW = 0, 1, 2, 3
BODY_NONE, BODY_CIRCLE, BODY_SPHERE = 0, 1, 2
MODE_HYBRID, MODE_DSMC, MODE_SHAKHOV = 0, 1, 2
FIELDS = ["N", "n", "ux", "uy", "uz", "T", "qx", "qy", "qz", "tau", "dtc", "ratio"]


class OrConfig(C.Structure):
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


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.or_init.argtypes = [C.POINTER(OrConfig), C.POINTER(P)]
        L.or_set_particles.argtypes = [P, P, P, C.c_int64]
        L.or_step.argtypes = [P, C.c_int]
        L.or_num_particles.argtypes = [P]
        L.or_num_particles.restype = C.c_int64
        L.or_get_particles.argtypes = [P, P, P, P]
        L.or_moments.argtypes = [P, C.c_int, P, C.c_int]
        L.or_get_step_record.argtypes = [P, P, P, P, P]
        L.or_get_cell_start.argtypes = [P, P]
        L.or_get_sigc_max.argtypes = [P, P]
        L.or_get_sample.argtypes = [P, P, P]
        L.or_dt.argtypes = [P]
        L.or_dt.restype = C.c_double
        L.or_step_index.argtypes = [P]
        L.or_step_index.restype = C.c_int64
        L.or_get_totals.argtypes = [P, P]
        L.or_set_threads.argtypes = [P, C.c_int]
        L.or_select_pair.argtypes = [C.c_int64, P, C.c_double, C.c_double, P, P]
        L.or_subcell_order.argtypes = [C.POINTER(OrConfig), C.c_int64, P, C.c_int64, P, P]
        L.or_get_threads.argtypes = [P]
        L.or_get_surface.argtypes = [P, P, P]
        L.or_mesh_locate.argtypes = [P, P, C.c_int64, P]
        L.or_mesh_geometry.argtypes = [P, P, P, P]
        L.or_get_volumes.argtypes = [P, P]
        L.or_free.argtypes = [P]
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_u01_from_words.argtypes = [C.c_uint32, C.c_uint32]
        L.or_u01_from_words.restype = C.c_double
        L.or_sigc.argtypes = [C.POINTER(OrConfig), C.c_double]
        L.or_sigc.restype = C.c_double
        L.or_collide_cell.argtypes = [C.POINTER(OrConfig), C.c_int64, C.c_uint32, C.c_double,
                                      C.c_double, P, P, C.c_int64, P, P]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def make_config(cfg: dict):
    """Marshal a config dict into the oracle's struct.  Returns (struct, keepalive)."""
    s = OrConfig()
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
    vol = cfg.get("cell_volume")
    keep = None
    if vol is not None:
        keep = np.ascontiguousarray(vol, dtype=np.float64)
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


def philox(ctr, key):
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(o))
    return o


def u01(a, b):
    return lib().or_u01_from_words(a, b)


def sigc(cfg, cr):
    s, _ = make_config(cfg)
    return lib().or_sigc(C.byref(s), cr)


def select_pair(N, u1, u2, soff=None):
    """The (i, j) slots of one NTC candidate from its uniforms u1, u2."""
    i = np.zeros(1, dtype=np.int64)
    j = np.zeros(1, dtype=np.int64)
    so = None if soff is None else np.ascontiguousarray(soff, dtype=np.int64)
    rc = lib().or_select_pair(int(N), _ptr(so), float(u1), float(u2), _ptr(i), _ptr(j))
    if rc != 0:
        raise ValueError("or_select_pair failed")
    return int(i[0]), int(j[0])


def subcell_order(cfg, cell, pos):
    """(order, soff): the stable order by sub-cell of particles pos [dim][N]
    of cell `cell` and the sub-cell offsets (cfg["subcells"] >= 2)."""
    s, keep = make_config(cfg)
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    N = pos.shape[1]
    order = np.zeros(max(N, 1), dtype=np.int64)
    soff = np.zeros(9, dtype=np.int64)
    rc = lib().or_subcell_order(C.byref(s), int(cell), _ptr(pos), N, _ptr(order), _ptr(soff))
    if rc != 0:
        raise ValueError("or_subcell_order failed")
    return order[:N], soff


def collide_cell(cfg, step, cell, volume, dt_G, sigc_max, vel):
    """One homogeneous collision step of one cell; vel is (3, N), returned updated."""
    s, _ = make_config(cfg)
    v = np.ascontiguousarray(vel, dtype=np.float64).copy()
    N = v.shape[1]
    sm = np.array([sigc_max], dtype=np.float64)
    rec = np.zeros(4, dtype=np.int64)
    res = np.zeros(max(N, 1), dtype=np.uint8)
    rc = lib().or_collide_cell(C.byref(s), step, cell, volume, dt_G, _ptr(sm), _ptr(v), N,
                               _ptr(rec), _ptr(res))
    assert rc == 0
    return v, float(sm[0]), rec, res[:N]


class Oracle:
    """One flow instance stepped by the oracle."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.dim = cfg["dim"]
        self.ncells = int(cfg["n"][0] * cfg["n"][1] * cfg["n"][2])
        s, keep = make_config(cfg)
        h = C.c_void_p()
        rc = lib().or_init(C.byref(s), C.byref(h))
        if rc != 0:
            raise ValueError(f"or_init failed: {rc}")
        self.h = h

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_free(self.h)
            self.h = None

    def set_particles(self, pos, vel):
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        vel = np.ascontiguousarray(vel, dtype=np.float64)
        M = vel.shape[1]
        rc = lib().or_set_particles(self.h, _ptr(pos), _ptr(vel), M)
        if rc != 0:
            raise ValueError(f"or_set_particles failed: {rc}")

    def step(self, n=1):
        rc = lib().or_step(self.h, n)
        assert rc == 0

    @property
    def M(self):
        return lib().or_num_particles(self.h)

    @property
    def dt(self):
        return lib().or_dt(self.h)

    @property
    def step_index(self):
        return lib().or_step_index(self.h)

    def particles(self):
        M = self.M
        pos = np.zeros((self.dim, M))
        vel = np.zeros((3, M))
        cell = np.zeros(M, dtype=np.uint32)
        lib().or_get_particles(self.h, _ptr(pos), _ptr(vel), _ptr(cell))
        return pos, vel, cell

    def moments(self, kind=0):
        out = np.zeros((len(FIELDS), self.ncells))
        lib().or_moments(self.h, kind, _ptr(out), len(FIELDS))
        return out

    def record(self):
        cell4 = np.zeros((4, self.ncells), dtype=np.int64)
        n_old = np.zeros(1, dtype=np.int64)
        lib().or_get_step_record(self.h, _ptr(cell4), None, None, _ptr(n_old))
        res = np.zeros(max(int(n_old[0]), 1), dtype=np.uint8)
        perm = np.zeros(max(self.M, 1), dtype=np.uint32)
        lib().or_get_step_record(self.h, None, _ptr(res), _ptr(perm), None)
        return cell4, res[: int(n_old[0])], perm[: self.M]

    def cell_start(self):
        st = np.zeros(self.ncells + 1, dtype=np.uint32)
        lib().or_get_cell_start(self.h, _ptr(st))
        return st

    def sigc_max(self):
        out = np.zeros(self.ncells)
        lib().or_get_sigc_max(self.h, _ptr(out))
        return out

    def sample(self):
        out = np.zeros((8, self.ncells))
        ns = np.zeros(1, dtype=np.int64)
        lib().or_get_sample(self.h, _ptr(out), _ptr(ns))
        return out, int(ns[0])

    def surface(self):
        """(tallies [7][n_surf] = hits, momentum to the wall x/y/z, energy to
        the wall, momentum along the inward normal, momentum along e_theta;
        sampled time)."""
        ns = int(self.cfg.get("n_surf", 0))
        out = np.zeros((7, max(ns, 1)))
        t = np.zeros(1)
        lib().or_get_surface(self.h, _ptr(out), _ptr(t))
        return out[:, :ns], float(t[0])

    def set_threads(self, n):
        """Threads of the per-cell loop (identical results for any count);
        returns the count in effect (1 without OpenMP)."""
        lib().or_set_threads(self.h, int(n))
        return int(lib().or_get_threads(self.h))

    def totals(self):
        out = np.zeros(4, dtype=np.int64)
        lib().or_get_totals(self.h, _ptr(out))
        return dict(removed=int(out[0]), injected=int(out[1]), move_capped=int(out[2]),
                    ar_capped=int(out[3]))

    def volumes(self):
        out = np.zeros(self.ncells)
        lib().or_get_volumes(self.h, _ptr(out))
        return out

    def mesh_locate(self, pos):
        """O-grid: the cell of each point of pos [2][n] (face-crossing walk), -1 outside."""
        pos = np.ascontiguousarray(pos, dtype=np.float64)
        n = pos.shape[1]
        out = np.zeros(max(n, 1), dtype=np.int64)
        rc = lib().or_mesh_locate(self.h, _ptr(pos), n, _ptr(out))
        if rc != 0:
            raise ValueError("not an O-grid context")
        return out[:n]

    def mesh_geometry(self):
        """O-grid: (nodes [(nr + ghost_layers + 1) * nt][2], faces [ncells][4][3], L [ncells])."""
        nr, nt = self.cfg["n"][0], self.cfg["n"][1]
        nn = (nr + max(int(self.cfg["ghost_layers"]), 0) + 1) * nt
        nodes = np.zeros((nn, 2))
        faces = np.zeros((self.ncells, 4, 3))
        L = np.zeros(self.ncells)
        rc = lib().or_mesh_geometry(self.h, _ptr(nodes), _ptr(faces), _ptr(L))
        if rc != 0:
            raise ValueError("not an O-grid context")
        return nodes, faces, L
