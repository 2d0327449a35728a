"""FP64 CPU oracle for the DEM step (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's CPU
baseline leg import this package.  The product path (the CUDA library and its
binding) never does.  The arithmetic lives in ``dem_oracle.c``; this module
only marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

PRED_FP64 = 0
PRED_FIXED_F32 = 1
PRED_ABS_F32 = 2


WALL_RECT, WALL_LINE = 0, 1


class Wall(C.Structure):
    """Rectangle p + s u + t v (u perpendicular to v) or segment p + s u,
    s, t in [0, 1]."""
    _fields_ = [
        ("kind", C.c_int32),
        ("pad", C.c_int32),
        ("p", C.c_double * 3),
        ("u", C.c_double * 3),
        ("v", C.c_double * 3),
    ]


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("g", C.c_double * 3),
        ("dt", C.c_double),
        ("E", C.c_double),
        ("poisson", C.c_double),
        ("density", C.c_double),
        ("restitution", C.c_double),
        ("mu_d", C.c_double),
        ("periodic", C.c_int32 * 3),
        ("floor_wall", C.c_int32),
        ("ncell", C.c_int32 * 3),
        ("predicate", C.c_int32),
        ("kn_literal", C.c_int32),
        ("brute_force", C.c_int32),
        ("stencil", C.c_int32),
        ("nwalls", C.c_int32),
        ("walls", C.POINTER(Wall)),
    ]


class ContactInfo(C.Structure):
    _fields_ = [
        ("F", C.c_double * 3),
        ("nF", C.c_double * 3),
        ("n", C.c_double * 3),
        ("kt", C.c_double),
        ("scale", C.c_double),
        ("delta_n", C.c_double),
        ("ratio", C.c_double),
        ("capped", C.c_int32),
        ("pad", C.c_int32),
    ]


INFO_DTYPE = np.dtype([("F", "<f8", 3), ("nF", "<f8", 3), ("n", "<f8", 3),
                       ("kt", "<f8"), ("scale", "<f8"),
                       ("delta_n", "<f8"), ("ratio", "<f8"), ("capped", "<i4"),
                       ("pad", "<i4")])
assert INFO_DTYPE.itemsize == C.sizeof(ContactInfo)

_libs = {}


def lib(parallel: bool = False):
    """The serial oracle library, or its OpenMP build (same results, all
    host cores) with parallel=True."""
    if parallel not in _libs:
        path = _build.build(parallel=parallel)
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_restitution.restype = C.c_double
        L.orc_restitution.argtypes = [C.c_double]
        L.orc_alpha.restype = C.c_double
        L.orc_alpha.argtypes = [C.c_double]
        L.orc_kn.restype = C.c_double
        L.orc_kn.argtypes = [C.POINTER(Params), C.c_double, C.c_double]
        L.orc_order.restype = C.c_int
        L.orc_order.argtypes = [C.POINTER(Params), C.c_int64, dp, ip, ip]
        L.orc_contacts.restype = C.c_int64
        L.orc_contacts.argtypes = [C.POINTER(Params), C.c_int64, dp, dp,
                                   C.c_int64, ip, ip]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.POINTER(Params), C.c_int64, dp, dp, dp, dp,
                               C.c_int64, ip, ip, dp, dp,
                               C.c_int64, C.POINTER(C.c_int64), ip, ip, dp,
                               C.c_void_p, dp, dp]
        _libs[parallel] = L
    return _libs[parallel]


def make_params(L, dt, E=3e9, poisson=0.3, density=1200.0, restitution=0.5,
                mu_d=0.3, periodic=(1, 1, 1), floor_wall=0, g=(0.0, 0.0, 0.0),
                ncell=None, predicate=PRED_FP64, kn_literal=0,
                brute_force=0, r_max=None, stencil=1, walls=()) -> Params:
    """Fill a Params struct.  ``ncell`` defaults to the largest grid whose
    cells are at least 2 r_max (1 + 1e-5) / stencil wide.  ``walls``: a
    sequence of (kind, p, u, v) with kind WALL_RECT or WALL_LINE (v unused
    for a line)."""
    p = Params()
    L = [float(v) for v in (L if np.ndim(L) else (L, L, L))]
    for a in range(3):
        p.L[a] = L[a]
        p.g[a] = float(g[a])
        p.periodic[a] = int(periodic[a])
    if ncell is None:
        if r_max is None:
            raise ValueError("ncell or r_max required")
        ncell = [max(1, int(np.floor(L[a] * stencil / (2.0 * r_max * (1.0 + 1e-5)))))
                 for a in range(3)]
    for a in range(3):
        p.ncell[a] = int(ncell[a])
    p.dt = float(dt)
    p.E = float(E)
    p.poisson = float(poisson)
    p.density = float(density)
    p.restitution = float(restitution)
    p.mu_d = float(mu_d)
    p.floor_wall = int(floor_wall)
    p.predicate = int(predicate)
    p.kn_literal = int(kn_literal)
    p.brute_force = int(brute_force)
    p.stencil = int(stencil)
    walls = list(walls)
    p.nwalls = len(walls)
    if walls:
        arr = (Wall * len(walls))()
        for k, (kind, pw, uw, vw) in enumerate(walls):
            arr[k].kind = int(kind)
            for a in range(3):
                arr[k].p[a] = float(pw[a])
                arr[k].u[a] = float(uw[a])
                arr[k].v[a] = float(vw[a]) if vw is not None else 0.0
        p.walls = C.cast(arr, C.POINTER(Wall))
        p._walls_keepalive = arr  # the struct only holds a pointer
    return p


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _i(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def restitution(alpha: float) -> float:
    return lib().orc_restitution(float(alpha))


def alpha(e: float) -> float:
    return lib().orc_alpha(float(e))


def kn(p: Params, r1: float, r2: float) -> float:
    return lib().orc_kn(C.byref(p), float(r1), float(r2))


def order(p: Params, x: np.ndarray):
    """Return (cell, order): linear cell per id and ids sorted by
    (Morton code of the cell, id)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    n = x.shape[0]
    cell = np.zeros(n, np.int32)
    order = np.zeros(n, np.int32)
    rc = lib().orc_order(C.byref(p), n, _d(x), _i(cell), _i(order))
    if rc:
        raise RuntimeError("orc_order failed")
    return cell, order


def contacts(p: Params, x: np.ndarray, r: np.ndarray, cap: int | None = None,
             parallel: bool = False):
    x = np.ascontiguousarray(x, dtype=np.float64)
    r = np.ascontiguousarray(r, dtype=np.float64)
    n = x.shape[0]
    cap = cap or max(64, 32 * n)
    lo = np.zeros(cap, np.int32)
    hi = np.zeros(cap, np.int32)
    cnt = lib(parallel).orc_contacts(C.byref(p), n, _d(x), _d(r), cap, _i(lo), _i(hi))
    if cnt < 0:
        raise RuntimeError(f"orc_contacts failed ({cnt})")
    return lo[:cnt].copy(), hi[:cnt].copy()


class State:
    """Particle state in id order plus the contact history."""

    def __init__(self, x, v, w, r, floor_wall=False, nwalls=0):
        self.x = np.array(x, dtype=np.float64, order="C")
        self.v = np.array(v, dtype=np.float64, order="C")
        self.w = np.array(w, dtype=np.float64, order="C")
        self.r = np.array(r, dtype=np.float64, order="C")
        n = self.x.shape[0]
        self.lo = np.zeros(0, np.int32)
        self.hi = np.zeros(0, np.int32)
        self.dt = np.zeros((0, 3), np.float64)
        nw = (1 if floor_wall else 0) + int(nwalls)
        # per particle and wall (the floor first): delta_t history
        self.wall_dt = np.zeros((n, nw, 3), np.float64) if nw else None

    @property
    def n(self):
        return self.x.shape[0]


def step(p: Params, s: State, cap: int | None = None, parallel: bool = False):
    """Advance ``s`` by one step in place.  Returns a dict with the forces
    and torques used in the step and per-contact info of the new list.
    parallel=True runs the OpenMP build (same results, bit for bit)."""
    n = s.n
    cap = cap or max(64, 32 * n)
    lo = np.zeros(cap, np.int32)
    hi = np.zeros(cap, np.int32)
    dto = np.zeros((cap, 3), np.float64)
    info = np.zeros(cap, INFO_DTYPE)
    F = np.zeros((n, 3), np.float64)
    T = np.zeros((n, 3), np.float64)
    nc = C.c_int64(0)
    lo_in = np.ascontiguousarray(s.lo, np.int32)
    hi_in = np.ascontiguousarray(s.hi, np.int32)
    dt_in = np.ascontiguousarray(s.dt, np.float64).reshape(-1, 3)
    if lo_in.size == 0:
        lo_in = np.zeros(1, np.int32)
        hi_in = np.zeros(1, np.int32)
        dt_in = np.zeros((1, 3), np.float64)
        n_in = 0
    else:
        n_in = s.lo.size
    wall = s.wall_dt
    rc = lib(parallel).orc_step(C.byref(p), n, _d(s.x), _d(s.v), _d(s.w), _d(s.r),
                        n_in, _i(lo_in), _i(hi_in), _d(dt_in),
                        _d(wall) if wall is not None else None,
                        cap, C.byref(nc), _i(lo), _i(hi), _d(dto),
                        info.ctypes.data_as(C.c_void_p), _d(F), _d(T))
    if rc:
        raise RuntimeError(f"orc_step failed ({rc})")
    k = nc.value
    s.lo = lo[:k].copy()
    s.hi = hi[:k].copy()
    s.dt = dto[:k].copy()
    return {"F": F, "T": T, "lo": s.lo, "hi": s.hi, "dt": s.dt,
            "info": info[:k].copy()}
