"""GB300 DEM library: Python binding of the C ABI in include/dem.h.

Argument marshalling only.  Every step of the method runs in the CUDA
kernels of ``libdem_gb300.so``; PyTorch supplies device memory (through the
allocator hook) and the CUDA stream.  There is no CPU fallback: the functions
raise if the library is missing or a call fails.

The module-level ``dem_*`` functions mirror the C entry points one to one;
``Context`` bundles them for convenience.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libdem_gb300.so")

ABI_VERSION = 5  # the include/dem.h this binding marshals for
DEM_OK, DEM_ERR_ARG, DEM_ERR_ALLOC, DEM_ERR_CUDA, DEM_ERR_CAPACITY = 0, 1, 2, 3, 4
DEM_ERR_NONFINITE, DEM_ERR_TIMEOUT, DEM_ERR_STATE = 5, 6, 7
DEM_FP64, DEM_MIXED, DEM_FP32 = 0, 1, 2
DEM_HOST, DEM_DEVICE = 0, 1
DEM_COLLIDE_COMPACT, DEM_COLLIDE_FUSED, DEM_COLLIDE_TWOLOOP = 0, 1, 2
DEM_NSTATS = 10
PRECISIONS = {"fp64": DEM_FP64, "mixed": DEM_MIXED, "fp32": DEM_FP32}
STATUS_NAMES = {0: "DEM_OK", 1: "DEM_ERR_ARG", 2: "DEM_ERR_ALLOC", 3: "DEM_ERR_CUDA",
                4: "DEM_ERR_CAPACITY", 5: "DEM_ERR_NONFINITE", 6: "DEM_ERR_TIMEOUT",
                7: "DEM_ERR_STATE"}


class DemError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class dem_material(C.Structure):
    _fields_ = [("E", C.c_double), ("poisson", C.c_double), ("density", C.c_double),
                ("restitution", C.c_double), ("mu_d", C.c_double)]


class dem_wall(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("p", C.c_double * 3),
                ("u", C.c_double * 3), ("v", C.c_double * 3)]


DEM_WALL_RECT, DEM_WALL_LINE = 0, 1


class dem_box(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("periodic", C.c_int32 * 3),
                ("floor_wall", C.c_int32), ("g", C.c_double * 3), ("dt", C.c_double),
                ("material", C.c_int32), ("ncell", C.c_int32 * 3),
                ("max_particles", C.c_int64), ("r_max", C.c_double),
                ("nwalls", C.c_int32), ("walls", C.POINTER(dem_wall)),
                ("r_split", C.c_double), ("skin", C.c_double)]


class dem_tuning(C.Structure):
    _fields_ = [("ms_per_step", C.c_double), ("skin_over_rmax", C.c_double),
                ("cell_scale", C.c_double), ("rsplit_quantile", C.c_double),
                ("block", C.c_int32), ("graph_steps", C.c_int32), ("trials", C.c_int32),
                ("pad", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class dem_config(C.Structure):
    _fields_ = [("nboxes", C.c_int32), ("boxes", C.POINTER(dem_box)),
                ("nmaterials", C.c_int32), ("materials", C.POINTER(dem_material)),
                ("precision", C.c_int32), ("collide", C.c_int32),
                ("kn_literal", C.c_int32), ("row_capacity", C.c_int32),
                ("graph_steps", C.c_int32), ("block", C.c_int32),
                ("l2_fetch", C.c_int32), ("stream", C.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN),
                ("alloc_ctx", C.c_void_p)]


_lib = None


def lib() -> C.CDLL:
    """Load libdem_gb300.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() "
                          "or python -m paper_1503_03553_gb300.build")
    L = C.CDLL(LIB_PATH)
    vp, dp, ip, i64p = C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_int32), C.POINTER(C.c_int64)
    sig = {
        "dem_abi_version": (C.c_int32, []),
        "dem_create": (C.c_int, [C.POINTER(dem_config), C.POINTER(vp)]),
        "dem_destroy": (C.c_int, [vp]),
        "dem_set_particles": (C.c_int, [vp, C.c_int32, C.c_int64, vp, vp, vp, vp, C.c_int32]),
        "dem_set_state": (C.c_int, [vp, C.c_int32, vp, vp, vp, C.c_int32]),
        "dem_step": (C.c_int, [vp, C.c_int64]),
        "dem_get_state": (C.c_int, [vp, C.c_int32, vp, vp, vp, vp, vp, C.c_int32]),
        "dem_get_count": (C.c_int, [vp, C.c_int32, i64p]),
        "dem_get_contacts": (C.c_int, [vp, C.c_int32, C.c_int64, i64p, ip, ip, dp]),
        "dem_set_contacts": (C.c_int, [vp, C.c_int32, C.c_int64, ip, ip, dp]),
        "dem_get_contact_forces": (C.c_int, [vp, C.c_int32, C.c_int64, i64p, ip, ip, dp, dp]),
        "dem_get_order": (C.c_int, [vp, C.c_int32, ip, ip]),
        "dem_get_grid": (C.c_int, [vp, C.c_int32, ip]),
        "dem_get_stats": (C.c_int, [vp, C.c_int32, dp]),
        "dem_get_phase_times": (C.c_int32, [vp, dp, C.c_int32]),
        "dem_set_timing": (C.c_int, [vp, C.c_int32]),
        "dem_launches_per_step": (C.c_int32, [vp]),
        "dem_get_resort_stats": (C.c_int, [vp, i64p]),
        "dem_autotune_layout": (C.c_int, [vp, C.c_int64, C.POINTER(dem_tuning)]),
        "dem_get_layout": (C.c_int, [vp, C.c_int32, ip, dp, dp]),
        "dem_measure_fma_rates": (C.c_int, [dp, dp, vp]),
        "dem_autotune": (C.c_int, [vp, C.c_int64, dp, ip, ip]),
        "dem_sync": (C.c_int, [vp]),
        "dem_last_error": (C.c_char_p, [vp]),
        "dem_alpha_of_restitution": (C.c_double, [C.c_double]),
        "dem_restitution_of_alpha": (C.c_double, [C.c_double]),
        "dem_contacts_static": (C.c_int, [C.c_int64, vp, vp, dp, ip, ip, C.c_int64, vp,
                                          i64p, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    if L.dem_abi_version() != ABI_VERSION:
        raise ImportError(f"{LIB_PATH} has ABI version {L.dem_abi_version()}, the binding "
                          f"expects {ABI_VERSION}: rebuild it")
    _lib = L
    return L


def _check(ctx, status: int):
    if status != DEM_OK:
        msg = lib().dem_last_error(ctx)
        raise DemError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------------------
# array marshalling
# ---------------------------------------------------------------------------
def _ptr(a, where: int, dtype=np.float64, elems=None, name="array"):
    """Return (pointer, keepalive) for a numpy array (host) or a torch tensor
    (device, on the current CUDA device).  elems: the number of elements the
    C call reads or writes there; an array of another size is refused before
    the call (a short one would be read or written past its end)."""
    if a is None:
        return None, None
    if where == DEM_DEVICE:
        import torch
        if not (isinstance(a, torch.Tensor) and a.is_cuda):
            raise TypeError(f"{name}: device arrays must be CUDA tensors")
        want = torch.float64 if dtype == np.float64 else torch.int32
        if a.dtype != want or not a.is_contiguous():
            raise TypeError(f"{name}: device array must be contiguous {want}")
        if a.device.index != torch.cuda.current_device():
            raise ValueError(f"{name} must be on the current CUDA device")
        if elems is not None and a.numel() != elems:
            raise ValueError(f"{name} must hold {elems} elements, not {a.numel()}")
        return C.c_void_p(a.data_ptr()), a
    arr = np.ascontiguousarray(a, dtype=dtype)
    if elems is not None and arr.size != elems:
        raise ValueError(f"{name} must hold {elems} elements, not {arr.size}")
    return C.c_void_p(arr.ctypes.data), arr


# ---------------------------------------------------------------------------
# C entry points, same names
# ---------------------------------------------------------------------------
def dem_abi_version() -> int:
    return lib().dem_abi_version()


def dem_alpha_of_restitution(eps: float) -> float:
    return lib().dem_alpha_of_restitution(float(eps))


def dem_restitution_of_alpha(alpha: float) -> float:
    return lib().dem_restitution_of_alpha(float(alpha))


def dem_contacts_static(x, radius, L, periodic, ncell, pairs, stream=None) -> int:
    """Contact list of one small box with no device allocation (see the
    C declaration).  x: CUDA float64 (n, 3); radius: CUDA float64 (n,);
    pairs: CUDA int32 (cap, 2) receiving (id_lo, id_hi).  Returns the count."""
    import torch
    for t, dt in ((x, torch.float64), (radius, torch.float64), (pairs, torch.int32)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == dt and t.is_contiguous()):
            raise TypeError("x, radius must be contiguous CUDA float64; pairs CUDA int32")
    if x.ndim != 2 or x.shape[1] != 3:
        raise ValueError("x must have shape (n, 3)")
    n = int(x.shape[0])
    if radius.ndim != 1 or radius.shape[0] != n:
        raise ValueError("radius must have shape (n,) with n = x.shape[0]")
    if pairs.ndim != 2 or pairs.shape[1] != 2:
        raise ValueError("pairs must have shape (cap, 2)")
    if not (x.device == radius.device == pairs.device):
        raise ValueError("x, radius and pairs must be on one device")
    if x.device.index != torch.cuda.current_device():
        raise ValueError("x, radius and pairs must be on the current CUDA device")
    Ld = (C.c_double * 3)(*[float(v) for v in L])
    per = (C.c_int32 * 3)(*[int(v) for v in periodic])
    nc = (C.c_int32 * 3)(*[int(v) for v in ncell])
    cnt = C.c_int64(0)
    s = stream if stream is not None else torch.cuda.current_stream()
    st = lib().dem_contacts_static(n, C.c_void_p(x.data_ptr()), C.c_void_p(radius.data_ptr()),
                                   Ld, per, nc, int(pairs.shape[0]), C.c_void_p(pairs.data_ptr()),
                                   C.byref(cnt), C.c_void_p(s.cuda_stream))
    _check(None, st)
    return cnt.value


def dem_create(cfg: dem_config) -> C.c_void_p:
    out = C.c_void_p()
    st = lib().dem_create(C.byref(cfg), C.byref(out))
    _check(None, st)
    return out


def dem_destroy(ctx) -> None:
    _check(ctx, lib().dem_destroy(ctx))


def dem_set_particles(ctx, box: int, x, v, omega, radius, where: int = DEM_HOST):
    """x, v, omega: (n, 3); radius: (n,); n is x's first dimension."""
    n = int(x.shape[0])
    px, kx = _ptr(x, where, elems=3 * n, name="x")
    pv, kv = _ptr(v, where, elems=3 * n, name="v")
    pw, kw = _ptr(omega, where, elems=3 * n, name="omega")
    pr, kr = _ptr(radius, where, elems=n, name="radius")
    _check(ctx, lib().dem_set_particles(ctx, box, n, px, pv, pw, pr, where))


def dem_set_state(ctx, box: int, x=None, v=None, omega=None, where: int = DEM_HOST):
    """Each given array: (n, 3) with n the box's particle count."""
    n = dem_get_count(ctx, box)
    px, kx = _ptr(x, where, elems=3 * n, name="x")
    pv, kv = _ptr(v, where, elems=3 * n, name="v")
    pw, kw = _ptr(omega, where, elems=3 * n, name="omega")
    _check(ctx, lib().dem_set_state(ctx, box, px, pv, pw, where))


def dem_step(ctx, nsteps: int) -> None:
    _check(ctx, lib().dem_step(ctx, int(nsteps)))


def dem_get_count(ctx, box: int) -> int:
    n = C.c_int64()
    _check(ctx, lib().dem_get_count(ctx, box, C.byref(n)))
    return n.value


def dem_get_state(ctx, box: int, x=None, v=None, omega=None, force=None,
                  torque=None, where: int = DEM_HOST):
    """Fill the given arrays (n x 3 float64, numpy for DEM_HOST, CUDA
    tensors for DEM_DEVICE)."""
    n = dem_get_count(ctx, box)
    names = ("x", "v", "omega", "force", "torque")
    for a, name in zip((x, v, omega, force, torque), names):
        if a is not None and where == DEM_HOST:
            if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
                raise TypeError(f"{name}: host outputs must be C-contiguous float64 numpy arrays")
    ptrs = [_ptr(a, where, elems=3 * n, name=name)[0]
            for a, name in zip((x, v, omega, force, torque), names)]
    _check(ctx, lib().dem_get_state(ctx, box, *ptrs, where))


def dem_get_contacts(ctx, box: int, cap: Optional[int] = None):
    """Return (id_lo, id_hi, delta_t) sorted by (id_lo, id_hi)."""
    n = C.c_int64()
    if cap is None:
        st = lib().dem_get_contacts(ctx, box, 0, C.byref(n), None, None, None)
        if st not in (DEM_OK, DEM_ERR_CAPACITY):
            _check(ctx, st)
        cap = n.value
    lo = np.zeros(max(cap, 1), np.int32)
    hi = np.zeros(max(cap, 1), np.int32)
    dt = np.zeros((max(cap, 1), 3), np.float64)
    _check(ctx, lib().dem_get_contacts(ctx, box, cap, C.byref(n),
                                       lo.ctypes.data_as(C.POINTER(C.c_int32)),
                                       hi.ctypes.data_as(C.POINTER(C.c_int32)),
                                       dt.ctypes.data_as(C.POINTER(C.c_double))))
    k = n.value
    return lo[:k].copy(), hi[:k].copy(), dt[:k].copy()


def dem_get_contact_forces(ctx, box: int):
    """Return (id_lo, id_hi, F, nF) of the last step, sorted by (id_lo, id_hi)."""
    n = C.c_int64()
    st = lib().dem_get_contact_forces(ctx, box, 0, C.byref(n), None, None, None, None)
    if st not in (DEM_OK, DEM_ERR_CAPACITY):
        _check(ctx, st)
    cap = n.value
    lo = np.zeros(max(cap, 1), np.int32)
    hi = np.zeros(max(cap, 1), np.int32)
    F = np.zeros((max(cap, 1), 3))
    nF = np.zeros((max(cap, 1), 3))
    _check(ctx, lib().dem_get_contact_forces(
        ctx, box, cap, C.byref(n), lo.ctypes.data_as(C.POINTER(C.c_int32)),
        hi.ctypes.data_as(C.POINTER(C.c_int32)), F.ctypes.data_as(C.POINTER(C.c_double)),
        nF.ctypes.data_as(C.POINTER(C.c_double))))
    k = n.value
    return lo[:k].copy(), hi[:k].copy(), F[:k].copy(), nF[:k].copy()


def dem_set_contacts(ctx, box: int, id_lo, id_hi, delta_t):
    lo = np.ascontiguousarray(id_lo, np.int32)
    hi = np.ascontiguousarray(id_hi, np.int32)
    dt = np.ascontiguousarray(delta_t, np.float64).reshape(-1, 3)
    _check(ctx, lib().dem_set_contacts(ctx, box, lo.size,
                                       lo.ctypes.data_as(C.POINTER(C.c_int32)),
                                       hi.ctypes.data_as(C.POINTER(C.c_int32)),
                                       dt.ctypes.data_as(C.POINTER(C.c_double))))


def dem_get_order(ctx, box: int):
    n = dem_get_count(ctx, box)
    ids = np.zeros(max(n, 1), np.int32)
    cells = np.zeros(max(n, 1), np.int32)
    _check(ctx, lib().dem_get_order(ctx, box, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                                    cells.ctypes.data_as(C.POINTER(C.c_int32))))
    return ids[:n].copy(), cells[:n].copy()


def dem_get_grid(ctx, box: int):
    nc = (C.c_int32 * 3)()
    _check(ctx, lib().dem_get_grid(ctx, box, nc))
    return tuple(nc)


def dem_get_stats(ctx, box: int) -> np.ndarray:
    out = np.zeros(DEM_NSTATS, np.float64)
    _check(ctx, lib().dem_get_stats(ctx, box, out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def dem_set_timing(ctx, on: bool) -> None:
    _check(ctx, lib().dem_set_timing(ctx, 1 if on else 0))


def dem_get_phase_times(ctx) -> np.ndarray:
    out = np.zeros(8, np.float64)
    k = lib().dem_get_phase_times(ctx, out.ctypes.data_as(C.POINTER(C.c_double)), 8)
    return out[:k].copy()


def dem_autotune(ctx, steps: int = 32):
    """Pick the fastest block size and graph length on the live state;
    returns (best ms per step, block, graph_steps)."""
    ms = C.c_double()
    blk = C.c_int32()
    gs = C.c_int32()
    _check(ctx, lib().dem_autotune(ctx, int(steps), C.byref(ms), C.byref(blk), C.byref(gs)))
    return ms.value, blk.value, gs.value


def dem_autotune_layout(ctx, steps: int = 32) -> dict:
    """Search skin, cell grid, size split, block size and graph length on
    the live particles (the state is put back); returns the choice."""
    t = dem_tuning()
    _check(ctx, lib().dem_autotune_layout(ctx, int(steps), C.byref(t)))
    return {f: getattr(t, f) for f, _ in dem_tuning._fields_ if f != "pad"}


def dem_measure_fma_rates(stream=None) -> dict:
    """Measured FP32 and FP64 FMA peaks of the current GPU [TFLOP/s]."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    a, b = C.c_double(), C.c_double()
    _check(None, lib().dem_measure_fma_rates(C.byref(a), C.byref(b), C.c_void_p(s.cuda_stream)))
    return {"fp32_tflops": a.value, "fp64_tflops": b.value}


def dem_get_layout(ctx, box: int = 0) -> dict:
    nc = (C.c_int32 * 3)()
    skin = C.c_double()
    rs = C.c_double()
    _check(ctx, lib().dem_get_layout(ctx, box, nc, C.byref(skin), C.byref(rs)))
    return {"ncell": tuple(nc), "skin": skin.value, "r_split": rs.value}


def dem_launches_per_step(ctx) -> int:
    return lib().dem_launches_per_step(ctx)


def dem_get_resort_stats(ctx) -> dict:
    """Re-sorts so far, kernels a re-sort adds, candidate pairs in the
    current list, steps so far (contact-list pipeline)."""
    out = (C.c_int64 * 4)()
    _check(ctx, lib().dem_get_resort_stats(ctx, out))
    return {"resorts": out[0], "launches_per_resort": out[1], "candidates": out[2],
            "steps": out[3]}


def dem_sync(ctx) -> None:
    _check(ctx, lib().dem_sync(ctx))


def dem_last_error(ctx) -> str:
    m = lib().dem_last_error(ctx)
    return m.decode() if m else ""


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------
class Context:
    """Owns one dem_ctx.  ``boxes`` are objects with the fields of
    ``synth.Box`` (L, periodic, floor_wall, g, dt, E, poisson, density,
    restitution, mu_d, r_max, n; optional walls, r_split, skin) or dicts
    with the same keys.  ``skins`` overrides the boxes' candidate-list skins
    [m] (0 = search every step)."""

    def __init__(self, boxes: Sequence, precision="mixed", collide=DEM_COLLIDE_COMPACT,
                 kn_literal=0, row_capacity=0, graph_steps=0, block=0,
                 l2_fetch=0, capacities: Optional[Sequence[int]] = None,
                 r_max: Optional[Sequence[float]] = None,
                 ncell: Optional[Sequence] = None, torch_alloc: bool = True,
                 skins: Optional[Sequence[float]] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self._torch = torch
        L = lib()
        nb = len(boxes)
        self._mats = (dem_material * nb)()
        self._boxes = (dem_box * nb)()
        for k, b in enumerate(boxes):
            g = (lambda name, default=None: getattr(b, name) if hasattr(b, name) else b.get(name, default))
            m = self._mats[k]
            m.E, m.poisson, m.density = g("E"), g("poisson"), g("density")
            m.restitution, m.mu_d = g("restitution"), g("mu_d")
            bx = self._boxes[k]
            Ls = g("L")
            for a in range(3):
                bx.L[a] = float(Ls[a])
                bx.periodic[a] = int(g("periodic")[a])
                bx.g[a] = float(g("g", (0.0, 0.0, 0.0))[a])
                bx.ncell[a] = int(ncell[k][a]) if ncell is not None else 0
            bx.floor_wall = int(g("floor_wall", 0))
            bx.dt = float(g("dt"))
            bx.material = k
            bx.max_particles = int(capacities[k]) if capacities is not None else int(g("n"))
            bx.r_max = float(r_max[k]) if r_max is not None else float(g("r_max"))
            bx.r_split = float(g("r_split", 0.0) or 0.0)
            bx.skin = float(skins[k]) if skins is not None else float(g("skin", 0.0) or 0.0)
            walls = list(g("walls", ()) or ())
            bx.nwalls = len(walls)
            if walls:
                arr = (dem_wall * len(walls))()
                for q, (kind, pw, uw, vw) in enumerate(walls):
                    arr[q].kind = int(kind)
                    for a in range(3):
                        arr[q].p[a] = float(pw[a])
                        arr[q].u[a] = float(uw[a])
                        arr[q].v[a] = float(vw[a]) if vw is not None else 0.0
                bx.walls = C.cast(arr, C.POINTER(dem_wall))
                self._wall_arrays = getattr(self, "_wall_arrays", []) + [arr]
        cfg = dem_config()
        cfg.nboxes = nb
        cfg.boxes = self._boxes
        cfg.nmaterials = nb
        cfg.materials = self._mats
        cfg.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        cfg.collide = int(collide)
        cfg.kn_literal = int(kn_literal)
        cfg.row_capacity = int(row_capacity)
        cfg.graph_steps = int(graph_steps)
        cfg.block = int(block)
        cfg.l2_fetch = int(l2_fetch)
        self.stream = torch.cuda.current_stream()
        cfg.stream = C.c_void_p(self.stream.cuda_stream)
        self._device = torch.cuda.current_device()
        if torch_alloc:
            dev, stream = self._device, self.stream

            def _alloc(nbytes, _ctx):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except Exception:
                    return None

            def _free(ptr, _ctx):
                torch.cuda.caching_allocator_delete(ptr)
            self._alloc = ALLOC_FN(_alloc)
            self._free = FREE_FN(_free)
        else:
            self._alloc = ALLOC_FN()
            self._free = FREE_FN()
        cfg.alloc = self._alloc
        cfg.free = self._free
        self.ctx = dem_create(cfg)
        self.nboxes = nb

    # lifecycle ------------------------------------------------------------
    def close(self):
        if getattr(self, "ctx", None):
            dem_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # calls ---------------------------------------------------------------
    def set_particles(self, box, x, v, w, r, where=DEM_HOST):
        dem_set_particles(self.ctx, box, x, v, w, r, where)

    def set_state(self, box, x=None, v=None, w=None, where=DEM_HOST):
        dem_set_state(self.ctx, box, x, v, w, where)

    def step(self, n=1):
        dem_step(self.ctx, n)

    def count(self, box=0):
        return dem_get_count(self.ctx, box)

    def get_state(self, box=0):
        n = self.count(box)
        out = {k: np.zeros((n, 3)) for k in ("x", "v", "w", "F", "T")}
        dem_get_state(self.ctx, box, out["x"], out["v"], out["w"], out["F"], out["T"])
        return out

    def contacts(self, box=0):
        return dem_get_contacts(self.ctx, box)

    def contact_forces(self, box=0):
        return dem_get_contact_forces(self.ctx, box)

    def set_contacts(self, box, lo, hi, dt):
        dem_set_contacts(self.ctx, box, lo, hi, dt)

    def order(self, box=0):
        return dem_get_order(self.ctx, box)

    def grid(self, box=0):
        return dem_get_grid(self.ctx, box)

    def stats(self, box=0):
        return dem_get_stats(self.ctx, box)

    def sync(self):
        dem_sync(self.ctx)

    def launches_per_step(self):
        return dem_launches_per_step(self.ctx)

    def resort_stats(self):
        return dem_get_resort_stats(self.ctx)

    def autotune_layout(self, steps=32):
        return dem_autotune_layout(self.ctx, steps)

    def layout(self, box=0):
        return dem_get_layout(self.ctx, box)

    def autotune(self, steps=32):
        return dem_autotune(self.ctx, steps)

    def set_timing(self, on=True):
        dem_set_timing(self.ctx, on)

    def phase_times(self):
        return dem_get_phase_times(self.ctx)
