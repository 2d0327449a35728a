"""Seeded synthetic particle sets for the DEM workloads.

This module draws inputs only: radii, positions, velocities, materials and
box sizes.  It holds none of the method's arithmetic (no contact law, no
cell search of its own); dense packings are made by a plain overlap-removal
relaxation on top of scipy's periodic k-d tree.

Workloads (sizes, distributions and steps follow the benchmark definitions):

  W1  1,000 monodisperse spheres, r = 5 um, periodic cube at packing 0.3,
      non-overlapping uniform placement, v ~ N(0, 0.1 m/s), w = 0.
  W2  1,000,000 polydisperse spheres, r lognormal (median 4 um, sigma_log
      0.25, clipped to [2, 8] um), periodic cube at packing 0.55 with random
      overlaps <= 1 % of the smaller radius, v ~ N(0, 0.05 m/s),
      w ~ N(0, 1e3 rad/s).  Built from a relaxed periodic tile repeated
      k x k x k times (ids shuffled), which keeps the packing fraction,
      radius distribution and contact statistics of a full relaxation.
  W3  bidisperse (r = 3 and 6 um, 50/50) spheres, lower half of the box at
      packing 0.55, upper half at 0.05, floor at z = 0, periodic x/y,
      gravity -9.81 m/s^2 along z, v ~ N(0, 0.05 m/s).
  W4  many independent periodic boxes, counts log-uniform in [200, 20000],
      per-box restitution U[0.3, 0.9], friction U[0.1, 0.6], radii lognormal
      (median 4 um, sigma_log 0.2, clipped [2, 8] um), packing U[0.2, 0.5].
  W5  spheres with r ~ U[3, 5] um at packing 0.60, relaxed to overlaps of
      about 1e-3 r, v = w = 0.

Radii are rounded to float32 values so that every precision mode of the
library and the FP64 oracle see the same sizes.  Time steps are fixed
numbers chosen as 1/50 of the Hertz contact duration of the smallest
particle pair at the impact speed sqrt(2) sigma_v (W1: 2.296e-9 s).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

SEED_BASE = 1503035530

# shared material of W1-W3 and W5
E_DEFAULT = 3e9
POISSON_DEFAULT = 0.3
DENSITY_DEFAULT = 1200.0


@dataclasses.dataclass
class Box:
    """One independent simulation box (positions etc. in id order)."""
    x: np.ndarray            # (n, 3) float64 [m]
    v: np.ndarray            # (n, 3) float64 [m/s]
    w: np.ndarray            # (n, 3) float64 [rad/s]
    r: np.ndarray            # (n,)   float64, float32-representable [m]
    L: tuple                 # box edge lengths [m]
    periodic: tuple = (1, 1, 1)
    floor_wall: int = 0
    g: tuple = (0.0, 0.0, 0.0)
    dt: float = 1e-9
    E: float = E_DEFAULT
    poisson: float = POISSON_DEFAULT
    density: float = DENSITY_DEFAULT
    restitution: float = 0.5
    mu_d: float = 0.3
    walls: tuple = ()        # (kind, p, u, v): 0 = rectangle, 1 = line
    r_split: float = 0.0     # size-binned search: radius above which a
                             # particle searches +-2 cells (0 = off)
    skin: float = 0.0        # candidate-list skin [m] (0 = search every step)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def r_max(self) -> float:
        return float(self.r.max()) if self.n else 0.0


def rng_for(k: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + k))


def _f32(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def _lognormal_radii(rng, n, median, sigma_log, rmin, rmax):
    r = median * np.exp(sigma_log * rng.standard_normal(n))
    return _f32(np.clip(r, rmin, rmax))


def _box_for(r, phi, aspect=(1.0, 1.0, 1.0)):
    vol = float(np.sum(4.0 / 3.0 * math.pi * r ** 3)) / phi
    s = (vol / (aspect[0] * aspect[1] * aspect[2])) ** (1.0 / 3.0)
    return tuple(s * a for a in aspect)


def relax_overlaps(x, r, L, periodic=(1, 1, 1), target=0.01, beta=0.9,
                   max_iter=20000):
    """Push overlapping spheres apart until every overlap is at most
    ``target`` times the smaller radius.  Non-periodic axes have hard walls
    at 0 and L.  A Jacobi sweep moves each member of an overlapping pair by
    beta/2 of the overlap along the centre line; a Verlet list with a skin
    of half the median radius is rebuilt from scipy's k-d tree when any
    sphere has moved more than half the skin."""
    from scipy.spatial import cKDTree

    x = np.array(x, dtype=np.float64)
    n = len(r)
    if n < 2:
        return x
    L = np.asarray(L, dtype=np.float64)
    per = np.asarray(periodic, dtype=bool)
    rmax = float(r.max())
    skin = 0.5 * float(np.median(r))
    box = np.where(per, L, 4.0 * L + 8 * rmax)  # non-periodic: never wraps
    ref = None
    I = J = None
    for _ in range(max_iter):
        if ref is None or np.max(np.abs(_min_image(x - ref, L, per))) > 0.5 * skin:
            xt = np.where(per, np.mod(x, L), x + 2 * rmax)
            tree = cKDTree(xt, boxsize=box)
            pr = tree.query_pairs(2 * rmax + skin, output_type="ndarray")
            I, J = pr[:, 0], pr[:, 1]
            ref = x.copy()
        d = _min_image(x[J] - x[I], L, per)
        dist = np.sqrt(np.einsum("ij,ij->i", d, d))
        ov = r[I] + r[J] - dist
        m = ov > 0
        i, j, d, dist, ov = I[m], J[m], d[m], dist[m], ov[m]
        rel = ov / np.minimum(r[i], r[j]) if ov.size else np.zeros(0)
        # walls on non-periodic axes
        wall_disp = np.zeros_like(x)
        wall_bad = 0.0
        for a in range(3):
            if per[a]:
                continue
            lo = r - x[:, a]
            hi = x[:, a] + r - L[a]
            wall_bad = max(wall_bad, float(np.max(lo / r)), float(np.max(hi / r)))
            wall_disp[:, a] += np.where(lo > 0, beta * lo, 0.0)
            wall_disp[:, a] -= np.where(hi > 0, beta * hi, 0.0)
        worst = max(float(rel.max()) if rel.size else 0.0, wall_bad)
        if worst <= target:
            break
        u = d / dist[:, None] * (0.5 * beta * ov)[:, None]
        disp = wall_disp
        for a in range(3):
            disp[:, a] += np.bincount(j, u[:, a], n) - np.bincount(i, u[:, a], n)
        x = x + disp
        x = np.where(per, np.mod(x, L), x)
    return x


def _min_image(d, L, per):
    return np.where(per, d - L * np.round(d / L), d)


def _gauss(rng, n, sigma, remove_mean=True):
    v = sigma * rng.standard_normal((n, 3))
    if remove_mean and n > 0:
        v -= v.mean(axis=0)
    return v


def rsa_placement(rng, r, L, max_tries=200000):
    """Random sequential addition of non-overlapping spheres (packing well
    below the RSA limit)."""
    from scipy.spatial import cKDTree

    n = len(r)
    L = np.asarray(L, dtype=np.float64)
    x = np.zeros((n, 3))
    placed = 0
    rmax = float(r.max())
    tree = None
    batch = []
    for k in range(n):
        for _ in range(max_tries):
            c = rng.random(3) * L
            ok = True
            if tree is not None:
                for q in tree.query_ball_point(c, 2 * rmax):
                    d = c - x[q]
                    d -= L * np.round(d / L)
                    if np.dot(d, d) < (r[k] + r[q]) ** 2:
                        ok = False
                        break
            if ok:
                for q in batch:
                    d = c - x[q]
                    d -= L * np.round(d / L)
                    if np.dot(d, d) < (r[k] + r[q]) ** 2:
                        ok = False
                        break
            if ok:
                break
        else:
            raise RuntimeError("RSA placement failed")
        x[k] = c
        batch.append(k)
        placed += 1
        if len(batch) >= 64:
            tree = cKDTree(np.mod(x[:placed], L), boxsize=L)
            batch = []
    return x


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def w1_monodisperse(n: int = 1000, seed: int = 1) -> Box:
    """W1: plain FP64 method case."""
    rng = rng_for(seed)
    r = _f32(np.full(n, 5e-6))
    L = _box_for(r, 0.3)
    x = rsa_placement(rng, r, L)
    v = _gauss(rng, n, 0.1)
    w = np.zeros((n, 3))
    return Box(x=x, v=v, w=w, r=r, L=L, dt=2.296e-9, restitution=0.5,
               mu_d=0.3)


def _dense_tile(rng, n, phi, radii_fn, target, beta=0.9):
    """Relaxed periodic tile.  The relaxation converges pairs onto exact
    touching (overlaps of 1e-20 m); a final Gaussian jitter of 0.005 target
    r_min per component, after relaxing to 0.95 target, leaves the overlaps
    random and still below target."""
    r = radii_fn(rng, n)
    L = _box_for(r, phi)
    x = rng.random((n, 3)) * np.asarray(L)
    x = relax_overlaps(x, r, L, target=0.95 * target, beta=beta)
    x = np.mod(x + 0.005 * target * float(r.min()) * rng.standard_normal(x.shape),
               np.asarray(L))
    return x, r, L


def _tile(rng, x, r, L, k):
    n0 = len(r)
    offs = np.array([(i, j, l) for l in range(k) for j in range(k) for i in range(k)],
                    dtype=np.float64) * np.asarray(L)
    X = (x[None, :, :] + offs[:, None, :]).reshape(-1, 3)
    R = np.tile(r, k ** 3)
    perm = rng.permutation(n0 * k ** 3)  # ids unrelated to position
    return X[perm], R[perm], tuple(k * l for l in L)


def tiling(n: int, tile_n: int = 8000) -> tuple:
    """(k, n0): a box of n > tile_n particles is k^3 copies of one relaxed
    tile of n0 particles (n rounded to k^3 n0); (1, n) otherwise."""
    if n <= tile_n:
        return 1, n
    k = max(1, int(round((n / tile_n) ** (1.0 / 3.0))))
    return k, int(round(n / k ** 3))


def w2_polydisperse(n: int = 1_000_000, seed: int = 2, tile_n: int = 8000,
                    phi: float = 0.55) -> Box:
    """W2: dense polydisperse periodic box (the throughput workload).  For
    n <= tile_n the box is one relaxed tile; larger n repeats a relaxed tile
    k^3 times with n = k^3 * n_tile (n is rounded to that form)."""
    rng = rng_for(seed)
    radii = lambda g, m: _lognormal_radii(g, m, 4e-6, 0.25, 2e-6, 8e-6)
    if n <= tile_n:
        x, r, L = _dense_tile(rng, n, phi, radii, 0.01)
    else:
        k, n0 = tiling(n, tile_n)
        x0, r0, L0 = _dense_tile(rng, n0, phi, radii, 0.01)
        x, r, L = _tile(rng, x0, r0, L0, k)
    m = len(r)
    v = _gauss(rng, m, 0.05)
    w = 1e3 * rng.standard_normal((m, 3))
    return Box(x=x, v=v, w=w, r=r, L=L, dt=1.0e-9, restitution=0.5, mu_d=0.3)


def wide_polydisperse(n: int = 1_000_000, seed: int = 6, tile_n: int = 8000,
                      phi: float = 0.5) -> Box:
    """Dense periodic box with radii spanning a factor 8 (log-normal,
    median 3 um, log-sd 0.5, clipped to [1, 8] um): the regime where one
    cell size, set by the largest particle, gives the small particles long
    candidate loops.  Built like W2 (relaxed tile, repeated k^3 times)."""
    rng = rng_for(seed)
    radii = lambda g, m: _lognormal_radii(g, m, 3e-6, 0.5, 1e-6, 8e-6)
    if n <= tile_n:
        x, r, L = _dense_tile(rng, n, phi, radii, 0.01)
    else:
        k = max(1, int(round((n / tile_n) ** (1.0 / 3.0))))
        n0 = int(round(n / k ** 3))
        x0, r0, L0 = _dense_tile(rng, n0, phi, radii, 0.01)
        x, r, L = _tile(rng, x0, r0, L0, k)
    m = len(r)
    v = _gauss(rng, m, 0.05)
    w = 1e3 * rng.standard_normal((m, 3))
    return Box(x=x, v=v, w=w, r=r, L=L, dt=1.0e-9, restitution=0.5, mu_d=0.3)


def lattice_gas(n: int = 131072, seed: int = 7, jitter: float = 0.05) -> Box:
    """The initialisation stage of the paper's runs (Sec. 5.2): particles
    created on a uniform cubic lattice with small random offsets, none in
    contact.  W2's radius law; lattice spacing 2.2 r_max, so that offsets of
    up to +-jitter r_max per component leave every pair apart; the first n
    sites of a k^3 lattice, periodic box of k spacings."""
    rng = rng_for(seed)
    r = _lognormal_radii(rng, n, 4e-6, 0.25, 2e-6, 8e-6)
    a = 2.2 * 8e-6
    k = int(math.ceil(n ** (1.0 / 3.0) - 1e-9))
    idx = np.arange(n)
    site = np.stack([idx % k, (idx // k) % k, idx // (k * k)], axis=1).astype(np.float64)
    x = (site + 0.5) * a + jitter * 8e-6 * rng.uniform(-1.0, 1.0, (n, 3))
    L = (k * a,) * 3
    v = _gauss(rng, n, 0.05)
    w = 1e3 * rng.standard_normal((n, 3))
    return Box(x=x, v=v, w=w, r=r, L=L, dt=1.0e-9, restitution=0.5, mu_d=0.3)


def w3_bidisperse_floor(n: int = 8_000_000, seed: int = 3,
                        column_n: int = 20000) -> Box:
    """W3: bidisperse spheres (r = 3 and 6 um, 50/50 by number) in a cube,
    lower half at packing 0.55, upper half at 0.05, floor at z = 0, gravity
    along -z, periodic in x and y.  Built from one relaxed column (periodic
    in x and y, hard floor and lid during the relaxation) of about column_n
    spheres, repeated k x k times in x and y with shuffled ids."""
    rng = rng_for(seed)
    mean_vol = 4.0 / 3.0 * math.pi * 0.5 * ((3e-6) ** 3 + (6e-6) ** 3)
    Lc = (n * mean_vol / 0.30) ** (1.0 / 3.0)  # average packing (0.55+0.05)/2
    k = max(1, int(round(math.sqrt(n / column_n))))
    cl = (Lc / k, Lc / k, Lc)
    n_col = int(round(n / (k * k)))
    n_dense = int(round(n_col * 0.55 / 0.60))
    n_dil = n_col - n_dense
    r = _f32(np.where(rng.random(n_col) < 0.5, 3e-6, 6e-6))
    x = rng.random((n_col, 3)) * np.asarray(cl)
    x[:n_dense, 2] *= 0.5
    x[n_dense:, 2] = Lc / 2 + x[n_dense:, 2] * 0.5
    x = relax_overlaps(x, r, cl, periodic=(1, 1, 0), target=0.01)
    offs = np.array([(i, j, 0) for j in range(k) for i in range(k)],
                    dtype=np.float64) * np.asarray(cl)
    X = (x[None] + offs[:, None]).reshape(-1, 3)
    R = np.tile(r, k * k)
    perm = rng.permutation(len(R))
    X, R = X[perm], R[perm]
    m = len(R)
    v = _gauss(rng, m, 0.05, remove_mean=False)
    w = np.zeros((m, 3))
    return Box(x=X, v=v, w=w, r=R, L=(Lc, Lc, Lc), periodic=(1, 1, 0),
               floor_wall=1, g=(0.0, 0.0, -9.81), dt=1.5e-9, restitution=0.5,
               mu_d=0.3)


def _w4_box(args):
    """One box of W4 (top level so that a process pool can run it)."""
    seed, b, nmin, nmax = args
    rng = np.random.Generator(np.random.PCG64([SEED_BASE + seed, b]))
    n = int(round(math.exp(rng.uniform(math.log(nmin), math.log(nmax)))))
    phi = float(rng.uniform(0.2, 0.5))
    r = _lognormal_radii(rng, n, 4e-6, 0.2, 2e-6, 8e-6)
    L = _box_for(r, phi)
    # jittered simple-cubic lattice start: few overlaps, fast relaxation
    m = int(math.ceil(n ** (1.0 / 3.0)))
    grid = np.stack(np.meshgrid(np.arange(m), np.arange(m), np.arange(m), indexing="ij"),
                    -1).reshape(-1, 3)
    sites = grid[rng.permutation(len(grid))[:n]].astype(np.float64)
    x = (sites + 0.5 + 0.1 * rng.standard_normal((n, 3))) * (np.asarray(L) / m)
    x = relax_overlaps(np.mod(x, np.asarray(L)), r, L, target=0.01)
    v = _gauss(rng, n, 0.05)
    w = np.zeros((n, 3))
    return Box(x=x, v=v, w=w, r=r, L=L, dt=1.0e-9,
               restitution=float(rng.uniform(0.3, 0.9)),
               mu_d=float(rng.uniform(0.1, 0.6)))


def w4_batched(nboxes: int = 512, seed: int = 4, nmin: int = 200,
               nmax: int = 20000, processes: int = 0) -> list:
    """W4: independent periodic boxes with their own counts and materials.
    Box b draws from its own stream (seed, b), so the set does not depend on
    how many worker processes build it (`processes` > 1 uses a spawn pool)."""
    jobs = [(seed, b, nmin, nmax) for b in range(nboxes)]
    if processes and processes > 1 and nboxes > 1:
        import multiprocessing as mp
        with mp.get_context("spawn").Pool(processes) as pool:
            return pool.map(_w4_box, jobs, chunksize=max(1, nboxes // (4 * processes)))
    return [_w4_box(j) for j in jobs]


def w5_precision(n: int = 4_000_000, seed: int = 5, tile_n: int = 8000) -> Box:
    """W5: dense packing 0.60 relaxed to overlaps around 1e-3 r, at rest."""
    rng = rng_for(seed)
    radii = lambda g, m: _f32(g.uniform(3e-6, 5e-6, m))
    if n <= tile_n:
        x, r, L = _dense_tile(rng, n, 0.60, radii, 0.002)
    else:
        k = max(1, int(round((n / tile_n) ** (1.0 / 3.0))))
        n0 = int(round(n / k ** 3))
        x0, r0, L0 = _dense_tile(rng, n0, 0.60, radii, 0.002)
        x, r, L = _tile(rng, x0, r0, L0, k)
    m = len(r)
    return Box(x=x, v=np.zeros((m, 3)), w=np.zeros((m, 3)), r=r, L=L,
               dt=2.0e-9, restitution=0.5, mu_d=0.3)


# ---------------------------------------------------------------------------
# inputs in a precision mode's representation
# ---------------------------------------------------------------------------
def quantize(x):
    """Positions rounded to the 2^-60 m fixed-point grid of DEM_MIXED."""
    return np.ldexp(np.round(np.ldexp(np.asarray(x, np.float64), 60)), -60)


def grid_for(box, stencil: int = 1, skin: float = 0.0):
    """Cells per axis: the largest grid whose cells are at least
    (2 r_max + skin)(1 + 1e-5) / stencil wide (the library's automatic grid
    for the same box)."""
    hmin = (2.0 * box.r_max + skin) * (1.0 + 1e-5) / stencil
    return [max(1, int(math.floor(box.L[a] / hmin))) for a in range(3)]


def prepared(box: Box, precision: str) -> Box:
    """Copy of ``box`` whose state is exactly what the library stores in the
    given precision mode, so that the library and any other consumer start
    from bit-identical inputs: positions wrapped into periodic axes and
    rounded to the mode's position type (2^-60 m fixed point for "mixed",
    float32 for "fp32"); velocities and angular velocities rounded to
    float32 in "mixed" and "fp32" (their storage type there); radii are
    float32 values already."""
    b = dataclasses.replace(box)
    x = np.array(box.x, np.float64)
    L = np.asarray(box.L)
    per = np.asarray(box.periodic, bool)
    x = np.where(per, np.mod(x, L), x)
    v = np.array(box.v, np.float64)
    w = np.array(box.w, np.float64)
    if precision == "mixed":
        x = quantize(x)
        x = np.where(per & (x >= L), x - L, x)
    elif precision == "fp32":
        x = x.astype(np.float32).astype(np.float64)
        x = np.where(per & (x >= L.astype(np.float32)), 0.0, x)
    if precision in ("mixed", "fp32"):
        v = _f32(v)
        w = _f32(w)
    b.x = x
    b.v = v
    b.w = w
    b.r = np.array(box.r, np.float64)
    return b
