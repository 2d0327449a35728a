"""Input generators: shapes, distributions and packing of the workloads."""
import math

import numpy as np

from paper_1503_03553_gb300 import synth


def _phi(b):
    return float(np.sum(4.0 / 3.0 * math.pi * b.r ** 3) / np.prod(b.L))


def test_w1_shape_and_no_overlap():
    b = synth.w1_monodisperse(n=300, seed=1)
    assert b.x.shape == (300, 3) and np.all(b.r == np.float32(5e-6))
    from scipy.spatial import cKDTree
    t = cKDTree(b.x, boxsize=b.L)
    d, _ = t.query(b.x, k=2)
    assert np.all(d[:, 1] >= 2 * 5e-6 * (1 - 1e-12))
    assert abs(_phi(b) - 0.3) < 1e-9
    assert np.allclose(b.v.mean(0), 0, atol=1e-12)


def test_w2_packing_and_radii():
    b = synth.w2_polydisperse(n=4000, seed=2)
    assert abs(_phi(b) - 0.55) < 1e-9
    assert b.r.min() >= np.float32(2e-6) and b.r.max() <= np.float32(8e-6)
    assert np.all(b.r.astype(np.float32).astype(np.float64) == b.r)
    assert abs(np.median(b.r) - 4e-6) < 0.2e-6
    # overlaps at most 1 % of the smaller radius
    from scipy.spatial import cKDTree
    L = np.asarray(b.L)
    t = cKDTree(np.mod(b.x, L), boxsize=L)
    pr = t.query_pairs(2 * b.r.max(), output_type="ndarray")
    d = b.x[pr[:, 1]] - b.x[pr[:, 0]]
    d -= L * np.round(d / L)
    ov = b.r[pr[:, 0]] + b.r[pr[:, 1]] - np.linalg.norm(d, axis=1)
    rel = ov / np.minimum(b.r[pr[:, 0]], b.r[pr[:, 1]])
    assert rel.max() <= 0.01 + 1e-12
    assert np.sum(ov > 0) > b.n  # a contact network exists


def test_w2_tiling_keeps_statistics():
    b = synth.w2_polydisperse(n=8 * 1000, seed=3, tile_n=1000)
    assert b.n == 8000
    assert abs(_phi(b) - 0.55) < 1e-9
    assert len(np.unique(b.x, axis=0)) == b.n


def test_w4_boxes_vary():
    boxes = synth.w4_batched(nboxes=6, seed=4, nmin=200, nmax=2000)
    ns = [b.n for b in boxes]
    assert min(ns) >= 200 and max(ns) <= 2000
    assert len({b.restitution for b in boxes}) == 6
    for b in boxes:
        assert 0.2 <= _phi(b) <= 0.5 + 1e-9
        assert 0.1 <= b.mu_d <= 0.6


def test_wide_polydisperse_radii_span_a_factor_8():
    b = synth.wide_polydisperse(n=3000, seed=6)
    assert abs(_phi(b) - 0.5) < 1e-9
    assert b.r.min() >= np.float32(1e-6) and b.r.max() <= np.float32(8e-6)
    assert np.sum(b.r < 1.5e-6) > 0 and np.sum(b.r > 6e-6) > 0
    assert abs(np.median(b.r) - 3e-6) < 0.2e-6


def test_lattice_gas_has_no_contacts():
    b = synth.lattice_gas(n=3000, seed=7)
    assert b.n == 3000
    from scipy.spatial import cKDTree
    L = np.asarray(b.L)
    t = cKDTree(np.mod(b.x, L), boxsize=L)
    d, _ = t.query(np.mod(b.x, L), k=2)
    assert np.all(d[:, 1] > 2 * b.r.max())


def test_w2_tiling_of_large_boxes():
    """A W2 box above one tile is k^3 shifted copies of one relaxed tile,
    its ids in random order (the bench's 1 M box: 5^3 tiles of 8,000)."""
    assert synth.tiling(1_000_000) == (5, 8000)
    assert synth.tiling(512_000) == (4, 8000)
    assert synth.tiling(3000) == (1, 3000)
    tile = synth.w2_polydisperse(n=1000, seed=7, tile_n=1000)
    big = synth.w2_polydisperse(n=8000, seed=7, tile_n=1000)
    assert big.n == 8000 and np.allclose(big.L, 2 * np.asarray(tile.L))
    assert np.array_equal(np.sort(big.r), np.sort(np.tile(tile.r, 8)))
    # every particle sits at a tile particle's position shifted by whole tiles
    L0 = np.asarray(tile.L)
    frac = np.mod(big.x, L0)
    key = lambda x: np.round(np.mod(x, L0) / L0 * 2 ** 20).astype(np.int64)
    a = {tuple(k) for k in key(tile.x)}
    assert all(tuple(k) in a for k in key(frac))
    assert not np.array_equal(big.r[:1000], tile.r)  # ids are not in tile order
