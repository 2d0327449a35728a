"""Size-binned contact search (a box with r_split > 0) against the oracle.

The cells of a size-binned box are sized for its small particles (at least
max(2 r_split, r_max) (1 + 1e-5) wide): small particles search +-1 cell for
partners up to r_split, large ones +-2 cells for all partners (Sec. 3.3: the
cell size trades the candidate loop against the cells visited).  The
contacts of any pair lie within +-2 cells of such a grid, so the oracle's
cell search with a +-2 stencil on the same grid is the reference: sort order
and contact set bit for bit, forces within the tolerances of
tests/parity.py.
"""
import dataclasses
import math

import numpy as np
import pytest

from paper_1503_03553_gb300 import synth
from parity import check_one_step, gpu_run, oracle_params, oracle_run, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle as O  # noqa: E402
import paper_1503_03553_gb300 as D  # noqa: E402


def binned_grid(box, r_split):
    """The library's grid for a size-binned box (ncell = 0 picks it)."""
    h = max(2.0 * r_split, box.r_max) * (1.0 + 1e-5)
    return [max(1, int(math.floor(box.L[a] / h))) for a in range(3)]


def _one(box, precision, r_split, **kw):
    b = prepared(dataclasses.replace(box, r_split=r_split), precision)
    ncell = binned_grid(b, r_split)
    assert min(ncell) >= 5
    g = gpu_run([b], precision, [ncell], **kw)[0]
    o = oracle_run(b, precision, ncell, stencil=2)
    return b, g, o


@pytest.fixture(scope="module")
def dense3k():
    return synth.w2_polydisperse(n=3000, seed=41)


@pytest.fixture(scope="module")
def dense20k():
    return synth.w2_polydisperse(n=20000, seed=42, tile_n=20000)


@pytest.mark.parametrize("precision", ["mixed", "fp64", "fp32"])
@pytest.mark.parametrize("r_split", [5.0e-6, 6.0e-6])
def test_one_step_matches_oracle(dense3k, precision, r_split):
    b, g, o = _one(dense3k, precision, r_split)
    large = b.r.astype(np.float32) > np.float32(r_split)
    assert 0.02 * b.n < large.sum() < 0.3 * b.n
    # pairs of every class: small-small, small-large, large-large
    lo, hi = o["lo"], o["hi"]
    kinds = large[lo].astype(int) + large[hi].astype(int)
    assert all(np.sum(kinds == k) > 0 for k in (0, 1, 2))
    if precision == "fp32":
        # FP32 positions lose the overlap: exact contacts only (as for the
        # single-class search)
        assert np.array_equal(g["order"], o["order"])
        assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    else:
        check_one_step(b, g, o, precision)


def test_one_step_20k_several_tiles(dense20k):
    b, g, o = _one(dense20k, "mixed", 5.0e-6)
    check_one_step(b, g, o, "mixed")


def test_grid_set_by_r_max_and_wide_radii():
    """Radii 1-8 um with r_split 3 um: the cells (r_max wide) are set by
    the +-2 reach of the largest pair, not by 2 r_split."""
    rng = synth.rng_for(43)
    radii = lambda g, m: synth._lognormal_radii(g, m, 3e-6, 0.5, 1e-6, 8e-6)
    x, r, L = synth._dense_tile(rng, 4000, 0.5, radii, 0.01)
    box = synth.Box(x=x, v=synth._gauss(rng, len(r), 0.05), w=1e3 * rng.standard_normal((len(r), 3)),
                    r=r, L=L)
    b, g, o = _one(box, "mixed", 3.0e-6)
    assert binned_grid(b, 3.0e-6)[0] == int(math.floor(L[0] / (b.r_max * (1 + 1e-5))))
    check_one_step(b, g, o, "mixed")


def test_open_axis_floor_and_gravity(dense3k):
    """Open z with the floor: the +-2 stencil stops at the box's open ends."""
    box = dataclasses.replace(dense3k, periodic=(1, 1, 0), floor_wall=1, g=(0.0, 0.0, -9.81))
    b, g, o = _one(box, "mixed", 5.0e-6)
    check_one_step(b, g, o, "mixed")


def test_history_over_steps_tracks_single_class(dense3k):
    """Ten FP64 steps size-binned and ten with one size class (cells 2 r_max
    wide): the same contacts and, up to the rounding of sums taken in
    another order, the same positions, velocities and delta_t.  (In FP32
    arithmetic that rounding, 1e-7 of a force, can flip a contact sitting
    on the contact threshold or the Coulomb limit, whose damping, ~ dn^(1/4),
    or cap then moves its particles far more; the MIXED form's history is
    checked against the oracle below.)"""
    b = prepared(dataclasses.replace(dense3k, r_split=5.0e-6), "fp64")
    one = prepared(dense3k, "fp64")
    s = gpu_run([b], "fp64", [binned_grid(b, 5.0e-6)], steps=10)[0]
    h = 2.0 * one.r_max * (1.0 + 1e-5)
    c = gpu_run([one], "fp64", [[int(math.floor(one.L[a] / h)) for a in range(3)]], steps=10)[0]
    assert np.array_equal(s["lo"], c["lo"]) and np.array_equal(s["hi"], c["hi"])
    L = np.asarray(b.L)
    dx = s["state"]["x"] - c["state"]["x"]
    dx -= L * np.round(dx / L)
    assert np.abs(dx).max() < 1e-17
    scale = np.abs(c["state"]["v"]).max()
    assert np.allclose(s["state"]["v"], c["state"]["v"], rtol=0, atol=1e-10 * scale)
    assert np.allclose(s["dt"], c["dt"], rtol=1e-9, atol=1e-12 * np.abs(c["dt"]).max())


def test_history_carried_matches_oracle(dense3k):
    """Three size-binned steps, then a fourth from the GPU's own state and
    contact history against the oracle started from the same (the delta_t
    of pairs found by the large-particle search is carried over)."""
    r_split = 5.0e-6
    b = prepared(dataclasses.replace(dense3k, r_split=r_split), "mixed")
    ncell = binned_grid(b, r_split)
    ctx = D.Context([b], precision="mixed", ncell=[ncell])
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(3)
        st = ctx.get_state(0)
        lo, hi, dt = ctx.contacts(0)
        ctx.step(1)
        g = dict(state=ctx.get_state(0))
        g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
        g["flo"], g["fhi"], g["Fc"], g["nFc"] = ctx.contact_forces(0)
        g["order"], g["cells"] = ctx.order(0)
    finally:
        ctx.close()
    b2 = prepared(b, "mixed")
    b2.x, b2.v, b2.w = st["x"], st["v"], st["w"]
    s = O.State(b2.x, b2.v, b2.w, b2.r)
    s.lo, s.hi, s.dt = lo, hi, dt
    p = oracle_params(b2, "mixed", ncell, stencil=2)
    cell, order = O.order(p, b2.x)
    v0, w0 = s.v.copy(), s.w.copy()
    out = O.step(p, s)
    out.update(order=order, cell=cell, x=s.x, v=s.v, w=s.w, v0=v0, w0=w0, params=p)
    large = b.r.astype(np.float32) > np.float32(r_split)
    carried = np.isin(out["lo"].astype(np.int64) * b.n + out["hi"], lo.astype(np.int64) * b.n + hi)
    assert carried.sum() > 0.5 * len(out["lo"])
    assert np.any(carried & (large[out["lo"]] | large[out["hi"]]))
    check_one_step(b2, g, out, "mixed")


def test_size_binned_and_plain_boxes_in_one_context(dense3k):
    plain = prepared(synth.w2_polydisperse(n=2000, seed=44), "mixed")
    binned = prepared(dataclasses.replace(dense3k, r_split=5.5e-6), "mixed")
    h = 2.0 * plain.r_max * (1.0 + 1e-5)
    ncells = [binned_grid(binned, 5.5e-6), [int(math.floor(plain.L[a] / h)) for a in range(3)]]
    gs = gpu_run([binned, plain], "mixed", ncells)
    check_one_step(binned, gs[0], oracle_run(binned, "mixed", ncells[0], stencil=2), "mixed")
    check_one_step(plain, gs[1], oracle_run(plain, "mixed", ncells[1]), "mixed")


def test_auto_grid_and_graph_replay_bit_identical(dense3k):
    b = prepared(dataclasses.replace(dense3k, r_split=5.0e-6), "mixed")
    ctx = D.Context([b], precision="mixed")
    try:
        assert list(ctx.grid(0)) == binned_grid(b, 5.0e-6)
    finally:
        ctx.close()
    ncell = binned_grid(b, 5.0e-6)
    a = gpu_run([b], "mixed", [ncell], steps=40, graph_steps=16)[0]
    c = gpu_run([b], "mixed", [ncell], steps=40, graph_steps=-1)[0]
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(a["state"][k], c["state"][k]), k
    assert np.array_equal(a["dt"], c["dt"])


def test_bad_size_binned_configurations_rejected(dense3k):
    b = dataclasses.replace(dense3k, r_split=5.0e-6)
    with pytest.raises(D.DemError) as e:  # per-particle Collide forms keep one class
        D.Context([b], precision="mixed", collide=D.DEM_COLLIDE_FUSED)
    assert e.value.status == D.DEM_ERR_ARG
    with pytest.raises(D.DemError) as e:  # r_split above r_max
        D.Context([dataclasses.replace(b, r_split=2.0 * b.r_max)], precision="mixed")
    assert e.value.status == D.DEM_ERR_ARG
    with pytest.raises(D.DemError) as e:  # a periodic axis of 4 cells
        D.Context([b], precision="mixed", ncell=[(4, 6, 6)])
    assert e.value.status == D.DEM_ERR_ARG
    with pytest.raises(D.DemError) as e:  # cells narrower than 2 r_split
        D.Context([b], precision="mixed", ncell=[(20, 20, 20)])
    assert e.value.status == D.DEM_ERR_ARG
