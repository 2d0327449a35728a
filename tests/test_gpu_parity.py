"""CUDA path against the FP64 oracle (needs a GB300).

Each test runs the library through its C ABI (ctypes binding), runs the
oracle on the same seeded input, and compares: sort order and contact set
bit for bit; forces, torques and delta_t per contact and per particle within
the tolerances stated in tests/parity.py.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1503_03553_gb300 import synth

from parity import check_one_step, force_errors, gpu_run, grid_for, oracle_run, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _one(box, precision, **kw):
    b = prepared(box, precision)
    ncell = grid_for(b)
    g = gpu_run([b], precision, [ncell], **kw)[0]
    o = oracle_run(b, precision, ncell)
    return b, g, o


@pytest.fixture(scope="module")
def dense3k():
    return synth.w2_polydisperse(n=3000, seed=21)


@pytest.fixture(scope="module")
def dense20k():
    # several thousand-thread tiles and a ragged tail
    return synth.w2_polydisperse(n=20000, seed=22, tile_n=20000)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_one_step_dense_small(dense3k, precision):
    b, g, o = _one(dense3k, precision)
    m = check_one_step(b, g, o, precision)
    assert m["contacts"] > b.n


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_one_step_dense_20k(dense20k, precision):
    b, g, o = _one(dense20k, precision)
    check_one_step(b, g, o, precision)


def test_one_step_monodisperse_fp64():
    box = synth.w1_monodisperse(n=1000, seed=23)
    # push particles together so that contacts exist
    box.x = box.x * 0.0 + box.x
    b, g, o = _one(box, "fp64")
    check_one_step(b, g, o, "fp64")


@pytest.mark.parametrize("n", [1, 2, 33, 257, 4097])
def test_ragged_small_counts(n):
    # the first n particles of a dense box: same box and grid, few contacts
    box = synth.w2_polydisperse(n=6000, seed=24, tile_n=6000)
    sel = slice(0, n)
    box.x, box.v, box.w, box.r = box.x[sel], box.v[sel], box.w[sel], box.r[sel]
    b, g, o = _one(box, "mixed")
    check_one_step(b, g, o, "mixed")


def test_empty_box_steps():
    import paper_1503_03553_gb300 as D
    box = synth.w2_polydisperse(n=500, seed=25)
    ctx = D.Context([box], precision="mixed")
    try:
        z = np.zeros((0, 3))
        ctx.set_particles(0, z, z, z, np.zeros(0))
        ctx.step(3)
        assert ctx.count(0) == 0
        assert len(ctx.contacts(0)[0]) == 0
    finally:
        ctx.close()


def test_history_carried_over_two_steps(dense3k):
    """Step 2 from the GPU's own state and contact history agrees with the
    oracle started from the same state and history (delta_t remap)."""
    import paper_1503_03553_gb300 as D
    precision = "mixed"
    b = prepared(dense3k, precision)
    ncell = grid_for(b)
    ctx = D.Context([b], precision=precision, ncell=[ncell])
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        for _ in range(3):
            ctx.step(1)
        st = ctx.get_state(0)
        lo, hi, dt = ctx.contacts(0)
        b2 = prepared(b, precision)
        b2.x, b2.v, b2.w = st["x"], st["v"], st["w"]
        ctx.step(1)
        g = dict(state=ctx.get_state(0))
        g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
        g["flo"], g["fhi"], g["Fc"], g["nFc"] = ctx.contact_forces(0)
        g["order"], g["cells"] = ctx.order(0)
    finally:
        ctx.close()
    p_state = O.State(b2.x, b2.v, b2.w, b2.r)
    p_state.lo, p_state.hi, p_state.dt = lo, hi, dt
    from parity import oracle_params
    p = oracle_params(b2, precision, ncell)
    cell, order = O.order(p, b2.x)
    v0, w0 = p_state.v.copy(), p_state.w.copy()
    out = O.step(p, p_state)
    out.update(order=order, cell=cell, x=p_state.x, v=p_state.v, w=p_state.w,
               v0=v0, w0=w0, params=p)
    carried = np.isin(out["lo"].astype(np.int64) * b.n + out["hi"], lo.astype(np.int64) * b.n + hi)
    assert carried.sum() > 0.5 * len(out["lo"])  # most contacts persist
    check_one_step(b2, g, out, precision)


def test_graph_replay_bit_identical(dense3k):
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b)
    a = gpu_run([b], "mixed", [ncell], steps=40, graph_steps=16)[0]
    c = gpu_run([b], "mixed", [ncell], steps=40, graph_steps=-1)[0]
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(a["state"][k], c["state"][k]), k
    assert np.array_equal(a["dt"], c["dt"])


def test_batched_equals_box_by_box():
    boxes = synth.w4_batched(nboxes=4, seed=26, nmin=200, nmax=3000)
    boxes = [prepared(b, "mixed") for b in boxes]
    ncells = [grid_for(b) for b in boxes]
    together = gpu_run(boxes, "mixed", ncells, steps=5)
    for k, b in enumerate(boxes):
        alone = gpu_run([b], "mixed", [ncells[k]], steps=5)[0]
        for key in ("x", "v", "w", "F", "T"):
            assert np.array_equal(together[k]["state"][key], alone["state"][key]), (k, key)


def test_batched_boxes_match_oracle():
    boxes = synth.w4_batched(nboxes=3, seed=27, nmin=200, nmax=2000)
    boxes = [prepared(b, "mixed") for b in boxes]
    ncells = [grid_for(b) for b in boxes]
    gs = gpu_run(boxes, "mixed", ncells)
    for b, nc, g in zip(boxes, ncells, gs):
        o = oracle_run(b, "mixed", nc)
        check_one_step(b, g, o, "mixed")


def test_checkpoint_resume_bit_exact(dense3k):
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b)
    ref = gpu_run([b], "mixed", [ncell], steps=20, graph_steps=-1)[0]
    ctx = D.Context([b], precision="mixed", ncell=[ncell], graph_steps=-1)
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(10)
        st = ctx.get_state(0)
        lo, hi, dt = ctx.contacts(0)
    finally:
        ctx.close()
    ctx = D.Context([b], precision="mixed", ncell=[ncell], graph_steps=-1)
    try:
        ctx.set_particles(0, st["x"], st["v"], st["w"], b.r)
        ctx.set_contacts(0, lo, hi, dt)
        ctx.step(10)
        st2 = ctx.get_state(0)
    finally:
        ctx.close()
    for k in ("x", "v", "w"):
        assert np.array_equal(st2[k], ref["state"][k]), k


def test_multi_step_statistics_track_oracle(dense3k):
    """Trajectories are chaotic; kinetic energy and mean coordination after
    50 steps agree within 1 %."""
    prec = "mixed"
    b = prepared(dense3k, prec)
    ncell = grid_for(b)
    g = gpu_run([b], prec, [ncell], steps=50)[0]
    p = __import__("parity").oracle_params(b, prec, ncell)
    s = O.State(b.x, b.v, b.w, b.r)
    for _ in range(50):
        O.step(p, s)
    m = b.density * 4.0 / 3.0 * math.pi * b.r ** 3
    ke_o = 0.5 * np.sum(m * np.sum(s.v ** 2, 1))
    ke_g = g["stats"][0]
    assert abs(ke_g - ke_o) <= 0.01 * ke_o
    z_o = 2.0 * len(s.lo) / b.n
    assert abs(g["stats"][6] - z_o) <= 0.01 * z_o


def test_floor_and_gravity_match_oracle():
    box = synth.w3_bidisperse_floor(n=6000, seed=28, column_n=6000)
    b, g, o = _one(box, "mixed")
    check_one_step(b, g, o, "mixed")
    b, g, o = _one(box, "fp64")
    check_one_step(b, g, o, "fp64")


def test_fp32_mode_exact_contacts_and_reported_error(dense3k):
    """DEM_FP32 keeps absolute FP32 positions: its contact set and sort order
    match the oracle's FP32 rule bit for bit, but the overlap carries FP32
    rounding of the position (~6e-8 |x|), so its force error is reported
    against the FP64 oracle and is larger than DEM_MIXED's."""
    b = prepared(dense3k, "fp32")
    ncell = grid_for(b)
    g = gpu_run([b], "fp32", [ncell])[0]
    o = oracle_run(b, "fp32", ncell)
    assert np.array_equal(g["order"], o["order"])
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"])
    e32 = force_errors(b, g, o, "fp32")
    bm = prepared(dense3k, "mixed")
    gm = gpu_run([bm], "mixed", [grid_for(bm)])[0]
    om = oracle_run(bm, "mixed", grid_for(bm))
    em = force_errors(bm, gm, om, "mixed")
    assert e32["contact_sets_equal"] and em["contact_sets_equal"]
    assert e32["median_rel_err"] < 1e-2
    assert em["max_err_over_scale"] < 1e-5
    assert e32["max_err_over_scale"] > em["max_err_over_scale"]


def test_precision_modes_ranked_on_relaxed_dense_packing():
    """Precision stress (packing 0.60 at rest, overlaps ~1e-3 r): after 200
    steps, re-evaluate one step from each mode's own state with the FP64
    oracle; DEM_MIXED stays within 1e-5 of the term scale while DEM_FP32
    does not."""
    box = synth.w5_precision(n=4000, seed=29)
    res = {}
    for prec in ("mixed", "fp32"):
        import paper_1503_03553_gb300 as D
        b = prepared(box, prec)
        ncell = grid_for(b)
        ctx = D.Context([b], precision=prec, ncell=[ncell])
        try:
            ctx.set_particles(0, b.x, b.v, b.w, b.r)
            ctx.step(200)
            st = ctx.get_state(0)
            lo, hi, dt = ctx.contacts(0)
            snap = prepared(b, prec)
            snap.x, snap.v, snap.w = st["x"], st["v"], st["w"]
            ctx.step(1)
            g = dict(state=ctx.get_state(0))
            g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
            g["flo"], g["fhi"], g["Fc"], g["nFc"] = ctx.contact_forces(0)
        finally:
            ctx.close()
        from parity import oracle_params
        p = oracle_params(snap, prec, ncell)
        s = O.State(snap.x, snap.v, snap.w, snap.r)
        s.lo, s.hi, s.dt = lo, hi, dt
        out = O.step(p, s)
        out["params"] = p
        res[prec] = force_errors(snap, g, out, prec)
    assert res["mixed"]["contact_sets_equal"] and res["fp32"]["contact_sets_equal"]
    assert res["mixed"]["p99_err_over_scale"] < 1e-5
    assert res["fp32"]["p99_err_over_scale"] > 10 * res["mixed"]["p99_err_over_scale"]


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_fused_algorithm1_matches_oracle(dense3k, precision):
    """DEM_COLLIDE_FUSED (the paper's Algorithm 1: search and force in one
    pass per particle, each pair evaluated by both of its particles)."""
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, precision)
    ncell = grid_for(b)
    g = gpu_run([b], precision, [ncell], collide=D.DEM_COLLIDE_FUSED)[0]
    o = oracle_run(b, precision, ncell)
    check_one_step(b, g, o, precision)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_twoloop_collide_matches_oracle(dense3k, precision):
    """DEM_COLLIDE_TWOLOOP (the paper's improvement, Sec. 3.4: a first loop
    keeps the contact partners, a second loop computes their forces)."""
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, precision)
    ncell = grid_for(b)
    g = gpu_run([b], precision, [ncell], collide=D.DEM_COLLIDE_TWOLOOP)[0]
    o = oracle_run(b, precision, ncell)
    check_one_step(b, g, o, precision)


def test_twoloop_and_fused_bit_identical_over_steps(dense3k):
    """The two per-particle forms find the same contacts and sum them in the
    same order: identical states, contacts and histories after 5 steps."""
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b)
    t = gpu_run([b], "mixed", [ncell], steps=5, collide=D.DEM_COLLIDE_TWOLOOP)[0]
    f = gpu_run([b], "mixed", [ncell], steps=5, collide=D.DEM_COLLIDE_FUSED)[0]
    assert np.array_equal(t["lo"], f["lo"]) and np.array_equal(t["hi"], f["hi"])
    for k in ("x", "v", "w"):
        assert np.array_equal(t["state"][k], f["state"][k])
    assert np.array_equal(t["dt"], f["dt"])


def test_fused_and_compact_agree_over_steps(dense3k):
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b)
    f = gpu_run([b], "mixed", [ncell], steps=5, collide=D.DEM_COLLIDE_FUSED)[0]
    c = gpu_run([b], "mixed", [ncell], steps=5)[0]
    # same contact sets every step; sums in another order differ in rounding
    assert np.array_equal(f["lo"], c["lo"]) and np.array_equal(f["hi"], c["hi"])
    assert np.allclose(f["state"]["x"], c["state"]["x"], rtol=0, atol=1e-15)
    scale = np.abs(c["state"]["v"]).max()
    assert np.allclose(f["state"]["v"], c["state"]["v"], rtol=0, atol=1e-5 * scale)
    assert np.allclose(f["dt"], c["dt"], rtol=1e-4, atol=1e-4 * np.abs(c["dt"]).max())


def test_autotune_picks_a_valid_config_and_keeps_results_exact(dense3k):
    """The autotuner only changes launch shapes: a tuned context and an
    untuned one give bit-identical states for the same number of steps."""
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b)
    ctx = D.Context([b], precision="mixed", ncell=[ncell])
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ms, blk, gs = ctx.autotune(steps=8)
        assert ms > 0 and blk in (128, 256, 512) and gs in (8, 16, 32)
        # per block size and graph length g: g warm-up steps + the timed steps
        ran = 3 * sum(g + max(8 // g, 1) * g for g in (8, 16, 32))
        tuned = ctx.get_state(0)
    finally:
        ctx.close()
    ref = gpu_run([b], "mixed", [ncell], steps=ran)[0]["state"]
    for k in ("x", "v", "w"):
        assert np.array_equal(tuned[k], ref[k]), k
