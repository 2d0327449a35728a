"""The candidate-list pipeline with a skin (dem_box.skin > 0).

A re-sort keeps every pair within r_i + r_j + skin; the steps after it apply
the contact rule to those pairs only, and the next re-sort comes when a
particle has moved far enough for a pair outside the list to reach contact.
The contact set is then the cell search's whatever the skin, and the force
sum runs in partner-id order, so a run with a skin is bit for bit the run
that searches every step (skin 0) on the same cell grid.  These tests check
that on several workloads and forms, check single steps between re-sorts and
steps that re-sort against the oracle, and check the graph form (re-sort
kernels in a conditional node) against direct launches.
"""
import dataclasses

import numpy as np
import pytest

from paper_1503_03553_gb300 import synth

from parity import check_one_step, gpu_run, grid_for, oracle_run, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SKIN_SMALL = 0.02e-6   # re-sorts every few tens of steps on these boxes
SKIN_LARGE = 0.4e-6


@pytest.fixture(scope="module")
def dense3k():
    return synth.w2_polydisperse(n=3000, seed=21)


def _same(a, b, keys=("x", "v", "w", "F", "T")):
    for k in keys:
        assert np.array_equal(a["state"][k], b["state"][k]), k
    assert np.array_equal(a["lo"], b["lo"]) and np.array_equal(a["hi"], b["hi"])
    assert np.array_equal(a["dt"], b["dt"])
    assert np.array_equal(a["Fc"], b["Fc"]) and np.array_equal(a["nFc"], b["nFc"])


@pytest.mark.parametrize("precision", ["mixed", "fp64", "fp32"])
def test_skin_runs_bit_identical_to_search_every_step(dense3k, precision):
    b = prepared(dense3k, precision)
    ncell = grid_for(b, skin=SKIN_LARGE)
    steps = 150
    ref = gpu_run([b], precision, [ncell], steps=steps, skins=[0.0])[0]
    assert ref["resorts"]["resorts"] == steps
    for skin in (SKIN_SMALL, SKIN_LARGE):
        g = gpu_run([b], precision, [ncell], steps=steps, skins=[skin])[0]
        rs = g["resorts"]
        assert 1 <= rs["resorts"] < steps, rs
        if skin == SKIN_SMALL:
            assert rs["resorts"] >= 3, rs  # the history crosses several re-sorts
        assert rs["candidates"] >= len(g["lo"])
        _same(g, ref)


def test_skin_graph_equals_direct_launches(dense3k):
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b, skin=SKIN_SMALL)
    a = gpu_run([b], "mixed", [ncell], steps=64, graph_steps=16, skins=[SKIN_SMALL])[0]
    c = gpu_run([b], "mixed", [ncell], steps=64, graph_steps=-1, skins=[SKIN_SMALL])[0]
    assert a["resorts"]["resorts"] == c["resorts"]["resorts"] >= 2
    _same(a, c)


def _stepwise(b, precision, ncell, skin, nmax):
    """Step one at a time until a step that re-sorts (after the first) and
    a step that does not have been seen; returns, for each, the state and
    history before it and the library's results of it."""
    import paper_1503_03553_gb300 as D
    ctx = D.Context([b], precision=precision, ncell=[ncell], skins=[skin], graph_steps=-1)
    found = {}
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(1)
        for _ in range(nmax):
            before = ctx.resort_stats()["resorts"]
            st = ctx.get_state(0)
            hist = ctx.contacts(0)
            ctx.step(1)
            kind = "resort" if ctx.resort_stats()["resorts"] > before else "kept"
            if kind in found:
                if len(found) == 2:
                    break
                continue
            g = dict(state=ctx.get_state(0))
            g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
            g["flo"], g["fhi"], g["Fc"], g["nFc"] = ctx.contact_forces(0)
            g["order"], g["cells"] = ctx.order(0)
            found[kind] = (st, hist, g)
            if len(found) == 2:
                break
    finally:
        ctx.close()
    return found


@pytest.mark.parametrize("l2_fetch", [-1, 32, 128])
def test_l2_fetch_setting_leaves_results_unchanged(dense3k, l2_fetch):
    """The context's L2 fetch granularity (dem_config.l2_fetch; the library
    sets 64 bytes unless told otherwise) is a hint to the memory system:
    every result is the same, bit for bit, whatever it is set to."""
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b, skin=SKIN_SMALL)
    ref = gpu_run([b], "mixed", [ncell], steps=40, skins=[SKIN_SMALL])[0]
    g = gpu_run([b], "mixed", [ncell], steps=40, skins=[SKIN_SMALL], l2_fetch=l2_fetch)[0]
    _same(ref, g)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_steps_between_and_at_resorts_match_oracle(dense3k, precision):
    b = prepared(dense3k, precision)
    ncell = grid_for(b, skin=SKIN_SMALL)
    found = _stepwise(b, precision, ncell, SKIN_SMALL, 400)
    assert set(found) == {"resort", "kept"}, sorted(found)
    for kind, (st, hist, g) in found.items():
        b2 = prepared(b, precision)
        b2.x, b2.v, b2.w = st["x"], st["v"], st["w"]
        o = oracle_run(b2, precision, ncell, hist=hist)
        # a step without a re-sort keeps the last re-sort's slot order
        check_one_step(b2, g, o, precision, check_order=(kind == "resort"))


def test_skin_batched_equals_box_by_box_and_no_skin():
    boxes = synth.w4_batched(nboxes=4, seed=26, nmin=300, nmax=3000)
    boxes = [prepared(b, "mixed") for b in boxes]
    ncells = [grid_for(b, skin=SKIN_SMALL) for b in boxes]
    skins = [SKIN_SMALL] * len(boxes)
    together = gpu_run(boxes, "mixed", ncells, steps=60, skins=skins)
    plain = gpu_run(boxes, "mixed", ncells, steps=60, skins=[0.0] * len(boxes))
    for k, b in enumerate(boxes):
        alone = gpu_run([b], "mixed", [ncells[k]], steps=60, skins=[SKIN_SMALL])[0]
        for key in ("x", "v", "w", "F", "T"):
            assert np.array_equal(together[k]["state"][key], alone["state"][key]), (k, key)
            assert np.array_equal(together[k]["state"][key], plain[k]["state"][key]), (k, key)


@pytest.mark.parametrize("workload", ["floor_gravity", "rectangles_and_line"])
def test_skin_with_floor_gravity_and_walls(workload):
    from test_gpu_walls import walled_box
    if workload == "floor_gravity":
        box = synth.w3_bidisperse_floor(n=6000, seed=28, column_n=6000)
    else:
        box = walled_box()
    b = prepared(box, "mixed")
    # the walls cross the packing and kick particles hard: a wider skin
    ncell = grid_for(b, skin=SKIN_LARGE)
    ref = gpu_run([b], "mixed", [ncell], steps=80, skins=[0.0])[0]
    g = gpu_run([b], "mixed", [ncell], steps=80, skins=[SKIN_LARGE])[0]
    assert g["resorts"]["resorts"] < 80
    _same(g, ref)


def test_skin_with_size_binned_search(dense3k):
    b = prepared(dataclasses.replace(dense3k, r_split=5.5e-6), "mixed")
    ncell = grid_for(b, skin=SKIN_SMALL)
    ref = gpu_run([b], "mixed", [ncell], steps=60, skins=[0.0])[0]
    g = gpu_run([b], "mixed", [ncell], steps=60, skins=[SKIN_SMALL])[0]
    assert g["resorts"]["resorts"] < 60
    _same(g, ref)


def test_skin_checkpoint_resume_bit_exact(dense3k):
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b, skin=SKIN_SMALL)
    ref = gpu_run([b], "mixed", [ncell], steps=40, skins=[SKIN_SMALL])[0]
    ctx = D.Context([b], precision="mixed", ncell=[ncell], skins=[SKIN_SMALL])
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(20)
        st = ctx.get_state(0)
        lo, hi, dt = ctx.contacts(0)
    finally:
        ctx.close()
    ctx = D.Context([b], precision="mixed", ncell=[ncell], skins=[SKIN_SMALL])
    try:
        ctx.set_particles(0, st["x"], st["v"], st["w"], b.r)
        ctx.set_contacts(0, lo, hi, dt)
        ctx.step(20)
        st2 = ctx.get_state(0)
    finally:
        ctx.close()
    for k in ("x", "v", "w"):
        assert np.array_equal(st2[k], ref["state"][k]), k


def test_skin_rejected_configurations(dense3k):
    import paper_1503_03553_gb300 as D
    b = prepared(dense3k, "mixed")
    with pytest.raises(D.DemError) as e:
        D.Context([b], precision="mixed", skins=[-1e-7])
    assert e.value.status == D.DEM_ERR_ARG
    with pytest.raises(D.DemError) as e:
        D.Context([b], precision="mixed", skins=[1e-7], collide=D.DEM_COLLIDE_FUSED)
    assert e.value.status == D.DEM_ERR_ARG
    # cells sized for no skin are too narrow for one
    with pytest.raises(D.DemError) as e:
        D.Context([b], precision="mixed", ncell=[grid_for(b)], skins=[2e-6])
    assert e.value.status == D.DEM_ERR_ARG


def _run_with_set_state(b, skin, ncell, shift):
    """Ten steps, then the positions read back, moved by `shift` metres
    along x and set again (dem_set_state), then twenty steps."""
    import paper_1503_03553_gb300 as D
    ctx = D.Context([b], precision="mixed", ncell=[ncell], skins=[skin])
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(10)
        st = ctx.get_state(0)
        x = st["x"].copy()
        x[:, 0] += shift
        before = ctx.resort_stats()["resorts"]
        ctx.set_state(0, x, st["v"], st["w"])
        ctx.step(1)
        resorted = ctx.resort_stats()["resorts"] > before
        ctx.step(19)
        out = dict(state=ctx.get_state(0))
        out["lo"], out["hi"], out["dt"] = ctx.contacts(0)
        out["flo"], out["fhi"], out["Fc"], out["nFc"] = ctx.contact_forces(0)
    finally:
        ctx.close()
    return out, resorted


@pytest.mark.parametrize("shift_over_skin", [0.0, 0.1, 3.0])
def test_set_state_positions_tracked_like_a_step(dense3k, shift_over_skin):
    """New positions from the host keep the candidate list when every
    particle stayed within the skin limit and re-sort otherwise; either way
    the run is bit for bit the run that re-sorts every step."""
    b = prepared(dense3k, "mixed")
    ncell = grid_for(b, skin=SKIN_LARGE)
    shift = shift_over_skin * SKIN_LARGE
    ref, _ = _run_with_set_state(b, 0.0, ncell, shift)
    g, resorted = _run_with_set_state(b, SKIN_LARGE, ncell, shift)
    if shift_over_skin >= 1.0:
        assert resorted
    elif shift_over_skin == 0.0:
        assert not resorted
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(g["state"][k], ref["state"][k]), k
    assert np.array_equal(g["lo"], ref["lo"]) and np.array_equal(g["dt"], ref["dt"])
    assert np.array_equal(g["Fc"], ref["Fc"])
