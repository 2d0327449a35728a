"""Layout tuner (dem_autotune_layout): it searches skin, cell grid, size
split, block size and graph length on the live particles, keeps the fastest,
and puts the state back.  After it, a step on the chosen layout gives the
oracle's contact set and sort order on the same grid (with the +-2 stencil
when it chose a size split) and forces within the parity tolerances."""
import dataclasses

import numpy as np
import pytest

from paper_1503_03553_gb300 import synth

from parity import check_one_step, oracle_run, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.mark.parametrize("workload", ["w2_dense", "radii_1_8um"])
def test_layout_tuner_keeps_state_and_matches_oracle(workload):
    import paper_1503_03553_gb300 as D
    if workload == "w2_dense":
        box = synth.w2_polydisperse(n=8000, seed=81)
    else:
        box = synth.wide_polydisperse(n=8000, seed=82)
    b = prepared(box, "mixed")
    ctx = D.Context([b], precision="mixed")
    try:
        ctx.set_particles(0, b.x, b.v, b.w, b.r)
        ctx.step(3)
        before = ctx.get_state(0)
        hist = ctx.contacts(0)
        t = ctx.autotune_layout(steps=24)
        assert t["trials"] >= 8 and t["ms_per_step"] > 0
        assert t["block"] in (128, 256, 512) and t["graph_steps"] in (8, 16, 32)
        after = ctx.get_state(0)
        for k in ("x", "v", "w"):
            assert np.array_equal(before[k], after[k]), k
        lo, hi, dt = ctx.contacts(0)
        assert np.array_equal(lo, hist[0]) and np.array_equal(hi, hist[1])
        assert np.array_equal(dt, hist[2])
        lay = ctx.layout(0)
        ctx.step(1)
        g = dict(state=ctx.get_state(0))
        g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
        g["flo"], g["fhi"], g["Fc"], g["nFc"] = ctx.contact_forces(0)
        g["order"], g["cells"] = ctx.order(0)
    finally:
        ctx.close()
    b2 = dataclasses.replace(prepared(b, "mixed"), r_split=lay["r_split"])
    b2.x, b2.v, b2.w = before["x"], before["v"], before["w"]
    o = oracle_run(b2, "mixed", list(lay["ncell"]), stencil=2 if lay["r_split"] > 0 else 1,
                   hist=hist)
    # the first step after the tuner re-sorts: the order is the oracle's
    check_one_step(b2, g, o, "mixed")
