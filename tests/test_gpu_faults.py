"""Failures the library reports through status codes, provoked on the host
(no GPU fault): a contact row too small for the packing, a non-finite value
injected into the state, and bad arguments.  Each device-side error is
sticky until the context is destroyed."""
import numpy as np
import pytest

from paper_1503_03553_gb300 import synth

from parity import grid_for, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1503_03553_gb300 as D  # noqa: E402


@pytest.fixture(scope="module")
def box():
    return prepared(synth.w2_polydisperse(n=3000, seed=61), "mixed")


def _ctx(box, **kw):
    ctx = D.Context([box], precision="mixed", ncell=[grid_for(box)], **kw)
    ctx.set_particles(0, box.x, box.v, box.w, box.r)
    return ctx


def test_row_capacity_overflow_is_reported_and_sticky(box):
    ctx = _ctx(box, row_capacity=2)
    try:
        with pytest.raises(D.DemError) as e:
            ctx.step(1)
        assert e.value.status == D.DEM_ERR_CAPACITY
        with pytest.raises(D.DemError) as e2:
            ctx.step(1)
        assert e2.value.status == D.DEM_ERR_CAPACITY
    finally:
        ctx.close()


def test_nonfinite_velocity_is_reported(box):
    ctx = _ctx(box)
    try:
        ctx.step(2)
        st = ctx.get_state(0)
        v = st["v"].copy()
        v[17, 1] = np.nan
        ctx.set_state(0, v=v)
        with pytest.raises(D.DemError) as e:
            ctx.step(1)
        assert e.value.status == D.DEM_ERR_NONFINITE
        with pytest.raises(D.DemError):
            ctx.sync()
    finally:
        ctx.close()


def test_bad_arguments_are_rejected(box):
    ctx = _ctx(box)
    try:
        with pytest.raises(D.DemError) as e:
            ctx.set_particles(3, box.x, box.v, box.w, box.r)  # no box 3
        assert e.value.status == D.DEM_ERR_ARG
        r = box.r.copy()
        r[5] = 1.0  # larger than r_max
        with pytest.raises(D.DemError) as e:
            ctx.set_particles(0, box.x, box.v, box.w, r)
        assert e.value.status == D.DEM_ERR_ARG
        with pytest.raises(D.DemError) as e:
            D.dem_step(ctx.ctx, -1)
        assert e.value.status == D.DEM_ERR_ARG
        ctx.step(1)  # the context is still usable
    finally:
        ctx.close()


def test_too_few_cells_rejected_at_create(box):
    with pytest.raises(D.DemError) as e:
        D.Context([box], precision="mixed", ncell=[(2, 2, 2)])
    assert e.value.status == D.DEM_ERR_ARG
