"""Device arrays at the boundary: dem_set_particles, dem_set_state and
dem_get_state take CUDA tensors (DEM_DEVICE) as well as host arrays, with
the same results bit for bit; arrays of the wrong size or on another device
are refused before the C call."""
import numpy as np
import pytest

from paper_1503_03553_gb300 import synth

from parity import grid_for, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

SKIN = 0.02e-6


@pytest.fixture(scope="module")
def box():
    return prepared(synth.w2_polydisperse(n=3000, seed=21), "mixed")


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _state_dev(D, ctx, n):
    out = [torch.full((n, 3), np.nan, dtype=torch.float64, device="cuda") for _ in range(5)]
    D.dem_get_state(ctx.ctx, 0, *out, where=D.DEM_DEVICE)
    return {k: t.cpu().numpy() for k, t in zip(("x", "v", "w", "F", "T"), out)}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_device_arrays_give_the_host_arrays_results(box, precision):
    import paper_1503_03553_gb300 as D
    b = prepared(synth.w2_polydisperse(n=3000, seed=21), precision)
    ncell = grid_for(b, skin=SKIN)
    runs = []
    for where in (D.DEM_HOST, D.DEM_DEVICE):
        ctx = D.Context([b], precision=precision, ncell=[ncell], skins=[SKIN])
        try:
            if where == D.DEM_HOST:
                ctx.set_particles(0, b.x, b.v, b.w, b.r)
            else:
                ctx.set_particles(0, _dev(b.x), _dev(b.v), _dev(b.w), _dev(b.r), where=where)
            ctx.step(10)
            mid = ctx.get_state(0)
            # new velocities (and the same positions) through the same route
            v2 = mid["v"] * 0.5
            if where == D.DEM_HOST:
                ctx.set_state(0, mid["x"], v2, None)
            else:
                ctx.set_state(0, _dev(mid["x"]), _dev(v2), None, where=where)
            ctx.step(10)
            runs.append(ctx.get_state(0) if where == D.DEM_HOST else _state_dev(D, ctx, b.n))
        finally:
            ctx.close()
    host, dev = runs
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(host[k], dev[k]), k


def test_wrong_device_arrays_are_refused(box):
    import paper_1503_03553_gb300 as D
    ncell = grid_for(box, skin=SKIN)
    ctx = D.Context([box], precision="mixed", ncell=[ncell], skins=[SKIN])
    try:
        ctx.set_particles(0, box.x, box.v, box.w, box.r)
        n = box.n
        short = torch.zeros((n - 1, 3), dtype=torch.float64, device="cuda")
        with pytest.raises(ValueError, match="x must hold"):
            ctx.set_state(0, short, None, None, where=D.DEM_DEVICE)
        with pytest.raises(ValueError, match="omega must hold"):
            D.dem_get_state(ctx.ctx, 0, None, None, short, None, None, where=D.DEM_DEVICE)
        with pytest.raises(TypeError):
            ctx.set_state(0, torch.zeros((n, 3), dtype=torch.float32, device="cuda"), None, None,
                          where=D.DEM_DEVICE)
        with pytest.raises(ValueError, match="radius must hold"):
            ctx.set_particles(0, _dev(box.x), _dev(box.v), _dev(box.w), _dev(box.r[:-1]),
                              where=D.DEM_DEVICE)
        with pytest.raises(ValueError, match="x must hold"):
            ctx.set_state(0, box.x[:-1], None, None)  # host arrays are checked too
        ctx.step(1)  # the context is unharmed
        assert np.all(np.isfinite(ctx.get_state(0)["x"]))
    finally:
        ctx.close()
