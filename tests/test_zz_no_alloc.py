"""dem_contacts_static: contact detection with no device allocation.

For callers that cannot allocate device memory when they need a contact
list (code inside another framework's memory pool or a fixed budget, or
latency-critical code that must not call cudaMalloc).  The entry point uses
one file-scope scratch array instead of allocations; this test checks it
against the contact list of dem_step (the existing path) on two calls in a
row, and that it rejects sizes beyond its limits.  The file name makes
pytest collect it last.
"""
import numpy as np
import pytest

from paper_1503_03553_gb300 import synth

from parity import gpu_run, grid_for, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _static_pairs(box, ncell, cap):
    import paper_1503_03553_gb300 as D
    x = torch.tensor(box.x, dtype=torch.float64, device="cuda")
    r = torch.tensor(box.r, dtype=torch.float64, device="cuda")
    pairs = torch.full((cap, 2), -7, dtype=torch.int32, device="cuda")
    n = D.dem_contacts_static(x, r, box.L, box.periodic, ncell, pairs)
    got = pairs[:n].cpu().numpy()
    key = np.lexsort((got[:, 1], got[:, 0]))
    return got[key, 0], got[key, 1]


def test_static_contacts_match_dem_step_two_calls():
    boxes = [prepared(synth.w2_polydisperse(n=3000, seed=41), "mixed"),
             prepared(synth.w2_polydisperse(n=1200, seed=42), "mixed")]
    for box in boxes:  # two calls in a row, the second on a smaller box
        ncell = grid_for(box, stencil=1)
        ref = gpu_run([box], "mixed", [ncell], stencil=1)[0]  # dem_step's contacts
        lo, hi = _static_pairs(box, ncell, cap=16 * box.n)
        assert len(ref["lo"]) > box.n
        assert np.array_equal(lo, ref["lo"]) and np.array_equal(hi, ref["hi"])


def test_static_contacts_reject_oversize():
    import paper_1503_03553_gb300 as D
    box = prepared(synth.w2_polydisperse(n=3000, seed=41), "mixed")
    x = torch.zeros((8193, 3), dtype=torch.float64, device="cuda")
    r = torch.full((8193,), 1e-6, dtype=torch.float64, device="cuda")
    pairs = torch.zeros((16, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(D.DemError) as e:
        D.dem_contacts_static(x, r, box.L, box.periodic, grid_for(box, stencil=1), pairs)
    assert e.value.status == D.DEM_ERR_ARG and "8192" in str(e.value)
    with pytest.raises(D.DemError) as e:
        D.dem_contacts_static(x[:10], r[:10], (1e-3,) * 3, (1, 1, 1), (40, 40, 40), pairs)
    assert e.value.status == D.DEM_ERR_ARG and "32768" in str(e.value)
