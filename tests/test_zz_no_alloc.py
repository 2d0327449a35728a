"""dem_contacts_static: contact detection with no device allocation.

For callers that cannot allocate device memory when they need a contact
list: code inside another framework's memory pool or a fixed budget, or
latency-critical code that must not call cudaMalloc (it can synchronise the
device).  The entry point uses one file-scope scratch array instead of
allocations.  These tests check it against the FP64 oracle's contact set
(the same single-precision contact rule on the same grid) and against the
contact list of dem_step (the allocating path) on two calls in a row, on a
box with an open axis, and its error paths: sizes beyond its limits, a
radius above half a cell or not positive, a non-finite position, a cap below
the contact count, and host memory.  The file name makes pytest collect it
last.
"""
import ctypes as C
import dataclasses

import numpy as np
import pytest

import oracle as O
from paper_1503_03553_gb300 import synth

from parity import gpu_run, grid_for, oracle_params, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


def _tensors(box, cap):
    x = torch.tensor(box.x, dtype=torch.float64, device="cuda")
    r = torch.tensor(box.r, dtype=torch.float64, device="cuda")
    pairs = torch.full((cap, 2), -7, dtype=torch.int32, device="cuda")
    return x, r, pairs


def _sorted(got):
    key = np.lexsort((got[:, 1], got[:, 0]))
    return got[key, 0], got[key, 1]


def _static_pairs(box, ncell, cap):
    import paper_1503_03553_gb300 as D
    x, r, pairs = _tensors(box, cap)
    n = D.dem_contacts_static(x, r, box.L, box.periodic, ncell, pairs)
    return _sorted(pairs[:n].cpu().numpy())


def _oracle_pairs(box, ncell):
    p = oracle_params(box, "mixed", ncell)
    lo, hi = O.contacts(p, box.x, box.r)
    key = np.lexsort((hi, lo))
    return lo[key], hi[key]


def test_static_contacts_match_oracle_and_dem_step_two_calls():
    boxes = [prepared(synth.w2_polydisperse(n=3000, seed=41), "mixed"),
             prepared(synth.w2_polydisperse(n=1200, seed=42), "mixed")]
    for box in boxes:  # two calls in a row, the second on a smaller box
        ncell = grid_for(box, stencil=1)
        lo, hi = _static_pairs(box, ncell, cap=16 * box.n)
        olo, ohi = _oracle_pairs(box, ncell)
        assert len(olo) > box.n
        assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)
        ref = gpu_run([box], "mixed", [ncell], stencil=1)[0]  # dem_step's contacts
        assert np.array_equal(lo, ref["lo"]) and np.array_equal(hi, ref["hi"])


def test_static_contacts_open_axis():
    """One non-periodic axis: cells clamp at the open faces."""
    box = prepared(dataclasses.replace(synth.w2_polydisperse(n=2500, seed=43),
                                       periodic=(1, 1, 0)), "mixed")
    ncell = grid_for(box, stencil=1)
    lo, hi = _static_pairs(box, ncell, cap=16 * box.n)
    olo, ohi = _oracle_pairs(box, ncell)
    assert len(olo) > 0
    assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)
    ref = gpu_run([box], "mixed", [ncell], stencil=1)[0]
    assert np.array_equal(lo, ref["lo"]) and np.array_equal(hi, ref["hi"])


def test_static_contacts_cap_below_count():
    import paper_1503_03553_gb300 as D
    box = prepared(synth.w2_polydisperse(n=2000, seed=44), "mixed")
    ncell = grid_for(box, stencil=1)
    olo, ohi = _oracle_pairs(box, ncell)
    cap = len(olo) // 2
    x, r, pairs = _tensors(box, cap)
    with pytest.raises(D.DemError) as e:
        D.dem_contacts_static(x, r, box.L, box.periodic, ncell, pairs)
    assert e.value.status == D.DEM_ERR_CAPACITY
    got = pairs.cpu().numpy()
    assert np.all(got[:, 0] >= 0)  # every row up to cap written
    truth = set(zip(olo.tolist(), ohi.tolist()))
    rows = list(zip(got[:, 0].tolist(), got[:, 1].tolist()))
    assert len(set(rows)) == cap and set(rows) <= truth


def test_static_contacts_reject_bad_radius_and_position():
    import paper_1503_03553_gb300 as D
    box = prepared(synth.w2_polydisperse(n=1500, seed=45), "mixed")
    ncell = grid_for(box, stencil=1)
    hmin = min(box.L[a] / ncell[a] for a in range(3))
    cases = []
    big = box.r.copy()
    big[17] = 0.6 * hmin
    cases.append((box.x, big, D.DEM_ERR_ARG, "half"))
    zero = box.r.copy()
    zero[3] = 0.0
    cases.append((box.x, zero, D.DEM_ERR_ARG, "zero"))
    nan = box.x.copy()
    nan[5, 1] = np.nan
    cases.append((nan, box.r, D.DEM_ERR_NONFINITE, "non-finite"))
    for xx, rr, status, word in cases:
        x = torch.tensor(xx, dtype=torch.float64, device="cuda")
        r = torch.tensor(rr, dtype=torch.float64, device="cuda")
        pairs = torch.zeros((16 * box.n, 2), dtype=torch.int32, device="cuda")
        with pytest.raises(D.DemError) as e:
            D.dem_contacts_static(x, r, box.L, box.periodic, ncell, pairs)
        assert e.value.status == status and word in str(e.value), str(e.value)
    # the scratch array keeps nothing from a failed call: a good call after
    lo, hi = _static_pairs(box, ncell, cap=16 * box.n)
    olo, ohi = _oracle_pairs(box, ncell)
    assert np.array_equal(lo, olo) and np.array_equal(hi, ohi)


def test_static_contacts_reject_host_memory_and_bad_shapes():
    import paper_1503_03553_gb300 as D
    box = prepared(synth.w2_polydisperse(n=500, seed=46), "mixed")
    ncell = grid_for(box, stencil=1)
    hx = np.ascontiguousarray(box.x)
    hr = np.ascontiguousarray(box.r)
    hp = np.zeros((64, 2), np.int32)
    cnt = C.c_int64(0)
    st = D.lib().dem_contacts_static(
        box.n, C.c_void_p(hx.ctypes.data), C.c_void_p(hr.ctypes.data),
        (C.c_double * 3)(*box.L), (C.c_int32 * 3)(*box.periodic), (C.c_int32 * 3)(*ncell),
        64, C.c_void_p(hp.ctypes.data), C.byref(cnt), None)
    assert st == D.DEM_ERR_ARG and "device memory" in D.dem_last_error(None)
    x, r, pairs = _tensors(box, 64)
    with pytest.raises(ValueError):
        D.dem_contacts_static(x, r[:-1], box.L, box.periodic, ncell, pairs)
    with pytest.raises(ValueError):
        D.dem_contacts_static(x, r, box.L, box.periodic, ncell, pairs.reshape(-1))


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
