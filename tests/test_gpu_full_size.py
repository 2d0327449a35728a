"""Parity at full size: the W2 workload of 1,000,000 polydisperse spheres
(packing 0.55) as `bench.py` builds it, and the W3 workload of 8,000,000
bidisperse spheres (dense and dilute halves, floor, gravity).

One step of the library against one step of the FP64 oracle over every
particle and contact (sort order and contact set bit for bit, forces,
torques and delta_t within the tolerances of tests/parity.py), and the
benchmark's launch form (CUDA graphs of 16 steps, candidate-list skin)
bit-identical to direct launches and to the search of every step over 32
steps.
"""
import numpy as np
import pytest

from paper_1503_03553_gb300 import synth
from parity import check_one_step, gpu_run, grid_for, oracle_run, prepared

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)


@pytest.fixture(scope="module")
def w2_full():
    b = prepared(synth.w2_polydisperse(n=1_000_000, seed=2), "mixed")
    assert b.n == 1_000_000
    return b


SKIN = 0.04e-6  # the benchmark's skin (bench.py --skin-um)


def test_full_size_one_step_matches_oracle(w2_full):
    ncell = grid_for(w2_full, skin=SKIN)
    g = gpu_run([w2_full], "mixed", [ncell], skins=[SKIN])[0]
    o = oracle_run(w2_full, "mixed", ncell, parallel=True)
    m = check_one_step(w2_full, g, o, "mixed")
    assert m["contacts"] > w2_full.n  # the dense contact network of the workload


def test_full_size_graph_replay_bit_identical(w2_full):
    ncell = grid_for(w2_full, skin=SKIN)
    a = gpu_run([w2_full], "mixed", [ncell], steps=32, graph_steps=16, skins=[SKIN])[0]
    c = gpu_run([w2_full], "mixed", [ncell], steps=32, graph_steps=-1, skins=[SKIN])[0]
    z = gpu_run([w2_full], "mixed", [ncell], steps=32, graph_steps=16, skins=[0.0])[0]
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(a["state"][k], c["state"][k]), k
        assert np.array_equal(a["state"][k], z["state"][k]), k
    assert np.array_equal(a["lo"], c["lo"]) and np.array_equal(a["hi"], c["hi"])
    assert np.array_equal(a["dt"], c["dt"])
    assert a["resorts"]["resorts"] < 32 and z["resorts"]["resorts"] == 32


def test_w3_full_size_one_step_matches_oracle():
    """8,000,000 bidisperse spheres, floor and gravity, open top: every
    contact and particle against the oracle (its OpenMP build)."""
    b = prepared(synth.w3_bidisperse_floor(n=8_000_000, seed=3), "mixed")
    assert b.n > 7_900_000
    ncell = grid_for(b, skin=SKIN)
    g = gpu_run([b], "mixed", [ncell], skins=[SKIN])[0]
    o = oracle_run(b, "mixed", ncell, parallel=True)
    m = check_one_step(b, g, o, "mixed")
    assert m["contacts"] > b.n // 2
