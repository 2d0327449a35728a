"""Parity at the benchmark's full size: the W2 workload of 1,000,000
polydisperse spheres (packing 0.55), as `bench.py` builds it.

One step of the library against one step of the FP64 oracle over every
particle and contact (sort order and contact set bit for bit, forces,
torques and delta_t within the tolerances of tests/parity.py), and the
benchmark's launch form (CUDA graphs of 16 steps) bit-identical to direct
launches over 32 steps.
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


def test_full_size_one_step_matches_oracle(w2_full):
    ncell = grid_for(w2_full)
    g = gpu_run([w2_full], "mixed", [ncell])[0]
    o = oracle_run(w2_full, "mixed", ncell)
    m = check_one_step(w2_full, g, o, "mixed")
    assert m["contacts"] > w2_full.n  # the dense contact network of the workload


def test_full_size_graph_replay_bit_identical(w2_full):
    ncell = grid_for(w2_full)
    a = gpu_run([w2_full], "mixed", [ncell], steps=32, graph_steps=16)[0]
    c = gpu_run([w2_full], "mixed", [ncell], steps=32, graph_steps=-1)[0]
    for k in ("x", "v", "w", "F", "T"):
        assert np.array_equal(a["state"][k], c["state"][k]), k
    assert np.array_equal(a["lo"], c["lo"]) and np.array_equal(a["hi"], c["hi"])
    assert np.array_equal(a["dt"], c["dt"])
