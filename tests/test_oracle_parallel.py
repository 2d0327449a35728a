"""The OpenMP build of the oracle (liboracle_omp.so, all host cores) gives
the serial oracle's results bit for bit: contact sets, forces, torques,
delta_t and the state after each step, over several steps with history, on
a periodic box, a box with an open axis, floor, gravity and walls, and with
the FP64 and fixed-point FP32 contact rules."""
import dataclasses
import os

import numpy as np
import pytest

import oracle as O
from paper_1503_03553_gb300 import synth

from parity import oracle_params, prepared


def _walled(n, seed):
    b = synth.w2_polydisperse(n=n, seed=seed)
    L = float(b.L[0])
    walls = ((0, (0.0, 0.0, 0.30 * L), (L, 0.0, 0.2 * L), (0.0, L, 0.0)),
             (1, (0.0, 0.5 * L, 0.8 * L), (L, 0.1 * L, 0.0), None))
    return dataclasses.replace(b, periodic=(1, 1, 0), floor_wall=1, g=(0.0, 0.0, -9.81),
                               walls=walls)


@pytest.mark.parametrize("case", ["periodic_fixed", "periodic_fp64", "walls_fixed"])
def test_openmp_oracle_bit_identical(case, monkeypatch):
    monkeypatch.setenv("OMP_NUM_THREADS", str(max(2, min(8, os.cpu_count() or 2))))
    if case == "walls_fixed":
        box = _walled(4000, 71)
    else:
        box = synth.w2_polydisperse(n=8000, seed=70)
    prec = "fp64" if case == "periodic_fp64" else "mixed"
    b = prepared(box, prec)
    p = oracle_params(b, prec, [max(3, int(b.L[a] // (2.0 * b.r_max * (1 + 1e-5)))) for a in range(3)])
    nw = len(getattr(b, "walls", ()))
    ss = [O.State(b.x, b.v, b.w, b.r, floor_wall=bool(b.floor_wall), nwalls=nw) for _ in range(2)]
    for _ in range(4):
        outs = [O.step(p, ss[0]), O.step(p, ss[1], parallel=True)]
        a, c = outs
        assert len(a["lo"]) > b.n // 2
        for k in ("lo", "hi", "dt", "F", "T"):
            assert np.array_equal(a[k], c[k]), k
        assert np.array_equal(a["info"], c["info"])
        for k in ("x", "v", "w"):
            assert np.array_equal(getattr(ss[0], k), getattr(ss[1], k)), k
        if ss[0].wall_dt is not None:
            assert np.array_equal(ss[0].wall_dt, ss[1].wall_dt)
    lo_s, hi_s = O.contacts(p, ss[0].x, b.r)
    lo_p, hi_p = O.contacts(p, ss[0].x, b.r, parallel=True)
    assert np.array_equal(lo_s, lo_p) and np.array_equal(hi_s, hi_p)
