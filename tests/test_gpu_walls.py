"""GPU parity of rectangle and line walls (Sec. 3.3 item 5; Sec. 4.2 kernels
CollideRectangle and CollideLine) against the FP64 oracle.

The box: a dense polydisperse packing, periodic in x and y, open in z with
the floor, gravity, two rectangles crossing the packing (one tilted, one
vertical-ish) and a line; many particles overlap a wall, some at an edge or
a corner of a rectangle.
"""
import dataclasses

import numpy as np
import pytest

from paper_1503_03553_gb300 import synth
from parity import check_one_step, gpu_run, grid_for, oracle_run, prepared

pytestmark = pytest.mark.gpu


def walled_box(n=3000, seed=31):
    b = synth.w2_polydisperse(n=n, seed=seed)
    L = float(b.L[0])
    walls = (
        (0, (0.0, 0.0, 0.30 * L), (L, 0.0, 0.2 * L), (0.0, L, 0.0)),
        (0, (0.2 * L, 0.1 * L, 0.55 * L), (0.5 * L, 0.0, 0.0), (0.0, 0.3 * L, 0.3 * L)),
        (1, (0.0, 0.5 * L, 0.8 * L), (L, 0.1 * L, 0.0), None),
    )
    return dataclasses.replace(b, periodic=(1, 1, 0), floor_wall=1, g=(0.0, 0.0, -9.81),
                               walls=walls)


@pytest.fixture(scope="module")
def walled():
    return walled_box()


def _wall_contacts(b):
    """How many particles touch each wall (FP64 geometry, for the test's own
    sanity: the configuration must exercise faces, edges and the line)."""
    counts = []
    for kind, p, u, v in b.walls:
        p, u = np.asarray(p), np.asarray(u)
        d = b.x - p
        s = np.clip(d @ u / (u @ u), 0, 1)
        q = p + s[:, None] * u
        if kind == 0:
            v = np.asarray(v)
            t = np.clip(d @ v / (v @ v), 0, 1)
            q = q + t[:, None] * v
        counts.append(int(np.sum(np.linalg.norm(q - b.x, axis=1) < b.r)))
    return counts


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_walls_one_step_match_oracle(walled, precision):
    b = prepared(walled, precision)
    assert all(c > 5 for c in _wall_contacts(b))
    ncell = grid_for(b)
    g = gpu_run([b], precision, [ncell])[0]
    o = oracle_run(b, precision, ncell)
    check_one_step(b, g, o, precision)


def test_walls_history_over_steps_tracks_oracle(walled):
    """Ten steps: the wall histories carried on the GPU keep per-particle
    forces within tolerance of the oracle's ten steps (compared through
    the kinetic energy and the mean height, which the walls and gravity
    set)."""
    import oracle as O
    from parity import oracle_params
    b = prepared(walled, "fp64")
    ncell = grid_for(b)
    g = gpu_run([b], "fp64", [ncell], steps=10)[0]
    s = O.State(b.x, b.v, b.w, b.r, floor_wall=True, nwalls=len(b.walls))
    p = oracle_params(b, "fp64", ncell)
    for _ in range(10):
        O.step(p, s)
    m = synth.DENSITY_DEFAULT * 4 / 3 * np.pi * b.r ** 3
    ke_g = 0.5 * np.sum(m[:, None] * g["state"]["v"] ** 2)
    ke_o = 0.5 * np.sum(m[:, None] * s.v ** 2)
    assert ke_g == pytest.approx(ke_o, rel=1e-6)
    assert np.allclose(g["state"]["x"][:, 2], s.x[:, 2], rtol=0, atol=1e-12)


def test_walled_and_plain_boxes_in_one_context(walled):
    """A context holding a box with walls and one without: each box matches
    the oracle run on it alone (the wall kernel and the wall histories skip
    the plain box)."""
    plain = synth.w2_polydisperse(n=2000, seed=32)
    boxes = [prepared(walled, "mixed"), prepared(plain, "mixed")]
    ncells = [grid_for(b) for b in boxes]
    gs = gpu_run(boxes, "mixed", ncells)
    for b, g, nc in zip(boxes, gs, ncells):
        check_one_step(b, g, oracle_run(b, "mixed", nc), "mixed")
