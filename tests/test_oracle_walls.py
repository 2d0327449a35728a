"""Pins of the oracle's rectangle and line walls (Sec. 3.3 item 5: walls are
rectangles and straight lines, and a particle-wall force is computed like a
particle-particle force; Sec. 4.2 kernels CollideRectangle and CollideLine).

A wall acts as a body of infinite radius and mass at rest, touching the
particle at the wall's point closest to the particle's centre.  The pins:
a rectangle lying in z = 0 reproduces the flat floor; a sphere rolls down an
inclined rectangle at the textbook 5/7 g sin(theta); a head-on bounce on a
line, and on a rectangle's edge, returns the restitution of the normal law;
the force on a sphere near a rectangle's corner points along the line from
the corner to the centre.
"""
import math

import numpy as np
import pytest

import oracle as O

E, SIG, RHO = 3e9, 0.3, 1200.0
E_STAR = E / (2.0 * (1.0 - SIG * SIG))
G = E / (2.0 * (1.0 + SIG))
G_STAR = G / (2.0 * (2.0 - SIG))
HERTZ_TC = 0.8 * 1.25 ** 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)
R = 5e-6


def mass(r):
    return RHO * 4.0 / 3.0 * math.pi * r ** 3


def hertz_kn(r_star):
    return 4.0 / 3.0 * E_STAR * math.sqrt(r_star)


def _rest_overlap(normal_force):
    return (normal_force / hertz_kn(R)) ** (2.0 / 3.0)


def _step_dt(normal_force):
    m = mass(R)
    d = _rest_overlap(normal_force)
    k_lin = 1.5 * hertz_kn(R) * math.sqrt(d)
    kt = 8.0 * math.sqrt(R * d) * G_STAR
    return min(2 * math.pi * math.sqrt(m / k_lin), 2 * math.pi * math.sqrt(m / (3.5 * kt))) / 50.0


def test_rectangle_in_the_floor_plane_is_the_floor():
    """A sphere launched sliding on a rectangle spanning the plane z = 0
    follows the trajectory it has on the built-in floor."""
    g, u0, mu = 9.81, 1e-3, 0.3
    d = _rest_overlap(mass(R) * g)
    dt = _step_dt(mass(R) * g)
    L = 1e-3
    x0 = np.array([[L / 2, L / 2, R - d]])
    v0 = np.array([[u0, 0.3 * u0, 0.0]])
    floor = O.State(x0, v0, np.zeros((1, 3)), np.array([R]), floor_wall=True)
    rect = O.State(x0, v0, np.zeros((1, 3)), np.array([R]), nwalls=1)
    common = dict(periodic=(0, 0, 0), g=(0, 0, -g), mu_d=mu, r_max=R)
    pf = O.make_params((L, L, L), dt, floor_wall=1, **common)
    pr = O.make_params((L, L, L), dt, walls=[(O.WALL_RECT, (-L, -L, 0.0), (3 * L, 0, 0),
                                              (0, 3 * L, 0))], **common)
    for _ in range(3000):
        a = O.step(pf, floor)
        b = O.step(pr, rect)
    assert np.allclose(rect.x, floor.x, rtol=0, atol=1e-15)
    assert np.allclose(rect.v, floor.v, rtol=1e-9, atol=1e-12 * u0)
    assert np.allclose(rect.w, floor.w, rtol=1e-9, atol=1e-12 * u0 / R)
    assert np.allclose(b["F"], a["F"], rtol=1e-9, atol=1e-9 * mass(R) * g)


@pytest.mark.parametrize("theta_deg", [15.0, 25.0])
def test_rolling_down_an_inclined_rectangle(theta_deg):
    """Friction large enough to roll (mu > 2/7 tan theta): the centre
    accelerates at 5/7 g sin(theta) along the slope and rolls without
    slipping (v = r w)."""
    th = math.radians(theta_deg)
    g, mu = 9.81, 0.6
    down = np.array([math.cos(th), 0.0, -math.sin(th)])   # along the slope
    n_up = np.array([math.sin(th), 0.0, math.cos(th)])    # plane normal
    W = 2e-3
    corner = np.array([0.0, -W / 2, 2e-3]) - 0.5 * W * down
    d = _rest_overlap(mass(R) * g * math.cos(th))
    dt = _step_dt(mass(R) * g * math.cos(th))
    c0 = corner + 0.3 * W * down + np.array([0.0, W / 2, 0.0]) + (R - d) * n_up
    s = O.State(c0[None, :], np.zeros((1, 3)), np.zeros((1, 3)), np.array([R]), nwalls=1)
    L = 1e-2
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), g=(0, 0, -g), mu_d=mu,
                      r_max=R, ncell=(1, 1, 1),
                      walls=[(O.WALL_RECT, corner, W * down, (0.0, W, 0.0))])
    t_settle = 3000 * dt
    ts, vs = [], []
    t = 0.0
    for _ in range(12000):
        O.step(p, s)
        t += dt
        if t > t_settle:
            ts.append(t)
            vs.append(float(np.dot(s.v[0], down)))
    a_fit = np.polyfit(np.array(ts), np.array(vs), 1)[0]
    a_roll = 5.0 / 7.0 * g * math.sin(th)
    assert a_fit == pytest.approx(a_roll, rel=2e-2)
    # no slip: the contact point's velocity along the slope is ~0
    w_axis = np.cross(n_up, down)  # rolling down turns about +y for this slope
    slip = np.dot(s.v[0], down) - R * np.dot(s.w[0], w_axis)
    assert abs(slip) < 2e-2 * abs(np.dot(s.v[0], down))
    # the sphere stays on the plane at its static overlap
    gap = np.dot(s.x[0] - corner, n_up) - R
    assert gap == pytest.approx(-d, rel=5e-2)


def _bounce(wall, c0, v0_vec, eps, frac=50):
    """Head-on impact of one sphere on a wall without gravity; returns the
    rebound speed over the impact speed and the contact time over the
    Hertz contact time of the same normal law (m* = m, R* = r)."""
    m = mass(R)
    v0 = float(np.linalg.norm(v0_vec))
    kn = hertz_kn(R)
    tc = HERTZ_TC * (m ** 2 / (kn ** 2 * v0)) ** 0.2
    dt = tc / frac
    L = 1e-2
    s = O.State(c0[None, :], v0_vec[None, :], np.zeros((1, 3)), np.array([R]), nwalls=1)
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), restitution=eps, mu_d=0.3,
                      r_max=R, ncell=(1, 1, 1), walls=[wall])
    started, steps = False, 0
    for _ in range(int(10 * frac)):
        out = O.step(p, s)
        touching = np.linalg.norm(out["F"][0]) > 0.0
        if touching:
            started = True
            steps += 1
        elif started:
            break
    return -float(np.dot(s.v[0], v0_vec)) / v0 ** 2, steps * dt / tc


@pytest.mark.parametrize("eps", [0.5, 0.9])
def test_bounce_on_a_line(eps):
    """A sphere moving along -z hits a line along y: it rebounds with the
    restitution of the normal law and touches for the Hertz contact time."""
    v0 = 0.1
    line = (O.WALL_LINE, (5e-3, 4e-3, 5e-3), (0.0, 2e-3, 0.0), None)
    c0 = np.array([5e-3, 5e-3, 5e-3 + R + 0.2 * v0 * 1e-9])
    e, t_rel = _bounce(line, c0, np.array([0.0, 0.0, -v0]), eps)
    assert e == pytest.approx(eps, abs=1e-2)
    if eps == 0.9:
        assert t_rel == pytest.approx(1.0, abs=0.05)


def test_bounce_on_a_rectangle_edge():
    """Approached within its own plane, a rectangle is touched at its edge:
    the bounce is that of a line."""
    v0, eps = 0.1, 0.5
    rect = (O.WALL_RECT, (4e-3, 4e-3, 5e-3), (1e-3, 0.0, 0.0), (0.0, 2e-3, 0.0))
    c0 = np.array([5e-3 + R + 1e-11, 5e-3, 5e-3])   # beyond the edge x = 5e-3
    e_edge, _ = _bounce(rect, c0, np.array([-v0, 0.0, 0.0]), eps)
    line = (O.WALL_LINE, (5e-3, 4e-3, 5e-3), (0.0, 2e-3, 0.0), None)
    e_line, _ = _bounce(line, c0, np.array([-v0, 0.0, 0.0]), eps)
    assert e_edge == pytest.approx(e_line, rel=1e-12)
    assert e_edge == pytest.approx(eps, abs=1e-2)


def test_force_at_a_rectangle_corner():
    """A sphere overlapping only a rectangle's corner is pushed along the
    line from the corner to its centre, with the Hertz force of the overlap
    (at rest: no damping, no tangential part)."""
    corner = np.array([1e-3, 1e-3, 1e-3])
    rect = (O.WALL_RECT, corner, (1e-4, 0.0, 0.0), (0.0, 1e-4, 0.0))
    direction = np.array([-1.0, -2.0, 2.0]) / 3.0     # away from the rectangle
    dn = 2e-9
    c0 = corner + (R - dn) * direction
    s = O.State(c0[None, :], np.zeros((1, 3)), np.zeros((1, 3)), np.array([R]), nwalls=1)
    L = 1e-2
    p = O.make_params((L, L, L), 1e-9, periodic=(0, 0, 0), r_max=R, ncell=(1, 1, 1),
                      walls=[rect])
    out = O.step(p, s)
    F = out["F"][0]
    assert np.allclose(F / np.linalg.norm(F), direction, atol=1e-9)
    assert np.linalg.norm(F) == pytest.approx(hertz_kn(R) * dn ** 1.5, rel=1e-6)
    assert np.allclose(out["T"][0], 0.0, atol=1e-9 * np.linalg.norm(F) * R)
