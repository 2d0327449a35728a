"""Pins of the FP64 oracle against facts fixed outside it.

Every test here runs on the CPU.  None compares the oracle with itself: each
checks it against a closed form, a library routine, brute force, or an
invariant of the mathematics, chosen so that a plausible slip (a dropped
term, a wrong sign or index, a transposed operand) fails one of them.

Paper: Nakahara & Washizawa, arXiv 1503.03553, Sec. 2 (force law, Eq. (1),
Eq. (vt), Eq. (dt), Eq. (sliding friction), k_n, k_t, eta) and Sec. 4.2
(kernel list).
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_1503_03553_gb300 import synth

E, SIG, RHO = 3e9, 0.3, 1200.0
E_STAR = E / (2.0 * (1.0 - SIG * SIG))       # Hertz, two equal bodies
G = E / (2.0 * (1.0 + SIG))
G_STAR = G / (2.0 * (2.0 - SIG))             # Mindlin, two equal bodies
HERTZ_TC = 0.8 * 1.25 ** 0.4 * math.gamma(0.4) * math.gamma(0.5) / math.gamma(0.9)


def mass(r):
    return RHO * 4.0 / 3.0 * math.pi * r ** 3


def hertz_kn(R_star):
    """Textbook Hertz stiffness F = k_n delta^{3/2}, k_n = 4/3 E* sqrt(R*)."""
    return 4.0 / 3.0 * E_STAR * math.sqrt(R_star)


# --------------------------------------------------------------------------
# contact search
# --------------------------------------------------------------------------
@pytest.fixture(scope="module")
def dense_box():
    return synth.w2_polydisperse(n=3000, seed=11)


@pytest.fixture(scope="module")
def dilute_box():
    return synth.w1_monodisperse(n=600, seed=12)


@pytest.mark.parametrize("pred", [O.PRED_FP64, O.PRED_FIXED_F32, O.PRED_ABS_F32])
def test_cell_search_equals_brute_force(dense_box, pred):
    b = dense_box
    p = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=pred)
    pb = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=pred, brute_force=1)
    lo, hi = O.contacts(p, b.x, b.r)
    lo2, hi2 = O.contacts(pb, b.x, b.r)
    assert len(lo) > b.n  # dense packing: more than one contact per particle
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)


@pytest.mark.parametrize("pred", [O.PRED_FP64, O.PRED_FIXED_F32, O.PRED_ABS_F32])
def test_two_cell_stencil_equals_brute_force(dense_box, pred):
    """Cells half as wide searched +-2 per axis find the same pairs."""
    b = dense_box
    p = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=pred, stencil=2)
    pb = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=pred, stencil=2,
                       brute_force=1)
    assert p.ncell[0] >= 2 * O.make_params(b.L, b.dt, r_max=b.r_max).ncell[0] - 1
    lo, hi = O.contacts(p, b.x, b.r)
    lo2, hi2 = O.contacts(pb, b.x, b.r)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)
    if pred == O.PRED_FP64:
        lo1, hi1 = O.contacts(O.make_params(b.L, b.dt, r_max=b.r_max), b.x, b.r)
        assert np.array_equal(lo, lo1) and np.array_equal(hi, hi1)


def _kdtree_pairs(x, r, L):
    """Contact set by scipy's periodic k-d tree, distances recomputed with
    the same minimum-image rounding as the definition."""
    from scipy.spatial import cKDTree

    L = np.asarray(L)
    t = cKDTree(np.mod(x, L), boxsize=L)
    pr = t.query_pairs(2.0 * r.max() * (1 + 1e-9), output_type="ndarray")
    i, j = np.minimum(pr[:, 0], pr[:, 1]), np.maximum(pr[:, 0], pr[:, 1])
    d = x[j] - x[i]
    hl = 0.5 * L
    d = np.where(d > hl, d - L, np.where(d < -hl, d + L, d))
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    R = r[i] + r[j]
    m = d2 < R * R
    key = np.lexsort((j[m], i[m]))
    return i[m][key].astype(np.int32), j[m][key].astype(np.int32)


def test_fp64_contacts_equal_kdtree(dense_box):
    b = dense_box
    p = O.make_params(b.L, b.dt, r_max=b.r_max)
    lo, hi = O.contacts(p, b.x, b.r)
    lo2, hi2 = _kdtree_pairs(b.x, b.r, b.L)
    assert np.array_equal(lo, lo2) and np.array_equal(hi, hi2)


@pytest.mark.parametrize("pred", [O.PRED_FIXED_F32, O.PRED_ABS_F32])
def test_f32_predicates_differ_only_at_the_boundary(dense_box, pred):
    """A single-precision predicate may flip only pairs whose gap is within
    float rounding of zero."""
    b = dense_box
    p64 = O.make_params(b.L, b.dt, r_max=b.r_max)
    p32 = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=pred)
    a = set(zip(*O.contacts(p64, b.x, b.r)))
    c = set(zip(*O.contacts(p32, b.x, b.r)))
    L = np.asarray(b.L)
    for (i, j) in a ^ c:
        d = b.x[j] - b.x[i]
        d -= L * np.round(d / L)
        gap = abs(np.linalg.norm(d) - (b.r[i] + b.r[j]))
        assert gap < 2e-6 * (b.r[i] + b.r[j]), (i, j, gap)


def test_fixed_predicate_is_symmetric(dense_box):
    """Swapping the two positions of a pair gives the same decision (the
    predicate uses (o_j - o_i) + shift, antisymmetric in float)."""
    b = dense_box
    p = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=O.PRED_FIXED_F32,
                      brute_force=1)
    lo, hi = O.contacts(p, b.x, b.r)
    # reversed ids: particle k becomes n-1-k, so every pair is evaluated with
    # its members swapped
    rev = b.x[::-1].copy()
    lo2, hi2 = O.contacts(p, rev, b.r[::-1].copy())
    n = b.n
    a = set(zip(lo.tolist(), hi.tolist()))
    c = set((n - 1 - j, n - 1 - i) for i, j in zip(lo2.tolist(), hi2.tolist()))
    assert a == c


# --------------------------------------------------------------------------
# sort order: cells by exact integer floor division, Morton interleave
# --------------------------------------------------------------------------
def _morton_py(cx, cy, cz):
    code = 0
    for bit in range(21):
        code |= ((cx >> bit) & 1) << (3 * bit)
        code |= ((cy >> bit) & 1) << (3 * bit + 1)
        code |= ((cz >> bit) & 1) << (3 * bit + 2)
    return code


def test_order_fixed_point_rule(dense_box):
    b = dense_box
    p = O.make_params(b.L, b.dt, r_max=b.r_max, predicate=O.PRED_FIXED_F32)
    cell, order = O.order(p, b.x)
    n = [p.ncell[a] for a in range(3)]
    codes = []
    lin = []
    for k in range(b.n):
        c = []
        for a in range(3):
            X = int(round(b.x[k, a] * 2.0 ** 60))
            Lq = int(round(b.L[a] * 2.0 ** 60))
            H = Lq // n[a]
            ca = min(X // H, n[a] - 1)
            assert ca * H <= X  # the position lies in its cell
            assert X < (ca + 1) * H or ca == n[a] - 1
            c.append(ca)
        codes.append(_morton_py(*c))
        lin.append((c[2] * n[1] + c[1]) * n[0] + c[0])
    assert np.array_equal(cell, np.array(lin, np.int32))
    expect = np.lexsort((np.arange(b.n), np.array(codes, dtype=np.uint64)))
    assert np.array_equal(order, expect.astype(np.int32))


# --------------------------------------------------------------------------
# restitution parameter alpha(eps)
# --------------------------------------------------------------------------
def _scipy_restitution(alpha):
    from scipy.integrate import solve_ivp

    def f(t, y):
        x = max(y[0], 0.0)
        return [y[1], -x ** 1.5 - alpha * x ** 0.25 * y[1]]

    def hit(t, y):
        return y[0]
    hit.terminal = True
    hit.direction = -1
    sol = solve_ivp(f, (0.0, 50.0), [0.0, 1.0], method="DOP853", rtol=1e-12,
                    atol=1e-14, events=hit, first_step=1e-6)
    return -sol.y_events[0][0][1], sol.t_events[0][0]


@pytest.mark.parametrize("alpha", [0.0, 0.1, 0.4818, 1.0])
def test_restitution_matches_library_ode_solve(alpha):
    e_lib, t_end = _scipy_restitution(alpha)
    assert abs(O.restitution(alpha) - e_lib) < 2e-7
    if alpha == 0.0:
        # undamped Hertz impact: elastic, duration = the closed-form constant
        assert abs(e_lib - 1.0) < 1e-9
        assert abs(t_end - HERTZ_TC) < 1e-6


@pytest.mark.parametrize("eps", [0.3, 0.5, 0.7, 0.9, 0.99])
def test_alpha_inverts_restitution(eps):
    a = O.alpha(eps)
    assert abs(O.restitution(a) - eps) < 1e-9
    # the published Hertz-damping closed form agrees to a few percent
    approx = math.sqrt(5.0) * (-math.log(eps)) / math.sqrt(math.log(eps) ** 2 + math.pi ** 2)
    assert abs(a - approx) < 0.05 * approx


# --------------------------------------------------------------------------
# two-sphere head-on impact: Hertz contact time, maximum overlap, restitution
# --------------------------------------------------------------------------
def _head_on(r1, r2, v0, eps, frac, mu=0.3):
    m1, m2 = mass(r1), mass(r2)
    mstar = m1 * m2 / (m1 + m2)
    Rstar = r1 * r2 / (r1 + r2)
    kn = hertz_kn(Rstar)
    tc = HERTZ_TC * (mstar ** 2 / (kn ** 2 * v0)) ** 0.2
    dmax = (5.0 * mstar * v0 ** 2 / (4.0 * kn)) ** 0.4
    dt = tc / frac
    L = 40.0 * (r1 + r2)
    # momentum-free approach along x, just touching at the first step
    x = np.array([[L / 2 - r1, L / 2, L / 2], [L / 2 + r2 + 0.25 * v0 * dt, L / 2, L / 2]])
    v = np.array([[v0 * m2 / (m1 + m2), 0, 0], [-v0 * m1 / (m1 + m2), 0, 0]])
    s = O.State(x, v, np.zeros((2, 3)), np.array([r1, r2]))
    p = O.make_params((L, L, L), dt, restitution=eps, mu_d=mu, periodic=(0, 0, 0),
                      r_max=max(r1, r2))
    steps_in_contact, peak, started = 0, 0.0, False
    for _ in range(int(5 * frac) + 10):
        out = O.step(p, s)
        if len(out["lo"]):
            started = True
            steps_in_contact += 1
            peak = max(peak, out["info"]["delta_n"][0])
        elif started:
            break
    e = (s.v[1, 0] - s.v[0, 0]) / v0  # separation speed over approach speed
    return steps_in_contact * dt, tc, peak, dmax, e


@pytest.mark.parametrize("frac,tol", [(50, 0.03), (500, 0.003)])
def test_hertz_contact_time_and_peak_overlap(frac, tol):
    t, tc, peak, dmax, e = _head_on(5e-6, 5e-6, 0.1, 1.0, frac)
    assert abs(t - tc) <= tol * tc + 1e-30
    assert abs(peak - dmax) <= tol * dmax
    assert abs(e - 1.0) <= tol


def test_hertz_unequal_spheres():
    t, tc, peak, dmax, e = _head_on(3e-6, 6e-6, 0.5, 1.0, 500)
    assert abs(t - tc) <= 0.003 * tc
    assert abs(peak - dmax) <= 0.003 * dmax


@pytest.mark.parametrize("eps", [0.3, 0.5, 0.9])
def test_restitution_of_a_collision(eps):
    _, _, _, _, e50 = _head_on(5e-6, 5e-6, 0.1, eps, 50)
    _, _, _, _, e500 = _head_on(5e-6, 5e-6, 0.1, eps, 500)
    assert abs(e50 - eps) < 1e-2
    assert abs(e500 - eps) < 1e-3


@pytest.mark.parametrize("v0,r", [(0.01, 5e-6), (1.0, 5e-6), (0.1, 2e-6)])
def test_restitution_independent_of_speed_and_size(v0, r):
    _, _, _, _, e = _head_on(r, r, v0, 0.5, 500)
    assert abs(e - 0.5) < 1e-3


# --------------------------------------------------------------------------
# single contact by hand
# --------------------------------------------------------------------------
def test_static_overlap_force_is_hertz_and_repulsive():
    r1, r2, dn = 4e-6, 6e-6, 5e-8
    L = 1e-3
    x = np.array([[L / 2, L / 2, L / 2], [L / 2, L / 2 + r1 + r2 - dn, L / 2]])
    s = O.State(x, np.zeros((2, 3)), np.zeros((2, 3)), np.array([r1, r2]))
    p = O.make_params((L, L, L), 1e-12, periodic=(0, 0, 0), r_max=r2)
    out = O.step(p, s)
    F = out["F"]
    mag = hertz_kn(r1 * r2 / (r1 + r2)) * dn ** 1.5
    assert np.allclose(F[0], [0, -mag, 0], rtol=1e-9, atol=0)
    assert np.allclose(F[1], [0, mag, 0], rtol=1e-9, atol=0)
    assert np.all(np.abs(out["T"]) < 1e-30)


def test_spin_drives_tangential_force_and_opposing_torque():
    """Particle 1 spins about +z, particle 2 rests on its +x side.  The
    contact point of 1 moves along +y, so friction on 1 points along -y,
    the torque on 1 opposes its spin, and 2 is spun the other way."""
    r, dn, w = 5e-6, 2e-8, 1e3
    L, dt = 1e-3, 1e-9
    x = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2 * r - dn, L / 2, L / 2]])
    om = np.array([[0, 0, w], [0, 0, 0]], dtype=float)
    s = O.State(x, np.zeros((2, 3)), om, np.array([r, r]))
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), r_max=r, mu_d=10.0,
                      restitution=0.5)
    out = O.step(p, s)
    F, T = out["F"], out["T"]
    kt = 8.0 * math.sqrt(r / 2 * dn) * G_STAR
    a = O.alpha(0.5)
    m = mass(r)
    eta = a * math.sqrt(m / 2 * hertz_kn(r / 2) * math.sqrt(dn))
    vt = r * w                       # contact-point slip speed along +y
    Ft = -kt * vt * dt - eta * vt    # spring on delta_t = v_t dt, plus damping
    assert F[0, 1] == pytest.approx(Ft, rel=1e-9)
    assert F[1, 1] == pytest.approx(-Ft, rel=1e-9)
    # T = r n x F with n = +x: z-component r * F_y for both particles
    assert T[0, 2] == pytest.approx(r * Ft, rel=1e-9) and T[0, 2] < 0
    assert T[1, 2] == pytest.approx(r * Ft, rel=1e-9)
    assert out["dt"][0] == pytest.approx([0, vt * dt, 0], rel=1e-12)


def test_error_scale_counts_the_terms_of_the_velocity():
    """The parity tolerance's scale S_c: the magnitudes of the terms of
    Eq. (1), with eta v_t counted by the terms of Eq. (vt) (|v| + r1 |w1| +
    r2 |w2|).  A rolling contact: particle 1 translates along +y at u while
    spinning so that its contact point is at rest (v_t = 0): S_c keeps
    eta (u + r |w|), the size of the two cancelling parts."""
    r, dn = 5e-6, 2e-8
    L, dt = 1e-3, 1e-9
    u = 1e-3
    w = u / r
    x = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2 * r - dn, L / 2, L / 2]])
    v = np.array([[0, u, 0], [0, 0, 0]], dtype=float)
    # contact point of 1 (at +x r) moves with v + w x (r, 0, 0); w along +z
    # gives +y r w, so spin -z cancels the translation
    om = np.array([[0, 0, -w], [0, 0, 0]], dtype=float)
    s = O.State(x, v, om, np.array([r, r]))
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), r_max=r, mu_d=10.0)
    out = O.step(p, s)
    info = out["info"][0]
    kn = hertz_kn(r / 2)
    eta = O.alpha(0.5) * math.sqrt(mass(r) / 2 * kn * math.sqrt(dn))
    assert np.allclose(out["dt"][0], 0.0, atol=1e-25)  # the contact point does not slip
    expect = kn * dn ** 1.5 + eta * (u + r * w)       # v_n = 0, delta_t = 0
    assert info["scale"] == pytest.approx(expect, rel=1e-12)


def test_coulomb_cap_resets_history():
    """With a tiny mu the cap fires: |F_t| = mu |F_n| and k_t delta_t = -F_t."""
    r, dn, w = 5e-6, 2e-8, 1e3
    L, dt = 1e-3, 1e-9
    x = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2 * r - dn, L / 2, L / 2]])
    om = np.array([[0, 0, w], [0, 0, 0]], dtype=float)
    s = O.State(x, np.zeros((2, 3)), om, np.array([r, r]))
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), r_max=r, mu_d=1e-3)
    out = O.step(p, s)
    info = out["info"][0]
    n = info["n"]
    Fc = info["F"]
    Fn = np.dot(Fc, n) * n
    Ft = Fc - Fn
    assert info["capped"] == 1
    assert np.linalg.norm(Ft) == pytest.approx(1e-3 * np.linalg.norm(Fn), rel=1e-12)
    assert np.allclose(info["kt"] * out["dt"][0], -Ft, rtol=1e-12, atol=0)


# --------------------------------------------------------------------------
# sphere on the floor: sliding turns into rolling at 5/7 of the launch speed
# --------------------------------------------------------------------------
def test_sliding_to_rolling_on_floor():
    r, u0, mu, g = 5e-6, 1e-3, 0.3, 9.81
    m = mass(r)
    kn = hertz_kn(r)                   # wall: R* -> r
    d_eq = (m * g / kn) ** (2.0 / 3.0)
    k_lin = 1.5 * kn * math.sqrt(d_eq)
    kt = 8.0 * math.sqrt(r * d_eq) * G_STAR
    dt = min(2 * math.pi * math.sqrt(m / k_lin),
             2 * math.pi * math.sqrt(m / (3.5 * kt))) / 50.0
    L = 1e-3
    x = np.array([[L / 2, L / 2, r - d_eq]])
    s = O.State(x, np.array([[u0, 0.0, 0.0]]), np.zeros((1, 3)), np.array([r]),
                floor_wall=True)
    p = O.make_params((L, L, L), dt, periodic=(1, 1, 0), floor_wall=1,
                      g=(0, 0, -g), mu_d=mu, restitution=0.5, r_max=r)
    t_roll = 2 * u0 / (7 * mu * g)
    t, t_hit = 0.0, None
    while t < 2.0 * t_roll:
        O.step(p, s)
        t += dt
        slip = s.v[0, 0] - r * s.w[0, 1]
        if t_hit is None and slip < 1e-3 * u0:
            t_hit = t
    assert t_hit is not None
    assert abs(t_hit - t_roll) < 0.03 * t_roll
    assert s.v[0, 0] == pytest.approx(5.0 / 7.0 * u0, rel=5e-3)
    assert s.w[0, 1] == pytest.approx(5.0 / 7.0 * u0 / r, rel=5e-3)


# --------------------------------------------------------------------------
# invariants on a dense box
# --------------------------------------------------------------------------
def _total_momentum(s):
    m = RHO * 4.0 / 3.0 * math.pi * s.r ** 3
    return (m[:, None] * s.v).sum(0), (m[:, None] * np.abs(s.v)).sum()


def test_momentum_conserved(dense_box):
    b = dense_box
    s = O.State(b.x, b.v, b.w, b.r)
    p = O.make_params(b.L, b.dt, r_max=b.r_max)
    P0, scale = _total_momentum(s)
    for _ in range(10):
        O.step(p, s)
    P1, _ = _total_momentum(s)
    assert np.all(np.abs(P1 - P0) < 1e-13 * scale)


def test_coulomb_inequality_every_contact(dense_box):
    b = dense_box
    s = O.State(b.x, b.v, b.w, b.r)
    p = O.make_params(b.L, b.dt, r_max=b.r_max, mu_d=0.1)
    capped = 0
    for _ in range(5):
        out = O.step(p, s)
        info = out["info"]
        n = info["n"]
        F = info["F"]
        Fn = (F * n).sum(1)[:, None] * n
        Ft = F - Fn
        nFt = np.linalg.norm(Ft, axis=1)
        nFn = np.linalg.norm(Fn, axis=1)
        # tolerance covers re-deriving F_t = F - (F.n) n from the total force
        assert np.all(nFt <= 0.1 * nFn * (1 + 1e-9) + 1e-300)
        c = info["capped"] == 1
        capped += int(c.sum())
        kd = np.linalg.norm(info["kt"][:, None] * out["dt"], axis=1)
        assert np.allclose(kd[c], 0.1 * nFn[c], rtol=1e-9)
    assert capped > 0


def _energy(s, p, info):
    m = RHO * 4.0 / 3.0 * math.pi * s.r ** 3
    I = 0.4 * m * s.r ** 2
    ke = 0.5 * (m * (s.v ** 2).sum(1)).sum() + 0.5 * (I * (s.w ** 2).sum(1)).sum()
    return ke


def test_elastic_frictionless_energy_conserved():
    """eps = 1, mu = 0: only the Hertz spring acts; kinetic plus elastic
    energy 2/5 k_n delta^{5/2} stays constant to O(dt^2)."""
    b = synth.w1_monodisperse(n=400, seed=13)
    s = O.State(b.x, b.v, b.w, b.r)
    p = O.make_params(b.L, b.dt / 5, r_max=b.r_max, restitution=1.0, mu_d=0.0)
    kn = hertz_kn(b.r[0] / 2)
    m = RHO * 4.0 / 3.0 * math.pi * s.r ** 3

    def total(s):
        lo, hi = O.contacts(p, s.x, s.r)
        d = s.x[hi] - s.x[lo]
        L = np.asarray(b.L)
        d -= L * np.round(d / L)
        dn = s.r[lo] + s.r[hi] - np.linalg.norm(d, axis=1)
        return 0.5 * (m * (s.v ** 2).sum(1)).sum() + (0.4 * kn * dn ** 2.5).sum()

    E0 = total(s)
    worst = 0.0
    for _ in range(300):
        O.step(p, s)
        worst = max(worst, abs(total(s) - E0) / E0)
    assert worst < 2e-3


def test_damping_dissipates(dense_box):
    """eps < 1, mu = 0: kinetic plus Hertz elastic energy decreases."""
    b = dense_box
    s = O.State(b.x, b.v, b.w, b.r)
    p = O.make_params(b.L, b.dt, r_max=b.r_max, restitution=0.3, mu_d=0.0)
    m = RHO * 4.0 / 3.0 * math.pi * s.r ** 3
    L = np.asarray(b.L)

    def total():
        lo, hi = O.contacts(p, s.x, s.r)
        d = s.x[hi] - s.x[lo]
        d -= L * np.round(d / L)
        dn = s.r[lo] + s.r[hi] - np.linalg.norm(d, axis=1)
        Rs = s.r[lo] * s.r[hi] / (s.r[lo] + s.r[hi])
        kn = 4.0 / 3.0 * E_STAR * np.sqrt(Rs)
        return 0.5 * (m * (s.v ** 2).sum(1)).sum() + (0.4 * kn * dn ** 2.5).sum()

    e0 = total()
    prev = e0
    for _ in range(40):
        O.step(p, s)
        e = total()
        assert e < prev * (1 + 1e-4)
        prev = e
    assert prev < 0.999 * e0


def test_history_erased_when_pair_separates():
    """Two spheres brushing past each other: delta_t is carried while in
    contact and the pair disappears from the list after separation."""
    r = 5e-6
    L = 1e-3
    dt = 2e-9
    x = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2 * r - 1e-8, L / 2 - 3 * r, L / 2]])
    v = np.array([[0, 0, 0], [0, 1.0, 0]], dtype=float)
    s = O.State(x, v, np.zeros((2, 3)), np.array([r, r]))
    p = O.make_params((L, L, L), dt, periodic=(0, 0, 0), r_max=r, mu_d=10.0)
    seen = False
    for _ in range(20000):
        out = O.step(p, s)
        if len(out["lo"]):
            seen = True
            assert np.linalg.norm(out["dt"][0]) > 0
        elif seen:
            break
    assert seen and len(s.lo) == 0


def test_history_projection_drops_normal_part():
    """Eq. (dt): the normal part of delta_t,old is removed before use.  Two
    spheres at rest along x with stored history (a, b, 0): the new history is
    (0, b, 0) and the tangential force is -k_t (0, b, 0)."""
    r, dn = 5e-6, 2e-8
    L = 1e-3
    x = np.array([[L / 2, L / 2, L / 2], [L / 2 + 2 * r - dn, L / 2, L / 2]])
    s = O.State(x, np.zeros((2, 3)), np.zeros((2, 3)), np.array([r, r]))
    a, bb = 3e-9, 2e-9
    s.lo = np.array([0], np.int32)
    s.hi = np.array([1], np.int32)
    s.dt = np.array([[a, bb, 0.0]])
    p = O.make_params((L, L, L), 1e-12, periodic=(0, 0, 0), r_max=r, mu_d=10.0)
    out = O.step(p, s)
    kt = 8.0 * math.sqrt(r / 2 * dn) * G_STAR
    assert out["dt"][0] == pytest.approx([0.0, bb, 0.0], abs=1e-24)
    assert out["F"][0, 1] == pytest.approx(-kt * bb, rel=1e-9)
    assert out["F"][0, 0] == pytest.approx(-hertz_kn(r / 2) * dn ** 1.5, rel=1e-9)
