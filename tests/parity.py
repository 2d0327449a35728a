"""Parity harness: one step of the CUDA library against the FP64 oracle.

Both sides start from the same seeded state in the library's storage
representation (``synth.prepared``): positions quantised to the 2^-60 m
fixed point (DEM_MIXED) or rounded to float32 (DEM_FP32), velocities and
angular velocities rounded to float32 in both of those modes, radii float32
values already; both sides use the same explicit cell grid, so the contact
predicate and the sort order can be compared bit for bit.

Two force tolerances are checked per contact c (oracle values):

  relative to the force (the stated criterion):
    |F_gpu - F_ora|  <= rtol |F_ora| + f_c
    |nF_gpu - nF_ora| <= rtol |F_ora| + f_c
  relative to the terms of Eq. (1) (a float sum's error is bounded by its
  terms, not by its result):
    |F_gpu - F_ora|  <= rtol S_c + f_c
    |nF_gpu - nF_ora| <= rtol S_c + f_c + 1e-6 |F_ora|
  S_c = k_n dn^1.5 + eta |v_n| + k_t |delta_t| + eta (|v| + r1 |w1| + r2 |w2|)
        (the magnitudes of the terms of Eq. (1), with v_t counted by the
        terms of Eq. (vt))
  f_c = 1e-9 k_n R*^1.5  (absolute floor)

with rtol = 1e-5 for FP32 force arithmetic and 1e-9 for FP64.  Both bounds
are asserted on every contact.  The contacts whose condition number
kappa_c = S_c / |F_ora| exceeds KAPPA_MAX are counted and reported: there the
terms of Eq. (1) cancel (a rolling contact, whose translational and
rotational parts of v_t nearly cancel, or a force near zero at the end of a
contact), an error of a few units of FP32 rounding in each term can exceed
rtol |F|, and a one-ulp change of the FP32 inputs can move the FP64
oracle's own force by as much (``oracle_sensitivity``,
``conditioning_report``).

Contacts whose Coulomb ratio lies within 1e-4 of 1 may be capped on one side
only, and contacts with an overlap below 1e-15 R* / rtol are below what an
FP64 overlap resolves to rtol in the damping force (eta ~ dn^{1/4}); both
kinds are counted and reported, not compared.  Per particle the bounds add up
over its contacts.
"""
from __future__ import annotations

import math

import numpy as np

import oracle as O
from paper_1503_03553_gb300.synth import grid_for, prepared, quantize  # noqa: F401

RTOL = {"mixed": 1e-5, "fp32": 1e-5, "fp64": 1e-9}
PRED = {"mixed": O.PRED_FIXED_F32, "fp64": O.PRED_FP64, "fp32": O.PRED_ABS_F32}
# contacts with S_c / |F| above this are ill-conditioned in FP32 (see above)
KAPPA_MAX = 10.0

STENCIL = 1  # neighbour cells per axis (+-1): cells of at least 2 r_max


def oracle_params(box, precision, ncell, brute_force=0, stencil=STENCIL):
    return O.make_params(box.L, box.dt, E=box.E, poisson=box.poisson,
                         density=box.density, restitution=box.restitution,
                         mu_d=box.mu_d, periodic=box.periodic,
                         floor_wall=box.floor_wall, g=box.g, ncell=ncell,
                         predicate=PRED[precision], brute_force=brute_force,
                         stencil=stencil, walls=getattr(box, "walls", ()))


def gpu_run(boxes, precision, ncells, steps=1, stencil=STENCIL, **kw):
    """Create a context for ``boxes``, set particles, run ``steps`` steps
    and collect everything per box (and the re-sort statistics under
    "resorts")."""
    import paper_1503_03553_gb300 as D

    assert stencil == 1, "the library searches +-1 neighbour cells"
    ctx = D.Context(boxes, precision=precision, ncell=ncells, **kw)
    try:
        for k, b in enumerate(boxes):
            ctx.set_particles(k, b.x, b.v, b.w, b.r)
        ctx.step(steps)
        out = []
        for k in range(len(boxes)):
            st = ctx.get_state(k)
            lo, hi, dt = ctx.contacts(k)
            flo, fhi, F, nF = ctx.contact_forces(k)
            order, cells = ctx.order(k)
            out.append(dict(state=st, lo=lo, hi=hi, dt=dt, flo=flo, fhi=fhi, Fc=F,
                            nFc=nF, order=order, cells=cells, stats=ctx.stats(k),
                            resorts=ctx.resort_stats()))
        return out
    finally:
        ctx.close()


def oracle_run(box, precision, ncell, stencil=STENCIL, hist=None, parallel=False):
    """One oracle step from box's state; hist = (id_lo, id_hi, delta_t) is
    the contact history to start from (none: a fresh start); parallel=True
    runs the oracle's OpenMP build (the same results, bit for bit)."""
    p = oracle_params(box, precision, ncell, stencil=stencil)
    cell, order = O.order(p, box.x)
    s = O.State(box.x, box.v, box.w, box.r, floor_wall=bool(box.floor_wall),
                nwalls=len(getattr(box, "walls", ())))
    if hist is not None:
        s.lo, s.hi, s.dt = hist
    x0, v0, w0 = s.x.copy(), s.v.copy(), s.w.copy()
    out = O.step(p, s, parallel=parallel)
    out.update(order=order, cell=cell, x=s.x, v=s.v, w=s.w, x0=x0, v0=v0, w0=w0,
               params=p)
    if hist is not None:
        out["hist"] = hist
    return out


def _contact_bounds(box, o, rtol):
    info = o["info"]
    lo, hi = o["lo"], o["hi"]
    r = box.r
    Rs = r[lo] * r[hi] / (r[lo] + r[hi])
    kn_c = O.kn(o["params"], 1.0, 1.0) / math.sqrt(0.5)
    kn = kn_c * np.sqrt(Rs)
    floor = 1e-9 * kn * Rs ** 1.5
    bF = rtol * info["scale"] + floor
    return bF, floor


def _explain(box, g, o, idx):
    """Human-readable detail of selected contacts (for failure messages)."""
    info = o["info"]
    lines = []
    for k in idx:
        i, j = int(o["lo"][k]), int(o["hi"][k])
        lines.append(
            f"  c={k} ({i},{j}) r=({box.r[i]:.4g},{box.r[j]:.4g}) dn={info['delta_n'][k]:.6g} "
            f"scale={info['scale'][k]:.4g} ratio={info['ratio'][k]:.6g} capped={info['capped'][k]} "
            f"kt={info['kt'][k]:.4g}\n    F_ora={info['F'][k]} F_gpu={g['Fc'][k]}\n"
            f"    dt_ora={o['dt'][k]} dt_gpu={g['dt'][k]}\n"
            f"    x_i={o['x0'][i]} x_j={o['x0'][j]} v_i={o['v0'][i]} v_j={o['v0'][j]}")
    return "\n".join(lines)


def _wall_bounds(box, o, mass, rtol):
    """Per particle: rtol |F_wall| + 1e-9 k_n r^1.5 (k_n with R* = r), where
    F_wall is the oracle's total force less its pair contacts' forces and
    gravity (zero for a particle touching no wall, up to round-off)."""
    info = o["info"]
    Fp = np.zeros((box.n, 3))
    if len(o["lo"]):
        np.add.at(Fp, o["lo"], info["F"])
        np.add.at(Fp, o["hi"], -info["F"])
    Fw = o["F"] - Fp - mass[:, None] * np.asarray(box.g, float)[None, :]
    kn_c = O.kn(o["params"], 1.0, 1.0) / math.sqrt(0.5)
    return rtol * np.linalg.norm(Fw, axis=1) + 1e-9 * kn_c * box.r ** 2


def _explain_particles(box, g, o, idx, eP, bP):
    """Human-readable detail of selected particles (for failure messages)."""
    lines = []
    for i in idx:
        i = int(i)
        nc = int(np.sum(o["lo"] == i) + np.sum(o["hi"] == i))
        lines.append(f"  particle {i}: err {eP[i]:.4g} bound {bP[i]:.4g} contacts {nc} "
                     f"F_ora={o['F'][i]} F_gpu={g['state']['F'][i]} r={box.r[i]:.4g} "
                     f"x={o['x0'][i]}")
    return "\n".join(lines)


def check_one_step(box, g, o, precision, allow_dont_care=True, check_order=True):
    """Compare one step; returns a metrics dict, raises AssertionError.
    check_order=False skips the sort order and cells (a step of the
    candidate-list pipeline that did not re-sort keeps the order of the
    last re-sort)."""
    rtol = RTOL[precision]
    m = {}
    # 1. sort order and contact set: bit-exact
    if check_order:
        assert np.array_equal(g["order"], o["order"]), "sort order differs"
        assert np.array_equal(g["cells"], o["cell"][o["order"]]), "cells differ"
    assert np.array_equal(g["lo"], o["lo"]) and np.array_equal(g["hi"], o["hi"]), (
        f"contact sets differ: gpu {len(g['lo'])} oracle {len(o['lo'])}")
    assert np.array_equal(g["flo"], o["lo"]) and np.array_equal(g["fhi"], o["hi"])
    nc = len(o["lo"])
    m["contacts"] = nc
    info = o["info"]
    bF, floor = _contact_bounds(box, o, rtol)
    # "don't care": a Coulomb ratio within 1e-4 of 1 (cap may fire on one
    # side only), or an overlap below 1e-15 R* / rtol: an FP64 overlap
    # carries ~4e-16 R of rounding and eta ~ dn^{1/4} turns that into more
    # than rtol of force below this size (1e-10 R* at rtol 1e-5)
    r = box.r
    Rs_all = r[o["lo"]] * r[o["hi"]] / (r[o["lo"]] + r[o["hi"]]) if nc else np.zeros(0)
    tiny = info["delta_n"] < (1e-15 / rtol) * Rs_all
    dont = ((np.abs(info["ratio"] - 1.0) < 1e-4) | tiny) if allow_dont_care else np.zeros(nc, bool)
    m["tiny_overlap"] = int(tiny.sum())
    m["dont_care"] = int(dont.sum())
    ok = ~dont
    eF = np.linalg.norm(g["Fc"] - info["F"], axis=1)
    enF = np.linalg.norm(g["nFc"] - info["nF"], axis=1)
    normF = np.linalg.norm(info["F"], axis=1)
    if nc:
        m["max_F_err_over_scale"] = float(np.max((eF / (info["scale"] + floor))[ok], initial=0))
        rel = eF / np.maximum(normF, 1e-300)
        m["p99_F_rel_err"] = float(np.percentile(rel[ok & (normF > 0)], 99)) if np.any(ok & (normF > 0)) else 0.0
        bad = ok & (eF > bF)
        assert not np.any(bad), (
            f"{int(bad.sum())} contact forces outside tolerance; worst "
            f"{float(np.max((eF / bF)[ok])):.3g} x bound\n" + _explain(box, g, o, np.where(bad)[0][:6]))
        bad = ok & (enF > bF + 1e-6 * normF)
        assert not np.any(bad), f"{int(bad.sum())} n x F outside tolerance"
        # the force-relative criterion: every well-conditioned contact
        kappa = info["scale"] / np.maximum(normF, 1e-300)
        well = ok & (kappa <= KAPPA_MAX)
        bN = rtol * normF + floor
        over = ok & (eF > bN)
        m["F_rel_max"] = float(np.max((eF / np.maximum(normF, 1e-300))[ok], initial=0))
        m["F_rel_p99"] = float(np.percentile((eF / np.maximum(normF, 1e-300))[ok], 99)) if ok.any() else 0.0
        m["F_rel_bound_max"] = float(np.max((eF / bN)[ok], initial=0))
        m["F_rel_bound_exceeded"] = int(over.sum())
        m["ill_conditioned"] = int((ok & ~well).sum())
        if precision != "fp32":
            bad = ok & (eF > bN)
            assert not np.any(bad), (
                f"{int(bad.sum())} contacts outside rtol |F| + floor ({int((bad & well).sum())} of "
                f"them well-conditioned); worst {float(np.max((eF / bN)[ok])):.3g} x bound\n"
                + _explain(box, g, o, np.where(bad)[0][:6]))
            bad = ok & (enF > bN)
            assert not np.any(bad), f"{int(bad.sum())} n x F outside rtol |F| + floor"
        # tangential history after the step
        lo, hi = o["lo"], o["hi"]
        v0, w0, r = o["v0"], o["w0"], box.r
        vscale = (np.linalg.norm(v0[lo], axis=1) + np.linalg.norm(v0[hi], axis=1)
                  + r[lo] * np.linalg.norm(w0[lo], axis=1) + r[hi] * np.linalg.norm(w0[hi], axis=1))
        kt = np.where(info["kt"] > 0, info["kt"], np.inf)
        bdt = rtol * (np.linalg.norm(o["dt"], axis=1) + box.dt * vscale + info["scale"] / kt) + 1e-30
        edt = np.linalg.norm(g["dt"] - o["dt"], axis=1)
        bad = ok & (edt > bdt)
        assert not np.any(bad), f"{int(bad.sum())} delta_t outside tolerance"
        m["max_dt_err_over_bound"] = float(np.max((edt / bdt)[ok], initial=0))
    # 2. per-particle totals
    n = box.n
    bP = np.zeros(n)
    np.add.at(bP, o["lo"], bF)
    np.add.at(bP, o["hi"], bF)
    mass = box.density * 4.0 / 3.0 * math.pi * box.r ** 3
    gmag = float(np.linalg.norm(box.g))
    bP += 1e-6 * mass * gmag + 1e-300
    walled = bool(box.floor_wall or len(getattr(box, "walls", ())))
    if walled:
        # the wall contacts of a particle, bounded like a particle contact:
        # rtol times their force plus the floor 1e-9 k_n R*^1.5 (R* = r);
        # their force is the oracle's total less its pair contacts and m g
        bW = _wall_bounds(box, o, mass, rtol)
        bP += bW + 1e-5 * np.linalg.norm(o["F"], axis=1) + 1e-5 * mass * gmag
    if dont.any():
        np.add.at(bP, o["lo"][dont], np.inf)
        np.add.at(bP, o["hi"][dont], np.inf)
    eP = np.linalg.norm(g["state"]["F"] - o["F"], axis=1)
    assert np.all(eP <= bP), (f"{int((eP > bP).sum())} particle forces outside tolerance\n"
                              + _explain_particles(box, g, o, np.where(eP > bP)[0][:4], eP, bP))
    if nc:
        # force-relative per particle: rtol times the sum of its contacts'
        # |F| plus their floors, for particles whose contacts are all
        # well-conditioned (the net force of a dense packing cancels, so the
        # scale is the sum of the magnitudes, not the net force)
        sF = np.zeros(n)
        np.add.at(sF, o["lo"], rtol * normF + floor)
        np.add.at(sF, o["hi"], rtol * normF + floor)
        sF += 1e-6 * mass * gmag + 1e-300
        if walled:
            sF += bW + 1e-5 * np.linalg.norm(o["F"], axis=1) + 1e-5 * mass * gmag
        cold = np.zeros(n, bool)
        notwell = ok & (kappa > KAPPA_MAX)
        cold[o["lo"][notwell]] = True
        cold[o["hi"][notwell]] = True
        dpart = np.zeros(n, bool)  # particles with a "don't care" contact
        dpart[o["lo"][dont]] = True
        dpart[o["hi"][dont]] = True
        m["particle_F_rel_bound_max"] = float(np.max((eP / sF)[~dpart], initial=0))
        m["particles_with_ill_conditioned_contacts"] = int(cold.sum())
        if precision != "fp32":
            assert np.all(eP[~dpart] <= sF[~dpart]), (
                f"{int((eP[~dpart] > sF[~dpart]).sum())} particle forces outside rtol sum|F| + floors")
    eT = np.linalg.norm(g["state"]["T"] - o["T"], axis=1)
    assert np.all(eT <= box.r * (bP + 1e-6 * np.linalg.norm(o["F"], axis=1)) * 2 + 1e-300), "torques"
    m["max_particle_F_err_over_bound"] = float(np.max(eP / bP))
    # 3. state after the step
    vs = np.linalg.norm(o["v"], axis=1) + box.dt / mass * bP
    ev = np.linalg.norm(g["state"]["v"] - o["v"], axis=1)
    vtol = (1e-6 if precision != "fp64" else 1e-12) * vs + box.dt / mass * bP
    assert np.all(ev <= vtol * 1.0001 + 1e-30), "velocities after the step"
    dx = g["state"]["x"] - o["x"]
    L = np.asarray(box.L)
    per = np.asarray(box.periodic, bool)
    dx = np.where(per, dx - L * np.round(dx / L), dx)
    ex = np.linalg.norm(dx, axis=1)
    xtol = box.dt * vtol * 2 + (1e-6 if precision == "fp32" else 0) * np.max(L) + 4 * 2.0 ** -60 + 1e-19
    assert np.all(ex <= xtol), f"positions after the step, worst {float(np.max(ex / xtol)):.3g}"
    return m


def force_errors(box, g, o, precision, detail=0):
    """Error statistics of one step against the oracle (no assertion):
    per contact |F_gpu - F_ora| / (S_c + f_c) with the term scale and floor,
    over the contacts both sides found (the sets must be equal).  detail > 0
    adds the `detail` worst contacts outside the "don't care" classes, each
    with its error split along and across the normal, overlap over R*,
    Coulomb ratio, cap flag, |F| and k_t |delta_t| over the scale, and the
    error of the delta_t after the step (when g has "dt")."""
    same = (len(g["lo"]) == len(o["lo"]) and np.array_equal(g["lo"], o["lo"])
            and np.array_equal(g["hi"], o["hi"]))
    if not same:
        return {"contact_sets_equal": False, "gpu_contacts": int(len(g["lo"])),
                "oracle_contacts": int(len(o["lo"]))}
    info = o["info"]
    if len(o["lo"]) == 0:
        return {"contact_sets_equal": True, "contacts": 0}
    _, floor = _contact_bounds(box, o, 1e-5)
    e = np.linalg.norm(g["Fc"] - info["F"], axis=1) / (info["scale"] + floor)
    nF = np.linalg.norm(info["F"], axis=1)
    rel = np.linalg.norm(g["Fc"] - info["F"], axis=1) / np.maximum(nF, 1e-300)
    ok = nF > 0
    # the "don't care" contacts of check_one_step (Coulomb ratio within 1e-4
    # of 1, or an overlap below 1e-15 R* / rtol), here at rtol 1e-5
    r = box.r
    Rs = r[o["lo"]] * r[o["hi"]] / (r[o["lo"]] + r[o["hi"]])
    dont = (np.abs(info["ratio"] - 1.0) < 1e-4) | (info["delta_n"] < 1e-10 * Rs)
    keep = ~dont
    worst = []
    if detail and keep.any():
        dF = g["Fc"] - info["F"]
        nrm = info["n"]
        en = np.abs(np.sum(dF * nrm, axis=1))
        et = np.linalg.norm(dF - np.sum(dF * nrm, axis=1)[:, None] * nrm, axis=1)
        den = info["scale"] + floor
        idx = np.flatnonzero(keep)
        idx = idx[np.argsort(-e[idx])][:detail]
        for k in idx:
            w = {"err": float(e[k]), "err_normal": float(en[k] / den[k]),
                 "err_tangential": float(et[k] / den[k]),
                 "dn_over_Rstar": float(info["delta_n"][k] / Rs[k]),
                 "ratio": float(info["ratio"][k]), "capped": int(info["capped"][k]),
                 "F_over_scale": float(nF[k] / info["scale"][k]),
                 "kt_dt_over_scale": float(info["kt"][k] * np.linalg.norm(o["dt"][k]) / info["scale"][k])}
            if "dt" in g:
                w["dt_err_rel"] = float(np.linalg.norm(g["dt"][k] - o["dt"][k]) /
                                        max(np.linalg.norm(o["dt"][k]), 1e-300))
            worst.append(w)
    fl = floor
    bN = 1e-5 * nF + fl
    eabs = np.linalg.norm(g["Fc"] - info["F"], axis=1)
    kappa = info["scale"] / np.maximum(nF, 1e-300)
    over = keep & (eabs > bN)
    rel_stats = {
        "F_rel_max": float(rel[keep].max()) if keep.any() else 0.0,
        "F_rel_p99": float(np.percentile(rel[keep], 99)) if keep.any() else 0.0,
        "F_rel_bound_max": float((eabs / bN)[keep].max()) if keep.any() else 0.0,
        "F_rel_bound_exceeded": int(over.sum()),
        "F_rel_bound_exceeded_frac": float(over.sum() / max(1, keep.sum())),
        "F_rel_bound_exceeded_kappa_le_10": int((over & (kappa <= 10.0)).sum()),
        "kappa_of_exceeders_min": float(kappa[over].min()) if over.any() else None,
        "kappa_of_exceeders_median": float(np.median(kappa[over])) if over.any() else None,
    }
    out = {"contact_sets_equal": True, "contacts": int(len(e)),
            "max_err_over_scale": float(e.max()),
            "p99_err_over_scale": float(np.percentile(e, 99)),
            "frac_within_1e-5": float(np.mean(e <= 1e-5)),
            "median_rel_err": float(np.median(rel[ok])) if ok.any() else 0.0,
            "dont_care": int(dont.sum()),
            "max_err_over_scale_cared": float(e[keep].max()) if keep.any() else 0.0,
            "frac_within_1e-5_cared": float(np.mean(e[keep] <= 1e-5)) if keep.any() else 1.0}
    out.update(rel_stats)
    if detail:
        out["worst_cared"] = worst
    return out


def oracle_sensitivity(box, o, precision, ncell, seed=0):
    """How far the FP64 oracle's own contact forces move when its inputs
    change by one FP32 unit: velocities and angular velocities (the FP32
    inputs of DEM_MIXED) scaled by 1 +- 2^-24 with random signs, one oracle
    step from the same positions and history.  Returns per contact
    |F_pert - F_ora| in the order of o["lo"] (the contact set is the same:
    the predicate reads positions only)."""
    rng = np.random.default_rng(seed)
    sgn = lambda a: 1.0 + np.ldexp(rng.choice([-1.0, 1.0], size=a.shape), -24)
    p = oracle_params(box, precision, ncell)
    s = O.State(box.x, box.v * sgn(box.v), box.w * sgn(box.w), box.r,
                floor_wall=bool(box.floor_wall), nwalls=len(getattr(box, "walls", ())))
    if "hist" in o:
        s.lo, s.hi, s.dt = o["hist"]
    out = O.step(p, s)
    assert np.array_equal(out["lo"], o["lo"]) and np.array_equal(out["hi"], o["hi"])
    return np.linalg.norm(out["info"]["F"] - o["info"]["F"], axis=1)


def conditioning_report(box, g, o, precision, ncell):
    """For the contacts outside 1e-5 |F_ora| + floor: their count, their
    condition numbers kappa = S_c / |F_ora|, and the ratio of the library's
    error to the oracle's own movement under a one-ulp FP32 change of its
    inputs (``oracle_sensitivity``)."""
    info = o["info"]
    nc = len(o["lo"])
    if nc == 0:
        return {"contacts": 0}
    _, floor = _contact_bounds(box, o, 1e-5)
    nF = np.linalg.norm(info["F"], axis=1)
    e = np.linalg.norm(g["Fc"] - info["F"], axis=1)
    r = box.r
    Rs = r[o["lo"]] * r[o["hi"]] / (r[o["lo"]] + r[o["hi"]])
    keep = ~((np.abs(info["ratio"] - 1.0) < 1e-4) | (info["delta_n"] < 1e-10 * Rs))
    over = keep & (e > 1e-5 * nF + floor)
    kappa = info["scale"] / np.maximum(nF, 1e-300)
    sens = oracle_sensitivity(box, o, precision, ncell)
    pert_over = keep & (sens > 1e-5 * nF + floor)
    ratio = e[over] / np.maximum(sens[over], 1e-300)
    return {
        "contacts": int(nc), "exceed_rel_1e-5": int(over.sum()),
        "exceed_frac": float(over.sum() / max(1, keep.sum())),
        "exceed_with_kappa_le_10": int((over & (kappa <= 10)).sum()),
        "kappa_exceeders_p10_median": ([float(np.percentile(kappa[over], 10)),
                                        float(np.median(kappa[over]))] if over.any() else None),
        "oracle_moved_beyond_rel_1e-5_by_one_ulp": int(pert_over.sum()),
        "exceeders_also_moved_by_one_ulp": int((over & pert_over).sum()),
        "gpu_err_over_one_ulp_move_median_p90": ([float(np.median(ratio)), float(np.percentile(ratio, 90))]
                                                 if over.any() else None),
    }
