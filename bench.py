"""Throughput of the GB300 DEM step: particle-steps per second.

Workload (default): 1,000,000 polydisperse spheres (lognormal radii, median
4 um, sigma_log 0.25, clipped to [2, 8] um), periodic box at packing 0.55
with overlaps up to 1 % of the smaller radius, v ~ N(0, 0.05 m/s),
w ~ N(0, 1e3 rad/s), material E = 3 GPa, Poisson 0.3, 1200 kg/m^3,
restitution 0.5, mu_D 0.3, dt = 1 ns.  One step = sort, contact search,
contact list, force, sum + integrate (all kernels of the library).

Prints one JSON line.  `value` is device-timed (CUDA events on the
library's stream) with the state resident in HBM; `e2e` runs the same steps
through the C ABI with host buffers (state in from pinned memory, state out
to pinned memory every step).  `--impl reference` times the FP64 CPU oracle
on the host cores instead (a periodic sub-box of the same workload).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       multi-GPU: python -m torch.distributed.run --nproc-per-node N bench.py --gpus N
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"  # the unit
# the headline metric: MIXED (FP32 force arithmetic) and FP64 forms at 1M
# particles within the 1e-5 force tolerance, batched boxes against one box
# at a time (the comparison legs under "compare")
METRIC_NAME = ("particle-steps/s @1M: FP32 vs FP64 GPU at force rel err\u22641e-5; "
               "batched vs 1-by-1")
L2_BYTES = 126.5 * 2 ** 20
# the candidate-list skin of the other workloads' legs (W3, W4, W5 and the
# tuner's starting layout), as a fraction of each box's largest radius
OTHER_SKIN_OVER_RMAX = 0.025


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_000_000)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64", "fp32"])
    ap.add_argument("--skin-um", type=float, default=0.04,
                    help="candidate-list skin in micrometres (0: search every step); "
                         "the default, 0.5 %% of the largest radius, is the layout "
                         "tuner's choice on this workload (its leg reports it)")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP64-GPU, parity and CPU-baseline side legs")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--no-batched", action="store_true", help="skip the W4 batched leg")
    ap.add_argument("--nboxes", type=int, default=512)
    ap.add_argument("--batched-steps", type=int, default=100)
    ap.add_argument("--w3", action="store_true",
                    help="add the 8M-particle floor/gravity leg (dense + dilute halves)")
    ap.add_argument("--w5", action="store_true",
                    help="add the W5 precision-stress leg (4 M spheres at packing 0.60, "
                         "10,000 steps of each form, oracle snapshots every 1,000 steps)")
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the particle-count sweep of the W2 workload (0.1 to 8 M)")
    ap.add_argument("--w5-n", type=int, default=4_000_000)
    ap.add_argument("--w5-steps", type=int, default=10_000)
    ap.add_argument("--w5-every", type=int, default=1_000)
    ap.add_argument("--w5-forms", default="mixed,fp32,fp64",
                    help="precision forms of the W5 leg, comma-separated")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index),
                                      f"--query-gpu={self.FIELDS}",
                                      "--format=csv,noheader,nounits"],
                                     capture_output=True, text=True, timeout=5).stdout
                for line in out.strip().splitlines():
                    self.rows.append([c.strip() for c in line.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic traffic model (bytes per particle-step, DEM_MIXED layout)
# ---------------------------------------------------------------------------
def phase_bytes(n, c_half, cand_half, ncells, resorts_per_step):
    """Unique bytes each phase must move, per step (DEM_MIXED layout): every
    array element read or written once; re-reads of neighbours' data served
    by the caches are not counted.  n particles, c_half contacts and
    cand_half candidate pairs per particle (each pair counted once), ncells
    cells.  The re-sort phases (sort, search, rows) run only in the steps
    that re-sort: their bytes are scaled by resorts_per_step."""
    C = c_half * n            # pairs in contact
    Cc = cand_half * n        # candidate pairs
    state = 24 + 16 + 16 + 16 + 4 + 4 + 4 + 4   # x, v, w, predicate record, id, cells
    sort = (ncells * (4 + 4 + 8 + 1 + 1 + 32)        # cell scan, ranges, flags, box reset
            + n * (4 + 4 + 4 + 1)                    # scatter
            + n * (4 + 4 + 2 * state + 4)            # reorder (state, previous slot)
            + ncells * 32)                           # cell bounding boxes
    search = (n * (16 + 4 + 4 + 4 + 4) + ncells * (8 + 32)
              + Cc * (4 + 8 + 8 + 8 + 4))            # rows, list pairs and ids, incoming rows
    rows = (n * (4 + 4 + 4 + 4)                      # blocks, incoming counts, previous slots
            + Cc * (8 + 8 + 2 * 4 + 8 + 8)           # pairs, incoming rows, row entries, old lists
            + C * (24 + 1)                           # history carried over
            + Cc * 2 * (8 + 8 + 24 + 1)              # commit of the list
            + n * (2 * state + 24))                  # commit of the state, positions of the sort
    pairs = (Cc * (8 + 1)                                 # list pairs and contact flags
             + n * (16 + 4 + 24 + 16 + 16)                # record, cell, x, v, w of the particles
             + C * (24 + 24 + 1 + 16 + 16))               # history in and out, flag, F, n x F
    sum_ = (n * (4 + 4 * 2 * cand_half)                   # row lengths and entries
            + 2 * Cc * 1                                  # contact flags of the row entries
            + C * (16 + 16)                               # F and n x F of each contact
            + n * (24 + 16 + 16 + 4 + 24 + 4)             # x, v, w, cell, skin test, rank cell
            + n * (24 + 16 + 16 + 16 + 4))                # x, v, w, record, cell written
    f = resorts_per_step
    return {"sort": sort * f, "search": search * f, "rows": rows * f, "pairs": pairs,
            "sum": sum_}


PHASES = ["sort", "search", "rows", "pairs", "sum"]
PHASE_KERNEL = {"pairs": "k_pairs", "sum": "k_gather_integrate"}


def _torch_setup(args):
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return torch, rank, world, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def combine_ranks(x, world):
    """Largest value over ranks (the timed region ends when the slowest rank
    ends).  Works on NCCL (GPU tensor) and gloo (CPU tensor) groups."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank, world, steps, secs):
    """Whole-job particle-steps/s: every rank advances its own replica."""
    return n_per_rank * world * steps / secs


def _max_over_ranks(x, world, torch):
    return combine_ranks(x, world)


def _workload(n, seed):
    from paper_1503_03553_gb300 import synth
    box = synth.w2_polydisperse(n=n, seed=seed)
    # the state in the library's storage representation (fixed-point
    # positions, float32 velocities) so that the parity leg and the oracle
    # see bit-identical inputs
    return box, synth.prepared(box, "mixed")


def _time_steps(ctx, torch, steps, world):
    s = ctx.stream
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _barrier(world)
    torch.cuda.synchronize()
    e0.record(s)
    ctx.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    _barrier(world)
    return e0.elapsed_time(e1) / 1e3


def _cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo), for the record."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return None


def _w2_construction(n):
    """How the W2 box of n particles is built (synth.w2_polydisperse)."""
    from paper_1503_03553_gb300 import synth
    k, n0 = synth.tiling(n)
    law = "radii log-normal (median 4 um, log-sd 0.25, clipped to 2-8 um)"
    if k == 1:
        return f"one relaxed tile of {n0} spheres, {law}"
    return (f"{k}^3 copies of one relaxed tile of {n0} spheres, {law}; "
            "particle ids in random order")


def _oracle_threads():
    return int(os.environ.get("OMP_NUM_THREADS") or os.cpu_count() or 1)


def _oracle_rate(box, seconds, max_steps=3, parallel=False, min_steps=1):
    """Time the FP64 oracle on this machine: steps 1..k from the box's state,
    k between min_steps and max_steps, stopping once `seconds` have passed.
    parallel=True runs its OpenMP build on all host cores.
    Returns (particle-steps/s, steps, seconds)."""
    import oracle as O
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import oracle_params
    from paper_1503_03553_gb300.synth import grid_for
    p = oracle_params(box, "mixed", grid_for(box))
    O.alpha(box.restitution)  # restitution solve outside the timed region
    O.lib(parallel)           # library load outside the timed region
    s = O.State(box.x, box.v, box.w, box.r)
    t0 = time.perf_counter()
    k = 0
    while True:
        O.step(p, s, parallel=parallel)
        k += 1
        dt = time.perf_counter() - t0
        if k >= max_steps or (k >= min_steps and dt >= seconds):
            break
    return box.n * k / dt, k, dt


def run_reference(args):
    """The FP64 CPU oracle as the reference arm, on all host cores (its
    OpenMP build: the serial oracle's results bit for bit), on the GPU arm's
    workload: the same W2 box of args.n particles, steps 1..K from its initial
    state after W warm-up steps.  When W + K steps of the full box would not
    end within about three minutes, each step is a sample: a periodic box of
    the same law (8,000-particle relaxed tiles) sized to fit."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    from paper_1503_03553_gb300 import synth
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import oracle_params
    from paper_1503_03553_gb300.synth import grid_for, prepared
    threads = _oracle_threads()
    full = prepared(synth.w2_polydisperse(n=args.n, seed=2), "mixed")
    rate1, _, _ = _oracle_rate(full, 0.0, max_steps=1, parallel=True)
    budget = 180.0
    n_s = int(min(full.n, 0.8 * rate1 * budget / max(1, args.steps + args.warmup)))
    if n_s >= full.n:
        box, what, same = full, "the full workload", True
    else:
        k = max(1, int((n_s / 8000) ** (1.0 / 3.0)))
        box = prepared(synth.w2_polydisperse(n=8000 * k ** 3, seed=2, tile_n=8000), "mixed")
        what, same = f"a sample: {k}^3 relaxed 8000-particle tiles of the same law", False
    p = oracle_params(box, "mixed", grid_for(box))
    s = O.State(box.x, box.v, box.w, box.r)
    for _ in range(args.warmup):
        O.step(p, s, parallel=True)
    # steps 1..K from the initial state, as the GPU arm times them
    s = O.State(box.x, box.v, box.w, box.r)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.step(p, s, parallel=True)
    dt = time.perf_counter() - t0
    value = box.n * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC_NAME, "value": value, "unit": METRIC,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded generator)",
        "config": {"workload": f"W2 polydisperse periodic box, {box.n} particles ({what}); "
                   "steps 1..K from the initial state",
                   "n": box.n, "same_workload_as_gpu_arm": same},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": threads, "kind": "oracle",
                         "cpu_model": _cpu_model(),
                         "sample": f"{args.steps} timed oracle steps of {box.n} particles "
                                   f"({what}), OpenMP build on {threads} threads"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
        return
    torch, rank, world, local = _torch_setup(args)
    import paper_1503_03553_gb300 as D
    if not os.path.exists(D.LIB_PATH):
        from paper_1503_03553_gb300 import build
        build.build()
    raw, box = _workload(args.n, 2 + rank)
    n = box.n
    from paper_1503_03553_gb300.synth import grid_for
    skin = args.skin_um * 1e-6
    ncell = grid_for(box, skin=skin)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = D.Context([box], precision=args.precision, ncell=[ncell], skins=[skin])
    # the workload is steps 1..K from the initial state: warm up from it,
    # then start again from it
    _reset(ctx, [box])
    ctx.step(args.warmup)
    _reset(ctx, [box])
    # ---- timed region: K steps, CUDA graphs, device time -------------------
    rs0 = ctx.resort_stats()
    with ClockSampler(local) as clk:
        secs = _time_steps(ctx, torch, args.steps, world)
    rs1 = ctx.resort_stats()
    resorts_timed = rs1["resorts"] - rs0["resorts"]
    secs = _max_over_ranks(secs, world, torch)
    value = job_throughput(n, world, args.steps, secs)
    # ---- the same K steps again, untimed: contacts and candidate pairs ---
    # along the trajectory (the packing relaxes: contacts fall during the run)
    _reset(ctx, [box])
    counts, chunk, done = [], max(1, args.steps // 20), 0
    while done < args.steps:
        k = min(chunk, args.steps - done)
        ctx.step(k)
        done += k
        counts.append((k, ctx.stats(0)[5], ctx.resort_stats()["candidates"]))
    contacts_total = sum(k * c for k, c, _ in counts)  # each chunk at its end count
    cands_total = sum(k * c for k, _, c in counts)
    c_half = contacts_total / args.steps / n
    cand_half = cands_total / args.steps / n
    # half contacts evaluated per second over the timed steps
    contact_evals = contacts_total * world / secs
    # ---- per-phase device time: the same K steps, direct launches ---------
    _reset(ctx, [box])
    ctx.set_timing(True)
    ctx.step(args.steps)
    ph = ctx.phase_times()
    ctx.set_timing(False)
    ncells = int(np.prod(ncell))
    pb = phase_bytes(n, c_half, cand_half, ncells, resorts_timed / args.steps)
    ph_ms = dict(zip(PHASES, ph.tolist()))
    peaks, src = _peaks()
    total_bytes = sum(pb.values())
    # the dominant kernel: of the two that run every step (the re-sort
    # kernels run in the steps that re-sort only), the slower
    dom = max(("pairs", "sum"), key=lambda k: ph_ms[k])
    achieved = pb[dom] / (ph_ms[dom] * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": PHASE_KERNEL[dom], "kernel_phase": dom,
            "achieved": achieved,
            "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None,
            "peak_source": src + " (MEASURED_PEAKS.json hbm_gbs; copy test, burst)",
            "algorithmic_bytes_per_launch": pb[dom],
            "kernel_ms": ph_ms[dom]}
    roof.update({"phase_ms": ph_ms, "phase_bytes": pb,
                 "candidates_per_particle": cand_half,
                 "resorts_per_step": resorts_timed / args.steps,
                 "step_algorithmic_bytes": total_bytes,
                 "step_frac_of_hbm": total_bytes / (secs / args.steps) / 1e9 / peaks["hbm_gbs"]})
    tr_path = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tr_path):
        # only while the kernels are the ones the counters were taken on
        try:
            import hashlib
            tr = json.load(open(tr_path))
            h = hashlib.sha256()
            for f in ("dem_kernels.cuh", "dem_common.cuh"):
                with open(os.path.join(ROOT, "paper_1503_03553_gb300", "csrc", f), "rb") as fh:
                    h.update(fh.read())
            if (tr.get("kernel") == PHASE_KERNEL[dom] and tr.get("precision") == args.precision
                    and tr.get("kernel_sha256") == h.hexdigest()):
                roof["traffic"] = tr["bytes_per_launch"] * n / tr["n"]
                roof["traffic_source"] = tr.get("source")
        except Exception:
            pass
    # ---- end to end through the C ABI with host buffers -----------------
    # every step: the state (x, v, w) from pinned host memory in, one step,
    # the new state back to pinned host memory
    pin = lambda: torch.empty((n, 3), dtype=torch.float64, pin_memory=True).numpy()
    hx, hv, hw = pin(), pin(), pin()
    _reset(ctx, [box])
    hx[:], hv[:], hw[:] = box.x, box.v, box.w
    _barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        D.dem_set_state(ctx.ctx, 0, hx, hv, hw)
        ctx.step(1)
        D.dem_get_state(ctx.ctx, 0, hx, hv, hw, None, None)
    e2e_secs = _max_over_ranks(time.perf_counter() - t0, world, torch)
    e2e = {"value": n * world * args.e2e_steps / e2e_secs, "unit": METRIC,
           "h2d_bytes_per_step": 3 * n * 3 * 8, "d2h_bytes_per_step": 3 * n * 3 * 8,
           "steps": args.e2e_steps}
    launches = ctx.launches_per_step() * args.steps + resorts_timed * rs1["launches_per_resort"]
    ctx.close()
    compare = {}
    cpu = None
    if rank == 0 and not args.no_compare:
        compare = _side_legs(args, D, torch, box, ncell, stream, skin)
        threads = _oracle_threads()
        rate, k, dt = _oracle_rate(box, args.cpu_seconds, max_steps=10, min_steps=10,
                                   parallel=True)
        rate1, k1, dt1 = _oracle_rate(box, 0.0, max_steps=1)
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
               "cpu_model": _cpu_model(),
               "sample": f"steps 1..{k} of the full {n}-particle workload, the oracle's "
                         f"OpenMP build on {threads} host threads, {dt:.1f} s",
               "single_thread": {"value": rate1, "unit": METRIC, "cores": 1,
                                 "sample": f"step 1 of the same workload, one host thread, "
                                           f"{dt1:.1f} s"}}
    if rank != 0:
        return
    line = {
        "metric": METRIC_NAME, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": secs / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "contact_evals_per_s": contact_evals,
        "dtype": {"mixed": "f32", "fp64": "f64", "fp32": "f32"}[args.precision],
        "data": "synthetic (seeded generator)",
        "config": {"workload": f"W2 polydisperse periodic box, {n} particles per GPU, "
                   "packing 0.55, dense contact network; steps 1..K from the initial "
                   "state (the packing relaxes: contacts fall during the run)",
                   "construction": _w2_construction(n),
                   "steps_from_initial_state": args.steps,
                   "n_per_gpu": n, "precision": args.precision,
                   "precision_detail": {"mixed": "FP32 force arithmetic; positions in 64-bit "
                                        "fixed point (2^-60 m); delta_t as float-float pairs",
                                        "fp64": "FP64 throughout",
                                        "fp32": "FP32 throughout"}[args.precision],
                   "ncell": ncell,
                   "skin_m": skin,
                   "resorts_in_timed_steps": resorts_timed,
                   "contacts_per_particle": c_half,
                   "l2": f"inputs larger than L2: a step touches {total_bytes / 1e6:.0f} MB "
                         f"of unique data vs {L2_BYTES / 1e6:.0f} MB L2",
                   "parallelism": f"{world} independent replica(s), one per GPU"},
        "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "clocks": clk.summary(),
        "compare": compare,
    }
    print(json.dumps(line))


def _reset(ctx, boxes):
    """Every box back to its initial particles (empty contact history)."""
    for k, b in enumerate(boxes):
        ctx.set_particles(k, b.x, b.v, b.w, b.r)


def _throughput(D, torch, stream, boxes, precision, ncells, steps, warmup=3, **kw):
    """Steps 1..steps of the workload from its initial state (after an
    untimed warm-up from the same state), device time."""
    with torch.cuda.stream(stream):
        ctx = D.Context(boxes, precision=precision, ncell=ncells, **kw)
    try:
        _reset(ctx, boxes)
        ctx.step(warmup)
        _reset(ctx, boxes)
        secs = _time_steps(ctx, torch, steps, 1)
    finally:
        ctx.close()
    n = sum(b.n for b in boxes)
    return {"value": n * steps / secs, "unit": METRIC, "steps": steps,
            "ms_per_step": secs / steps * 1e3}


def _side_legs(args, D, torch, box, ncell, stream, skin):
    """Comparison legs: the FP64 and FP32 GPU forms on the same workload, the
    force error of one step of each form against the FP64 oracle over every
    contact, the paper's Collide forms, the size-binned search, the paper's
    Fig. 4 regimes and batched boxes against a box-by-box loop.  A leg that
    fails is recorded with its error; the headline line is printed anyway."""
    out = {}

    def leg(name, fn):
        try:
            out[name] = fn()
        except Exception as e:  # recorded, not hidden: the line says which leg failed
            out[name] = {"error": f"{type(e).__name__}: {str(e)[:300]}"}

    leg("fp64_gpu", lambda: _fp64_leg(args, D, torch, stream, box, ncell, skin))
    leg("fp32_gpu", lambda: _throughput(D, torch, stream, [box], "fp32", [ncell], args.steps,
                                        skins=[skin]))
    leg("mixed_gpu_search_every_step", lambda: _throughput(D, torch, stream, [box], "mixed",
                                                           [ncell], args.steps, skins=[0.0]))
    leg("force_error_vs_fp64_oracle", lambda: _error_leg(out, box, ncell))
    leg("collide_fused_vs_compact", lambda: _fused_leg(args, D, torch, stream, box))
    leg("size_binned_search", lambda: _size_binned_leg(args, D, torch, stream, box, ncell))
    leg("fig4_kernel_times_131k", lambda: _fig4_leg(args, D, torch, stream))
    leg("layout_tuner", lambda: _tuner_leg(args, D, torch, stream, box, OTHER_SKIN_OVER_RMAX))
    if not args.no_batched:
        leg("batched", lambda: _batched_leg(args, D, torch, stream, OTHER_SKIN_OVER_RMAX))
    if args.w3:
        leg("w3_floor_8M", lambda: _w3_leg(args, D, torch, stream))
    if args.w5:
        leg("w5_precision", lambda: _w5_leg(args, D, torch, stream))
    if not args.no_sweep:
        leg("n_sweep", lambda: _sweep_leg(args, D, torch, stream, skin))
    return out


# FP64 operations (an FMA counts two) per pair in contact of the FP64 pair
# kernel, the contact rule on every candidate included: ncu thread-level
# DFMA/DADD/DMUL counts of one launch on the 512,000-particle W2 box
# (profiles/fp64_pairs_w2_512k.md)
FP64_FLOPS_PER_CONTACT = 320.0


def _fp64_leg(args, D, torch, stream, box, ncell, skin):
    """The plain FP64 form on the same workload and skin: throughput, and the
    roofline of its dominant kernel, the pair kernel, against the FP64 FMA
    rate measured on this GPU in this run (the form is bound by the FP64
    pipe, not by HBM)."""
    from paper_1503_03553_gb300.synth import prepared
    b = prepared(box, "fp64")
    res = _throughput(D, torch, stream, [b], "fp64", [ncell], args.steps, skins=[skin])
    ph = _phase_ms(D, torch, stream, [b], "fp64", [ncell], args.steps, skins=[skin])
    with torch.cuda.stream(stream):
        ctx = D.Context([b], precision="fp64", ncell=[ncell], skins=[skin])
    try:
        _reset(ctx, [b])
        contacts = 0.0
        for _ in range(args.steps):
            ctx.step(1)
            contacts += ctx.stats(0)[5]
    finally:
        ctx.close()
    peaks = D.dem_measure_fma_rates(stream)
    per_launch = FP64_FLOPS_PER_CONTACT * contacts / args.steps
    achieved = per_launch / (ph["pairs"] * 1e-3) / 1e12
    res["roofline"] = {"bound": "alu", "kernel": "k_pairs (FP64)", "achieved": achieved,
                       "peak": peaks["fp64_tflops"], "unit": "TFLOP/s",
                       "frac": achieved / peaks["fp64_tflops"],
                       "peak_source": "measured in this run (dem_measure_fma_rates: FP64 FMA)",
                       "flops_per_contact": FP64_FLOPS_PER_CONTACT,
                       "flops_source": "profiles/fp64_pairs_w2_512k.md (ncu DFMA/DADD/DMUL counts)",
                       "kernel_ms": ph["pairs"], "phase_ms": ph}
    res["alu_peaks_tflops"] = peaks
    return res


def _error_leg(out, box, ncell):
    """One step of each form against one FP64 oracle step over every
    contact; the MIXED form also through the parity test's full check."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from parity import (check_one_step, conditioning_report, force_errors, gpu_run, oracle_run,
                        prepared)
    errs = {}
    for prec in ("mixed", "fp32", "fp64"):
        b = prepared(box, prec)
        g = gpu_run([b], prec, [ncell])[0]
        o = oracle_run(b, prec, ncell)
        errs[prec] = force_errors(b, g, o, prec)
        if prec == "mixed":
            errs["mixed_conditioning"] = conditioning_report(b, g, o, prec, ncell)
            try:
                m = check_one_step(b, g, o, "mixed")
                out["force_parity_vs_fp64_oracle"] = {"pass": True, **m}
            except AssertionError as e:
                out["force_parity_vs_fp64_oracle"] = {"pass": False, "error": str(e)[:300]}
    return errs


def _sweep_leg(args, D, torch, stream, skin):
    """Particle-steps/s of the MIXED form against the particle count, W2
    radius law and packing (tiles of 8,000 relaxed spheres), the headline's
    skin, steps 1..200 from the initial state at every size (Sec. 5.2: the
    paper's speed-up is comparable for all sizes above 0.1 M)."""
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import grid_for, prepared
    rows = []
    for n in (100_000, 300_000, 1_000_000, 3_000_000, 8_000_000):
        box = prepared(synth.w2_polydisperse(n=n, seed=2), "mixed")
        nc = grid_for(box, skin=skin)
        steps = 200
        r = _throughput(D, torch, stream, [box], "mixed", [nc], steps, warmup=5, skins=[skin])
        r.update({"particles": box.n, "ncell": nc})
        rows.append(r)
    return rows


def _w3_leg(args, D, torch, stream):
    """W3: 8,000,000 bidisperse spheres, dense lower half and dilute upper
    half (divergence stress), floor and gravity: contact-list compaction vs
    the fused Algorithm 1, and the FP32 / FP64 forms."""
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import grid_for, prepared
    box = prepared(synth.w3_bidisperse_floor(n=8_000_000, seed=3), "mixed")
    skin = OTHER_SKIN_OVER_RMAX * box.r_max
    nc = grid_for(box)  # the per-particle forms and the search every step
    ncs = grid_for(box, skin=skin)
    res = {"particles": box.n, "ncell": nc, "ncell_with_skin": ncs, "skin_m": skin}
    k = 500  # the workload's steps, 1..500 from the initial state, every form
    res["steps"] = k
    res["mixed_compact"] = _throughput(D, torch, stream, [box], "mixed", [ncs], k, skins=[skin])
    res["mixed_compact"]["phase_ms"] = _phase_ms(D, torch, stream, [box], "mixed", [ncs], k,
                                                 skins=[skin])
    res["mixed_compact_search_every_step"] = _throughput(D, torch, stream, [box], "mixed",
                                                         [nc], k)
    res["mixed_fused"] = _throughput(D, torch, stream, [box], "mixed", [nc], k,
                                     collide=D.DEM_COLLIDE_FUSED)
    res["mixed_twoloop"] = _throughput(D, torch, stream, [box], "mixed", [nc], k,
                                       collide=D.DEM_COLLIDE_TWOLOOP)
    res["fp32_compact"] = _throughput(D, torch, stream, [prepared(box, "fp32")], "fp32", [ncs],
                                      k, skins=[skin])
    res["fp64_compact"] = _throughput(D, torch, stream, [prepared(box, "fp64")], "fp64", [ncs],
                                      k, skins=[skin])
    return res


def _w5_oracle(path):
    """Worker (spawned, no GPU): one FP64 oracle step from a saved GPU
    snapshot (state and contact history) and the error statistics of the
    GPU's forces of the same step."""
    import pickle
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O
    from parity import force_errors, oracle_params
    with open(path, "rb") as fh:
        b2, g, hist, prec, ncell = pickle.load(fh)
    os.remove(path)
    s = O.State(b2.x, b2.v, b2.w, b2.r)
    s.lo, s.hi, s.dt = hist
    p = oracle_params(b2, prec, ncell)
    out = O.step(p, s)
    out["params"] = p
    return force_errors(b2, g, out, prec, detail=5)


def _w5_leg(args, D, torch, stream):
    """W5 precision stress: spheres of radius U[3, 5] um at packing 0.60
    relaxed to overlaps of about 1e-3 r, at rest; each form runs the full
    step count, and every 'every' steps the force of one step from the
    form's own state and history is compared with the FP64 oracle
    re-evaluating that step (a full oracle run of this size is out of
    reach).  The oracle steps run in spawned host processes while the GPU
    continues."""
    import multiprocessing as mp
    import pickle
    import tempfile
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import grid_for, prepared
    raw = synth.w5_precision(n=args.w5_n, seed=5)
    res = {"particles": raw.n, "steps": args.w5_steps, "every": args.w5_every}
    tmp = tempfile.mkdtemp(prefix="w5_")
    workers = max(1, min(8, (os.cpu_count() or 2) - 2))
    pending = []
    with mp.get_context("spawn").Pool(workers) as pool:
        for prec in args.w5_forms.split(","):
            b = prepared(raw, prec)
            skin = OTHER_SKIN_OVER_RMAX * b.r_max
            nc = grid_for(b, skin=skin)
            with torch.cuda.stream(stream):
                ctx = D.Context([b], precision=prec, ncell=[nc], skins=[skin])
            try:
                ctx.set_particles(0, b.x, b.v, b.w, b.r)
                gpu_s = 0.0
                for k in range(args.w5_steps // args.w5_every):
                    gpu_s += _time_steps(ctx, torch, args.w5_every, 1)
                    st = ctx.get_state(0)
                    hist = ctx.contacts(0)
                    ctx.step(1)
                    g = {}
                    g["lo"], g["hi"], g["dt"] = ctx.contacts(0)
                    _, _, g["Fc"], _ = ctx.contact_forces(0)
                    b2 = prepared(b, prec)
                    b2.x, b2.v, b2.w = st["x"], st["v"], st["w"]
                    path = os.path.join(tmp, f"{prec}_{k}.pkl")
                    with open(path, "wb") as fh:
                        pickle.dump((b2, g, hist, prec, nc), fh, protocol=4)
                    del g, hist, st, b2
                    while sum(not r.ready() for _, _, r in pending) >= workers:
                        time.sleep(0.5)
                    pending.append((prec, (k + 1) * args.w5_every,
                                    pool.apply_async(_w5_oracle, (path,))))
                res[prec] = {"ms_per_step": 1e3 * gpu_s / args.w5_steps,
                             "contacts_at_end": int(ctx.stats(0)[5])}
            finally:
                ctx.close()
        for prec, step, r in pending:
            res[prec].setdefault("snapshots", []).append({"step": step, **r.get()})
    for prec in args.w5_forms.split(","):
        sn = res[prec]["snapshots"]
        res[prec]["worst_max_err_over_scale"] = max(x.get("max_err_over_scale", float("inf")) for x in sn)
        res[prec]["min_frac_within_1e-5"] = min(x.get("frac_within_1e-5", 0.0) for x in sn)
        res[prec]["worst_max_err_over_scale_cared"] = max(
            x.get("max_err_over_scale_cared", float("inf")) for x in sn)
        res[prec]["min_frac_within_1e-5_cared"] = min(x.get("frac_within_1e-5_cared", 0.0) for x in sn)
        res[prec]["contact_sets_equal"] = all(x["contact_sets_equal"] for x in sn)
        # the force-relative criterion, 1e-5 |F_ora| + 1e-9 k_n R*^1.5
        res[prec]["max_F_rel_bound_exceeded"] = max(x.get("F_rel_bound_exceeded", 0) for x in sn)
        res[prec]["worst_F_rel_bound_max"] = max(x.get("F_rel_bound_max", 0.0) for x in sn)
        res[prec]["max_F_rel_bound_exceeded_kappa_le_10"] = max(
            x.get("F_rel_bound_exceeded_kappa_le_10", 0) for x in sn)
    return res


def _phase_ms(D, torch, stream, boxes, precision, ncells, steps, **kw):
    """Per-phase device time averaged over steps 1..steps from the initial
    state (kernels launched one by one, events between phases)."""
    with torch.cuda.stream(stream):
        ctx = D.Context(boxes, precision=precision, ncell=ncells, **kw)
    try:
        _reset(ctx, boxes)
        ctx.step(3)
        _reset(ctx, boxes)
        ctx.set_timing(True)
        ctx.step(steps)
        return dict(zip(PHASES, ctx.phase_times().tolist()))
    finally:
        ctx.close()


def _contact_phase_ms(ph, fused):
    """The contact part of a step (the paper's Collide): the per-particle
    forms' one kernel (timed as the search phase); for the contact-list
    pipeline the search and rows of its re-sorts (averaged over the steps)
    and the pair kernel."""
    if fused:
        return ph["search"]
    return ph["search"] + ph["rows"] + ph["pairs"]


def _fused_leg(args, D, torch, stream, box):
    """The paper's comparison on this workload.  Its two per-particle Collide
    forms: Algorithm 1 as printed (search and force fused, each force as soon
    as its contact is found) and its improvement (Sec. 3.4: a first loop keeps
    the contact partners, a second computes their forces); against the split
    pipeline here (search, dense contact list, one thread per contact).
    'collide' is the contact part of the step: the per-particle kernel vs
    search + list + force."""
    from paper_1503_03553_gb300.synth import grid_for
    ncell = grid_for(box)  # the per-particle forms search every step: finest grid
    steps = args.steps
    out = {}
    coll = {}
    for name, form in (("fused", D.DEM_COLLIDE_FUSED), ("twoloop", D.DEM_COLLIDE_TWOLOOP)):
        out[f"{name}_step"] = _throughput(D, torch, stream, [box], "mixed", [ncell], steps,
                                          collide=form)
        pf = _phase_ms(D, torch, stream, [box], "mixed", [ncell], steps, collide=form)
        coll[name] = _contact_phase_ms(pf, fused=True)
    pc = _phase_ms(D, torch, stream, [box], "mixed", [ncell], steps)
    coll["compact"] = _contact_phase_ms(pc, fused=False)
    out.update({"collide_ms_fused": coll["fused"], "collide_ms_twoloop": coll["twoloop"],
                "collide_ms_compact": coll["compact"],
                "twoloop_speedup_over_fused": coll["fused"] / coll["twoloop"],
                "collide_speedup_of_compaction": coll["fused"] / coll["compact"]})
    return out


def _size_binned_leg(args, D, torch, stream, box, ncell):
    """Size-binned contact search (dem_box.r_split, Sec. 3.3's cell-size
    trade-off) against the one-class search: step time and the search phase
    (both search kernels) on this W2 box and on a box with radii spanning a
    factor 8 (1-8 um), each at the library's automatic grid."""
    import dataclasses
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import prepared
    steps = args.steps
    wide = prepared(synth.wide_polydisperse(n=box.n, seed=6), "mixed")
    out = {}
    for name, b0, splits in (("w2", box, (0.0, 5.5e-6, 6e-6)), ("radii_1_8um", wide, (0.0, 4e-6, 5e-6))):
        rows = []
        for rs in splits:
            b = dataclasses.replace(b0, r_split=rs)
            r = _throughput(D, torch, stream, [b], "mixed", None, steps)
            ph = _phase_ms(D, torch, stream, [b], "mixed", None, steps)
            r.update({"r_split_um": rs * 1e6, "search_ms": ph["search"], "sort_ms": ph["sort"]})
            rows.append(r)
        out[name] = {"particles": b0.n, "rows": rows}
    return out


FIG4_PARTICLES = 131072  # the particle count of the paper's Fig. 4 (Sec. 5.2)


def paper_figures():
    """The figures the paper prints for this comparison (Sec. 5.1, 5.2), read
    from tests/golden/paper_figures.txt: context beside the measurements."""
    path = os.path.join(ROOT, "tests", "golden", "paper_figures.txt")
    out = {}
    with open(path) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            name, value, unit, where = (x.strip() for x in line.split("|"))
            try:
                value = float(value)
            except ValueError:
                pass
            out[name] = {"value": value, "unit": unit, "where": where}
    return out


def _fig4_leg(args, D, torch, stream):
    """The paper's kernel-time comparison (Sec. 5.2, Fig. 4) at its size,
    131,072 particles: dense (W2 law and packing, left graph) and the
    initialisation stage, where no particles touch (lattice gas, right
    graph); per-phase ms of the previous Collide (Algorithm 1 as printed,
    fused), the paper's two-loop Collide and the contact-list pipeline."""
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import grid_for, prepared
    n = FIG4_PARTICLES
    pf = paper_figures()
    out = {"paper": {"collide_speedup_two_loop_over_fused":
                     pf["collide_speedup_two_loop_over_fused"],
                     "hardware": pf["gpu"]}}
    for name, b0 in (("dense", synth.w2_polydisperse(n=n, seed=2)),
                     ("initialisation_no_contacts", synth.lattice_gas(n=n, seed=7))):
        b = prepared(b0, "mixed")
        nc = grid_for(b)
        rows = {"particles": b.n}
        for form_name, form in (("fused_previous", D.DEM_COLLIDE_FUSED),
                                ("twoloop_paper", D.DEM_COLLIDE_TWOLOOP),
                                ("contact_list", D.DEM_COLLIDE_COMPACT)):
            ph = _phase_ms(D, torch, stream, [b], "mixed", [nc], 200, collide=form)
            ph["collide"] = _contact_phase_ms(ph, fused=form != D.DEM_COLLIDE_COMPACT)
            rows[form_name] = {k: round(v, 5) for k, v in ph.items()}
        rows["twoloop_speedup_over_fused_collide"] = (rows["fused_previous"]["collide"] /
                                                      rows["twoloop_paper"]["collide"])
        out[name] = rows
    return out


def _w4_boxes(args):
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import prepared
    procs = max(1, min(16, os.cpu_count() or 1))
    return [prepared(b, "mixed") for b in synth.w4_batched(nboxes=args.nboxes, processes=procs)]


_W4 = {}


def _w4_cached(args):
    """W4's boxes, generated once per run (the tuner and batched legs)."""
    if "b" not in _W4:
        _W4["b"] = _w4_boxes(args)
    return _W4["b"]


def _batched_leg(args, D, torch, stream, skin_frac):
    """W4: many independent periodic boxes in one context (one launch per
    kernel for all boxes, CUDA graphs) against the same boxes stepped one
    context at a time; every box keeps a skin of the same fraction of its
    largest radius as the W2 line."""
    from paper_1503_03553_gb300.synth import grid_for
    boxes = _w4_cached(args)
    skins = [skin_frac * b.r_max for b in boxes]
    ncells = [grid_for(b, skin=sk) for b, sk in zip(boxes, skins)]
    steps = args.batched_steps
    res = {"boxes": len(boxes), "particles": int(sum(b.n for b in boxes)), "steps": steps,
           "skin_over_rmax": skin_frac}
    res["batched"] = _throughput(D, torch, stream, boxes, "mixed", ncells, steps, skins=skins)
    total = 0.0
    for b, nc, sk in zip(boxes, ncells, skins):
        with torch.cuda.stream(stream):
            ctx = D.Context([b], precision="mixed", ncell=[nc], skins=[sk])
        try:
            _reset(ctx, [b])
            ctx.step(3)
            _reset(ctx, [b])
            total += _time_steps(ctx, torch, steps, 1)
        finally:
            ctx.close()
    res["box_by_box"] = {"value": res["particles"] * steps / total, "unit": METRIC,
                         "ms_per_step": total / steps * 1e3}
    res["speedup"] = res["batched"]["value"] / res["box_by_box"]["value"]
    return res


def _tuner_leg(args, D, torch, stream, box, skin_frac):
    """The layout tuner (dem_autotune_layout: skin, cell grid, size split,
    block size, graph length) on W2, on a W3-law box of 1,000,000
    particles (floor and gravity) and on W4's boxes: its choice, and steps
    1..K from the initial state with the bench's default layout and with the
    tuned one (a new context with the chosen skin and grid per box)."""
    import dataclasses
    from paper_1503_03553_gb300 import synth
    from paper_1503_03553_gb300.synth import grid_for, prepared
    steps = args.steps
    cases = [("w2", [box])]
    cases.append(("w3_1M", [prepared(synth.w3_bidisperse_floor(n=1_000_000), "mixed")]))
    if not args.no_batched:
        cases.append(("w4", _w4_cached(args)))
    out = {}
    for name, boxes in cases:
        skins = [skin_frac * b.r_max for b in boxes]
        ncells = [grid_for(b, skin=sk) for b, sk in zip(boxes, skins)]
        res = {"particles": int(sum(b.n for b in boxes)), "boxes": len(boxes)}
        res["default"] = _throughput(D, torch, stream, boxes, "mixed", ncells, steps, skins=skins)
        with torch.cuda.stream(stream):
            ctx = D.Context(boxes, precision="mixed", ncell=ncells, skins=skins)
        try:
            _reset(ctx, boxes)
            res["choice"] = ctx.autotune_layout(steps=max(steps, 32))
            lay = [ctx.layout(k) for k in range(len(boxes))]
        finally:
            ctx.close()
        tb = [dataclasses.replace(b, r_split=lay[k]["r_split"]) for k, b in enumerate(boxes)]
        res["tuned"] = _throughput(D, torch, stream, tb, "mixed", [l["ncell"] for l in lay], steps,
                                   skins=[l["skin"] for l in lay],
                                   block=res["choice"]["block"],
                                   graph_steps=res["choice"]["graph_steps"])
        res["tuned_layout_box0"] = lay[0]
        out[name] = res
    return out


if __name__ == "__main__":
    main()
