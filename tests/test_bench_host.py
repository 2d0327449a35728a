"""Host logic of bench.py that needs no GPU: a failing comparison leg is
recorded in the line instead of stopping the benchmark."""
import os
import sys
import types

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_failing_leg_is_recorded(monkeypatch):
    calls = []

    def ok(name):
        def f(*a, **k):
            calls.append(name)
            return {"leg": name}
        return f

    def boom(*a, **k):
        raise RuntimeError("no such workload")

    monkeypatch.setattr(bench, "_throughput", ok("throughput"))
    monkeypatch.setattr(bench, "_error_leg", ok("errors"))
    monkeypatch.setattr(bench, "_fused_leg", boom)
    monkeypatch.setattr(bench, "_size_binned_leg", ok("size_binned"))
    monkeypatch.setattr(bench, "_fig4_leg", ok("fig4"))
    monkeypatch.setattr(bench, "_batched_leg", ok("batched"))
    monkeypatch.setattr(bench, "_tuner_leg", ok("tuner"))
    monkeypatch.setattr(bench, "_fp64_leg", ok("fp64"))
    args = types.SimpleNamespace(steps=10, no_batched=False, w3=False, w5=False, no_sweep=True)
    out = bench._side_legs(args, None, None, None, None, None, 0.0)
    assert out["collide_fused_vs_compact"]["error"].startswith("RuntimeError: no such workload")
    assert out["fp64_gpu"] == {"leg": "fp64"} and out["batched"] == {"leg": "batched"}
    assert out["fp32_gpu"] == {"leg": "throughput"}
    assert "fig4" in calls and "size_binned" in calls  # the legs after the failure still ran
    assert out["layout_tuner"] == {"leg": "tuner"}


def test_reference_arm_prints_one_line(capsys, monkeypatch):
    """--impl reference: the oracle on the host cores, one JSON line with
    the GPU arm's metric and unit, no host-device copies, and a
    cpu_baseline describing the run; ranks other than 0 print nothing."""
    import json
    args = types.SimpleNamespace(n=8000, steps=2, warmup=1, gpus=1)
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    bench.run_reference(args)
    lines = capsys.readouterr().out.strip().splitlines()
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["metric"] == bench.METRIC_NAME and line["unit"] == bench.METRIC
    assert line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["config"]["n"] == 8000 and line["config"]["same_workload_as_gpu_arm"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"],
                           "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == line["value"] and cb["cores"] >= 1
