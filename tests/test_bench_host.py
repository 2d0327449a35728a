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
