"""The bench line's contract on the CPU: the reference arm (the oracle on
every host core) prints one JSON line with the keys the harness reads."""
import argparse
import contextlib
import io
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line_has_the_contract_keys(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setattr(bench, "REF_SAMPLE_N", 16)  # a 16^3 sample keeps the test short
    args = argparse.Namespace(gpus=1, steps=2, warmup=3, grid=256)
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(args, 0, None)
    lines = [l for l in out.getvalue().splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["steps"] == 2 and d["higher_is_better"] is True
    assert "workload" in d["config"] and "256^3" in d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"].startswith("oracle") and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_prints_nothing_on_other_ranks():
    sys.path.insert(0, ROOT)
    import bench
    out = io.StringIO()
    with contextlib.redirect_stdout(out):
        bench.run_reference(argparse.Namespace(gpus=2, steps=1, warmup=3, grid=256), 1, None)
    assert out.getvalue() == ""
