"""The bench line's contract on a small grid: one JSON line with the keys the
measurement needs (metric, value, roofline, flops, e2e, clocks, launches),
and numbers that agree with one another."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_keys_and_consistency():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--n", "128", "--steps", "5", "--warmup", "3",
           "--no-cpu-baseline", "--no-ensemble", "--no-paper-shapes", "--no-err", "--no-tc", "--e2e-reps", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "step_roofline", "flops", "kernels", "e2e",
              "clocks", "gpu_launches"):
        assert k in d, k
    assert d["metric"].endswith("128^3 FP32") and d["config"]["n"] == 128
    assert d["steps"] == 5 and d["warmup"] >= 3 and d["n_gpus"] == 1
    # value = points x steps / time
    assert d["value"] == pytest.approx(128 ** 3 / (d["ms_per_step"] / 1e3) / 1e6, rel=1e-6)
    r = d["roofline"]
    assert r["bound"] == "hbm" and 0 < r["frac"] < 1.2 and r["achieved"] == pytest.approx(r["frac"] * r["peak"])
    assert 0 < d["flops"]["frac"] < 1.0 and d["flops"]["peak_tflops"] > 10
    e = d["e2e"]
    assert 0 < e["value"] <= d["value"] * 1.05 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] == 16 * d["steps"]
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
