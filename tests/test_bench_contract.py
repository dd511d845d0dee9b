"""bench.py's JSON line on the GPU: one line with the keys the measurement
contract asks for, consistent with each other (a short run of the default
workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_line_has_the_contract_keys():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "3",
           "--no-cpu-baseline", "--no-16bit", "--no-1024", "--naive-calls", "0"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3 and d["higher_is_better"] is True
    assert d["unit"] == "GCUPS" and d["value"] > 0 and d["dtype"] == "f32" and "workload" in d["config"]
    # value = cell updates per second of the timed step
    nx, ny, nz = d["config"]["grid_xyz"]
    assert abs(d["value"] - nx * ny * nz * d["config"]["steps_per_call"] / (d["ms_per_step"] * 1e-3) / 1e9) \
        < 1e-6 * d["value"]
    rf = d["roofline"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in rf, k
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-9
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert d["gpu_launches"] >= 1
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    ir = d.get("issue_roofline")
    if ir is not None:  # measured instruction count x GCUPS against the SMs' issue rate
        assert 0 < ir["frac"] <= 1.0 and abs(ir["frac"] - ir["achieved"] / ir["peak"]) < 1e-9
