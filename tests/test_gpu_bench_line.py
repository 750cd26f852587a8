"""The bench line on the GPU: `bench.py` on the small profiling workload
prints one JSON line with the keys the measurement contract asks for, and
its numbers are consistent with each other."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
pytestmark = pytest.mark.gpu


def _run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py")] + list(args), cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_bench_line_has_the_contract_keys():
    d = _run("--workload", "small", "--steps", "2", "--warmup", "3", "--no-cpu-baseline", "--e2e-steps", "1")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 2 and d["warmup"] == 3 and d["higher_is_better"] is True
    pts = d["config"]["points"]
    # value = point-stages per second of the timed steps
    assert abs(d["value"] - 4 * pts / (d["ms_per_step"] * 1e-3)) <= 1e-6 * d["value"]
    r = d["roofline"]
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s" and 0.0 < r["frac"] < 1.2
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9
    assert abs(r["achieved"] - r["flops_per_point_stage"] * pts / (d["stage_kernel_ms"] * 1e-3) / 1e12) \
        <= 1e-9 * r["achieved"]
    e = d["e2e"]
    assert e["value"] > 0 and e["h2d_bytes_per_step"] == e["d2h_bytes_per_step"] == 25 * pts * 8 + 25 * 8 * (
        d["config"]["ghost_cells"])
    assert d["gpu_launches"] > 0 and d["clocks"]["sm_mhz"] > 0
    # the CUDA-graph path runs the same kernels: within 20 % of the launch path per step
    gr = d["graph"]
    assert gr["value"] > 0 and abs(gr["ms_per_step"] - d["ms_per_step"]) <= 0.2 * d["ms_per_step"]
    # measured FMA peaks: FP64 below the nominal unit-count peak, FP32 far above FP64
    pk = r["peak_measured"]
    assert 0.5 * r["peak"] < pk["fp64_tflops"] <= 1.05 * r["peak"] and pk["fp32_tflops"] > 20 * pk["fp64_tflops"]
    m = d["mixed"]
    assert m["speedup_vs_fp64"] > 1.0 and m["max_rel_state_error_vs_fp64"] < 1e-5
    assert set(m["rms_state_error_per_field"]) == set(m["rel_state_error_per_field"])
