"""bench.py's native lines on the GPU at reduced sizes: every key of the output contract, the roofline,
the host-buffer (end-to-end) figures with their byte counts, and the CPU oracle baseline."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(args):
    r = subprocess.run([sys.executable, "bench.py"] + args, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout[-2000:]
    return lines[0]


def test_native_line_contract(kirin_lib):
    n, steps = 65536, 3
    line = _run(["--n", str(n), "--steps", str(steps), "--warmup", "3", "--cpu-seconds", "1"])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "e2e", "gpu_launches", "clocks", "roofline",
                "cpu_baseline"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == steps and line["warmup"] == 3
    assert line["value"] > 1e11 and line["ms_per_step"] > 0 and line["higher_is_better"] is True
    assert line["scaling"] == "weak" and line["vs_baseline"] is None and line["data"] == "synthetic"
    assert f"N={n}" in line["config"]["workload"]
    assert line["gpu_launches"] >= 2 * steps
    e2e = line["e2e"]
    assert e2e["value"] > 0 and e2e["unit"] == line["unit"]
    assert e2e["h2d_bytes_per_step"] == n * 7 * 8  # m, x, v in FP64
    assert e2e["d2h_bytes_per_step"] == n * 7 * 8  # acc, jerk, pot in FP64
    clk = line["clocks"]
    assert clk["sm_max_mhz"] > 0 and isinstance(clk["reasons"], list)
    roof = line["roofline"]
    assert roof["bound"] == "alu" and roof["unit"] == "TFLOP/s" and roof["peak"] > 0
    assert 0.1 < roof["frac"] < 1.2 and roof["achieved"] == pytest.approx(roof["frac"] * roof["peak"])
    assert roof["traffic"] is None  # the stored counters are for the N = 2^20 launch only
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] > 0 and cb["sample"]
    err = line["mixed_vs_oracle_rel_err"]
    assert err["acc"]["median"] <= 1e-6 and err["acc"]["max"] <= 1e-5 and err["pot"]["median"] <= 1e-6
    assert line["fp64"]["mixed_speedup"] > 1.0
    # the other workloads ride on the same line, each with its clocks and an oracle parity summary
    for name in ("small", "block", "ensemble", "adjoint"):
        sub = line[name]
        assert "error" not in sub, (name, sub)
        assert sub["value"] > 0 and sub["clocks"]["sm_max_mhz"] > 0 and sub["parity"], name
        sr = sub["roofline"]
        assert sr["bound"] == "alu" and sr["unit"] == "TFLOP/s" and 0 < sr["frac"] < 1.2, name
        assert sr["achieved"] == pytest.approx(sr["frac"] * sr["peak"]), name
    blk = line["block"]
    assert blk["t_end"] == 0.125 and blk["fp64"]["t_end"] == 0.125 and blk["block_steps"] > 1000
    assert blk["parity"]["x_final_device_vs_host_loop_rel_diff"] < 1e-6
    assert blk["parity"]["x_final_mixed_vs_fp64_rel_diff"] < 1e-6
    assert line["small"]["parity"]["x_after_10_steps_rel_diff"] < 1e-9
    assert blk["parity"]["start_evaluation_256_i_vs_oracle"]["acc"]["max"] <= 1e-5
    assert abs(blk["dE_E"]) < 1e-6 and abs(blk["fp64"]["dE_E"]) < 1e-6
    # the host-stepped histogram run sums large blocks in other launch shapes: a step-size decision near
    # its threshold may differ by rounding, so the counts agree to a few steps
    assert abs(sum(h["steps"] for h in blk["n_active_histogram"].values()) - blk["block_steps"]) <= 0.005 * blk["block_steps"]
    assert line["small"]["parity"]["first_evaluation_vs_oracle"]["acc"]["max"] <= 1e-5
    assert all(e["max"] <= 1e-5 for q, e in line["ensemble"]["parity"].items() if q.startswith("acc"))
    assert line["adjoint"]["parity"]["acc_pot_vs_oracle"]["acc"]["max"] <= 1e-5


def test_small_workload_line(kirin_lib):
    line = _run(["--workload", "small", "--steps", "2", "--warmup", "3"])
    assert line["value"] > 0 and line["steps"] >= 2 and "N=1024" in line["config"]["workload"]
    assert line["fp64"]["value"] > 0
