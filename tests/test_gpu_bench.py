"""GPU: bench.py's JSON line on a tiny configuration carries every key of the benchmark contract."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_keys(cuda):
    cmd = [sys.executable, "bench.py", "--buses", "100", "--columns", "4096", "--steps", "3", "--warmup", "3",
           "--no-learned", "--no-other", "--no-scenario", "--no-batch", "--no-poly", "--no-zip", "--no-large",
           "--fp64-sample", "64", "--cpu-seconds", "1", "--check-columns", "64", "--train-columns", "8192",
           "--epochs", "10"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "clocks", "gpu_launches"):
        assert k in d, k
    assert d["value"] > 0 and d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3
    # The headline step is the learned-start solve: the fused inference (it reads S itself) and one
    # sparse launch.
    assert d["headline_start"] == "learned" and d["gpu_launches"] == 6
    assert d["flat_start"]["gpu_launches"] == 3  # one sparse launch per step
    lh = d["learned_start_headline"]
    assert lh["fallback_columns"] == 0 and lh["converged"] == 4096 and lh["mean_sweeps"] < d["flat_start"]["mean_sweeps"]
    for k in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert k in d["roofline"], k
    assert 0 < d["roofline"]["frac"] < 1.5
    for k in ("sm_mhz", "sm_max_mhz", "reasons"):
        assert k in d["clocks"], k
    for k in ("value", "unit", "h2d_bytes_per_step", "d2h_bytes_per_step"):
        assert k in d["e2e"], k
    assert d["e2e"]["h2d_bytes_per_step"] == 4096 * 99 * 16
    for k in ("value", "unit", "cores", "kind", "sample"):
        assert k in d["cpu_baseline"], k
    assert d["accuracy"]["max_abs_err_pu"] <= 1e-8 and d["flat_start"]["max_abs_err_pu"] <= 1e-8
    small = d["small_feeder"]  # 34 buses x 1,440 columns, every column against the oracle
    for name, bound in (("fp64", 1e-9), ("mixed_sparse", 1e-8), ("mixed_dense", 1e-8)):
        r = small[name]
        assert r["converged"] == 1440 and r["columns_checked"] == 1440, name
        assert r["max_abs_err_pu"] <= bound, (name, r["max_abs_err_pu"])
        assert r["value"] > 0 and r["host_ms_per_call"] >= r["ms_per_call"] * 0.5, name
    t1 = d["table1_100_bus"]  # 100 buses over the one-minute year, sampled columns against the oracle
    assert t1["converged"] == 525600 and t1["columns_checked"] == 1024
    assert t1["max_abs_err_pu"] <= 1e-8 and t1["value"] > 0
