"""bench.py on the GPU: one short run, and the JSON line carries every key of
the measurement contract with sane values."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_bench_line_has_the_contract_keys(cuda_lib):
    r = subprocess.run([sys.executable, "bench.py", "--steps", "50", "--warmup", "3",
                        "--no-extras", "--no-cpu-baseline", "--no-autotune"],
                       cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "roofline", "e2e", "gpu_launches", "clocks"):
        assert key in line, key
    assert line["n_gpus"] == 1 and line["steps"] == 50 and line["warmup"] == 3
    assert line["unit"] == "pairs/s" and line["value"] > 1e10
    assert line["higher_is_better"] is True and line["scaling"] == "weak"
    assert line["config"]["workload"] == "bandwidth_2p28"
    roof = line["roofline"]
    for key in ("bound", "achieved", "peak", "unit", "frac", "traffic"):
        assert key in roof, key
    assert roof["bound"] == "hbm" and roof["unit"] == "GB/s"
    assert 0.5 < roof["frac"] < 1.1
    # the copy peak re-measured on this machine, beside the file's
    assert 1000 < roof["peak_live_copy"] < 10000 and 0.5 < roof["frac_of_live_copy"] < 1.1
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 4 * (1 << 28)
    assert e2e["d2h_bytes_per_step"] == 8 * (1 << 28)
    assert 0 < e2e["value"] < line["value"]
    assert line["gpu_launches"] >= 50
    assert line["wait_timeouts"] == 0
    assert {"sm_mhz", "sm_max_mhz", "reasons", "mem_mhz"} <= set(line["clocks"])
