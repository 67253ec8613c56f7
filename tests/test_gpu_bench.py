"""bench.py's one-line JSON contract on a small workload (1M triangles): the
keys, the roofline arithmetic, the end-to-end byte counts, the kernel launch
count and the oracle baseline object."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.gpu
def test_bench_json_line():
    steps, warmup = 6, 3
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--workload", "thacker_paraboloid_1m",
                        "--steps", str(steps), "--warmup", str(warmup), "--e2e-steps", "2", "--cpu-budget", "1",
                        "--batched-steps", "0", "--adjoint-steps", "0"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1, r.stdout[-2000:]
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == steps and d["warmup"] == warmup
    assert d["higher_is_better"] is True and d["scaling"] == "weak" and d["vs_baseline"] is None
    assert d["dtype"] == "f32" and d["unit"] == "cell-updates/s"
    cells = d["config"]["cells"]
    assert d["config"]["workload"] == "thacker_paraboloid_1m" and cells > 900_000
    assert d["value"] > 0
    assert abs(d["value"] - cells * 1e3 / d["ms_per_step"]) <= 1e-6 * d["value"]
    rf = d["roofline"]
    assert rf["bound"] == "hbm" and rf["unit"] == "GB/s" and rf["peak"] > 0
    assert abs(rf["frac"] - rf["achieved"] / rf["peak"]) < 1e-3
    dom = rf["kernel"]
    assert abs(rf["achieved"] - rf["algo_bytes_per_launch"] / (rf["kernel_avg_ms"][dom] * 1e6)) <= 0.01 * rf["achieved"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 3 * 4 * cells and e["d2h_bytes_per_step"] == 3 * 4 * cells
    assert e["f64_host"]["h2d_bytes_per_step"] == 3 * 8 * cells
    assert d["gpu_launches"] == 3 * steps          # stage 1, stage 2, epilogue per step
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["value"] > 0 and c["cores"] >= 1 and c["unit"] == d["unit"] and c["sample"]
    assert set(d["clocks"]) >= {"sm_mhz", "sm_max_mhz", "reasons"}
