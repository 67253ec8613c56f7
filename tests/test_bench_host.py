"""Host-side logic of bench.py (no GPU): the kernel-source digest that ties an
ncu summary to the kernels it measured, the traffic lookup, the workload table
and the roofline arithmetic."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_digest_ignores_comments_and_whitespace_only():
    code = "int f(int x) {\n    return x + 1;   // add one\n}\n"
    same = "// header comment\nint f(int x)\n{\n  return x + 1;\n}\n"
    other = "int f(int x) {\n    return x + 2;   // add one\n}\n"
    assert bench.code_digest([code]) == bench.code_digest([same])
    assert bench.code_digest([code]) != bench.code_digest([other])
    assert bench.code_digest([code, same]) != bench.code_digest([code])


def test_profiled_traffic_matches_the_committed_summary():
    # the committed FP32 summary was taken on the current kernel source
    t1 = bench.profiled_traffic("thacker_paraboloid_40m", 32, "stage1")
    t2 = bench.profiled_traffic("thacker_paraboloid_40m", 32, "stage2")
    assert t1 is not None and t2 is not None
    cells = 39_997_568
    assert 60 * cells < t1 < 120 * cells and 90 * cells < t2 < 140 * cells     # bytes per launch
    assert bench.profiled_traffic("flat_basin_allwet_40m", 32, "stage2") is None
    assert bench.profiled_traffic("thacker_paraboloid_40m", 32, "nonexistent") is None


def test_workload_table():
    for name, w in bench.WORKLOADS.items():
        kind = w.get("kind", "thacker")
        assert kind in bench.FP64_FLOPS_PER_CELL_STEP, name
        assert bench.workload_hthr(name) in (1e-5, 1e-3)
    assert bench.workload_hthr("coast_basin_5m") == 1e-3
    m, s = bench.workload_inputs("coast_basin_5m", 40)        # small sample of the coast generator
    assert abs(m.nc - 2 * 40 * 40) < 0.2 * 2 * 40 * 40 and s.H.shape == (m.nc,)


def test_roofline_of_fused_and_unfused_profiles():
    """The dominant kernel's achieved bandwidth is its algorithmic bytes per launch
    over its mean launch time; an unfused step (the RK updates as kernels of their
    own) reports every kernel against the same peak and the step's bytes summed
    over its four kernels."""
    nc = 1_000_000
    peak, _ = bench.measured_peaks()
    fused = {"stage1": (10, 10.0), "stage2": (10, 12.0), "post_step": (10, 0.1), "bed_update": (0, 0.0)}
    r = bench.roofline_of(fused, nc, 32, "thacker_paraboloid_40m", 2.3)
    assert r["kernel"] == "stage2" and r["bound"] == "hbm"
    assert abs(r["achieved"] - 76 * nc / 1.2e-3 / 1e9) < 0.1
    assert abs(r["frac"] - r["achieved"] / peak) < 1e-4
    assert abs(r["step_algo_gbs"] - 140 * nc / 2.3e-3 / 1e9) < 0.1
    assert "per_kernel_gbs" not in r
    unfused = {"stage1": (10, 10.0), "stage2": (0, 0.0), "rk_update1": (10, 3.0), "residual_w1": (10, 10.0),
               "rk_update2": (10, 3.0), "post_step": (10, 0.1)}
    u = bench.roofline_of(unfused, nc, 32, "thacker_paraboloid_40m", 2.7)
    assert u["kernel"] == "stage1"
    assert abs(u["step_algo_gbs"] - (64 + 40 + 64 + 52) * nc / 2.7e-3 / 1e9) < 0.1
    assert abs(u["per_kernel_gbs"]["rk_update1"] - 40 * nc / 0.3e-3 / 1e9) < 0.1
    assert abs(u["per_kernel_gbs"]["rk_update2"] - 52 * nc / 0.3e-3 / 1e9) < 0.1
    # FP64 reports the FP64 units' roofline on the counted flops
    f = bench.roofline_of(fused, nc, 64, "thacker_paraboloid_40m", 2.3)
    assert f["bound"] == "alu" and f["unit"] == "TFLOP/s"
    flops = 0.5 * bench.FP64_FLOPS_PER_CELL_STEP["thacker"] * nc
    assert abs(f["achieved"] - flops / 1.2e-3 / 1e12) < 1e-4
