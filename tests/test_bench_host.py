"""Host-side logic of bench.py (no GPU): the kernel-source digest that ties an
ncu summary to the kernels it measured, the traffic lookup, and the workload
table."""
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
