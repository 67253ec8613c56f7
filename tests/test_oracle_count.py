"""The operation-counting build of the oracle (oracle/op_count.hpp), whose
counts give the FP64 roofline's algorithmic flops, runs the oracle's own
arithmetic: the time step it computes equals the plain oracle's bit for bit,
and the counts grow with the number of cells."""
import oracle as O
from paper_2002_04889_gb300 import inputs as I


def test_counting_build_runs_the_same_arithmetic():
    m = I.thacker_mesh(n=30)
    s = I.thacker_initial_state(m)
    c = O.count_step_ops(m, (s.H, s.Hu, s.Hv), h_threshold=1e-5, cfl=0.9)
    r = O.OracleMesh.from_mesh(m).run(O.params(h_threshold=1e-5, cfl=0.9), (s.H, s.Hu, s.Hv, 0.0), 1)
    assert c["dt"] == r["dts"][0]
    assert c["sqrt"] > 0 and c["div"] > 0 and c["mul"] > c["div"]


def test_counts_scale_with_cells():
    a = I.flat_basin_mesh(20, 1.0, 10.0)
    b = I.flat_basin_mesh(40, 2.0, 10.0)           # same dx, four times the cells
    sa = I.gaussian_hump_state(a, 0.0, 0.5, 0.0, 0.0, 10.0)
    sb = I.gaussian_hump_state(b, 0.0, 0.5, 0.0, 0.0, 10.0)
    ca = O.count_step_ops(a, (sa.H, sa.Hu, sa.Hv))
    cb = O.count_step_ops(b, (sb.H, sb.Hu, sb.Hv))
    for k in ("add", "sub", "mul", "div", "sqrt"):
        assert 3.5 * ca[k] < cb[k] < 4.5 * ca[k], k
