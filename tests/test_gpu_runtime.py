"""Runtime entry points around the evaluation: the measured pipe throughputs
(roofline denominators) and the real-space residency cap."""
import numpy as np
import pytest

import oracle
from workloads import KERNEL_S, KERNEL_W, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_07844_gb300 as p
    return p


def test_pipe_peaks_are_measured_and_ordered(pkg):
    """FP64 multiply-adds are far slower than FP32 ones on this part, and a
    double-float multiply-add (~15 FP32 instructions) lies in between; every
    figure is below the unit-count peak at the reported maximum clock."""
    m = pkg.hse.hse_measure_pipe_peaks()
    assert m["n_sm"] > 0 and m["sm_clock_mhz"] > 0
    clk = m["sm_clock_mhz"] * 1e6
    fp32_units = m["n_sm"] * 128 * 2 * clk / 1e12
    assert 0.3 * fp32_units < m["fp32_tflops"] <= 1.05 * fp32_units
    assert m["fp64_tflops"] > 0 and m["fp32_tflops"] > 8 * m["fp64_tflops"]
    assert m["fp64_tflops"] < m["df64_tflops"] < m["fp32_tflops"] / 4
    print("pipe peaks:", m)


@pytest.mark.parametrize("bps", [1, 3])
def test_real_residency_cap_keeps_results(pkg, bps):
    """A persistent real-space grid of bps blocks per SM gives the same sums
    (up to the order of the partner atomics), alone and with overlapped halves
    (tol 1e-10: equal to well within tol / 10)."""
    mask = KERNEL_S | KERNEL_W
    pr = problem(mask, 20000, 1.0, "near_wall", 36)
    src = torch.from_numpy(pr.src).cuda()
    st = torch.from_numpy(pr.strengths).cuda()
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=20.0, rc=0.0, P=0, tol=1e-10)
    try:
        base = plan.eval(src, st).cpu().numpy()
        plan.set_real_residency(bps)
        capped = plan.eval(src, st).cpu().numpy()
        plan.set_overlap(True)
        both = plan.eval(src, st).cpu().numpy()
        assert plan.stats()["overlapped"]
    finally:
        plan.close()
    # the order of the partner atomics changes: FP64 ones at rounding level,
    # the FP32 outer shell's float4 ones at ~1e-7 of its small terms
    assert oracle.rel_rms(capped, base) < 1e-11
    assert oracle.rel_rms(both, base) < 1e-11
    with pytest.raises(pkg.HseError):
        h = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=20.0, rc=0.1, P=8, tol=0.0)
        try:
            h.set_real_residency(-1)
        finally:
            h.close()
