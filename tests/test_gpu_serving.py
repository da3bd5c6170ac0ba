"""Serving with continuous batching: requests of mixed kernel, size, precision
and distribution overlap on the GPU, and each result equals the same request
evaluated alone (same plan parameters) and the FP64 direct sum within its
tolerance."""
import numpy as np
import pytest

import oracle
from workloads import KERNEL_S, KERNEL_T, KERNEL_W, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_07844_gb300 as p
    return p


def _requests():
    rng = np.random.default_rng(1802078444)
    masks = [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W]
    out = []
    for i in range(12):
        mask = masks[i % 4]
        n = int(np.exp(rng.uniform(np.log(1000), np.log(12000))))
        dist = "near_wall" if i % 2 else "uniform"
        tol = 1e-10 if i % 3 else 1e-5
        out.append((mask, n, dist, tol, i))
    return out


def test_mix_equals_alone_and_oracle(pkg):
    srv = pkg.hse.Server(n_slots=3)
    try:
        _mix_equals_alone(pkg, srv)
    finally:
        srv.close()


def _mix_equals_alone(pkg, srv):
    reqs = []
    for mask, n, dist, tol, i in _requests():
        pr = problem(mask, n, 1.0, dist, 60, sub=i)
        prec = pkg.HSE_MIXED if tol >= 1e-6 else pkg.HSE_FP64
        src = torch.from_numpy(pr.src).cuda()
        st = torch.from_numpy(pr.strengths).cuda()
        t = srv.submit(mask, src, st, tol, prec)
        reqs.append((t, pr, prec, tol, src, st))
    for t, *_ in reqs:
        assert srv.wait(t, 300.0) == pkg.hse.HSE_OK
    stats = srv.stats()
    assert stats["completed"] == len(reqs) and stats["failed"] == 0
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    assert stats["plans_created"] + stats["plan_hits"] >= len(reqs)
    for t, pr, prec, tol, src, st in reqs:
        mixed = srv.result(t).cpu().numpy()
        # the plan the server used, read back through the ABI; the same call
        # the server makes (xi given, r_c, P, M from tol) gives the same plan
        used = srv.request_params(t)
        plan = pkg.Plan(pr.mask, (1.0, 1.0, 1.0), xi=used["xi"], rc=0.0, P=0, tol=tol, precision=prec)
        for k in ("xi", "rc", "P", "M", "Mt", "rc64", "eta", "precision", "kernel_mask"):
            assert plan.params[k] == used[k], k
        alone = plan.eval(src, st).cpu().numpy()
        plan.close()
        # same plan parameters: only the atomic summation order can differ
        # (FP64 atomics; float4 atomics for the FP32 outer shell of FP64 plans)
        assert oracle.rel_rms(mixed, alone) < (tol / 10 if prec == pkg.HSE_FP64 else 1e-6)
        # error over all targets (Sec. 6): sampled norms of the heavy-tailed
        # reference fluctuate more than the error
        ref = oracle.direct(pr.mask, pr.src, pr.strengths)
        assert oracle.rel_rms(mixed, ref) < tol


def test_prewarm_makes_the_first_request_a_cache_hit(pkg):
    """A prewarmed plan is resident before the first request that needs it:
    that request is admitted as a plan-cache hit, no plan is built inside its
    latency, and its result equals the direct sum within tol."""
    pr = problem(KERNEL_W, 4000, 1.0, "near_wall", 62)
    src = torch.from_numpy(pr.src).cuda()
    st = torch.from_numpy(pr.strengths).cuda()
    srv = pkg.hse.Server(n_slots=2)
    try:
        srv.prewarm(KERNEL_W, 4000, 1e-8, pkg.HSE_FP64)
        srv.prewarm(KERNEL_W, 4000, 1e-8, pkg.HSE_FP64)  # already resident: no second plan
        s0 = srv.stats()
        assert s0["plans_created"] == 1 and s0["plan_build_s"] > 0
        srv.reset_stats()
        t = srv.submit(KERNEL_W, src, st, 1e-8, pkg.HSE_FP64)
        assert srv.wait(t, 300.0) == pkg.hse.HSE_OK
        s1 = srv.stats()
        assert s1["plan_hits"] == 1 and s1["plans_created"] == 1 and s1["plan_build_s"] == 0.0
        ref = oracle.direct(KERNEL_W, pr.src, pr.strengths)
        assert oracle.rel_rms(srv.result(t).cpu().numpy(), ref) < 1e-8
        # an unknown ticket has no parameters
        with pytest.raises(pkg.HseError):
            srv.request_params(t + 1000)
    finally:
        srv.close()


def test_mixed_stokeslet_requests_take_a_double_float_fourier_part_when_large(pkg):
    """HSE_MIXED half-space stokeslet requests whose modelled FP32 rounding of
    the Fourier part (2.5e-8 sqrt(N)) exceeds tol/3 run their Fourier part in
    double-float; small ones, and other kernels, keep FP32 grids."""
    srv = pkg.hse.Server(n_slots=2)
    try:
        tickets = []
        for mask, n in ((KERNEL_S, 30000), (KERNEL_S, 4000), (KERNEL_W, 30000)):
            pr = problem(mask, n, 1.0, "uniform", 63, sub=n)
            src = torch.from_numpy(pr.src).cuda()
            st = torch.from_numpy(pr.strengths).cuda()
            tickets.append((srv.submit(mask, src, st, 1e-5, pkg.HSE_MIXED), pr, src, st))
        ffts = []
        for t, pr, _, _ in tickets:
            assert srv.wait(t, 300.0) == pkg.hse.HSE_OK
            ffts.append(srv.request_params(t)["fft"])
            n = pr.src.shape[1]
            idx = np.sort(np.random.default_rng(3).choice(n, min(n, 800), replace=False))
            ref = oracle.direct(pr.mask, pr.src, pr.strengths, pr.src[:, idx])
            u = srv.result(t).cpu().numpy()
            err = np.sqrt(np.mean(np.sum((u[:, idx] - ref) ** 2, axis=0)) / np.mean(np.sum(u ** 2, axis=0)))
            assert err < 1e-5
        assert ffts == [pkg.HSE_FFT_DF64, pkg.HSE_FFT_CUFFT, pkg.HSE_FFT_CUFFT]
    finally:
        srv.close()


def test_bounded_wait_and_memory_admission(pkg):
    pr = problem(KERNEL_S, 200_000, 1.0, "uniform", 61)
    src = torch.from_numpy(pr.src).cuda()
    st = torch.from_numpy(pr.strengths).cuda()
    srv = pkg.hse.Server(n_slots=1)
    t = srv.submit(KERNEL_S, src, st, 1e-10, pkg.HSE_FP64)
    # a host-side wait with a short limit returns a timeout, not a hang
    assert srv.wait(t, 1e-4) == pkg.hse.HSE_ERR_TIMEOUT
    assert srv.wait(t, 300.0) == pkg.hse.HSE_OK
    srv.close()
    # a request whose grids cannot fit the server's budget is refused at submission
    small = pkg.hse.Server(n_slots=1, mem_budget_bytes=16 << 20)
    with pytest.raises(pkg.HseError) as e:
        small.submit(KERNEL_S, src, st, 1e-10, pkg.HSE_FP64)
    assert e.value.status == pkg.hse.HSE_ERR_OOM
    small.close()
