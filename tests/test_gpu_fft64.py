"""Double-float (df64) transforms of the FP64 Fourier part (Sec. 4 steps
FFT - scale - IFFT) against cuFFT double on the same plan and inputs: every
kernel mask, line lengths with radices 4, 2, 5 and 3 (including lengths not
divisible by 4), the wide line passes with radix 8 (512, 576 and 640 points),
the fallback to cuFFT for lengths with other prime factors,
and the mode switch rules.  Both runs share the spread and the gather, so the
comparison isolates the transforms and the scaling."""
import numpy as np
import pytest

import oracle
from workloads import KERNEL_S, KERNEL_T, KERNEL_W, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FREE = oracle.FREE_SPACE


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_07844_gb300 as p
    return p


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def fourier_both(pkg, plan, pr):
    src, st = dev(pr.src), dev(pr.strengths)
    plan.set_fft(pkg.HSE_FFT_CUFFT)
    assert plan.params["fft"] == pkg.HSE_FFT_CUFFT
    _, ref = plan.eval_parts(src, st, real=False)
    ref = host(ref)
    plan.set_fft(pkg.HSE_FFT_DF64)
    assert plan.params["fft"] == pkg.HSE_FFT_DF64
    _, u = plan.eval_parts(src, st, real=False)
    return host(u), ref


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W, KERNEL_S | KERNEL_T | KERNEL_W,
                                  KERNEL_S | KERNEL_W | FREE])
@pytest.mark.parametrize("M", [18, 33, 68])  # Mt = 30, 45, 80: lines 4.3.5, 2.5.3.3, 4.4.2.5 (x2 for z)
def test_df64_matches_cufft(pkg, mask, M):
    pr = problem(mask & 7, 3000, 1.0, "near_wall", 70 + M)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=6.0, rc=0.5, P=12, tol=0.0, M=M)
    assert plan.params["fft"] == pkg.HSE_FFT_DF64  # explicit parameters: df64 by default
    u, ref = fourier_both(pkg, plan, pr)
    # ~48-bit arithmetic: the difference is rounding, far below any tolerance
    assert rel(u, ref) < 1e-12
    assert float(np.abs(u - ref).max() / np.abs(ref).max()) < 1e-12
    plan.close()


def test_df64_bench_shape(pkg):
    # the benchmark's line length (Mt = 320: 640 points, wide passes forward
    # 2.8.8.5, inverse 8.8.5.2) at a reduced count
    mask = KERNEL_S | KERNEL_W
    pr = problem(mask, 20000, 1.0, "near_wall", 79)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=87.0, rc=0.0552, P=18, tol=0.0, M=302)
    u, ref = fourier_both(pkg, plan, pr)
    assert rel(u, ref) < 1e-12
    plan.close()


@pytest.mark.parametrize("M", [238, 270])
def test_df64_wide_lines(pkg, M):
    # lines of 512 and 576 points (Mt = 256, 288) take the wide line passes
    # (N / 8 threads per line, radix 8): forward 2.8.8.4 and 2.8.4.3.3,
    # inverse 8.8.4.2 and 8.4.3.3.2
    mask = KERNEL_S | KERNEL_W
    pr = problem(mask, 20000, 1.0, "near_wall", 80 + M % 7)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=87.0, rc=0.0552, P=18, tol=0.0, M=M)
    assert plan.params["Mt"] == M + 18
    u, ref = fourier_both(pkg, plan, pr)
    assert rel(u, ref) < 1e-12
    assert float(np.abs(u - ref).max() / np.abs(ref).max()) < 1e-12
    plan.close()


def test_df64_unsupported_length_falls_back(pkg):
    # Mt = 28: lines of 56 = 8 x 7 have a factor the df64 transforms lack
    plan = pkg.Plan(KERNEL_S, (1.0, 1.0, 1.0), xi=5.0, rc=0.5, P=12, tol=0.0, M=16)
    assert plan.params["fft"] == pkg.HSE_FFT_CUFFT
    with pytest.raises(pkg.HseError):
        plan.set_fft(pkg.HSE_FFT_DF64)
    assert plan.params["fft"] == pkg.HSE_FFT_CUFFT
    pr = problem(KERNEL_S, 500, 1.0, "uniform", 80)
    u = host(plan.eval(dev(pr.src), dev(pr.strengths)))
    assert np.isfinite(u).all()
    plan.close()


def test_df64_mode_rules(pkg):
    # FP32 plans take cuFFT single unless a double-float Fourier part is asked
    # for; tight tolerances keep cuFFT double
    mixed = pkg.Plan(KERNEL_S, (1.0, 1.0, 1.0), xi=10.0, tol=1e-5, precision=pkg.HSE_MIXED)
    assert mixed.params["fft"] == pkg.HSE_FFT_CUFFT
    b32 = mixed.params["grid_bytes"]
    mixed.set_fft(pkg.HSE_FFT_DF64)
    assert mixed.params["fft"] == pkg.HSE_FFT_DF64
    assert mixed.params["grid_bytes"] > 1.5 * b32  # 8-byte grids and tables
    mixed.set_fft(pkg.HSE_FFT_CUFFT)
    assert mixed.params["fft"] == pkg.HSE_FFT_CUFFT
    mixed.close()
    tight = pkg.Plan(KERNEL_W, (1.0, 1.0, 1.0), xi=10.0, tol=1e-13)
    assert tight.params["fft"] == pkg.HSE_FFT_CUFFT
    tight.close()
    loose = pkg.Plan(KERNEL_W, (1.0, 1.0, 1.0), xi=10.0, tol=1e-8)
    assert loose.params["fft"] == pkg.HSE_FFT_DF64
    loose.set_fft(pkg.HSE_FFT_AUTO)
    assert loose.params["fft"] == pkg.HSE_FFT_DF64
    loose.close()


def test_df64_full_eval_vs_oracle(pkg):
    # whole evaluation with df64 transforms against the direct half-space sum
    mask = KERNEL_S | KERNEL_T | KERNEL_W
    pr = problem(mask, 600, 1.0, "near_wall", 81)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=10.0, tol=1e-9)
    assert plan.params["fft"] == pkg.HSE_FFT_DF64
    u = host(plan.eval(dev(pr.src), dev(pr.strengths)))
    ref = oracle.direct(mask, pr.src, pr.strengths)
    assert rel(u, ref) < 1e-9
    plan.close()


@pytest.mark.parametrize("mask", [KERNEL_S | KERNEL_W, KERNEL_T])
def test_df64_at_the_tightest_automatic_tolerance(pkg, mask):
    # tol = 1e-12 is the tightest tolerance the automatic rule serves with df64:
    # the whole evaluation (df64 grids and transforms) must meet it against the
    # direct half-space sum, as the cuFFT-double path does
    pr = problem(mask, 1500, 1.0, "near_wall", 82)
    ref = oracle.direct(mask, pr.src, pr.strengths)
    src, st = dev(pr.src), dev(pr.strengths)
    plan = pkg.Plan(mask, (1.0, 1.0, 1.0), xi=8.0, tol=1e-12)
    assert plan.params["fft"] == pkg.HSE_FFT_DF64
    e_df = rel(host(plan.eval(src, st)), ref)
    plan.set_fft(pkg.HSE_FFT_CUFFT)
    e_cu = rel(host(plan.eval(src, st)), ref)
    plan.close()
    assert e_df < 1e-12 and e_cu < 1e-12
    assert e_df < 2.0 * e_cu + 1e-14


def test_mixed_plan_with_double_float_fourier_part(pkg):
    """Half-space stokeslets spread through the box: with FP32 grids the
    Fourier part loses ~2.5e-8 sqrt(N) of the velocity (FP32 rounding at low
    wave numbers, where the image system cancels the long-range field and the
    kernel scales by ~1/k^2).  An HSE_MIXED plan with HSE_FFT_DF64 keeps FP32
    real space and matches the FP64 plan's Fourier part far more closely, and
    the whole evaluation meets tol against the direct sum."""
    n = 60000
    pr = problem(KERNEL_S, n, 1.0, "uniform", 83)
    src, st = dev(pr.src), dev(pr.strengths)
    m = pkg.Plan(KERNEL_S, (1.0, 1.0, 1.0), xi=28.0, tol=1e-5, precision=pkg.HSE_MIXED)
    prm = m.params
    d = pkg.Plan(KERNEL_S, (1.0, 1.0, 1.0), xi=prm["xi"], rc=prm["rc"], P=prm["P"], tol=0.0, M=prm["M"])
    try:
        _, f64 = d.eval_parts(src, st)
        u64 = host(d.eval(src, st))
        _, f32 = m.eval_parts(src, st)
        m.set_fft(pkg.HSE_FFT_DF64)
        _, fdf = m.eval_parts(src, st)
        u = host(m.eval(src, st))
    finally:
        m.close()
        d.close()
    urms = np.sqrt(np.mean(np.sum(u64 ** 2, axis=0)))
    e32 = np.sqrt(np.mean(np.sum((host(f32) - host(f64)) ** 2, axis=0))) / urms
    edf = np.sqrt(np.mean(np.sum((host(fdf) - host(f64)) ** 2, axis=0))) / urms
    print(f"Fourier part vs FP64, relative to |u|: FP32 grids {e32:.2e}, double-float grids {edf:.2e}")
    assert edf < 1e-8 and edf < e32 / 100
    idx = np.sort(np.random.default_rng(7).choice(n, 1500, replace=False))
    ref = oracle.direct(KERNEL_S, pr.src, pr.strengths, pr.src[:, idx])
    err = np.sqrt(np.mean(np.sum((u[:, idx] - ref) ** 2, axis=0))) / urms
    assert err < 1e-5
