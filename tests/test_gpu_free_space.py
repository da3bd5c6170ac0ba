"""Free-space variant (Sec. 2; kernel-mask bit HSE_FREE_SPACE) through the C
ABI against the oracle's free-space sums: spread grids and the real part to
FP64 rounding, the Fourier part to the numpy Alg. 1 (C1 at the sources, no
phi) and to the free-space smooth sum, full evaluations within tol, explicit
targets, mixed precision and batched instances."""
import numpy as np
import pytest

import oracle
from oracle import se_fourier as se
from workloads import KERNEL_S, KERNEL_T, KERNEL_W, problem

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FREE = oracle.FREE_SPACE
MASKS = [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W, KERNEL_S | KERNEL_T | KERNEL_W]


@pytest.fixture(scope="module")
def pkg():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1802_07844_gb300 as p
    assert p.HSE_FREE_SPACE == FREE
    return p


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("mask", MASKS)
def test_free_spread_grids(pkg, mask):
    pr = problem(mask, 150, 1.0, "uniform", 50)
    xi, M, P = 5.0, 14, 12
    plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=xi, rc=0.6, P=P, tol=0.0, M=M)
    g = host(plan.spread_grids(dev(pr.src), dev(pr.strengths)))
    h, Mt, _ = se.geometry(1.0, M, P, xi)
    ref = oracle.spread(mask | FREE, pr.src, pr.strengths, xi, h, P, Mt)
    assert g.shape == ref.shape
    assert float(np.abs(g - ref).max() / np.abs(ref).max()) < 1e-13
    plan.close()


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("prec", [0, 1])
def test_free_real_part(pkg, mask, prec):
    pr = problem(mask, 2000, 1.0, "near_wall", 51)
    xi, rc = 14.0, 0.3
    plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=xi, rc=rc, P=12, tol=0.0, M=40, precision=prec)
    if prec == 0:
        plan.set_rc64(rc)  # every pair in FP64: rounding-level parity
    ur, _ = plan.eval_parts(dev(pr.src), dev(pr.strengths))
    ref = (oracle.half_space_sum(mask | FREE, pr.src, pr.strengths, None, oracle.PART_REAL, xi, rc)
           + oracle.half_space_sum(mask | FREE, pr.src, pr.strengths, None, oracle.PART_SELF, xi))
    assert oracle.rel_rms(host(ur), ref) < (1e-13 if prec == 0 else 2e-6)
    plan.close()


@pytest.mark.parametrize("mask", MASKS)
def test_free_fourier_part(pkg, mask):
    pr = problem(mask, 300, 1.0, "uniform", 52)
    xi, M, P = 5.0, 16, 14
    plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=xi, rc=0.6, P=P, tol=0.0, M=M)
    _, uf = plan.eval_parts(dev(pr.src), dev(pr.strengths))
    assert plan.params["n_fft_out"] == 3
    ref = se.fourier_part(mask | FREE, pr.src, pr.strengths, xi, 1.0, M, P)
    assert oracle.rel_rms(host(uf), ref) < 1e-12
    plan.close()
    plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=8.0, rc=0.0, P=0, tol=1e-11)
    _, uf = plan.eval_parts(dev(pr.src), dev(pr.strengths))
    smooth = oracle.half_space_sum(mask | FREE, pr.src, pr.strengths, None, oracle.PART_SMOOTH, 8.0)
    assert oracle.rel_rms(host(uf), smooth) < 1e-10
    plan.close()


@pytest.mark.parametrize("mask", MASKS)
@pytest.mark.parametrize("dist", ["uniform", "near_wall"])
def test_free_full_eval(pkg, mask, dist):
    pr = problem(mask, 1500, 1.0, dist, 53)
    plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=9.0, rc=0.0, P=0, tol=1e-9)
    u = host(plan.eval(dev(pr.src), dev(pr.strengths)))
    ref = oracle.direct(mask | FREE, pr.src, pr.strengths)
    assert oracle.rel_rms(u, ref) < 1e-9
    # and it is not the half-space sum
    assert oracle.rel_rms(u, oracle.direct(mask, pr.src, pr.strengths)) > 1e-3
    plan.close()


def test_free_explicit_targets_and_mixed(pkg):
    mask = KERNEL_S | KERNEL_T | KERNEL_W
    pr = problem(mask, 3000, 1.0, "uniform", 54)
    rng = np.random.default_rng(55)
    tgt = np.stack([rng.uniform(0, 1, 700), rng.uniform(0, 1, 700), rng.uniform(0, 1, 700)])
    tgt[2, :10] = 0.0              # on the (absent) wall plane
    tgt[:, 10:30] = pr.src[:, :20]  # coincident with sources: pair skipped, self term added
    ref = oracle.direct(mask | FREE, pr.src, pr.strengths, tgt)
    for prec, tol in [(0, 1e-10), (1, 1e-5)]:
        plan = pkg.Plan(mask | FREE, (1.0, 1.0, 1.0), xi=12.0, rc=0.0, P=0, tol=tol, precision=prec)
        u = host(plan.eval(dev(pr.src), dev(pr.strengths), dev(tgt)))
        assert oracle.rel_rms(u, ref) < tol
        plan.close()


def test_free_batch(pkg):
    rng = np.random.default_rng(56)
    probs = []
    for i in range(16):
        mask = [KERNEL_S, KERNEL_T, KERNEL_W][i % 3] | FREE
        n = int(np.exp(rng.uniform(np.log(300), np.log(3000))))
        probs.append(problem(mask, n, 1.0, "uniform", 57, sub=i))
    items = [(p.mask, dev(p.src), dev(p.strengths)) for p in probs]
    b = pkg.hse.Batch(1e-8, 0)
    try:
        outs = [host(u) for u in b.eval(items)]
    finally:
        b.close()
    for p, u in zip(probs, outs):
        assert oracle.rel_rms(u, oracle.direct(p.mask, p.src, p.strengths)) < 1e-8
