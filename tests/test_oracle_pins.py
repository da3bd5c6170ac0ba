"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each test checks the oracle against mathematics or against statements of the
paper (arXiv 1802.07844): the no-slip condition the half-space formulas are
built to satisfy (Sec. 3), Blake's independent image system for a stokeslet
(Sec. 1, ref. JBlake1971), the derivative relations between singularities,
incompressibility, the Ewald identity of Sec. 4, the printed radial functions
of eq. (G_R) and the Appendix, the truncated-kernel transforms of Sec. 5.2,
spectral convergence of the Fourier part (Alg. 1) and the error estimates of
Tables 2-3 / the accuracy statement of Sec. 7.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from oracle import se_fourier as se
from workloads import KERNEL_S, KERNEL_T, KERNEL_W, problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(20240601)


# --------------------------------------------------------------------------
# independent closed forms (written here from the literature, not the oracle)
# --------------------------------------------------------------------------
def _s8(r, f):
    rn = np.linalg.norm(r)
    return f / rn + r * (r @ f) / rn ** 3


def blake(x, y, F):
    """Blake (1971): velocity (8 pi units, unit viscosity) of a stokeslet F at y
    above a no-slip wall z = 0:  S(r)F - S(R)F + 2 h D(R) F^I, R = x - y^I, with
    D_ik = d/dR_k [ h R_i/R^3 - (delta_i3/R + R_i R_3/R^3) ]."""
    h = y[2]
    r = x - y
    R = x - np.array([y[0], y[1], -y[2]])
    Rn = np.linalg.norm(R)
    D = np.zeros((3, 3))
    for i in range(3):
        for k in range(3):
            D[i, k] = (h * ((i == k) / Rn ** 3 - 3 * R[i] * R[k] / Rn ** 5) + (i == 2) * R[k] / Rn ** 3
                       - ((i == k) * R[2] + R[i] * (k == 2)) / Rn ** 3 + 3 * R[i] * R[2] * R[k] / Rn ** 5)
    FI = np.array([F[0], F[1], -F[2]])
    return _s8(r, F) - _s8(R, F) + 2 * h * D @ FI


def blake_dipole(x, y, g, q, step=1e-5):
    """D(g, q) = sum_k q_k d/dy_k [Blake velocity of force g at y] (central FD, Richardson)."""
    def d(hh):
        out = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = hh
            out += q[k] * (blake(x, y + e, g) - blake(x, y - e, g)) / (2 * hh)
        return out
    return (4 * d(step) - d(2 * step)) / 3


def _rand_targets(n, zlo=0.05, zhi=1.0):
    return np.stack([RNG.uniform(0, 1, n), RNG.uniform(0, 1, n), RNG.uniform(zlo, zhi, n)])


# --------------------------------------------------------------------------
# direct sum
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_T | KERNEL_W])
def test_no_slip_on_wall(mask):
    """Sec. 3: the representation satisfies u = 0 on the wall x3 = 0."""
    pr = problem(mask, 60, 1.0, "uniform", 11)
    wall = np.stack([RNG.uniform(0, 1, 40), RNG.uniform(0, 1, 40), np.zeros(40)])
    u_wall = oracle.direct(mask, pr.src, pr.strengths, wall)
    u_in = oracle.direct(mask, pr.src, pr.strengths, _rand_targets(40))
    assert np.abs(u_wall).max() <= 1e-13 * np.abs(u_in).max()


def test_no_slip_fails_with_printed_phi_T():
    """The stresslet correction as printed (coefficients 2, +2) leaves a wall
    residual; the reading used by the oracle (4, -4) removes it.  Checked on the
    wall trace of the image pair, independently of the oracle code."""
    g, q = RNG.standard_normal(3), RNG.standard_normal(3)
    y = np.array([0.3, 0.6, 0.25])
    x = np.array([0.7, 0.1, 0.0])
    yI = y * [1, 1, -1]
    gI, qI = g * [1, 1, -1], q * [1, 1, -1]
    r, rt = x - y, x - yI
    t8 = lambda v, a, b: -6 * v * (v @ a) * (v @ b) / np.linalg.norm(v) ** 5
    jump = t8(r, g, q) - t8(rt, gI, qI)  # normal component must be cancelled by phi
    rho = np.linalg.norm(rt)
    dG3 = -rt[2] / rho ** 3
    ddG = -np.eye(3) / rho ** 3 + 3 * np.outer(rt, rt) / rho ** 5
    h = y[2]
    printed = 2 * (2 * (gI @ qI) * dG3 + h * (gI @ ddG @ qI))
    reading = 4 * (gI @ qI) * dG3 - 4 * h * (gI @ ddG @ qI)
    assert abs(jump[0]) < 1e-14 and abs(jump[1]) < 1e-14
    assert abs(jump[2] + reading) < 1e-12 * abs(jump[2])
    assert abs(jump[2] + printed) > 1e-2 * abs(jump[2])


def test_blake_single_stokeslet():
    """Sec. 3 (Gimbutas form) agrees with Blake's image system for one stokeslet."""
    for trial in range(5):
        y = np.array([RNG.uniform(0, 1), RNG.uniform(0, 1), RNG.uniform(0.01, 1)])
        F = RNG.standard_normal(3)
        tg = _rand_targets(7, 0.0, 1.0)
        u = oracle.direct(KERNEL_S, y[:, None], F[:, None], tg)
        ub = np.stack([blake(tg[:, p], y, F) for p in range(tg.shape[1])], axis=1)
        assert oracle.rel_rms(u, ub) < 1e-13


def test_stokeslet_green_function_is_reciprocal():
    """Lorentz reciprocity of Stokes flow with a no-slip wall: the half-space
    stokeslet's Green's function satisfies G(x, y) = G(y, x)^T for any two
    points above the wall (a transposed index or a wrong sign in the image
    system breaks the symmetry)."""
    eye = np.eye(3)
    for trial in range(6):
        x = np.array([RNG.uniform(0, 1), RNG.uniform(0, 1), RNG.uniform(0.005, 0.6)])
        y = np.array([RNG.uniform(0, 1), RNG.uniform(0, 1), RNG.uniform(0.005, 0.6)])
        gxy = np.stack([oracle.direct(KERNEL_S, y[:, None], eye[:, j:j + 1], x[:, None])[:, 0] for j in range(3)],
                       axis=1)
        gyx = np.stack([oracle.direct(KERNEL_S, x[:, None], eye[:, j:j + 1], y[:, None])[:, 0] for j in range(3)],
                       axis=1)
        assert np.abs(gxy - gyx.T).max() < 1e-13 * np.abs(gxy).max()


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_T | KERNEL_W])
def test_invariant_under_shifts_parallel_to_the_wall(mask):
    """The half-space sums depend on x - y in the wall's plane and on the
    heights: shifting every source and target by (a1, a2, 0) leaves the
    velocities unchanged (a term using an absolute coordinate where a
    difference belongs breaks this)."""
    pr = problem(mask, 40, 1.0, "near_wall", 93)
    tg = _rand_targets(12, 0.0, 1.0)
    u = oracle.direct(mask, pr.src, pr.strengths, tg)
    shift = np.array([[0.37], [-0.21], [0.0]])
    us = oracle.direct(mask, pr.src + shift, pr.strengths, tg + shift)
    assert oracle.rel_rms(us, u) < 1e-13


@pytest.mark.parametrize("mask,degree", [(KERNEL_S, 1), (KERNEL_T, 2), (KERNEL_W, 2)])
def test_homogeneity_under_scaling(mask, degree):
    """Stokes flow has no length scale: with every position scaled by lam the
    stokeslet field scales by lam^-1 and the stresslet and rotlet fields by
    lam^-2 (their kernels have one more derivative), images and wall
    corrections included; the Ewald parts obey the same law with xi -> xi/lam
    (xi has units of inverse length).  A wrong power of r or a missing xi
    factor in any term breaks it."""
    pr = problem(mask, 30, 1.0, "near_wall", 94)
    tg = _rand_targets(9, 0.0, 1.0)
    lam, xi = 2.5, 7.0
    u = oracle.direct(mask, pr.src, pr.strengths, tg)
    us = oracle.direct(mask, lam * pr.src, pr.strengths, lam * tg)
    assert oracle.rel_rms(us * lam ** degree, u) < 1e-13
    for part in (oracle.PART_REAL, oracle.PART_SMOOTH):
        a = oracle.half_space_sum(mask, pr.src, pr.strengths, tg, part, xi, 0.0)
        b = oracle.half_space_sum(mask, lam * pr.src, pr.strengths, lam * tg, part, xi / lam, 0.0)
        assert oracle.rel_rms(b * lam ** degree, a) < 1e-12, part


def test_rotlet_from_blake_dipole():
    """Half-space rotlet = antisymmetric force dipole of the half-space stokeslet:
    W8 tau = -(D(g,q) - D(q,g)) with tau = g x q (W8 tau = 2 tau x r / r^3)."""
    for trial in range(4):
        y = np.array([RNG.uniform(0.2, 0.8), RNG.uniform(0.2, 0.8), RNG.uniform(0.05, 0.8)])
        g, q = RNG.standard_normal(3), RNG.standard_normal(3)
        tau = np.cross(g, q)
        tg = _rand_targets(5, 0.0, 1.0)
        u = oracle.direct(KERNEL_W, y[:, None], tau[:, None], tg)
        ref = np.stack([-(blake_dipole(tg[:, p], y, g, q) - blake_dipole(tg[:, p], y, q, g))
                        for p in range(tg.shape[1])], axis=1)
        assert oracle.rel_rms(u, ref) < 1e-7


def test_stresslet_from_blake_dipole():
    """Half-space stresslet with g perpendicular to q equals the symmetric force
    dipole of the half-space stokeslet: T8 (g x q) = -(D(g,q) + D(q,g)).  The
    traceless symmetric tensors are spanned by such pairs; the trace part is
    pinned by the no-slip and divergence tests."""
    for trial in range(4):
        y = np.array([RNG.uniform(0.2, 0.8), RNG.uniform(0.2, 0.8), RNG.uniform(0.05, 0.8)])
        g, q = RNG.standard_normal(3), RNG.standard_normal(3)
        q -= (q @ g) / (g @ g) * g
        st = np.concatenate([g, q])[:, None]
        tg = _rand_targets(5, 0.0, 1.0)
        u = oracle.direct(KERNEL_T, y[:, None], st, tg)
        ref = np.stack([-(blake_dipole(tg[:, p], y, g, q) + blake_dipole(tg[:, p], y, q, g))
                        for p in range(tg.shape[1])], axis=1)
        assert oracle.rel_rms(u, ref) < 1e-7


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W])
def test_divergence_free(mask):
    """Stokes flow is incompressible: Richardson-extrapolated central-difference
    divergence vanishes relative to the velocity gradient."""
    pr = problem(mask, 20, 1.0, "uniform", 12)
    x0 = _rand_targets(6, 0.1, 0.9)

    def div_at(hs):
        div = np.zeros(x0.shape[1])
        scale = np.zeros(x0.shape[1])
        for d in range(3):
            e = np.zeros((3, 1))
            e[d] = hs
            up = oracle.direct(mask, pr.src, pr.strengths, x0 + e)
            um = oracle.direct(mask, pr.src, pr.strengths, x0 - e)
            div += (up[d] - um[d]) / (2 * hs)
            scale += np.abs((up - um) / (2 * hs)).max(axis=0)
        return div, scale

    d1, scale = div_at(2e-4)
    d2, _ = div_at(4e-4)
    assert np.all(np.abs((4 * d1 - d2) / 3) < 1e-8 * scale)


# --------------------------------------------------------------------------
# free space (Sec. 2): the sums without the wall
# --------------------------------------------------------------------------
FREE = oracle.FREE_SPACE


def oseen_dipole(x, y, g, q, step=1e-5):
    """sum_k q_k d/dy_k [S8(x - y) g] (central FD, Richardson) -- the force
    dipole of the free-space stokeslet."""
    def d(hh):
        out = np.zeros(3)
        for k in range(3):
            e = np.zeros(3)
            e[k] = hh
            out += q[k] * (_s8(x - y - e, g) - _s8(x - y + e, g)) / (2 * hh)
        return out
    return (4 * d(step) - d(2 * step)) / 3


def test_free_space_stokeslet_is_oseen_tensor():
    """Sec. 2: the free-space stokeslet sum is the Oseen tensor S8(r) f summed
    over the other sources."""
    pr = problem(KERNEL_S, 12, 1.0, "uniform", 40)
    tg = _rand_targets(6, 0.0, 1.0)
    u = oracle.direct(KERNEL_S | FREE, pr.src, pr.strengths, tg)
    ref = np.zeros_like(u)
    for p in range(tg.shape[1]):
        for m in range(pr.src.shape[1]):
            ref[:, p] += _s8(tg[:, p] - pr.src[:, m], pr.strengths[:, m])
    assert oracle.rel_rms(u, ref) < 1e-14


def test_free_space_rotlet_and_stresslet_are_oseen_dipoles():
    """Free-space rotlet = antisymmetric and stresslet (g perpendicular to q) =
    symmetric force dipole of the Oseen tensor (finite differences in the
    source position)."""
    for trial in range(4):
        y = np.array([RNG.uniform(0.2, 0.8), RNG.uniform(0.2, 0.8), RNG.uniform(0.05, 0.8)])
        g, q = RNG.standard_normal(3), RNG.standard_normal(3)
        q -= (q @ g) / (g @ g) * g
        tg = _rand_targets(5, 0.0, 1.0)
        uw = oracle.direct(KERNEL_W | FREE, y[:, None], np.cross(g, q)[:, None], tg)
        ut = oracle.direct(KERNEL_T | FREE, y[:, None], np.concatenate([g, q])[:, None], tg)
        dgq = np.stack([oseen_dipole(tg[:, p], y, g, q) for p in range(tg.shape[1])], axis=1)
        dqg = np.stack([oseen_dipole(tg[:, p], y, q, g) for p in range(tg.shape[1])], axis=1)
        assert oracle.rel_rms(uw, -(dgq - dqg)) < 1e-7
        assert oracle.rel_rms(ut, -(dgq + dqg)) < 1e-7


@pytest.mark.parametrize("mask,order", [(KERNEL_S, 1), (KERNEL_T, 2), (KERNEL_W, 3)])
def test_free_space_is_far_wall_limit(mask, order):
    """Far from the wall the half-space sum (pinned above by no-slip and Blake)
    tends to the free-space sum: lifting every point by H leaves a difference
    O(H^-1) for the stokeslet (its image system decays like a stokeslet),
    O(H^-2) for the stresslet, and O(H^-3) for the rotlet (at O(H^-2) the image
    rotlet, -v/(2H^2) with v = (-tau2, tau1, 0), cancels the -x3 grad(phi_W)
    term, +v/(2H^2))."""
    pr = problem(mask, 40, 1.0, "uniform", 41)
    tg = _rand_targets(20, 0.0, 1.0)
    diffs = []
    for H in (1e2, 1e3):
        lift = np.array([[0.0], [0.0], [H]])
        uh = oracle.direct(mask, pr.src + lift, pr.strengths, tg + lift)
        uf = oracle.direct(mask | FREE, pr.src + lift, pr.strengths, tg + lift)
        diffs.append(oracle.rel_rms(uh, uf))
    ratio = diffs[0] / diffs[1]
    assert 10 ** order / 2 < ratio < 10 ** order * 2
    assert diffs[1] < 10.0 ** (-2 * order)


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W])
def test_free_space_divergence_free(mask):
    pr = problem(mask, 20, 1.0, "uniform", 42)
    x0 = _rand_targets(6, 0.1, 0.9)

    def div_at(hs):
        div = np.zeros(x0.shape[1])
        scale = np.zeros(x0.shape[1])
        for d in range(3):
            e = np.zeros((3, 1))
            e[d] = hs
            up = oracle.direct(mask | FREE, pr.src, pr.strengths, x0 + e)
            um = oracle.direct(mask | FREE, pr.src, pr.strengths, x0 - e)
            div += (up[d] - um[d]) / (2 * hs)
            scale += np.abs((up - um) / (2 * hs)).max(axis=0)
        return div, scale

    d1, scale = div_at(2e-4)
    d2, _ = div_at(4e-4)
    assert np.all(np.abs((4 * d1 - d2) / 3) < 1e-8 * scale)


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_T | KERNEL_W])
@pytest.mark.parametrize("xi", [2.5, 9.0])
def test_free_space_split_identity(mask, xi):
    """Sec. 4 for the free-space kernels: direct = real (no cut-off) + smooth + self."""
    pr = problem(mask, 80, 1.0, "uniform", 43)
    d = oracle.direct(mask | FREE, pr.src, pr.strengths)
    r, s, sf = oracle.ewald_split(mask | FREE, pr.src, pr.strengths, xi)
    assert oracle.rel_rms(r + s + sf, d) < 1e-13
    # the free-space parts differ from the half-space ones (images dropped)
    rh = oracle.ewald_split(mask, pr.src, pr.strengths, xi)[0]
    assert oracle.rel_rms(r, rh) > 1e-6


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W])
def test_free_space_fourier_part_converges_to_smooth_sum(mask):
    """Alg. 1 with C1 at the sources only (no images, no phi) computes the
    free-space smooth part: spectral convergence as k_inf/xi and P grow."""
    pr = problem(mask, 40, 1.0, "uniform", 44)
    xi = 4.0
    smooth = oracle.half_space_sum(mask | FREE, pr.src, pr.strengths, None, oracle.PART_SMOOTH, xi)
    errs = [oracle.rel_rms(se.fourier_part(mask | FREE, pr.src, pr.strengths, xi, 1.0, M, P), smooth)
            for M, P in [(12, 12), (16, 20)]]
    assert errs[0] < 2e-6
    assert errs[1] < 1e-10
    assert errs[1] < 1e-3 * errs[0]


# --------------------------------------------------------------------------
# Ewald split (Sec. 4, Appendix)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W])
@pytest.mark.parametrize("xi", [2.5, 9.0])
def test_split_identity(mask, xi):
    """Sec. 4: direct = real part (no cut-off) + smooth part + self term."""
    pr = problem(mask, 80, 1.0, "uniform", 13)
    d = oracle.direct(mask, pr.src, pr.strengths)
    r, s, sf = oracle.ewald_split(mask, pr.src, pr.strengths, xi)
    assert oracle.rel_rms(r + s + sf, d) < 1e-13


def test_split_identity_explicit_targets_with_coincident_points():
    """Explicit targets: pairs at exactly zero separation are dropped and get the self term."""
    pr = problem(KERNEL_S | KERNEL_W, 50, 1.0, "uniform", 14)
    tg = np.concatenate([pr.src[:, :10], _rand_targets(10, 0.0, 1.0)], axis=1)
    tg[2, -1] = 0.0
    d = oracle.direct(pr.mask, pr.src, pr.strengths, tg)
    r, s, sf = oracle.ewald_split(pr.mask, pr.src, pr.strengths, 5.0, 0.0, tg)
    assert oracle.rel_rms(r + s + sf, d) < 1e-13
    d_self = oracle.direct(pr.mask, pr.src, pr.strengths)
    assert np.allclose(d[:, :10], d_self[:, :10], rtol=1e-14, atol=0)


def test_self_term_value():
    """Appendix: the stokeslet self term is -4 xi/sqrt(pi) f; stresslet and rotlet have none."""
    pr = problem(KERNEL_S | KERNEL_T | KERNEL_W, 7, 1.0, "uniform", 15)
    xi = 3.3
    sf = oracle.half_space_sum(pr.mask, pr.src, pr.strengths, None, oracle.PART_SELF, xi)
    assert np.allclose(sf, -4 * xi / math.sqrt(math.pi) * pr.strengths[0:3], rtol=1e-15, atol=0)


def _paper_fprime(xi, r):
    """f = erf(xi r)/r and the derivatives printed in the Appendix (with exp(-xi^2 r^2))."""
    e = math.exp(-xi * xi * r * r)
    er = math.erf(xi * r)
    sp = math.sqrt(math.pi)
    f1 = 2 * xi * e / (sp * r) - er / r ** 2
    f2 = -4 * xi * e / (sp * r ** 2) - 4 * xi ** 3 * e / sp + 2 * er / r ** 3
    f3 = 4 * xi * e / (sp * r) * (3 / r ** 2 + 2 * xi ** 2 + 2 * xi ** 4 * r ** 2) - 6 * er / r ** 4
    return f1, f2, f3


@pytest.mark.parametrize("t", [0.5, 1.0, 1.7, 3.0])
def test_real_space_radial_functions_match_printed_forms(t):
    """Sec. 4 eq. (G_R): the oracle's erfc forms equal the printed brackets."""
    xi = 4.0
    r = t / xi
    f1, f2, f3 = _paper_fprime(xi, r)
    c = oracle.coefs(oracle.PART_REAL, xi, r)
    assert c["g0"] == pytest.approx(1 / r - math.erf(xi * r) / r, rel=1e-12)
    assert c["g1"] == pytest.approx(-(1 / r ** 3 + f1 / r), rel=1e-11)
    assert c["g2"] == pytest.approx(3 / r ** 5 + f1 / r ** 3 - f2 / r ** 2, rel=1e-10)
    assert c["g3"] == pytest.approx(-15 / r ** 7 - 3 * f1 / r ** 5 + 3 * f2 / r ** 4 - f3 / r ** 3, rel=1e-9)


def test_real_space_kernels_tend_to_plain_as_xi_vanishes():
    """Appendix: S^R, T^R, W^R and G_R reduce to the plain kernels as xi -> 0."""
    r = 0.37
    plain = oracle.coefs(oracle.PART_DIRECT, 0.0, r)
    real = oracle.coefs(oracle.PART_REAL, 1e-9, r)
    for k in plain:
        assert real[k] == pytest.approx(plain[k], rel=1e-8, abs=1e-12)


def test_smooth_functions_series_and_closed_forms_agree_and_differentiate():
    """F(s) = erf(xi sqrt s)/sqrt s: series (xi r < 1) and closed forms (xi r >= 1)
    join continuously, and F', F'', F''' are derivatives of F (central FD)."""
    xi = 3.0
    s_edge = 1.0 / xi ** 2
    lo = oracle.fsmooth(xi, s_edge * (1 - 1e-12))
    hi = oracle.fsmooth(xi, s_edge)
    assert np.allclose(lo, hi, rtol=1e-11)
    for s in [0.01, 0.05, 0.2, 0.6]:
        ds = 1e-5 * s
        Fp, Fm = oracle.fsmooth(xi, s + ds), oracle.fsmooth(xi, s - ds)
        F0 = oracle.fsmooth(xi, s)
        for k in range(3):
            assert (Fp[k] - Fm[k]) / (2 * ds) == pytest.approx(F0[k + 1], rel=1e-7, abs=1e-9 * abs(F0[k]))
    assert oracle.fsmooth(xi, 0.0)[0] == pytest.approx(2 * xi / math.sqrt(math.pi), rel=1e-15)


@pytest.mark.parametrize("kernel,mask", [("stokeslet", KERNEL_S), ("stresslet", KERNEL_T), ("rotlet", KERNEL_W)])
def test_real_space_truncation_error_within_table3_estimate(kernel, mask):
    """Sec. 6, Table 3 and Fig. 3 (N=2000, L=3, xi=4.67): the measured real-space
    truncation error of the half-space sum agrees with the free-space estimate
    with Q counting sources and images (the paper's half-space estimate adds a
    correction-term contribution it does not print, so agreement is checked
    within a band: at or below it for the stokeslet and stresslet, within a
    small factor for the rotlet)."""
    cfg = json.load(open(os.path.join(GOLDEN, "paper_error_experiments.json")))["real_experiment"]
    L, xi = cfg["L"], cfg["xi"]
    n = cfg["N"]
    pr = problem(mask, n, L, "uniform", 16)
    exact = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_REAL, xi, 0.0)
    g = pr.strengths[0:3]
    q = pr.strengths[3:6] if mask == KERNEL_T else None
    if mask == KERNEL_S:
        Q = np.sum(g ** 2)
    elif mask == KERNEL_T:
        Q = sum(np.sum((g[i] * q[j]) ** 2) for i in range(3) for j in range(3))
    else:
        Q = np.sum(g ** 2)
    Q *= 2.0  # sources and their images
    for rc in [0.35, 0.5, 0.65]:
        cut = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_REAL, xi, rc)
        err = np.sqrt(np.mean(np.sum((cut - exact) ** 2, axis=0)))
        e = math.exp(-xi * xi * rc * rc)
        if mask == KERNEL_S:
            est = math.sqrt(4 * Q * rc / L ** 3) * e
        elif mask == KERNEL_T:
            est = math.sqrt(112 * Q * xi ** 4 * rc ** 3 / (9 * L ** 3)) * e
        else:
            est = math.sqrt(8 * Q / (3 * L ** 3 * rc)) * e
        if mask == KERNEL_W:
            assert 0.3 * est < err < 3.5 * est
        else:
            assert 0.3 * est < err < 1.2 * est


@pytest.mark.parametrize("kernel,mask", [("stokeslet", KERNEL_S), ("stresslet", KERNEL_T), ("rotlet", KERNEL_W)])
def test_fourier_truncation_error_against_table2_estimate(kernel, mask):
    """Sec. 6, Table 2 and Fig. 2 (L = 3, xi = 3.49, k_inf = pi M / L): the
    measured Fourier-space truncation error of the half-space sum lies below
    the free-space estimate (Q over sources and images) for the stokeslet and
    stresslet, and close to it for the rotlet, whose neglected correction terms
    decay at the kernel's own rate.

    The truncation error alone is isolated as the paper prescribes (approximation
    errors made negligible): Alg. 1 runs on a fine grid (M = 37, P = 24, whose
    own error is ~1e-15 of the field) and the scaled spectra are cut at k_inf =
    pi M / L for the coarser M (modes with some |k_d| >= k_inf dropped, the cube
    a grid of M points resolves).  The exact Fourier part is the smooth sum
    K - K_R over all pairs (``PART_SMOOTH``).  N = 2000 sources keeps the CPU
    time down; the ratio error / estimate does not depend on N (both scale as
    sqrt(Q))."""
    cfg = json.load(open(os.path.join(GOLDEN, "paper_error_experiments.json")))["fourier_experiment"]
    L, xi = cfg["L"], cfg["xi"]
    Ms = [14, 20, 26]
    assert all(cfg["M_range"][0] <= M <= cfg["M_range"][1] for M in Ms)
    P, M_fine = 24, 37
    pr = problem(mask, 2000, L, "uniform", 18)
    u = oracle.direct(mask, pr.src, pr.strengths)
    exact = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_SMOOTH, xi, 0.0)
    rms = math.sqrt(np.mean(np.sum(u ** 2, axis=0)))
    g = pr.strengths[0:3]
    if mask == KERNEL_T:
        q = pr.strengths[3:6]
        Q = sum(np.sum((g[i] * q[j]) ** 2) for i in range(3) for j in range(3))
    else:
        Q = np.sum(g ** 2)  # the rotlet strength is tau = g x q itself
    Q *= 2.0  # sources and their images
    h, Mt, _ = se.geometry(L, M_fine, P, xi)
    R = math.sqrt(6.0) * Mt * h  # truncation radius of the kernels actually used
    res = se.fourier_part(mask, pr.src, pr.strengths, xi, L, M_fine, P, kmax=[math.pi * M / L for M in Ms])
    prev = np.inf
    for M, uf in zip(Ms, res):
        err = math.sqrt(np.mean(np.sum((uf - exact) ** 2, axis=0)))
        k = math.pi * M / L
        e = math.exp(-k * k / (4 * xi * xi))
        if mask == KERNEL_S:
            est = math.sqrt(Q) * R * k ** 3 / (xi ** 2 * math.pi * L) * e
        elif mask == KERNEL_T:
            est = math.sqrt(7 * Q / 6) * R * k ** 4 / (xi ** 2 * math.pi * L) * e
        else:
            est = math.sqrt(8 * xi ** 2 * Q / (3 * math.pi * L ** 3 * k)) * e
        print(f"Fig. 2 replay {kernel} M {M}: relative error {err / rms:.3e}, estimate {est / rms:.3e}")
        assert err < prev  # decreasing in k_inf
        prev = err
        if mask == KERNEL_W:
            assert 0.3 * est < err < 3.5 * est
        else:
            assert err < est


# --------------------------------------------------------------------------
# Fourier part (Sec. 5.2, Alg. 1)
# --------------------------------------------------------------------------
def test_truncated_kernel_transforms_by_quadrature():
    """Sec. 5.2: H^R and (corrected) B^R are the transforms of (1/r) 1{r<R} and r 1{r<R}."""
    from scipy.integrate import quad
    R = 2.3
    for k in [1e-4, 0.01, 0.3, 0.7, 3.1, 11.0]:
        hq = 4 * math.pi / k * quad(lambda r: math.sin(k * r), 0, R, limit=200)[0]
        bq = 4 * math.pi / k * quad(lambda r: r * r * math.sin(k * r), 0, R, limit=200)[0]
        assert se.h_trunc(np.array([k]), R)[0] == pytest.approx(hq, rel=1e-9)
        assert se.b_trunc(np.array([k]), R)[0] == pytest.approx(bq, rel=1e-9)
    assert se.b_trunc(np.array([0.0]), R)[0] == pytest.approx(math.pi * R ** 4, rel=1e-15)
    assert se.h_trunc(np.array([0.0]), R)[0] == pytest.approx(2 * math.pi * R ** 2, rel=1e-15)


def test_spread_grid_moments():
    """Alg. 1 step 5: each truncated Gaussian carries unit mass (h^3 sum) up to
    its truncation error, and is centred on its point."""
    xi, M, P = 4.0, 14, 16
    h, Mt, eta = se.geometry(1.0, M, P, xi)
    pr = problem(KERNEL_S, 1, 1.0, "uniform", 17)
    g = oracle.spread(KERNEL_S, pr.src, pr.strengths, xi, h, P, Mt)
    f = pr.strengths[:, 0]
    y = pr.src[:, 0]
    mass_c2 = h ** 3 * g[3].sum()  # C2 = f3 at the image point
    assert mass_c2 == pytest.approx(f[2], rel=1e-9)
    ox, oz = -0.5 * P * h, -Mt * h
    zc = oz + np.arange(2 * Mt) * h
    xc = ox + np.arange(Mt) * h
    wz = h ** 3 * g[3].sum(axis=(0, 1))
    wx = h ** 3 * g[3].sum(axis=(1, 2))
    assert (wz @ zc) / wz.sum() == pytest.approx(-y[2], abs=1e-9)
    assert (wx @ xc) / wx.sum() == pytest.approx(y[0], abs=1e-9)
    # C1 x-component: source and (negated) image masses cancel; z-components add
    assert h ** 3 * g[0].sum() == pytest.approx(0.0, abs=1e-9)
    assert h ** 3 * g[2].sum() == pytest.approx(2 * f[2], rel=1e-9)


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W])
def test_fourier_part_converges_to_smooth_sum(mask):
    """Alg. 1 computes the smooth part of the split: spectral convergence to the
    erf-screened direct sum (an independent real-space computation) as k_inf/xi
    and P grow together."""
    pr = problem(mask, 40, 1.0, "uniform", 3)
    xi = 4.0
    smooth = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_SMOOTH, xi)
    errs = [oracle.rel_rms(se.fourier_part(mask, pr.src, pr.strengths, xi, 1.0, M, P), smooth)
            for M, P in [(12, 12), (16, 20)]]
    assert errs[0] < 2e-6
    assert errs[1] < 1e-10
    assert errs[1] < 1e-3 * errs[0]


@pytest.mark.slow
def test_paper_parameters_reach_stated_accuracy():
    """Sec. 7: with P = 16 and the paper's (xi, r_c, M/L) at density 2500 the
    relative RMS error stays below 0.5e-8 (checked at L = 1, N = 2500)."""
    cfg = json.load(open(os.path.join(GOLDEN, "paper_parameters.json")))
    masks = {"stokeslet": KERNEL_S, "stresslet": KERNEL_T, "rotlet": KERNEL_W}
    L = 1.0
    n = int(cfg["density"] * L ** 3)
    for name, p in cfg["kernels"].items():
        mask = masks[name]
        pr = problem(mask, n, L, "uniform", 18)
        d = oracle.direct(mask, pr.src, pr.strengths)
        real = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_REAL, p["xi"], p["rc"])
        sf = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_SELF, p["xi"])
        uf = se.fourier_part(mask, pr.src, pr.strengths, p["xi"], L, int(p["M_over_L"] * L), cfg["P"])
        assert oracle.rel_rms(real + uf + sf, d) < cfg["rel_rms_bound"], name


# --------------------------------------------------------------------------
# cell lists (Sec. 5.1)
# --------------------------------------------------------------------------
def test_cells_invariants():
    pr = problem(KERNEL_S, 3000, 1.0, "near_wall", 19)
    ncell = np.array([7, 6, 9], np.int32)
    origin = np.zeros(3)
    inv = ncell / 1.0
    cid, perm, start = oracle.cells(pr.src, origin, inv, ncell)
    assert sorted(perm.tolist()) == list(range(3000))
    assert np.all(np.diff(start) >= 0) and start[0] == 0 and start[-1] == 3000
    c = np.stack([cid % 7, (cid // 7) % 6, cid // 42])
    lo = c / inv[:, None]
    hi = (c + 1) / inv[:, None]
    assert np.all(pr.src >= lo - 1e-15) and np.all(pr.src <= hi + 1e-15)
    for k in range(len(start) - 1):
        seg = perm[start[k]:start[k + 1]]
        assert np.all(cid[seg] == k)
        assert np.all(np.diff(seg) > 0)  # stable: original index order inside a cell


def test_neighbor_counts_vs_kdtree():
    from scipy.spatial import cKDTree
    pr = problem(KERNEL_S, 1500, 1.0, "near_wall", 20)
    rc = 0.08
    a, b = oracle.neighbor_counts(pr.src, rc)
    pts = pr.src.T
    tree = cKDTree(pts)
    pairs = tree.query_pairs(rc, output_type="ndarray")
    cnt = np.bincount(pairs.ravel(), minlength=1500)
    assert np.array_equal(a, cnt)
    imgs = pts * [1, 1, -1]
    cnt_i = np.array([len(x) for x in cKDTree(imgs).query_ball_point(pts, rc)])
    assert np.array_equal(b, cnt_i)


@pytest.mark.parametrize("mask", [KERNEL_S, KERNEL_T, KERNEL_W, KERNEL_S | KERNEL_W])
def test_fourier_derivative_variant_converges_to_smooth_sum(mask):
    """The derivative variant of Alg. 1 (harmonic potential spread as one scalar
    grid through window derivatives, grad(phi) gathered with the window's
    gradient) computes the same smooth part: spectral convergence to the smooth
    sum, and agreement with the paper's C2/C3/T2 route to well below the
    truncation error of either."""
    pr = problem(mask, 40, 1.0, "uniform", 3)
    xi = 4.0
    smooth = oracle.half_space_sum(mask, pr.src, pr.strengths, None, oracle.PART_SMOOTH, xi)
    errs, diffs = [], []
    for M, P in [(12, 12), (16, 20)]:
        a = se.fourier_part(mask, pr.src, pr.strengths, xi, 1.0, M, P)
        b = se.fourier_part_derivative(mask, pr.src, pr.strengths, xi, 1.0, M, P)
        errs.append(oracle.rel_rms(b, smooth))
        diffs.append(oracle.rel_rms(b, a))
    # at the coarse grid the two discretisations differ by about their error
    assert errs[0] < 5e-6
    assert diffs[0] < 3 * errs[0]
    assert errs[1] < 1e-10
    assert diffs[1] < 1e-10


def test_fourier_derivative_variant_free_space_is_alg1():
    """Without a wall there is no potential: the variant is Alg. 1 itself."""
    pr = problem(KERNEL_S | KERNEL_W, 30, 1.0, "uniform", 45)
    m = KERNEL_S | KERNEL_W | FREE
    a = se.fourier_part(m, pr.src, pr.strengths, 4.0, 1.0, 12, 12)
    b = se.fourier_part_derivative(m, pr.src, pr.strengths, 4.0, 1.0, 12, 12)
    assert oracle.rel_rms(b, a) < 1e-14
