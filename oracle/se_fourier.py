"""Numpy restatement of the Fourier-space part of the half-space Spectral Ewald
method (Alg. 1 of arXiv 1802.07844 and the precomputation of Sec. 5.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Slow and memory
hungry: meant for grids of a few tens of points per side.

Steps, in the paper's order:
  2-3  extended domain [0, L~) x [0, L~) x [-L~, L~), L~ = L + P h, grid of
       Mt x Mt x 2 Mt points, Mt = M + P;
  4    eta = P xi^2 h^2 / (c^2 pi), c = 0.95;
  5    spread C1 (2N points), C2, C3 (N image points) -- ``oracle.spread``;
  6    FFT zero-padded by 2 in every direction;
  7    truncated kernels H^R, B^R (R = sqrt(6) L~) sampled on a grid refined
       by s_f >= 1 + sqrt(6) in k, inverse-transformed, truncated to the
       padded box and transformed back (the three precomputation steps);
  8    multiply by A(k, xi) K^R(k) exp(-(1 - eta) k^2 / 4 xi^2);
  9    inverse FFT and truncation to the Mt x Mt x 2 Mt grid, giving T1, T2;
  10   trapezoidal quadrature with the same truncated Gaussian at each target:
       u_F = <T1> - x3 <T2>.

Free space (Sec. 2, mask bit FREE_SPACE): C1 is spread at the sources only,
there is no harmonic potential (phi = 0, T2 = 0), and u_F = <T1>.

Readings of the paper used here:
  * Continuous transform pair K^(k) = int K e^{-ik.x} dx; gradients map to i k.
    Then A^W = -2 i eps k (the printed +2 i eps k has the opposite sign to the
    printed W^R) and the harmonic corrections (Sec. 3) transform to
      phi^_S = 2 G^(-C2^ - i k.C3^),  phi^_T = G^(4 i k3 C2^ + 4 k C3^ k),
      phi^_W = 4 G^ i k.C2^,
    with G^ = H^R exp(-(1-eta) k^2/4xi^2); T1^ = K^ C1^ + e3 phi^,
    T2^ = i k phi^ (Sec. 5.2, eq. uF_stokeslet).
  * Quadrature weight h^3 with the unnormalised forward DFT; no extra
    (2 pi)^-3 factor (the printed one belongs to the continuous integral).
  * B^R(k) = 4 pi [(2 - R^2 k^2) cos Rk + 2 R k sin Rk - 2] / k^4, the
    transform of r 1{r < R} (the printed "R^2 k sin(R^2 k)" is a misprint);
    Taylor series 4 pi R^4 sum_n (-1)^n (Rk)^{2n} / ((2n+1)! (2n+4)) for Rk < 1.
  * Modes at the Nyquist index of any padded dimension are set to zero.
"""
from __future__ import annotations

import math

import numpy as np

from . import FREE_SPACE, KERNEL_S, KERNEL_T, KERNEL_W, spread

C_WINDOW = 0.95


def h_trunc(k, R):
    """H^R(k) = 8 pi (sin(R k / 2) / k)^2, the transform of (1/r) 1{r < R}."""
    k = np.asarray(k, np.float64)
    x = 0.5 * R * k
    sinc = np.where(x == 0.0, 1.0, np.sin(x) / np.where(x == 0.0, 1.0, x))
    return 8.0 * np.pi * (0.5 * R) ** 2 * sinc ** 2


def b_trunc(k, R):
    """B^R(k), the transform of r 1{r < R} (Sec. 5.2, corrected)."""
    k = np.asarray(k, np.float64)
    t = R * k
    out = np.empty_like(t)
    small = t < 1.0
    ts = t[small]
    ser = np.zeros_like(ts)
    for n in range(25):
        ser += (-1) ** n * ts ** (2 * n) / (math.factorial(2 * n + 1) * (2 * n + 4))
    out[small] = 4.0 * np.pi * R ** 4 * ser
    tl = t[~small]
    kl = k[~small]
    out[~small] = 4.0 * np.pi * ((2.0 - tl ** 2) * np.cos(tl) + 2.0 * tl * np.sin(tl) - 2.0) / kl ** 4
    return out


def geometry(L, M, P, xi):
    h = L / M
    Mt = M + P
    eta = P * xi ** 2 * h ** 2 / (C_WINDOW ** 2 * np.pi)
    return h, Mt, eta


def precompute_table(kind, Mt, h):
    """Truncated-kernel table on the 2x padded grid (Sec. 5.2, three steps).

    kind: 'H' or 'B'.  Returns the (2Mt, 2Mt, 4Mt) array of K^R values in numpy
    FFT order (real)."""
    Lt = Mt * h
    R = math.sqrt(6.0) * Lt
    nf = int(math.ceil((1.0 + math.sqrt(6.0)) * Mt))
    if nf % 2:
        nf += 1  # s_f Mt must be even
    shape_f = (nf, nf, 2 * nf)
    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape_f]
    KX, KY, KZ = np.meshgrid(*ks, indexing="ij")
    kabs = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    del KX, KY, KZ
    Khat = h_trunc(kabs, R) if kind == "H" else b_trunc(kabs, R)
    del kabs
    # step 2: inverse transform -> real-space values (the h^3 factors cancel)
    Kr = np.fft.ifftn(Khat)
    del Khat
    # truncate to the padded box: x, y in [-Mt, Mt), z in [-2Mt, 2Mt)
    pad = (2 * Mt, 2 * Mt, 4 * Mt)
    box = np.zeros(pad, np.complex128)
    idx = [np.r_[0:p // 2, n - p // 2:n] for p, n in zip(pad, shape_f)]
    dst = [np.r_[0:p // 2, p - p // 2:p] for p in pad]
    box[np.ix_(*dst)] = Kr[np.ix_(*idx)]
    # step 3: transform back on the padded grid
    return np.real(np.fft.fftn(box))


def _sym(c6):
    """6 stored components xx xy xz yy yz zz -> full 3x3 (symmetric)."""
    xx, xy, xz, yy, yz, zz = c6
    return [[xx, xy, xz], [xy, yy, yz], [xz, yz, zz]]


def fourier_part(mask, src, strengths, xi, L, M, P, tgt=None, kmax=None):
    """u_F at the targets (targets = sources when ``tgt`` is None).

    kmax: optional wave-number cut-off(s) k_inf (Sec. 6): the scaled spectra
    are zeroed wherever some |k_d| >= k_inf before the inverse transform,
    i.e. the Fourier integral is truncated to the cube a grid of spacing
    h = pi / k_inf resolves, while the discretisation (grid, window, P) stays
    that of (M, P).  A sequence of cut-offs returns one result per cut-off."""
    src = np.ascontiguousarray(src, np.float64)
    h, Mt, eta = geometry(L, M, P, xi)
    if not (0.0 < eta < 1.0):
        raise ValueError("eta must lie in (0, 1)")
    grids = spread(mask, src, strengths, xi, h, P, Mt)
    pad = (2 * Mt, 2 * Mt, 4 * Mt)
    Np = pad[0] * pad[1] * pad[2]

    def fft_pad(g):
        buf = np.zeros(pad)
        buf[:Mt, :Mt, :2 * Mt] = g
        return np.fft.fftn(buf)

    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in pad]
    K = np.meshgrid(*ks, indexing="ij")
    k2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    nyq = np.zeros(pad, bool)
    for d, n in enumerate(pad):
        sl = [slice(None)] * 3
        sl[d] = n // 2
        nyq[tuple(sl)] = True
    E = np.exp(-(1.0 - eta) * k2 / (4.0 * xi ** 2))
    s_fac = 1.0 + k2 / (4.0 * xi ** 2)
    TH = precompute_table("H", Mt, h)
    TB = precompute_table("B", Mt, h) if mask & (KERNEL_S | KERNEL_T) else None
    GF = E * TH  # G^ with the remaining screening

    T1 = [np.zeros(pad, np.complex128) for _ in range(3)]
    phi = np.zeros(pad, np.complex128)
    free = bool(mask & FREE_SPACE)  # Sec. 2: C1 at the sources only, no phi
    c = 0
    if mask & KERNEL_S:
        C1 = [fft_pad(grids[c + i]) for i in range(3)]
        kC1 = sum(K[i] * C1[i] for i in range(3))
        for j in range(3):  # A^S = -(k^2 I - k k)(1 + k^2/4xi^2)
            T1[j] += -s_fac * E * TB * (k2 * C1[j] - K[j] * kC1)
        if free:
            c += 3
        else:
            C2 = fft_pad(grids[c + 3])
            C3 = [fft_pad(grids[c + 4 + i]) for i in range(3)]
            c += 7
            phi += 2.0 * GF * (-C2 - 1j * sum(K[i] * C3[i] for i in range(3)))
    if mask & KERNEL_T:
        C1 = _sym([fft_pad(grids[c + i]) for i in range(6)])
        # A^T_jlm C_lm = -i (1 + k^2/4xi^2) [ (k_m d_jl + k_j d_lm + k_l d_mj) k^2 - 2 k_j k_l k_m ] C_lm
        trC = C1[0][0] + C1[1][1] + C1[2][2]
        Ck = [sum(C1[j][m] * K[m] for m in range(3)) for j in range(3)]
        kCk = sum(K[j] * Ck[j] for j in range(3))
        for j in range(3):
            T1[j] += -1j * s_fac * E * TB * (k2 * (2.0 * Ck[j] + K[j] * trC) - 2.0 * K[j] * kCk)
        if free:
            c += 6
        else:
            C2 = fft_pad(grids[c + 6])
            C3 = _sym([fft_pad(grids[c + 7 + i]) for i in range(6)])
            c += 13
            kC3k = sum(K[j] * C3[j][m] * K[m] for j in range(3) for m in range(3))
            phi += GF * (4j * K[2] * C2 + 4.0 * kC3k)
    if mask & KERNEL_W:
        C1 = [fft_pad(grids[c + i]) for i in range(3)]
        # A^W_jl = -2 i eps_jlm k_m :  (A^W C)_j = -2 i (C x k)_j
        cross = [C1[1] * K[2] - C1[2] * K[1], C1[2] * K[0] - C1[0] * K[2], C1[0] * K[1] - C1[1] * K[0]]
        for j in range(3):
            T1[j] += -2j * E * TH * cross[j]
        if free:
            c += 3
        else:
            C2 = [fft_pad(grids[c + 3 + i]) for i in range(2)]
            c += 5
            phi += 4.0 * GF * 1j * (K[0] * C2[0] + K[1] * C2[1])
    T1[2] = T1[2] + phi
    T2 = [1j * K[j] * phi for j in range(3)]
    tg = src if tgt is None else np.ascontiguousarray(tgt, np.float64)
    cuts = [None] if kmax is None else (list(kmax) if np.ndim(kmax) else [kmax])
    results = []
    for kc in cuts:
        drop = nyq if kc is None else (nyq | (np.abs(K[0]) >= kc) | (np.abs(K[1]) >= kc) | (np.abs(K[2]) >= kc))
        fields = [np.real(np.fft.ifftn(np.where(drop, 0.0, F)))[:Mt, :Mt, :2 * Mt] for F in T1 + T2]
        # step 10: quadrature at the targets with the same truncated Gaussian
        results.append(gather(fields, tg, xi, h, P, Mt, eta))
    del T1, T2
    return results if (kmax is not None and np.ndim(kmax)) else results[0]


def _support(c, o, h, P, n):
    i0 = int(math.floor((c - o) / h)) - P // 2 + 1
    return min(max(i0, 0), n - P)


def gather(fields, tgt, xi, h, P, Mt, eta):
    """u_F(x) = h^3 sum_j W(x - x_j) (T1(x_j) - x3 T2(x_j)) over the P^3 support."""
    pre = (2.0 * xi ** 2 / (np.pi * eta)) ** 1.5
    ox, oz = -0.5 * P * h, -Mt * h
    nt = tgt.shape[1]
    out = np.zeros((3, nt))
    for p in range(nt):
        x = tgt[:, p]
        i0 = _support(x[0], ox, h, P, Mt)
        j0 = _support(x[1], ox, h, P, Mt)
        k0 = _support(x[2], oz, h, P, 2 * Mt)
        gx = ox + (i0 + np.arange(P)) * h
        gy = ox + (j0 + np.arange(P)) * h
        gz = oz + (k0 + np.arange(P)) * h
        d2 = ((gx[:, None, None] - x[0]) ** 2 + (gy[None, :, None] - x[1]) ** 2
              + (gz[None, None, :] - x[2]) ** 2)
        w = pre * np.exp(-2.0 * xi ** 2 * d2 / eta) * h ** 3
        sl = (slice(i0, i0 + P), slice(j0, j0 + P), slice(k0, k0 + P))
        for d in range(3):
            out[d, p] = np.sum(w * fields[d][sl]) - x[2] * np.sum(w * fields[3 + d][sl])
    return out


# ---------------------------------------------------------------------------
# Variant with the wall corrections spread and gathered through window
# derivatives.  In the continuous method i k C^ is the transform of the
# divergence of the smeared field and k k C^ that of minus its second
# derivatives, so the harmonic potential can be spread as ONE scalar grid
#   D(x) = sum_images [ cs W + cv . grad W - ct : grad grad W ](x - y^I)
# with phi^ = G^ D^ (G^ = E H^R), and the gather of T2 = grad phi can use
# the window's gradient on the phi grid instead:  <grad phi>(x) =
# h^3 sum_j grad_x W(x - x_j) phi_j.  Both are the same integrals as Alg. 1's
# C2/C3 and T2 terms, discretised differently; they agree to the truncation
# error of the window (tests pin both against the smooth sum).
#   stokeslet: cs = -2 f3, cv = -2 y3 f^I           (phi_S = 2 G (-C2 - i k.C3))
#   stresslet: cv = (0, 0, 4 g.q), ct = 4 y3 sym(g^I q^I)
#                                                   (phi_T = G (4 i k3 C2 + 4 k C3 k))
#   rotlet:    cv = 4 (-tau2, tau1, 0)              (phi_W = 4 G i k.C2)
# ---------------------------------------------------------------------------
def _window(c, o, h, P, n, alpha):
    i0 = _support(c, o, h, P, n)
    d = o + (i0 + np.arange(P)) * h - c
    w = np.exp(-alpha * d * d)
    return i0, w, -2.0 * alpha * d * w, (4.0 * alpha * alpha * d * d - 2.0 * alpha) * w


def _correction_grid(mask, src, strengths, xi, h, P, Mt, eta):
    alpha = 2.0 * xi ** 2 / eta
    pre = (2.0 * xi ** 2 / (np.pi * eta)) ** 1.5
    ox, oz = -0.5 * P * h, -Mt * h
    D = np.zeros((Mt, Mt, 2 * Mt))
    n = src.shape[1]
    ia, ib = [0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]
    for m in range(n):
        y = src[:, m]
        yI = np.array([y[0], y[1], -y[2]])
        row = 0
        cs, cv, ct = 0.0, np.zeros(3), np.zeros(6)
        if mask & KERNEL_S:
            f = strengths[row:row + 3, m]
            row += 3
            cs += -2.0 * f[2]
            cv += -2.0 * y[2] * np.array([f[0], f[1], -f[2]])
        if mask & KERNEL_T:
            g, q = strengths[row:row + 3, m], strengths[row + 3:row + 6, m]
            row += 6
            gI, qI = g * [1, 1, -1], q * [1, 1, -1]
            cv[2] += 4.0 * (gI @ qI)
            ct += 4.0 * y[2] * np.array([0.5 * (gI[ia[c]] * qI[ib[c]] + gI[ib[c]] * qI[ia[c]]) for c in range(6)])
        if mask & KERNEL_W:
            tau = strengths[row:row + 3, m]
            cv += 4.0 * np.array([-tau[1], tau[0], 0.0])
        ix, wx, dx, ddx = _window(yI[0], ox, h, P, Mt, alpha)
        iy, wy, dy, ddy = _window(yI[1], ox, h, P, Mt, alpha)
        iz, wz, dz, ddz = _window(yI[2], oz, h, P, 2 * Mt, alpha)
        fac = [(wx, dx, ddx), (wy, dy, ddy), (wz, dz, ddz)]

        def term(ox_, oy_, oz_):
            return np.einsum('i,j,k->ijk', fac[0][ox_], fac[1][oy_], fac[2][oz_])
        blk = cs * term(0, 0, 0) + cv[0] * term(1, 0, 0) + cv[1] * term(0, 1, 0) + cv[2] * term(0, 0, 1)
        for c in range(6):
            o = [0, 0, 0]
            o[ia[c]] += 1
            o[ib[c]] += 1
            blk -= (1.0 if ia[c] == ib[c] else 2.0) * ct[c] * term(*o)
        D[ix:ix + P, iy:iy + P, iz:iz + P] += pre * blk
    return D


def fourier_part_derivative(mask, src, strengths, xi, L, M, P, tgt=None):
    """u_F at the targets by the derivative variant (see above): C1 as in Alg.
    1, the harmonic potential from one spread grid D, T2 never formed."""
    src = np.ascontiguousarray(src, np.float64)
    h, Mt, eta = geometry(L, M, P, xi)
    if not (0.0 < eta < 1.0):
        raise ValueError("eta must lie in (0, 1)")
    free = bool(mask & FREE_SPACE)
    grids = spread(mask, src, strengths, xi, h, P, Mt)
    pad = (2 * Mt, 2 * Mt, 4 * Mt)

    def fft_pad(g):
        buf = np.zeros(pad)
        buf[:Mt, :Mt, :2 * Mt] = g
        return np.fft.fftn(buf)

    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in pad]
    K = np.meshgrid(*ks, indexing="ij")
    k2 = K[0] ** 2 + K[1] ** 2 + K[2] ** 2
    nyq = np.zeros(pad, bool)
    for d, n in enumerate(pad):
        sl = [slice(None)] * 3
        sl[d] = n // 2
        nyq[tuple(sl)] = True
    E = np.exp(-(1.0 - eta) * k2 / (4.0 * xi ** 2))
    s_fac = 1.0 + k2 / (4.0 * xi ** 2)
    TH = precompute_table("H", Mt, h)
    TB = precompute_table("B", Mt, h) if mask & (KERNEL_S | KERNEL_T) else None
    T1 = [np.zeros(pad, np.complex128) for _ in range(3)]
    c = 0
    if mask & KERNEL_S:
        C1 = [fft_pad(grids[c + i]) for i in range(3)]
        c += 3 if free else 7
        kC1 = sum(K[i] * C1[i] for i in range(3))
        for j in range(3):
            T1[j] += -s_fac * E * TB * (k2 * C1[j] - K[j] * kC1)
    if mask & KERNEL_T:
        C1 = _sym([fft_pad(grids[c + i]) for i in range(6)])
        c += 6 if free else 13
        trC = C1[0][0] + C1[1][1] + C1[2][2]
        Ck = [sum(C1[j][m] * K[m] for m in range(3)) for j in range(3)]
        kCk = sum(K[j] * Ck[j] for j in range(3))
        for j in range(3):
            T1[j] += -1j * s_fac * E * TB * (k2 * (2.0 * Ck[j] + K[j] * trC) - 2.0 * K[j] * kCk)
    if mask & KERNEL_W:
        C1 = [fft_pad(grids[c + i]) for i in range(3)]
        c += 3 if free else 5
        cross = [C1[1] * K[2] - C1[2] * K[1], C1[2] * K[0] - C1[0] * K[2], C1[0] * K[1] - C1[1] * K[0]]
        for j in range(3):
            T1[j] += -2j * E * TH * cross[j]
    phi = np.zeros(pad, np.complex128)
    if not free:
        phi = E * TH * fft_pad(_correction_grid(mask, src, strengths, xi, h, P, Mt, eta))
        T1[2] = T1[2] + phi
    fields = [np.real(np.fft.ifftn(np.where(nyq, 0.0, F)))[:Mt, :Mt, :2 * Mt] for F in T1 + [phi]]
    tg = src if tgt is None else np.ascontiguousarray(tgt, np.float64)
    alpha = 2.0 * xi ** 2 / eta
    pre = (2.0 * xi ** 2 / (np.pi * eta)) ** 1.5 * h ** 3
    ox, oz = -0.5 * P * h, -Mt * h
    out = np.zeros((3, tg.shape[1]))
    for p in range(tg.shape[1]):
        x = tg[:, p]
        ix, wx, dx, _ = _window(x[0], ox, h, P, Mt, alpha)
        iy, wy, dy, _ = _window(x[1], ox, h, P, Mt, alpha)
        iz, wz, dz, _ = _window(x[2], oz, h, P, 2 * Mt, alpha)
        sl = (slice(ix, ix + P), slice(iy, iy + P), slice(iz, iz + P))
        W = pre * np.einsum('i,j,k->ijk', wx, wy, wz)
        for d in range(3):
            out[d, p] = np.sum(W * fields[d][sl])
        if not free:
            ph = fields[3][sl]
            # grad_x W(x - x_j) = -(dW/d(x_j - x)): minus the window derivative
            grad = [-pre * np.sum(np.einsum('i,j,k->ijk', *f) * ph)
                    for f in ((dx, wy, wz), (wx, dy, wz), (wx, wy, dz))]
            for d in range(3):
                out[d, p] -= x[2] * grad[d]
    return out
