"""CPU oracle for the half-space Stokes sums (arXiv 1802.07844).

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by the smoke
check in ``__graft_entry__`` and by the CPU-baseline leg of ``bench.py``; the
product path (the CUDA library and its Python binding) never imports it.  It
shares no code with the CUDA path.

Contents
  * ``hs_oracle.c``   -- plain FP64 C: direct half-space sums (Sec. 3) and
    free-space sums (Sec. 2, mask bit ``FREE_SPACE``), the
    real-space / smooth / self split (Sec. 4, Appendix), cell lists and
    brute-force neighbour counts (Sec. 5.1), the spread grids (Alg. 1 step 5).
  * ``se_fourier.py`` -- numpy restatement of the Fourier part (Alg. 1 steps
    2-10 and the truncated-kernel precomputation of Sec. 5.2), for small grids.

Units: all velocities are 8*pi times the physical velocity at unit viscosity.
Array layout: component-major, positions ``(3, n)``, strengths stacked in the
kernel order S (f, 3 rows), T (g then q, 6 rows), W (tau, 3 rows).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

KERNEL_S, KERNEL_T, KERNEL_W = 1, 2, 4
FREE_SPACE = 8  # mask bit: the free-space sums of Sec. 2 (no wall, no images, no corrections)
PART_DIRECT, PART_REAL, PART_SMOOTH, PART_SELF = 0, 1, 2, 3

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hs_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libhs_oracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            L.oracle_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_long,
                                     dp, dp, ctypes.c_long, dp, ctypes.c_int, dp]
            L.oracle_sum.restype = ctypes.c_int
            L.oracle_coefs.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, dp]
            L.oracle_coefs.restype = None
            L.oracle_fsmooth.argtypes = [ctypes.c_double, ctypes.c_double, dp]
            L.oracle_fsmooth.restype = None
            L.oracle_cells.argtypes = [ctypes.c_long, dp, dp, dp, ip, ip, ip, ip]
            L.oracle_cells.restype = ctypes.c_int
            L.oracle_neighbor_counts.argtypes = [ctypes.c_long, dp, ctypes.c_long, dp, ctypes.c_int,
                                                 ctypes.c_double, ip, ip]
            L.oracle_neighbor_counts.restype = ctypes.c_int
            L.oracle_spread.argtypes = [ctypes.c_int, ctypes.c_long, dp, dp, ctypes.c_double, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, dp]
            L.oracle_spread.restype = ctypes.c_int
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _i(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def n_strength_rows(mask: int) -> int:
    return (3 if mask & KERNEL_S else 0) + (6 if mask & KERNEL_T else 0) + (3 if mask & KERNEL_W else 0)


def half_space_sum(mask, src, strengths, tgt=None, part=PART_DIRECT, xi=0.0, rc=0.0):
    """One part of the half-space sum at the targets (Sec. 3 / Sec. 4).

    ``tgt=None`` means the targets are the sources (pair m = p excluded by
    index).  ``part``: PART_DIRECT (plain sum), PART_REAL (real-space parts,
    cut-off ``rc``; ``rc <= 0`` means none), PART_SMOOTH (K - K_R over all
    pairs), PART_SELF (stokeslet self term).  Returns ``(3, n_tgt)``."""
    src = _c64(src)
    strengths = _c64(strengths)
    n = src.shape[1]
    assert src.shape == (3, n) and strengths.shape == (n_strength_rows(mask), n)
    if tgt is None:
        t, nt, same = src, n, 1
    else:
        t = _c64(tgt)
        nt, same = t.shape[1], 0
    out = np.zeros((3, nt))
    rcode = lib().oracle_sum(int(mask), int(part), float(xi), float(rc), n, _d(src), _d(strengths), nt, _d(t),
                             same, _d(out))
    if rcode != 0:
        raise ValueError("oracle_sum rejected its arguments")
    return out


def direct(mask, src, strengths, tgt=None):
    """Plain FP64 O(N N_t) half-space sum (Sec. 3, eq. v_sum_halfspace); with
    the FREE_SPACE bit in ``mask`` the free-space sum of Sec. 2."""
    return half_space_sum(mask, src, strengths, tgt, PART_DIRECT)


def ewald_split(mask, src, strengths, xi, rc=0.0, tgt=None):
    """(real, smooth, self) parts of the Ewald split (Sec. 4)."""
    return (half_space_sum(mask, src, strengths, tgt, PART_REAL, xi, rc),
            half_space_sum(mask, src, strengths, tgt, PART_SMOOTH, xi),
            half_space_sum(mask, src, strengths, tgt, PART_SELF, xi))


def coefs(part, xi, rho):
    out = np.zeros(9)
    lib().oracle_coefs(int(part), float(xi), float(rho), _d(out))
    return dict(zip(["g0", "g1", "g2", "g3", "sa", "sb", "ta", "tb", "wa"], out))


def fsmooth(xi, s):
    out = np.zeros(4)
    lib().oracle_fsmooth(float(xi), float(s), _d(out))
    return out


def cells(pos, origin, inv_cell, ncell):
    """Cell ids, stably sorted permutation and cell starts (Sec. 5.1)."""
    pos = _c64(pos)
    n = pos.shape[1]
    origin = _c64(origin)
    inv_cell = _c64(inv_cell)
    nc = np.ascontiguousarray(ncell, dtype=np.int32)
    cid = np.zeros(n, np.int32)
    perm = np.zeros(n, np.int32)
    start = np.zeros(int(np.prod(nc.astype(np.int64))) + 1, np.int32)
    lib().oracle_cells(n, _d(pos), _d(origin), _d(inv_cell), _i(nc), _i(cid), _i(perm), _i(start))
    return cid, perm, start


def neighbor_counts(src, rc, tgt=None):
    src = _c64(src)
    n = src.shape[1]
    if tgt is None:
        t, nt, same = src, n, 1
    else:
        t = _c64(tgt)
        nt, same = t.shape[1], 0
    a = np.zeros(nt, np.int32)
    b = np.zeros(nt, np.int32)
    lib().oracle_neighbor_counts(n, _d(src), nt, _d(t), same, float(rc), _i(a), _i(b))
    return a, b


def spread(mask, src, strengths, xi, h, P, Mt):
    """Spread grids C1/C2/C3 of Alg. 1 step 5, shape (ncomp, Mt, Mt, 2 Mt)
    (C1 only with the FREE_SPACE bit)."""
    src = _c64(src)
    strengths = _c64(strengths)
    n = src.shape[1]
    if mask & FREE_SPACE:
        ncomp = (3 if mask & KERNEL_S else 0) + (6 if mask & KERNEL_T else 0) + (3 if mask & KERNEL_W else 0)
    else:
        ncomp = (7 if mask & KERNEL_S else 0) + (13 if mask & KERNEL_T else 0) + (5 if mask & KERNEL_W else 0)
    grids = np.zeros((ncomp, Mt, Mt, 2 * Mt))
    lib().oracle_spread(int(mask), n, _d(src), _d(strengths), float(xi), float(h), int(P), int(Mt), _d(grids))
    return grids


def rel_rms(u, u_ref):
    """Relative RMS error (Sec. 6): sqrt(sum |u - u_ref|^2) / sqrt(sum |u_ref|^2)."""
    u = np.asarray(u, np.float64)
    u_ref = np.asarray(u_ref, np.float64)
    return float(np.sqrt(np.sum((u - u_ref) ** 2)) / np.sqrt(np.sum(u_ref ** 2)))
