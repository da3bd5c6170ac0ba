"""Seeded synthetic inputs for the half-space Stokes sums.

This module only draws random numbers: it holds none of the method's
arithmetic and is shared by the tests, the oracle runs and ``bench.py``.

Recipe (the paper measures on random points only, Sec. 7; no dataset is
involved):
  * generator: numpy ``default_rng`` (PCG64), seed 1802078440 + workload index
    (+ instance index for batched or served workloads);
  * positions in the paper's frame, wall at z = 0: x, y uniform in [0, L);
    z uniform in (0, L] ("uniform") or truncated Exponential(mean 0.05) on
    (0, L] ("near_wall"), sampled by inverse CDF
    z = -mu ln(1 - u (1 - e^{-L/mu})), u in (0, 1];
  * strengths i.i.d. N(0, 1) per component: stokeslet f (3 rows),
    stresslet g (3 rows) and a unit orientation q = n / |n| with n ~ N(0,1)^3
    (3 rows), rotlet torque tau (3 rows).
All arrays are float64 and component-major: positions (3, n), strengths
stacked in the kernel order S, T, W.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

KERNEL_S, KERNEL_T, KERNEL_W = 1, 2, 4
SEED_BASE = 1802078440


def rng_for(index: int, sub: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + int(index) + 1_000_003 * int(sub))


def positions(rng: np.random.Generator, n: int, L: float = 1.0, dist: str = "uniform", mu: float = 0.05):
    x = rng.uniform(0.0, L, n)
    y = rng.uniform(0.0, L, n)
    u = 1.0 - rng.uniform(0.0, 1.0, n)  # in (0, 1]
    if dist == "uniform":
        z = L * u  # (0, L]
    elif dist == "near_wall":
        z = -mu * np.log1p(-u * (1.0 - np.exp(-L / mu)))
        z = np.clip(z, np.nextafter(0.0, 1.0), L)
    else:
        raise ValueError(dist)
    return np.stack([x, y, z])


def strengths(rng: np.random.Generator, mask: int, n: int):
    rows = []
    if mask & KERNEL_S:
        rows.append(rng.standard_normal((3, n)))
    if mask & KERNEL_T:
        g = rng.standard_normal((3, n))
        q = rng.standard_normal((3, n))
        q /= np.linalg.norm(q, axis=0, keepdims=True)
        rows += [g, q]
    if mask & KERNEL_W:
        rows.append(rng.standard_normal((3, n)))
    return np.ascontiguousarray(np.concatenate(rows, axis=0))


@dataclass
class Problem:
    mask: int
    src: np.ndarray
    strengths: np.ndarray
    L: float
    name: str


def problem(mask: int, n: int, L: float = 1.0, dist: str = "uniform", index: int = 0, sub: int = 0,
            name: str = "") -> Problem:
    rng = rng_for(index, sub)
    src = positions(rng, n, L, dist)
    st = strengths(rng, mask, n)
    return Problem(mask, src, st, L, name or f"{dist}_n{n}_mask{mask}")


# The five workloads: index, kernel mask, N, distribution, target tolerance.
WORKLOADS = {
    "hs_stokeslet_n1000_uniform": dict(index=0, mask=KERNEL_S, n=1000, dist="uniform", tol=1e-8),
    "hs_stokeslet_n100k_uniform": dict(index=1, mask=KERNEL_S, n=100_000, dist="uniform", tol=1e-10),
    "hs_stresslet_n100k_uniform": dict(index=1, mask=KERNEL_T, n=100_000, dist="uniform", tol=1e-10),
    "hs_stokeslet_rotlet_n1m_nearwall": dict(index=2, mask=KERNEL_S | KERNEL_W, n=1_000_000, dist="near_wall",
                                             tol=1e-10),
}


def workload(name: str, n: int | None = None) -> Problem:
    w = WORKLOADS[name]
    return problem(w["mask"], n if n is not None else w["n"], 1.0, w["dist"], w["index"], name=name)


def subsample(rng_index: int, n: int, k: int) -> np.ndarray:
    """Seeded subsample of k target indices out of n (sorted)."""
    rng = rng_for(rng_index, 777)
    return np.sort(rng.choice(n, size=min(k, n), replace=False))
