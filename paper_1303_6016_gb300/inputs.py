"""Seeded synthetic spin configurations (inputs only; no GFMC arithmetic).

The paper's workloads are classical spin configurations on an L x L x L simple
cubic lattice (Sec. 2.1; Sec. 5 runs 6^3 ... 32^3 lattices).  It uses no public
dataset, so every input here is synthetic and seeded:

* ``uniform_sphere``  -- each spin uniform on the unit sphere (a hot start),
* ``von_mises_fisher`` -- spins concentrated about +z with concentration kappa
  (a partially ordered start), drawn by the exact inverse CDF of the
  von Mises--Fisher distribution on S^2 (Wood, 1994),
* ``ferromagnet``     -- all spins along +z (theta = 0), the ordered state.

All return float64 arrays [N, 2] of (theta, phi), site = x + L*(y + L*z).
This module is shared by the tests, the benchmark and the smoke check; it
imports neither the CUDA binding nor the oracle.
"""
from __future__ import annotations

import numpy as np


def uniform_sphere(L: int, seed: int = 0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    N = L ** 3
    u = rng.random(N)
    v = rng.random(N)
    theta = np.arccos(1.0 - 2.0 * u)
    phi = 2.0 * np.pi * v
    return np.stack([theta, phi], axis=1)


def von_mises_fisher(L: int, kappa: float = 5.0, seed: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    N = L ** 3
    u = rng.random(N)
    v = rng.random(N)
    cos_t = 1.0 + np.log(u + (1.0 - u) * np.exp(-2.0 * kappa)) / kappa
    cos_t = np.clip(cos_t, -1.0, 1.0)
    theta = np.arccos(cos_t)
    phi = 2.0 * np.pi * v
    return np.stack([theta, phi], axis=1)


def ferromagnet(L: int) -> np.ndarray:
    return np.zeros((L ** 3, 2), dtype=np.float64)


def make(kind: str, L: int, seed: int = 0, kappa: float = 5.0) -> np.ndarray:
    if kind == "uniform":
        return uniform_sphere(L, seed)
    if kind == "vmf":
        return von_mises_fisher(L, kappa, seed)
    if kind == "fm":
        return ferromagnet(L)
    raise ValueError(f"unknown spin configuration kind {kind!r}")
