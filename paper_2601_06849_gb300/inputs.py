"""Seeded synthetic inputs for the ETD2RK-DS workloads.

This module only draws initial fields and problem parameters; it holds none of
the scheme's arithmetic. Both the CUDA path (through the tests and bench.py)
and the CPU oracle take their inputs from here, so the two see the same bits.

Grid: n interior points per axis on (0, 1), h = 1/(n+1), x_i = i h,
i = 1..n (Section 2.1); arrays are [comp][z][y][x] with x fastest.
Seeds: 20260106 + workload index, NumPy PCG64.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List

import numpy as np

SEED_BASE = 20260106


def grid(n: int) -> np.ndarray:
    """Interior node coordinates x_i = i/(n+1), i = 1..n."""
    return np.arange(1, n + 1, dtype=np.float64) / (n + 1)


def rng(workload: int, sub: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([SEED_BASE + workload, sub]))


def sine_mode(n: int, d: int, modes) -> np.ndarray:
    """prod_axis sin(k_axis pi x_axis) on the interior grid; modes = (kx, ky[, kz])."""
    x = grid(n)
    fx = np.sin(modes[0] * np.pi * x)
    fy = np.sin(modes[1] * np.pi * x)
    if d == 2:
        return np.einsum("j,i->ji", fy, fx)
    fz = np.sin(modes[2] * np.pi * x)
    return np.einsum("k,j,i->kji", fz, fy, fx)


def allen_cahn_2d(n: int, workload: int = 0) -> np.ndarray:
    """u0 = 0.5 sin(pi x) sin(pi y) + 0.01 N(0,1) on interior nodes, shape (1, n, n)."""
    u = 0.5 * sine_mode(n, 2, (1, 1)) + 0.01 * rng(workload).standard_normal((n, n))
    return u[None]


def fhn_uniform(n: int, d: int = 2, workload: int = 1, lo: float = -0.1, hi: float = 0.1) -> np.ndarray:
    """u0, v0 ~ U[lo, hi] independently, shape (2, n, ..)."""
    return rng(workload).uniform(lo, hi, size=(2,) + (n,) * d)


def gaussian_bump(n: int, d: int = 3, sigma: float = 0.1, center: float = 0.5) -> np.ndarray:
    """exp(-|x - c|^2 / sigma^2), c = (0.5, ..), shape (1, n, ..)."""
    x = grid(n) - center
    r2 = x[None, :] ** 2 + x[:, None] ** 2 if d == 2 else (
        x[None, None, :] ** 2 + x[None, :, None] ** 2 + x[:, None, None] ** 2)
    return np.exp(-r2 / sigma ** 2)[None]


def random_field(shape, workload: int, sub: int = 0, scale: float = 1.0) -> np.ndarray:
    """Standard-normal field times scale (edge-case and parity tests)."""
    return scale * rng(workload, sub).standard_normal(shape)


@dataclass
class EnsembleMember:
    n: int
    kappa_u: float
    tau: float
    u0: np.ndarray  # (2, n, n)


def fhn_ensemble(count: int = 512, workload: int = 3, n_choices=tuple(range(64, 513, 32))) -> List[EnsembleMember]:
    """Independent 2D FitzHugh-Nagumo instances: n uniform over n_choices,
    kappa_u log-uniform on [1e-4, 1e-2], tau uniform on [1e-3, 1e-2],
    fields U[-0.1, 0.1], each member seeded on its own."""
    g = rng(workload)
    ns = g.choice(np.array(n_choices), size=count)
    ku = np.exp(g.uniform(np.log(1e-4), np.log(1e-2), size=count))
    taus = g.uniform(1e-3, 1e-2, size=count)
    out = []
    for i in range(count):
        u0 = rng(workload, i + 1).uniform(-0.1, 0.1, size=(2, int(ns[i]), int(ns[i])))
        out.append(EnsembleMember(int(ns[i]), float(ku[i]), float(taus[i]), u0))
    return out
