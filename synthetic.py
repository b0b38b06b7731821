"""Seeded synthetic inputs shared by the tests, the benchmark, the oracle side and the CUDA side.

This module holds no arithmetic of the lattice Boltzmann method itself: it only draws the
macroscopic fields (density, velocity, temperature) and the workload parameters that both
implementations then turn into populations with their own equilibrium code. Every generator
takes an explicit seed.

Workloads (the paper's 1D normal shock of Sec. 4.2 and a 3D periodic box):

* ``tanh_blend``: q(x) = q1 + (q2 - q1) (1 + tanh((x - x0)/W)) / 2 over cell centres
  x = 0..L-1, x0 = L/2 -- the smooth stand-in for the paper's step initial condition.
* ``taylor_green``: rho = 1 + N(0, sigma^2) noise, theta = 1,
  u = A (sin X cos Y cos Z, -cos X sin Y cos Z, 0), X = 2 pi i / n.
* ``batched_shocks``: Mach numbers uniform in [lo, hi] and lengths drawn from a set.
* ``perturbed``: multiplicative +-frac uniform perturbation of a parameter vector.
* ``random_populations``: positive populations w_i (1 + eps N(0,1)) for unit tests.
"""
from __future__ import annotations

import numpy as np

SEED = 11086


def tanh_blend(L: int, width: float, q1: float, q2: float, x0: float | None = None) -> np.ndarray:
    x = np.arange(L, dtype=np.float64)
    x0 = L / 2.0 if x0 is None else x0
    return q1 + (q2 - q1) * 0.5 * (1.0 + np.tanh((x - x0) / width))


def step_blend(L: int, q1: float, q2: float) -> np.ndarray:
    """The initial condition of the paper's shock runs (Sec. 4.2): q1 on x < L/2, q2 beyond."""
    x = np.arange(L)
    return np.where(x < L // 2, q1, q2).astype(np.float64)


def taylor_green(n: int, amplitude: float = 0.05, noise: float = 1e-3, seed: int = SEED,
                 shape: tuple | None = None):
    """Fields on an (nz, ny, nx) grid (default n^3): rho (noisy), u (3, ...), theta."""
    nz, ny, nx = shape if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    rho = 1.0 + noise * rng.standard_normal((nz, ny, nx))
    X = 2.0 * np.pi * np.arange(nx) / nx
    Y = 2.0 * np.pi * np.arange(ny) / ny
    Z = 2.0 * np.pi * np.arange(nz) / nz
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    u = np.stack([amplitude * np.sin(Xg) * np.cos(Yg) * np.cos(Zg),
                  -amplitude * np.cos(Xg) * np.sin(Yg) * np.cos(Zg),
                  np.zeros_like(Xg)])
    theta = np.ones((nz, ny, nx))
    return rho, u, theta


def batched_shocks(count: int = 64, seed: int = SEED, ma_range=(1.2, 7.0),
                   lengths=(512, 1024, 2048, 4096, 8192)):
    rng = np.random.default_rng(seed)
    ma = rng.uniform(ma_range[0], ma_range[1], size=count)
    L = rng.choice(np.asarray(lengths), size=count)
    return ma, L


def perturbed(values, frac: float = 0.2, seed: int = SEED) -> np.ndarray:
    rng = np.random.default_rng(seed)
    values = np.asarray(values, dtype=np.float64)
    return values * (1.0 + rng.uniform(-frac, frac, size=values.shape))


def random_populations(w: np.ndarray, ncell: int, eps: float = 0.05, seed: int = SEED) -> np.ndarray:
    """(Q, ncell) populations w_i (1 + eps g), g standard normal, clipped positive."""
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((len(w), ncell))
    return np.asarray(w)[:, None] * np.clip(1.0 + eps * g, 0.05, None)
