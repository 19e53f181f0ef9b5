"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws numbers: it holds none of the solver's arithmetic.
Every field is float64 numpy in C order, x fastest: shape ``(n,)``,
``(ny, nx)`` or ``(nz, ny, nx)``.

Grid conventions (the same as the library's):
  * Dirichlet axis of n points on [lo, hi] includes both end nodes,
    spacing (hi - lo)/(n - 1); fields vanish on the boundary.
  * Periodic axis of n points on [lo, hi) holds n distinct points,
    spacing (hi - lo)/n.

Workloads (the paper uses no public dataset; these stand in for the
shapes of its experiments):
  1. 1D periodic [0, 2pi), N = 256, P = 1, CFL 1.5, 200 steps: sum of the
     Fourier modes k = 1..8 with N(0,1) cosine and sine amplitudes.
  2. 2D Dirichlet unit square 2048^2, P = 3, CFL 2, 500 steps: Gaussian pulse,
     centre U[0.3, 0.7]^2, width 0.02.
  3. 3D periodic [0, 2pi)^3, 256^3, P = 2, CFL 1.5, 200 steps: 16 distinct
     integer wave vectors 0 < |k| <= 12, N(0,1) amplitudes, U[0, 2pi) phases.
  4. Batch of 512 Dirichlet squares, n log-uniform in [64, 1024], P in
     {1, 2, 3}, CFL U[0.5, 4], Gaussian pulses, 200 steps.
  5. Adjoint: 2D Dirichlet 1024^2, P = 2, CFL 2, 400 steps, 64 receivers.
Seeds: workload k uses seed 1000 + k unless told otherwise.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def axis_coords(n: int, lo: float, hi: float, bc: str) -> np.ndarray:
    if bc == "dirichlet":
        return np.linspace(lo, hi, n)
    return lo + (hi - lo) * np.arange(n) / n


def spacing(n: int, lo: float, hi: float, bc: str) -> float:
    return (hi - lo) / (n - 1) if bc == "dirichlet" else (hi - lo) / n


def fourier_1d(n: int = 256, seed: int = 1001, kmax: int = 8) -> np.ndarray:
    rng = np.random.default_rng(seed)
    x = axis_coords(n, 0.0, 2 * np.pi, "periodic")
    a = rng.normal(size=kmax)
    b = rng.normal(size=kmax)
    u = np.zeros(n)
    for k in range(1, kmax + 1):
        u += a[k - 1] * np.cos(k * x) + b[k - 1] * np.sin(k * x)
    return u


def gaussian_2d(n: int = 2048, seed: int = 1002, width: float = 0.02, ny: int | None = None) -> np.ndarray:
    rng = np.random.default_rng(seed)
    ny = n if ny is None else ny
    cx, cy = rng.uniform(0.3, 0.7, size=2)
    x = axis_coords(n, 0.0, 1.0, "dirichlet")
    y = axis_coords(ny, 0.0, 1.0, "dirichlet")
    u = np.exp(-((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) / (2 * width ** 2))
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    return u


def fourier_3d(n: int = 256, seed: int = 1003, nmodes: int = 16, kmax: int = 12,
               shape: tuple[int, int, int] | None = None) -> tuple[np.ndarray, np.ndarray]:
    """Returns (field, modes) with modes rows (kx, ky, kz, amplitude, phase)."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape if shape is not None else (n, n, n)
    modes = []
    seen = set()
    while len(modes) < nmodes:
        k = tuple(int(v) for v in rng.integers(-kmax, kmax + 1, size=3))
        r2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
        if r2 == 0 or r2 > kmax ** 2 or k in seen:
            continue
        seen.add(k)
        modes.append((*k, rng.normal(), rng.uniform(0, 2 * np.pi)))
    modes = np.array(modes, dtype=np.float64)
    x = axis_coords(nx, 0.0, 2 * np.pi, "periodic")
    y = axis_coords(ny, 0.0, 2 * np.pi, "periodic")
    z = axis_coords(nz, 0.0, 2 * np.pi, "periodic")
    u = np.zeros((nz, ny, nx))
    for kx, ky, kz, amp, ph in modes:
        u += amp * np.cos(kx * x[None, None, :] + ky * y[None, :, None] + kz * z[:, None, None] + ph)
    return u, modes


@dataclass
class BatchProblem:
    n: int
    P: int
    cfl: float
    u0: np.ndarray


def batch_problems(count: int = 512, seed: int = 1004, nmin: int = 64, nmax: int = 1024,
                   width: float = 0.02, with_fields: bool = True) -> list[BatchProblem]:
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), size=count)).round().astype(int)
    Ps = rng.integers(1, 4, size=count)
    cfls = rng.uniform(0.5, 4.0, size=count)
    out = []
    for i in range(count):
        u0 = gaussian_2d(int(ns[i]), seed=seed * 7919 + i, width=width) if with_fields else None
        out.append(BatchProblem(int(ns[i]), int(Ps[i]), float(cfls[i]), u0))
    return out


def receivers_2d(n: int = 1024, count: int = 64, seed: int = 1005) -> np.ndarray:
    """Distinct interior grid nodes (iy, ix) of an n x n Dirichlet grid."""
    rng = np.random.default_rng(seed)
    picked = set()
    while len(picked) < count:
        iy, ix = (int(v) for v in rng.integers(1, n - 1, size=2))
        picked.add((iy, ix))
    return np.array(sorted(picked), dtype=np.int64)


def random_field(shape, seed: int) -> np.ndarray:
    return np.random.default_rng(seed).normal(size=shape)
