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


# --------------------------------------------------------------------------
# Embedded domains (Sec. 4.3): a convex domain q(x, y) < 0 cut out of a grid
# --------------------------------------------------------------------------
@dataclass
class EmbeddedGrid:
    """A convex domain embedded in an nx x ny grid of spacing (hx, hy).

    Node (i, j) sits at (x0 + i hx, y0 + j hy).  Row j holds the interior
    nodes r0[j]..r1[j] (empty when r0 > r1), with the boundary points at
    distances ra[j] before r0[j] and rb[j] after r1[j]; column i holds the
    rows c0[i]..c1[i] with gaps ca[i], cb[i].  ``mask`` marks the interior
    nodes, shape (ny, nx).
    """
    nx: int
    ny: int
    x0: float
    y0: float
    hx: float
    hy: float
    r0: np.ndarray
    r1: np.ndarray
    ra: np.ndarray
    rb: np.ndarray
    c0: np.ndarray
    c1: np.ndarray
    ca: np.ndarray
    cb: np.ndarray
    mask: np.ndarray

    def coords(self):
        x = self.x0 + self.hx * np.arange(self.nx)
        y = self.y0 + self.hy * np.arange(self.ny)
        return x, y


def _chords(a: float, bl: np.ndarray, cl: np.ndarray):
    """Roots t_lo < t_hi of a t^2 + bl t + cl (a > 0) for every entry; NaN where
    the line misses the domain."""
    disc = bl * bl - 4.0 * a * cl
    ok = disc > 0.0
    sq = np.sqrt(np.where(ok, disc, 0.0))
    lo = np.where(ok, (-bl - sq) / (2.0 * a), np.nan)
    hi = np.where(ok, (-bl + sq) / (2.0 * a), np.nan)
    return lo, hi


def conic_grid(n: int, lo: float, hi: float, q) -> EmbeddedGrid:
    """The domain q(x, y) = a x^2 + 2 b x y + c y^2 + d x + e y + f < 0 (a, c > 0,
    ac > b^2: an ellipse) on the n x n grid of [lo, hi]^2 including both ends.

    q = (a, b, c, d, e, f).  A node is interior when it lies strictly inside
    both the row's and the column's chord, more than 1e-9 of a spacing from
    either end; the gaps are the distances from the first and last interior
    node to the chord's ends.
    """
    a, b, c, d, e, f = (float(t) for t in q)
    h = (hi - lo) / (n - 1)
    xs = lo + h * np.arange(n)
    eps = 1e-9 * h
    rxa, rxb = _chords(a, 2 * b * xs + d, c * xs * xs + e * xs + f)      # x-chord of row y = xs[j]
    cya, cyb = _chords(c, 2 * b * xs + e, a * xs * xs + d * xs + f)      # y-chord of column x = xs[i]
    def outside(t, beyond):
        t = t[np.isfinite(t)]                      # rows or columns that meet the domain
        return t.size > 0 and bool(beyond(t).any())
    if (outside(rxa, lambda t: t <= lo) or outside(rxb, lambda t: t >= hi) or outside(cya, lambda t: t <= lo)
            or outside(cyb, lambda t: t >= hi)):
        raise ValueError("the domain must lie inside the grid")
    with np.errstate(invalid="ignore"):
        in_row = (xs[None, :] > rxa[:, None] + eps) & (xs[None, :] < rxb[:, None] - eps)
        in_col = (xs[:, None] > cya[None, :] + eps) & (xs[:, None] < cyb[None, :] - eps)
    mask = in_row & in_col                                               # mask[j, i]: row j, column i

    def lines(m, ta, tb):
        cnt = m.sum(axis=1)
        first = np.where(cnt > 0, m.argmax(axis=1), 1)
        last = np.where(cnt > 0, n - 1 - m[:, ::-1].argmax(axis=1), 0)
        if ((last - first + 1)[cnt > 0] != cnt[cnt > 0]).any():
            raise ValueError("the domain's intersection with a grid line is not one interval")
        ga = np.where(cnt > 0, xs[first] - ta, h)
        gb = np.where(cnt > 0, tb - xs[last], h)
        return first.astype(np.int64), last.astype(np.int64), ga, gb

    r0, r1, ra, rb = lines(mask, rxa, rxb)
    c0, c1, ca, cb = lines(mask.T, cya, cyb)
    return EmbeddedGrid(n, n, lo, lo, h, h, r0, r1, ra, rb, c0, c1, ca, cb, mask)


def ellipse_grid(n: int, half: float = 2.2) -> EmbeddedGrid:
    """The ellipse ((x + y)/4)^2 + (x - y)^2 < 1 of Sec. 4.3 (principal axes on
    the diagonals, semi-axes 2 sqrt 2 and 1/sqrt 2) in the grid of
    [-half, half]^2 (it spans |x|, |y| <= sqrt(17)/2 = 2.06)."""
    # (x + y)^2 / 16 + (x - y)^2 - 1 = (17/16)(x^2 + y^2) - (15/8) x y - 1
    return conic_grid(n, -half, half, (17.0 / 16.0, -15.0 / 16.0, 17.0 / 16.0, 0.0, 0.0, -1.0))


def disk_grid(n: int, radius: float = 1.0, half: float = 1.1) -> EmbeddedGrid:
    """The disk x^2 + y^2 < radius^2 in the grid of [-half, half]^2."""
    return conic_grid(n, -half, half, (1.0, 0.0, 1.0, 0.0, 0.0, -radius * radius))


def gaussian_embedded(g: EmbeddedGrid, seed: int = 1006, width: float = 0.15) -> np.ndarray:
    """Gaussian pulse with its centre drawn within 0.3 of the origin, zero
    outside the domain."""
    rng = np.random.default_rng(seed)
    cx, cy = rng.uniform(-0.3, 0.3, size=2)
    x, y = g.coords()
    X, Y = np.meshgrid(x, y)
    u = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width * width))
    return np.where(g.mask, u, 0.0)
