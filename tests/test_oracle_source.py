"""Pins of the oracle's source terms (Sec. 4.1; readings in the design doc).

* C in 1D is D, and in 2D it equals D_x v + D_y v - D_y D_x v - D_x D_y v
  (L^{-1} = 1 - D), composed here from the per-axis D;
* zero source reduces to the homogeneous stepping; the source enters
  linearly;
* the manufactured solution u = sin(pi x) sin(pi y) cos(w t) (source
  S = (2 pi^2 - w^2) sin(pi x) sin(pi y) cos(w t)) is reached at order 2 for
  P = 1 and 4 for P = 2 -- which fixes the sign and scale of the C[S] term
  (the printed form does not reach fourth order, see the reading);
* P = 3 is refused (no higher-order source terms are given).
"""
import numpy as np
import pytest

import oracle


def test_C_is_D_in_1d():
    v = np.random.default_rng(1).normal(size=50)
    assert np.abs(oracle.C(v, 0.8) - oracle.D_axis(v, 0, 0.8, "dirichlet", 2)).max() <= 1e-15


def test_C_in_2d_from_the_per_axis_operators():
    v = np.random.default_rng(2).normal(size=(17, 23))
    nu = (0.7, 1.1)
    Dx = lambda w: oracle.D_axis(w, 0, nu[0], "dirichlet", 2)      # axis 0 = x (x first)
    Dy = lambda w: oracle.D_axis(w, 1, nu[1], "dirichlet", 2)
    ref = Dx(v) + Dy(v) - Dy(Dx(v)) - Dx(Dy(v))
    assert np.abs(oracle.C(v, nu) - ref).max() <= 1e-14 * np.abs(ref).max()


def mode(n):
    x = np.linspace(0, 1, n)
    X, Y = np.meshgrid(x, x)
    return np.sin(np.pi * X) * np.sin(np.pi * Y)


def run_mode(n, P, M, T, w, scale=1.0):
    h = 1.0 / (n - 1)
    dt = T / M
    beta = oracle.beta_max(P)
    nu = beta / dt * h
    g = scale * (2 * np.pi ** 2 - w ** 2) * mode(n)
    f = np.cos(w * dt * np.arange(M + 1))
    return oracle.run_source(mode(n), M, nu, P, beta, dt ** 2, g, f)


def test_zero_source_is_the_homogeneous_stepping():
    n, P, M, dt = 41, 2, 7, 0.03
    beta = oracle.beta_max(P)
    nu = beta / dt / (n - 1)
    u0 = mode(n)
    got = oracle.run_source(u0, M, nu, P, beta, dt ** 2, np.zeros_like(u0), np.ones(M + 1))
    _, ref = oracle.run(u0, oracle.start(u0, nu, P, beta, "dirichlet"), M - 1, nu, P, beta, "dirichlet")
    assert np.abs(got - ref).max() <= 1e-14


def test_source_enters_linearly():
    n, P, M, T, w = 41, 2, 8, 0.4, 5.0
    u0 = np.zeros((n, n))
    h = 1.0 / (n - 1)
    beta = oracle.beta_max(P)
    nu = beta / (T / M) * h
    g = mode(n)
    f = np.cos(w * (T / M) * np.arange(M + 1))
    a = oracle.run_source(u0, M, nu, P, beta, (T / M) ** 2, g, f)
    b = oracle.run_source(u0, M, nu, P, beta, (T / M) ** 2, 3.0 * g, f)
    assert np.abs(b - 3.0 * a).max() <= 1e-13 * np.abs(b).max()


W = 5.0
TW = (np.pi / 2 + 2 * np.pi) / W        # cos(W T) = 0: the phase error shows at first order


@pytest.mark.parametrize("P,M1,M2,expect", [(1, 20, 40, 2), (2, 20, 40, 4)])
def test_manufactured_solution_converges_at_order_2P(P, M1, M2, expect):
    n = 321
    h = 1.0 / (n - 1)
    ex = mode(n) * np.cos(W * TW)
    e = [np.sqrt(h * h * np.sum((run_mode(n, P, M, TW, W) - ex) ** 2)) for M in (M1, M2)]
    rate = np.log2(e[0] / e[1])
    assert expect - 0.5 <= rate <= expect + 0.5, (P, e, rate)


def test_higher_orders_are_refused():
    with pytest.raises(ValueError):
        oracle.run_source(np.zeros((5, 5)), 2, 0.5, 3, oracle.beta_max(3), 0.01, np.zeros((5, 5)), np.zeros(3))
