"""Pins of the oracle's time-dependent Dirichlet data (Sec. 3.2): the
boundary values of D^m u come from (d_tt/c^2)^m of the data.

* zero data reduces to the homogeneous operator and stepping;
* D applied to zero with end values gL, gR is a pure boundary layer: it takes
  gL and gR at the end nodes and is a combination of d^j and d^{n-1-j} (the
  homogeneous solutions of the recurrences), checked by a least-squares fit;
* D is affine in the data: D_g v = D_0 v + D_g 0;
* the boundary values of D^p u for a mode of the data equal the truncated
  series of the symbol (s/(1+s))^p (D = -(d_xx/alpha^2)(1 - d_xx/alpha^2)^{-1});
* the stepping with the exact data of u = cos(k pi x) cos(k pi t) (nonzero on
  the boundary) converges at order 2P to it, like the homogeneous example,
  and at second order when the data's derivatives are left out.
"""
import numpy as np
import pytest

import oracle


def test_zero_data_is_the_homogeneous_operator():
    rng = np.random.default_rng(3)
    v = rng.normal(size=77)
    v[0] = v[-1] = 0.0
    assert np.abs(oracle.D_line_bc(v, 0.7, 0.0, 0.0) - oracle.D_axis(v, 0, 0.7, "dirichlet", 2)).max() <= 1e-15


@pytest.mark.parametrize("nu", [0.05, 0.6, 2.5])
def test_D_of_zero_is_a_boundary_layer(nu):
    n, gL, gR = 41, 0.7, -1.3
    e = oracle.D_line_bc(np.zeros(n), nu, gL, gR)
    assert abs(e[0] - gL) <= 1e-14 and abs(e[-1] - gR) <= 1e-14
    d = np.exp(-nu)
    j = np.arange(n)
    basis = np.stack([d ** j, d ** (n - 1 - j)], axis=1)
    coef, *_ = np.linalg.lstsq(basis, e, rcond=None)
    assert np.abs(basis @ coef - e).max() <= 1e-14


def test_D_is_affine_in_the_data():
    rng = np.random.default_rng(4)
    v = rng.normal(size=64)
    a = oracle.D_line_bc(v, 0.9, 0.4, 2.0)
    b = oracle.D_line_bc(v, 0.9, 0.0, 0.0) + oracle.D_line_bc(np.zeros(64), 0.9, 0.4, 2.0)
    assert np.abs(a - b).max() <= 1e-14


def test_zero_data_stepping_is_the_homogeneous_stepping():
    n, P, nsteps = 101, 2, 9
    beta = oracle.beta_max(P)
    x = np.linspace(0, 1, n)
    u0 = np.sin(np.pi * x) + 0.3 * np.sin(3 * np.pi * x)
    got = oracle.run_bc(u0, nsteps, 0.8, P, beta, np.zeros((nsteps + 1, 2, P + 1)))
    u1 = oracle.start(u0, 0.8, P, beta, "dirichlet")
    _, ref = oracle.run(u0, u1, nsteps - 1, 0.8, P, beta, "dirichlet")
    assert np.abs(got - ref).max() <= 1e-13


def standing_wave_data(k, T, M, P, beta, h):
    """gam[k, side, m] for u = cos(k pi x) cos(k pi t) on [0, 1], c = 1:
    (d_tt)^m u_side = (-(k pi)^2)^m u_side, scaled by alpha^{-2m}."""
    dt = T / M
    alpha = beta / dt
    t = dt * np.arange(M + 1)
    g = np.empty((M + 1, 2, P + 1))
    for m in range(P + 1):
        f = (-(k * np.pi) ** 2 / alpha ** 2) ** m * np.cos(k * np.pi * t)
        g[:, 0, m] = f
        g[:, 1, m] = np.cos(k * np.pi) * f
    return g


def error_bc(k, T, M, P, n=2001):
    beta = oracle.beta_max(P)
    x = np.linspace(0, 1, n)
    h = 1.0 / (n - 1)
    nu = beta / (T / M) * h
    u = oracle.run_bc(np.cos(k * np.pi * x), M, nu, P, beta, standing_wave_data(k, T, M, P, beta, h))
    exact = np.cos(k * np.pi * x) * np.cos(k * np.pi * T)
    return np.sqrt(h * np.sum((u - exact) ** 2))


@pytest.mark.parametrize("P,M1,M2", [(1, 40, 80), (2, 40, 80), (3, 20, 40)])
def test_exact_data_converges_at_order_2P(P, M1, M2):
    """u = cos(3 pi x) cos(3 pi t), t = 7/6 (cos(3 pi t) = 0, so the phase
    error shows at first order)."""
    e1, e2 = error_bc(3, 7.0 / 6.0, M1, P), error_bc(3, 7.0 / 6.0, M2, P)
    assert e2 > 1e-7
    rate = np.log2(e1 / e2)
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, e1, e2, rate)


def test_missing_derivative_data_costs_the_order():
    """The boundary values of D^p u matter: with the data's time derivatives
    left out (homogeneous D at the ends while the field is not zero there)
    the P = 2 run converges at about second order instead of fourth."""
    P, n, T = 2, 2001, 7.0 / 6.0
    beta = oracle.beta_max(P)
    x = np.linspace(0, 1, n)
    h = 1.0 / (n - 1)
    es = []
    for M in (40, 80):
        nu = beta / (T / M) * h
        g = standing_wave_data(3, T, M, P, beta, h)
        g[:, :, 1:] = 0.0
        u = oracle.run_bc(np.cos(3 * np.pi * x), M, nu, P, beta, g)
        es.append(np.sqrt(h * np.sum((u - np.cos(3 * np.pi * x) * np.cos(3 * np.pi * T)) ** 2)))
    assert np.log2(es[0] / es[1]) <= 2.6
    good = [error_bc(3, T, M, P, n) for M in (40, 80)]
    assert np.log2(good[0] / good[1]) >= 2 * P - 1.0 and good[1] < es[1] / 10


def test_boundary_values_of_a_mode():
    """For data cos(w t) the boundary values of D^p u are those of the
    symbol (s / (1 + s))^p, s = (w / alpha)^2, truncated at total order P in
    s: the sum over j = p..P of the series coefficients."""
    P, s = 4, 0.03
    data = np.array([[(-s) ** j for j in range(P + 1)], [2.0 * (-s) ** j for j in range(P + 1)]])
    g = oracle.bc_values(data, P)
    for p in range(1, P + 1):
        # (s/(1+s))^p = sum_{k>=0} (-1)^k C(p+k-1, k) s^{p+k}
        from math import comb
        series = sum((-1) ** k * comb(p + k - 1, k) * s ** (p + k) for k in range(0, P - p + 1))
        assert abs(g[p, 0] - series) <= 1e-16 and abs(g[p, 1] - 2 * series) <= 1e-16
    assert abs(g[1, 0] - s / (1 + s)) <= s ** (P + 1)
