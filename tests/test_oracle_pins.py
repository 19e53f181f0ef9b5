"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: numerical
quadrature of the paper's integrals, closed-form Fourier symbols, dense
Kronecker-product evaluation of the ADI formulas as the paper prints them,
values the paper prints (Tables 1 and 2, the explicit schemes of Secs. 3-4),
convergence orders and A-stability.  CPU only.
"""
from fractions import Fraction
from math import comb
from pathlib import Path

import numpy as np
import pytest

import oracle

GOLDEN = Path(__file__).resolve().parent / "golden"


def _read_golden(name):
    rows = []
    for line in (GOLDEN / name).read_text().splitlines():
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# Local quadrature (Sec. 2): J^L_j = (alpha/2) int_0^h e^{-alpha y} p(x_j - y) dy
# --------------------------------------------------------------------------
def _gl(npts=24):
    return np.polynomial.legendre.leggauss(npts)


def _lagrange(nodes, vals, y):
    out = np.zeros_like(y, dtype=float)
    for i, (xi, vi) in enumerate(zip(nodes, vals)):
        li = np.ones_like(y, dtype=float)
        for k, xk in enumerate(nodes):
            if k != i:
                li *= (y - xk) / (xi - xk)
        out += vi * li
    return out


@pytest.mark.parametrize("nu", [1e-3, 0.03, 0.4, 0.617, 1.7, 6.0])
@pytest.mark.parametrize("quad", [1, 2])
def test_weights_equal_exact_integral_of_interpolant(nu, quad):
    rng = np.random.default_rng(7)
    d, W0, W1, R = oracle.weights(nu, quad)
    assert d == pytest.approx(np.exp(-nu), rel=1e-15)
    h = 0.37
    alpha = nu / h
    g, gw = _gl(30)
    y = 0.5 * h * (g + 1.0)          # y in [0, h]
    wq = 0.5 * h * gw
    for _ in range(5):
        vm, v0, vp = rng.normal(size=3)
        if quad == 2:
            # quadratic through x_{j-1}, x_j, x_{j+1}, evaluated at x_j - y
            p = _lagrange([-h, 0.0, h], [vm, v0, vp], -y)
            S = vp - 2 * v0 + vm
        else:
            p = _lagrange([-h, 0.0], [vm, v0], -y)
            S = 0.0
        J_quad = 0.5 * alpha * np.sum(wq * np.exp(-alpha * y) * p)
        J_orc = 0.5 * (W0 * v0 + W1 * vm + R * S)
        assert J_orc == pytest.approx(J_quad, rel=1e-12, abs=1e-14)


# --------------------------------------------------------------------------
# L^{-1} against direct O(N^2) quadrature of the Green's-function integral
# --------------------------------------------------------------------------
def _stencil_L(k, n, periodic):
    """Nodes of the interpolant used by J^L on the cell [x_{k-1}, x_k]."""
    if periodic or k + 1 <= n - 1:
        return [k - 1, k, k + 1]
    return [k - 2, k - 1, k]


def _stencil_R(k, n, periodic):
    """Nodes of the interpolant used by J^R on the cell [x_k, x_{k+1}]."""
    if periodic or k - 1 >= 0:
        return [k - 1, k, k + 1]
    return [k, k + 1, k + 2]


def _cell_integral(alpha, h, nodes, vals, a_cell, xj, sign, g, gw):
    """(alpha/2) int_cell e^{-alpha |x_j - y|} p(y) dy with GL quadrature."""
    y = a_cell + 0.5 * h * (g + 1.0)
    p = _lagrange([k * h for k in nodes], vals, y)
    return 0.5 * alpha * np.sum(0.5 * h * gw * np.exp(-alpha * sign * (xj - y)) * p)


def _linv_brute(v, nu, periodic, quad):
    n = v.size
    h = 1.0
    alpha = nu / h
    g, gw = _gl(24)
    x = np.arange(n) * h
    val = (lambda k: v[k % n]) if periodic else (lambda k: v[k])
    w = np.zeros(n)
    if periodic:
        Lper = n * h
        fac = 1.0 / (1.0 - np.exp(-alpha * Lper))
        for j in range(n):
            IL = IR = 0.0
            for k in range(j - n + 1, j + 1):          # cells [x_{k-1}, x_k] left of x_j
                nodes = _stencil_L(k, n, True) if quad == 2 else [k - 1, k]
                IL += _cell_integral(alpha, h, nodes, [val(i) for i in nodes], (k - 1) * h, x[j], 1.0, g, gw)
            for k in range(j, j + n):                  # cells [x_k, x_{k+1}] right of x_j
                nodes = _stencil_R(k, n, True) if quad == 2 else [k, k + 1]
                IR += _cell_integral(alpha, h, nodes, [val(i) for i in nodes], k * h, x[j], -1.0, g, gw)
            w[j] = fac * (IL + IR)
        return w
    IL = np.zeros(n)
    IR = np.zeros(n)
    for j in range(n):
        for k in range(1, j + 1):
            nodes = _stencil_L(k, n, False) if quad == 2 else [k - 1, k]
            IL[j] += _cell_integral(alpha, h, nodes, [val(i) for i in nodes], (k - 1) * h, x[j], 1.0, g, gw)
        for k in range(j, n - 1):
            nodes = _stencil_R(k, n, False) if quad == 2 else [k, k + 1]
            IR[j] += _cell_integral(alpha, h, nodes, [val(i) for i in nodes], k * h, x[j], -1.0, g, gw)
    # homogeneous part A e^{-alpha(x-a)} + B e^{-alpha(b-x)} with w(a)=v(a), w(b)=v(b)
    mu = np.exp(-alpha * (n - 1) * h)
    M = np.array([[1.0, mu], [mu, 1.0]])
    A, B = np.linalg.solve(M, [v[0] - IL[0] - IR[0], v[-1] - IL[-1] - IR[-1]])
    return IL + IR + A * np.exp(-alpha * x) + B * np.exp(-alpha * (x[-1] - x))


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("quad", [1, 2])
@pytest.mark.parametrize("nu", [0.05, 0.7, 3.0])
@pytest.mark.parametrize("n", [3, 4, 9, 12])
def test_linv_equals_green_function_quadrature(bc, quad, nu, n):
    rng = np.random.default_rng(100 + n)
    v = rng.normal(size=n)
    w_orc = oracle.linv_line(v, nu, bc, quad)
    w_ref = _linv_brute(v, nu, bc == "periodic", quad)
    np.testing.assert_allclose(w_orc, w_ref, rtol=1e-12, atol=1e-13)


def test_dirichlet_ends_are_reproduced():
    """The corrected L^{-1} returns the data at both end nodes, so D v = 0 there."""
    rng = np.random.default_rng(3)
    v = rng.normal(size=33)
    w = oracle.linv_line(v, 0.8, "dirichlet", 2)
    assert w[0] == pytest.approx(v[0], abs=1e-14)
    assert w[-1] == pytest.approx(v[-1], abs=1e-14)


# --------------------------------------------------------------------------
# Fourier symbols (Sec. 3): D-hat = (k/alpha)^2 / (1 + (k/alpha)^2)
# --------------------------------------------------------------------------
def _weights_by_quadrature(nu):
    """(d, W0, W1, R) from numerical integrals of the Lagrange basis."""
    g, gw = _gl(30)
    t = 0.5 * nu * (g + 1.0)
    wt = 0.5 * nu * gw * np.exp(-t)
    s = -t / nu
    lm, l0, lp = s * (s - 1) / 2, (1 - s) * (1 + s), s * (s + 1) / 2   # nodes s=-1,0,1
    cm, c0, cp = (np.sum(wt * lm), np.sum(wt * l0), np.sum(wt * lp))
    # cm v_{j-1} + c0 v_j + cp v_{j+1} = W0 v_j + W1 v_{j-1} + R (v_{j+1} - 2 v_j + v_{j-1})
    R = cp
    W1 = cm - R
    W0 = c0 + 2 * R
    return np.exp(-nu), W0, W1, R


@pytest.mark.parametrize("nu", [0.02, 0.5, 1.333, 4.0])
@pytest.mark.parametrize("n", [16, 37, 256])
def test_periodic_symbol_is_the_geometric_series(nu, n):
    """Every Fourier mode is an eigenvector of the periodic L^{-1} with
    eigenvalue Re[(W0 + W1 e^{-i th} + R(2cos th - 2)) / (1 - d e^{-i th})]."""
    d, W0, W1, R = _weights_by_quadrature(nu)
    j = np.arange(n)
    for k in [0, 1, 3, n // 2]:
        th = 2 * np.pi * k / n
        sym = np.real((W0 + W1 * np.exp(-1j * th) + R * (2 * np.cos(th) - 2)) / (1 - d * np.exp(-1j * th)))
        for phase in (0.0, 0.9):
            v = np.cos(th * j + phase)
            np.testing.assert_allclose(oracle.linv_line(v, nu, "periodic", 2), sym * v, rtol=1e-12, atol=1e-13)


def test_periodic_preserves_constants():
    for nu in (0.01, 0.6, 5.0):
        np.testing.assert_allclose(oracle.linv_line(np.ones(21), nu, "periodic", 2), 1.0, rtol=1e-13)


@pytest.mark.parametrize("quad, order", [(1, 2.0), (2, 3.0)])
def test_symbol_converges_to_continuous_symbol(quad, order):
    """D_h -> D-hat = (k/alpha)^2/(1+(k/alpha)^2) as h -> 0 at fixed alpha, k.
    The relative error in D falls like h^2 for the linear interpolant and like
    h^3 for the quadratic one (at least second order, as Sec. 3.2 states)."""
    alpha, k, L = 3.0, 2.0, 2 * np.pi
    errs = []
    for n in (64, 128, 256, 512):
        h = L / n
        x = np.arange(n) * h
        v = np.cos(k * x)
        Dv = v - oracle.linv_line(v, alpha * h, "periodic", quad)
        Dhat = (k / alpha) ** 2 / (1 + (k / alpha) ** 2)
        errs.append(np.max(np.abs(Dv - Dhat * v)) / Dhat)
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - order) < 0.2) and abs(rates[-1] - order) < 0.1, (errs, rates)


# --------------------------------------------------------------------------
# Coefficients A_p (eq. update_P), Table 1 and the stability polynomial
# --------------------------------------------------------------------------
def test_Ap_match_explicit_schemes():
    rows = _read_golden("explicit_updates.txt")
    for beta in (0.3, 1.0, 1.2345, 2.0):
        A = oracle.Ap(3, beta)
        for row in rows:
            p = int(row[0])
            coefs = [Fraction(c) for c in row[1:]]
            ref = sum(float(c) * beta ** (2 * (i + 1)) for i, c in enumerate(coefs))
            assert A[p - 1] == pytest.approx(ref, rel=1e-14, abs=1e-15)


def test_beta_max_matches_table1():
    for P, _, printed in _read_golden("table1_beta_max.txt"):
        P, printed = int(P), float(printed)
        b = oracle.beta_max(P)
        # The roots of eq. (Stab_cond) round to the printed digits for P = 1, 4
        # and 5; P = 2 (root 1.48393, printed 1.4840) and P = 3 (root 1.23429,
        # printed 1.2345) are a little off in the last digits.
        tol = {2: 1e-4, 3: 3e-4}.get(P, 5e-5)
        assert abs(b - printed) <= tol, (P, b, printed)
        assert -np.sum(oracle.Ap(P, b)) == pytest.approx(4.0, abs=1e-10)


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
def test_stability_polynomial_within_cohn_schur_range(P):
    """0 <= S(beta, D) <= 4 for D in [0, 1], 0 < beta <= beta_max (Sec. 3.1)."""
    bm = oracle.beta_max(P)
    Dh = np.linspace(0, 1, 201)
    for beta in np.linspace(0.05, bm, 12):
        A = oracle.Ap(P, beta)
        S = -sum(A[p] * Dh ** (p + 1) for p in range(P))
        assert S.min() >= -1e-12 and S.max() <= 4 + 1e-9
    A = oracle.Ap(P, bm * 1.02)
    assert -np.sum(A) > 4.0


# --------------------------------------------------------------------------
# A-stability of the discrete operators
# --------------------------------------------------------------------------
@pytest.mark.parametrize("nu", [0.01, 0.3, 1.0, 4.0])
@pytest.mark.parametrize("n", [5, 12, 33])
def test_dirichlet_D_spectrum_in_unit_interval(nu, n):
    M = np.stack([oracle.D_axis(np.eye(n)[i], 0, nu, "dirichlet") for i in range(n)], axis=1)
    ev = np.linalg.eigvals(M)
    assert np.max(np.abs(ev.imag)) < 1e-10
    assert ev.real.min() > -1e-12 and ev.real.max() < 1.0


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("cfl", [1.0, 4.0, 10.0])
def test_energy_bounded_long_run(P, cfl):
    """10^4 steps at beta_max with rough data stay bounded (A-stability)."""
    n = 64
    rng = np.random.default_rng(11)
    u0 = rng.normal(size=n)
    beta = oracle.beta_max(P)
    nu = beta / cfl
    u1 = oracle.start(u0, nu, P, beta, "periodic")
    _, u = oracle.run(u0, u1, 10_000, nu, P, beta, "periodic")
    assert np.all(np.isfinite(u))
    assert np.abs(u).max() < 20 * np.abs(u0).max()


def test_energy_grows_beyond_beta_max():
    """The bound above has teeth: beta well above beta_max blows up."""
    n, P, cfl = 64, 2, 10.0
    u0 = np.cos(np.pi * np.arange(n))          # the highest mode
    beta = 1.3 * oracle.beta_max(P)
    nu = beta / cfl
    u1 = oracle.start(u0, nu, P, beta, "periodic")
    _, u = oracle.run(u0, u1, 400, nu, P, beta, "periodic")
    assert not np.all(np.abs(u) < 1e3)


# --------------------------------------------------------------------------
# Order 2P in time (Sec. 3 numerical results, eq. update_P)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("P, dts, n", [(1, (0.2, 0.1, 0.05), 1024),
                                       (2, (0.4, 0.2, 0.1), 2048),
                                       (3, (0.4, 0.2, 0.1), 4096)])
@pytest.mark.parametrize("start", ["exact", "convolution"])
def test_standing_wave_converges_at_order_2P(P, dts, n, start):
    L, T = 2 * np.pi, 4.0
    h = L / n
    x = np.arange(n) * h
    u0 = np.cos(x)                               # exact: cos(x) cos(t), c = 1
    beta = oracle.beta_max(P)
    errs = []
    for dt in dts:
        nu = beta / dt * h
        u1 = u0 * np.cos(dt) if start == "exact" else oracle.start(u0, nu, P, beta, "periodic")
        ns = int(round(T / dt))
        _, u = oracle.run(u0, u1, ns - 1, nu, P, beta, "periodic")
        errs.append(np.sqrt(h * np.sum((u - u0 * np.cos(ns * dt)) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(np.abs(rates - 2 * P) < 0.25 * P + 0.1), (errs, rates)


# --------------------------------------------------------------------------
# ADI composition (Sec. 4) against dense Kronecker products of the printed
# explicit schemes
# --------------------------------------------------------------------------
def _dense_D(n, nu, bc):
    return np.stack([oracle.D_axis(np.eye(n)[i], 0, nu, bc) for i in range(n)], axis=1)


def _explicit_F(C, D, P, beta):
    """The schemes printed after eq. (Full_2D) for P = 1, 2, 3."""
    b2, b4, b6 = beta ** 2, beta ** 4, beta ** 6
    F = -b2 * C
    if P >= 2:
        F = F - (b2 * D - b4 / 12 * C) @ C
    if P >= 3:
        F = F - (b2 * D @ D - b4 / 6 * C @ D + b6 / 360 * C @ C) @ C
    return F


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("P", [1, 2, 3])
def test_2d_F_matches_dense_adi_formula(bc, P):
    nx, ny = 7, 6
    nux, nuy = 0.45, 0.9
    beta = oracle.beta_max(P)
    Dx, Dy = _dense_D(nx, nux, bc), _dense_D(ny, nuy, bc)
    Ix, Iy = np.eye(nx), np.eye(ny)
    # C order (ny, nx): flat index = y*nx + x
    Lx_inv = np.kron(Iy, Ix - Dx)
    Ly_inv = np.kron(Iy - Dy, Ix)
    C = Ly_inv @ np.kron(Iy, Dx) + Lx_inv @ np.kron(Dy, Ix)      # eq. (C_def_ADI)
    D = np.eye(nx * ny) - Lx_inv @ Ly_inv                          # eq. (D_def_ADI)
    Fm = _explicit_F(C, D, P, beta)
    rng = np.random.default_rng(5)
    u = rng.normal(size=(ny, nx))
    F = oracle.F(u, (nux, nuy), P, beta, bc)
    np.testing.assert_allclose(F.ravel(), Fm @ u.ravel(), rtol=1e-11, atol=1e-12)


@pytest.mark.parametrize("P", [1, 2, 3])
def test_3d_F_matches_dense_adi_formula(P):
    nx, ny, nz = 4, 5, 6
    nus = (0.5, 0.8, 1.1)
    bc = "dirichlet"
    beta = oracle.beta_max(P)
    Dg = [_dense_D(n, nu, bc) for n, nu in zip((nx, ny, nz), nus)]
    I = [np.eye(n) for n in (nx, ny, nz)]
    # C order (nz, ny, nx)
    ops = [np.kron(I[2], np.kron(I[1], Dg[0])), np.kron(I[2], np.kron(Dg[1], I[0])),
           np.kron(Dg[2], np.kron(I[1], I[0]))]
    Id = np.eye(nx * ny * nz)
    Li = [Id - o for o in ops]
    C = Li[1] @ Li[2] @ ops[0] + Li[2] @ Li[0] @ ops[1] + Li[0] @ Li[1] @ ops[2]   # eq. (C_def_ADI_3)
    D = Id - Li[0] @ Li[1] @ Li[2]                                                 # eq. (D_def_ADI_3)
    Fm = _explicit_F(C, D, P, beta)
    rng = np.random.default_rng(6)
    u = rng.normal(size=(nz, ny, nx))
    F = oracle.F(u, nus, P, beta, bc)
    np.testing.assert_allclose(F.ravel(), Fm @ u.ravel(), rtol=1e-11, atol=1e-12)


def test_1d_F_is_sum_of_Ap_powers():
    """In 1D, F = sum_p A_p D^p (eq. update_P), D from repeated application."""
    rng = np.random.default_rng(8)
    u = rng.normal(size=40)
    for P in (1, 2, 3, 5):
        beta = 0.9 * oracle.beta_max(P)
        A = oracle.Ap(P, beta)
        ref = sum(A[p - 1] * oracle.D_axis(u, 0, 0.7, "dirichlet", power=p) for p in range(1, P + 1))
        np.testing.assert_allclose(oracle.F(u, 0.7, P, beta, "dirichlet"), ref, rtol=1e-12, atol=1e-13)


def test_adi_reduces_to_1d_for_field_constant_in_y():
    """Setting C = D recovers the 1D scheme (Sec. 4): with a field constant
    along a periodic y axis, D_y u = 0 and every row follows eq. update_P."""
    rng = np.random.default_rng(9)
    f = rng.normal(size=24)
    u = np.tile(f, (10, 1))
    for P in (1, 2, 3):
        beta = oracle.beta_max(P)
        F2 = oracle.F(u, (0.6, 0.6), P, beta, "periodic")
        F1 = oracle.F(f, 0.6, P, beta, "periodic")
        np.testing.assert_allclose(F2, np.tile(F1, (10, 1)), rtol=1e-11, atol=1e-12)


def test_table3_operation_counts():
    """Table 3: 1, 3, 6 applications of C or D for P = 1, 2, 3."""
    u = np.random.default_rng(1).normal(size=(6, 5))
    for P, expect in [(1, 1), (2, 3), (3, 6), (4, 10)]:
        _, nops = oracle.F(u, 0.5, P, 1.0, "dirichlet", return_nops=True)
        assert nops == expect


def test_start_value_taylor_accuracy():
    """u^1 = u^0 + F/2 matches u(dt) = cos(x) cos(dt) to O(dt^{2P+2}) (Sec. 3.2)."""
    n = 4096
    h = 2 * np.pi / n
    x = np.arange(n) * h
    u0 = np.cos(x)
    for P in (1, 2):
        beta = oracle.beta_max(P)
        errs = []
        for dt in (0.4, 0.2):
            u1 = oracle.start(u0, beta / dt * h, P, beta, "periodic")
            errs.append(np.max(np.abs(u1 - np.cos(dt) * u0)))
        rate = np.log2(errs[0] / errs[1])
        assert abs(rate - (2 * P + 2)) < 0.3, (P, errs, rate)


# --------------------------------------------------------------------------
# Table 2: the paper's 2D refinement study, reproduced value by value
# --------------------------------------------------------------------------
TABLE2_BETA = {1: 2.0, 2: 1.48, 3: 1.2}


def _table2_error(P, dt, beta, n=641, T=1.2):
    x = np.linspace(-1.0, 1.0, n)
    h = x[1] - x[0]
    X, Y = np.meshgrid(x, x)
    u0 = np.sin(np.pi * X) * np.sin(np.pi * Y)
    w = np.sqrt(2.0) * np.pi
    nu = beta / dt * h
    up, uc = u0, u0 * np.cos(w * dt)            # analytic start value (Sec. 3.2)
    errs = [np.sqrt(h * h * np.sum((uc - u0 * np.cos(w * dt)) ** 2))]
    for k in range(2, int(round(T / dt)) + 1):
        up, uc = uc, oracle.step(up, uc, nu, P, beta, "dirichlet")
        errs.append(np.sqrt(h * h * np.sum((uc - u0 * np.cos(w * k * dt)) ** 2)))
    return max(errs)


@pytest.mark.slow
@pytest.mark.parametrize("row", _read_golden("table2_adi_errors.txt"), ids=lambda r: f"P{r[0]}-dt{r[1]}")
def test_table2_errors_reproduced(row):
    """Every error of Table 2 within 1% (3 printed digits), with the quadratic
    local interpolant, beta = 2, 1.48, 1.2 and the analytic start value."""
    P, dt, err = int(row[0]), float(row[1]), float(row[2])
    ours = _table2_error(P, dt, TABLE2_BETA[P])
    assert ours == pytest.approx(err, rel=0.01)


def test_thread_count_does_not_change_the_oracle():
    """The oracle's parallel loops run over independent lines, so one thread
    and all threads give bitwise the same steps (the single-thread timing of
    the benchmark measures the same computation)."""
    from paper_1308_3214_gb300 import workloads
    n0 = oracle.num_threads()
    u = workloads.gaussian_2d(96, seed=1002, ny=80)
    beta = oracle.beta_max(3)
    try:
        oracle.set_threads(1)
        one = oracle.run(u, u, 4, beta / 2.0, 3, beta, "dirichlet")
        oracle.set_threads(max(n0, 2))
        many = oracle.run(u, u, 4, beta / 2.0, 3, beta, "dirichlet")
    finally:
        oracle.set_threads(n0)
    for a, b in zip(one, many):
        assert np.array_equal(a, b)
