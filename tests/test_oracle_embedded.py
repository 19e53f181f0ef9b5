"""Pins of the oracle's embedded-boundary path (Sec. 4.3: line objects).

A line object is the part of a grid line inside a domain: interior grid nodes
plus a boundary point at each end, off the grid, where the Dirichlet data sit.
The oracle's L^{-1} on it is checked against direct quadrature of the
Green's-function integral, against the rectangular line it must reduce to,
and through the whole 2D scheme against the exact standing mode of a disk.
CPU only.
"""
import numpy as np
import pytest

import oracle
from paper_1308_3214_gb300 import workloads

scipy_special = pytest.importorskip("scipy.special")


def _lagrange(nodes, vals, y):
    out = np.zeros_like(y)
    for i, (xi, vi) in enumerate(zip(nodes, vals)):
        li = np.ones_like(y)
        for k, xk in enumerate(nodes):
            if k != i:
                li *= (y - xk) / (xi - xk)
        out += vi * li
    return out


def _linv_obj_brute(v, h, da, db, alpha):
    """w_j = (alpha/2) int_a^b e^{-alpha|x_j - y|} p(y) dy + A e^{-alpha(x_j-a)} + B e^{-alpha(b-x_j)}.

    The integral runs cell by cell with 30-point Gauss-Legendre quadrature;
    the left-going part integrates, over cell k, the quadratic that the
    recurrence uses for destination k (x_{k-1}, x_k, x_{k+1}, shifted inward in
    the last cell), the right-going part the mirror rule; A, B make w vanish
    at both boundary points.
    """
    m = v.size
    N = m + 1
    x = np.concatenate([[0.0], da + h * np.arange(m), [da + h * (m - 1) + db]])
    u = np.concatenate([[0.0], v, [0.0]])
    g, gw = np.polynomial.legendre.leggauss(30)

    def cell(lo, hi, nodes, xj):
        y = 0.5 * (hi - lo) * (g + 1.0) + lo
        p = _lagrange(x[nodes], u[nodes], y)
        return 0.5 * alpha * np.sum(0.5 * (hi - lo) * gw * np.exp(-alpha * np.abs(xj - y)) * p)

    IL = np.zeros(N + 1)
    IR = np.zeros(N + 1)
    for j in range(N + 1):
        for k in range(1, j + 1):                     # cells [x_{k-1}, x_k] left of x_j
            nodes = [k - 1, k, k + 1] if k + 1 <= N else [k - 2, k - 1, k]
            IL[j] += cell(x[k - 1], x[k], nodes, x[j])
        for k in range(j, N):                         # cells [x_k, x_{k+1}] right of x_j
            nodes = [k - 1, k, k + 1] if k >= 1 else [k, k + 1, k + 2]
            IR[j] += cell(x[k], x[k + 1], nodes, x[j])
    mu = np.exp(-alpha * (x[N] - x[0]))
    A, B = np.linalg.solve([[1.0, mu], [mu, 1.0]], [-IL[0] - IR[0], -IL[N] - IR[N]])
    w = IL + IR + A * np.exp(-alpha * (x - x[0])) + B * np.exp(-alpha * (x[N] - x))
    return w[1:-1]


@pytest.mark.parametrize("m", [1, 2, 3, 6, 11])
@pytest.mark.parametrize("gaps", [(1.0, 1.0), (0.37, 0.81), (1e-3, 0.5), (0.9, 2e-4), (1.6, 0.05)])
@pytest.mark.parametrize("nu", [0.05, 0.8, 3.5])
def test_line_object_equals_green_function_quadrature(m, gaps, nu):
    rng = np.random.default_rng(31 * m + 7)
    h = 0.2
    alpha = nu / h
    da, db = gaps[0] * h, gaps[1] * h
    v = rng.normal(size=m)
    w = oracle.linv_obj(v, h, da, db, alpha)
    ref = _linv_obj_brute(v, h, da, db, alpha)
    np.testing.assert_allclose(w, ref, rtol=1e-11, atol=1e-12 * np.abs(v).max())


@pytest.mark.parametrize("m", [1, 2, 5, 40])
def test_unit_gaps_give_the_rectangular_dirichlet_line(m):
    """With both boundary points one spacing away, a line object is the
    rectangular Dirichlet line of m + 2 nodes with zero end values."""
    rng = np.random.default_rng(m)
    h, nu = 0.05, 0.9
    v = rng.normal(size=m)
    w = oracle.linv_obj(v, h, h, h, nu / h)
    ref = oracle.linv_line(np.concatenate([[0.0], v, [0.0]]), nu, "dirichlet", 2)[1:-1]
    np.testing.assert_allclose(w, ref, rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("gaps", [(1.0, 1.0), (0.3, 0.7), (1e-3, 1e-2), (1e-5, 0.99)])
@pytest.mark.parametrize("nu", [0.3, 1.0, 3.0])
def test_line_object_D_spectrum_in_unit_interval(gaps, nu):
    """D = 1 - L^{-1} on a line object has a real spectrum in [0, 1), as the
    rectangular Dirichlet line has (the ingredient of A-stability), for any
    end gaps."""
    m, h = 24, 0.1
    M = np.column_stack([oracle.linv_obj(e, h, gaps[0] * h, gaps[1] * h, nu / h) for e in np.eye(m)])
    ev = np.linalg.eigvals(np.eye(m) - M)
    assert np.abs(ev.imag).max() < 1e-10
    assert ev.real.min() > 0.0 and ev.real.max() < 1.0


def _rect_grid(n, xa, xb, ya, yb, lo=-1.1, hi=1.1):
    """An axis-aligned rectangle with its sides between grid lines."""
    h = (hi - lo) / (n - 1)
    xs = lo + h * np.arange(n)
    mx, my = (xs > xa) & (xs < xb), (xs > ya) & (xs < yb)
    ix, iy = np.flatnonzero(mx), np.flatnonzero(my)
    i64 = lambda a: np.asarray(a, dtype=np.int64)
    return workloads.EmbeddedGrid(
        n, n, lo, lo, h, h,
        i64(np.where(my, ix[0], 1)), i64(np.where(my, ix[-1], 0)),
        np.full(n, xs[ix[0]] - xa), np.full(n, xb - xs[ix[-1]]),
        i64(np.where(mx, iy[0], 1)), i64(np.where(mx, iy[-1], 0)),
        np.full(n, xs[iy[0]] - ya), np.full(n, yb - xs[iy[-1]]),
        my[:, None] & mx[None, :])


@pytest.mark.parametrize("P", [1, 2, 3])
def test_grid_aligned_rectangle_gives_the_rectangular_scheme(P):
    """A rectangle whose sides pass through grid nodes: every line object has
    unit gaps, and F is the rectangular Dirichlet F of the same grid."""
    n, h = 14, 0.1
    g = _rect_grid(n, -1.1 + 0.5 * h, 1.1 - 0.5 * h, -1.1 + 0.5 * h, 1.1 - 0.5 * h)
    g.ra[:] = g.rb[:] = g.ca[:] = g.cb[:] = g.hx            # sides on the outer nodes
    rng = np.random.default_rng(P)
    u = np.where(g.mask, rng.normal(size=(n, n)), 0.0)
    nu = 0.8
    beta = oracle.beta_max(P)
    Fe = oracle.F_embed(u, g, nu / g.hx, P, beta)
    Fr = oracle.F(u, nu, P, beta, "dirichlet")
    np.testing.assert_allclose(Fe, Fr, rtol=0, atol=1e-13 * np.abs(Fr).max())


def test_rectangle_operators_commute_and_stay_bounded():
    """On a rectangle off the grid lines the x and y line objects are the same
    on every row / column, so L_x^{-1} L_y^{-1} = L_y^{-1} L_x^{-1}, and the
    scheme stays bounded at CFL 10 (the A-stable regime of Sec. 4): no growth
    from step 250 to step 1000 (modes near the edge of the stability range
    oscillate with a large but fixed amplitude)."""
    g = _rect_grid(41, -0.9333, 0.8777, -0.7712, 0.9101)
    u = workloads.random_field((g.ny, g.nx), 9) * g.mask
    alpha = 1.4839 / (10 * g.hx)
    a = oracle.linv_axis_embed(oracle.linv_axis_embed(u, 1, g, alpha), 0, g, alpha)
    b = oracle.linv_axis_embed(oracle.linv_axis_embed(u, 0, g, alpha), 1, g, alpha)
    np.testing.assert_allclose(a, b, atol=1e-13 * np.abs(a).max())
    P = 2
    beta = oracle.beta_max(P)
    norms = [np.linalg.norm(oracle.run_embed(u, k, g, beta / (10 * g.hx), P, beta)) for k in (250, 500, 1000)]
    assert max(norms[1:]) < 1.5 * norms[0]


@pytest.mark.parametrize("P", [1, 2])
def test_disk_standing_mode_converges(P):
    """u = J_0(k r) cos(k t), J_0(k) = 0, is the exact solution on the unit disk
    with zero Dirichlet data.  Refining h and dt together at CFL 1, the error
    at t = 0.5 falls at second order (the boundary cells bound the spatial
    order), and the fourth-order scheme is the more accurate one."""
    k = scipy_special.jn_zeros(0, 1)[0]
    T = 0.5
    errs = []
    for n in (45, 89, 177):
        g = workloads.disk_grid(n)
        x, y = g.coords()
        r = np.hypot(*np.meshgrid(x, y))
        u0 = np.where(g.mask, scipy_special.j0(k * r), 0.0)
        ns = int(round(T / g.hx))
        beta = oracle.beta_max(P)
        u = oracle.run_embed(u0, ns, g, beta / (T / ns), P, beta)
        ex = np.where(g.mask, scipy_special.j0(k * r) * np.cos(k * T), 0.0)
        errs.append(np.sqrt(g.hx * g.hy * np.sum((u - ex) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.9, (errs, rates)
    ref = {1: 1.0e-4, 2: 2.0e-5}[P]                   # observed 9.4e-5 and 1.7e-5 at n = 177
    assert errs[-1] < ref


def test_ellipse_grid_is_consistent():
    """Rows and columns of the ellipse of Sec. 4.3 see the same interior nodes,
    each grid line meets the domain in one interval, and every gap lies in
    (0, h] from the chord's end to the nearest interior node."""
    g = workloads.ellipse_grid(61)
    assert (g.mask == g.mask.T).all()                 # the ellipse is symmetric in x <-> y
    for j in range(g.ny):
        idx = np.flatnonzero(g.mask[j])
        if idx.size:
            assert (g.r0[j], g.r1[j]) == (idx[0], idx[-1])
    live = g.r0 <= g.r1
    assert (g.ra[live] > 0).all() and (g.ra[live] <= g.hx * (1 + 1e-12)).all()
    assert (g.rb[live] > 0).all() and (g.rb[live] <= g.hx * (1 + 1e-12)).all()
    x, y = g.coords()
    X, Y = np.meshgrid(x, y)
    inside = ((X + Y) / 4) ** 2 + (X - Y) ** 2 < 1.0
    assert (g.mask <= inside).all() and (inside & ~g.mask).sum() == 0


def test_disk_time_convergence_at_fixed_fine_grid():
    """The same standing mode on a 201^2 grid (h = 0.011) with 4..16 steps to
    t = 0.5 (CFL 11 down to 2.8): the second-order scheme converges at order
    2 in dt; the fourth-order one starts at order 3 or more at the largest
    steps and is 8 times or more as accurate, until both meet the spatial
    error of the boundary cells."""
    k = scipy_special.jn_zeros(0, 1)[0]
    g = workloads.disk_grid(201)
    x, y = g.coords()
    r = np.hypot(*np.meshgrid(x, y))
    u0 = np.where(g.mask, scipy_special.j0(k * r), 0.0)
    T = 0.5
    ex = np.where(g.mask, scipy_special.j0(k * r) * np.cos(k * T), 0.0)
    errs = {}
    for P in (1, 2):
        beta = oracle.beta_max(P)
        errs[P] = np.array([np.sqrt(g.hx * g.hy * np.sum(
            (oracle.run_embed(u0, ns, g, beta / (T / ns), P, beta) - ex) ** 2)) for ns in (4, 8, 16)])
    r1 = np.log2(errs[1][:-1] / errs[1][1:])
    r2 = np.log2(errs[2][:-1] / errs[2][1:])
    assert r1.min() > 1.9, (errs[1], r1)
    assert r2[0] > 3.0, (errs[2], r2)
    assert (errs[1] / errs[2]).min() > 8.0
