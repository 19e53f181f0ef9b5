"""GPU parity of the embedded-boundary path (Sec. 4.3) with the oracle.

Float64 on both sides.  Tolerance: relative L2 1e-12, or 100 eps64 h / g_min
when larger: the weights of a cell next to a boundary point at distance g
from the first interior node carry a factor h / g (the quadratic through two
nodes g apart), so two correct float64 evaluations of the same operator can
differ by about that factor times the rounding unit.
"""
import numpy as np
import pytest

import oracle
from paper_1308_3214_gb300 import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


def _tol(g):
    live_r, live_c = g.r0 <= g.r1, g.c0 <= g.c1
    gmin = min(g.ra[live_r].min(), g.rb[live_r].min(), g.ca[live_c].min(), g.cb[live_c].min())
    return max(1e-12, 100 * EPS64 * g.hx / gmin)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _solver(g, cfl, P):
    from paper_1308_3214_gb300 import molt
    return molt.EmbedSolver(g, dt=cfl * g.hx, P=P)


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("shape", [("ellipse", 61), ("ellipse", 257), ("disk", 90)])
@pytest.mark.parametrize("axis", [0, 1])
def test_linv_matches_oracle(shape, axis):
    g = workloads.ellipse_grid(shape[1]) if shape[0] == "ellipse" else workloads.disk_grid(shape[1])
    s = _solver(g, 1.7, 2)
    alpha = oracle.beta_max(2) / (1.7 * g.hx)
    v = workloads.random_field((g.ny, g.nx), 11 + axis) * g.mask
    got = s.linv(_dev(v), axis).cpu().numpy()
    ref = oracle.linv_axis_embed(v, axis, g, alpha)
    assert _rel(got, ref) <= _tol(g)
    assert not got[~g.mask].any()                      # nothing written outside the domain
    s.close()


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("cfl", [0.8, 3.0])
def test_F_matches_oracle(P, cfl):
    g = workloads.ellipse_grid(73)
    s = _solver(g, cfl, P)
    u = workloads.gaussian_embedded(g, seed=1006 + P, width=0.3)
    got = s.apply_F(_dev(u)).cpu().numpy()
    ref = oracle.F_embed(u, g, oracle.beta_max(P) / (cfl * g.hx), P, oracle.beta_max(P))
    assert _rel(got, ref) <= _tol(g)
    s.close()


@pytest.mark.parametrize("nsteps", [1, 2, 3, 4, 12])
def test_time_stepping_matches_oracle(nsteps):
    """start, then nsteps - 1 steps in place: every rotation of the three
    level buffers ends with (u^{n-1}, u^n) back in the caller's tensors."""
    g = workloads.ellipse_grid(65)
    P, cfl = 2, 1.5
    s = _solver(g, cfl, P)
    u0 = workloads.gaussian_embedded(g, seed=1006, width=0.25)
    up = _dev(u0)
    uc = s.start(up)
    s.step(up, uc, nsteps - 1)
    beta = oracle.beta_max(P)
    alpha = beta / (cfl * g.hx)
    ref_cur = oracle.run_embed(u0, nsteps, g, alpha, P, beta)
    ref_prev = oracle.run_embed(u0, nsteps - 1, g, alpha, P, beta)
    assert _rel(uc.cpu().numpy(), ref_cur) <= 10 * _tol(g)
    assert _rel(up.cpu().numpy(), ref_prev) <= 10 * _tol(g)
    s.close()


def test_solve_host_matches_oracle_on_a_large_ellipse():
    """801^2 grid (rows of up to 750 interior nodes): 3 steps from host memory."""
    g = workloads.ellipse_grid(801)
    P, cfl = 2, 2.0
    s = _solver(g, cfl, P)
    u0 = workloads.gaussian_embedded(g, seed=1006, width=0.15)
    got = s.solve_host(u0, 3)
    beta = oracle.beta_max(P)
    ref = oracle.run_embed(u0, 3, g, beta / (cfl * g.hx), P, beta)
    assert _rel(got, ref) <= 10 * _tol(g)
    s.close()


def test_longest_line_object():
    """A disk whose middle row holds 2045 interior nodes (the kernel's limit is 2046)."""
    g = workloads.disk_grid(2249, radius=1.0, half=1.1)
    assert (g.r1 - g.r0 + 1).max() <= 2046 and (g.r1 - g.r0 + 1).max() > 2000
    s = _solver(g, 1.0, 1)
    v = workloads.random_field((g.ny, g.nx), 5) * g.mask
    alpha = oracle.beta_max(1) / g.hx
    for axis in (0, 1):
        got = s.linv(_dev(v), axis).cpu().numpy()
        assert _rel(got, oracle.linv_axis_embed(v, axis, g, alpha)) <= _tol(g)
    s.close()


@pytest.mark.parametrize("P", [1, 2])
def test_disk_standing_mode_converges_on_the_gpu(P):
    """J_0(k r) cos(k t) with J_0(k) = 0 on the unit disk: second-order
    convergence at CFL 1 to t = 0.5, as the oracle shows."""
    special = pytest.importorskip("scipy.special")
    k = special.jn_zeros(0, 1)[0]
    T = 0.5
    errs = []
    for n in (89, 177, 353):
        g = workloads.disk_grid(n)
        x, y = g.coords()
        r = np.hypot(*np.meshgrid(x, y))
        ns = int(round(T / g.hx))
        s = _solver(g, T / ns / g.hx, P)
        u = s.solve_host(np.where(g.mask, special.j0(k * r), 0.0), ns)
        s.close()
        ex = np.where(g.mask, special.j0(k * r) * np.cos(k * T), 0.0)
        errs.append(np.sqrt(g.hx * g.hy * np.sum((u - ex) ** 2)))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert rates.min() > 1.9, (errs, rates)


# ---------------------------------------------------------------------------
# mixed precision: float32 sweeps of the difference form of D, time levels as
# float32 pairs.  A recurrence with decay d = exp(-alpha h) sums about
# 1/(1 - d) terms that matter, so one application of D carries a relative
# error of order eps32 (1 + 1/(1 - d)) in |D v|; L^{-1} v = v - D v inherits it
# scaled by |D v| / |L^{-1} v|; F (2P sweeps) compounds 2P of them; n steps add
# one F error each, 8 eps32 (1 + 1/(1 - d)) 2P sum_k |F_k| / |u_n|.  The cells
# next to a boundary point enter through second divided differences whose
# weights and coefficients are formed in float64 on the host, so no h / g
# factor reaches the float32 arithmetic.  The float64 bound is added to each.
# ---------------------------------------------------------------------------
EPS32 = 2.0 ** -24


def _mixed_unit(cfl, P):
    d = np.exp(-oracle.beta_max(P) / cfl)
    return EPS32 * (1.0 + 1.0 / (1.0 - d))


def _mixed(g, cfl, P):
    from paper_1308_3214_gb300 import molt
    return molt.EmbedSolver(g, dt=cfl * g.hx, P=P, prec="mixed")


@pytest.mark.parametrize("shape", [("ellipse", 61), ("ellipse", 257), ("disk", 90)])
@pytest.mark.parametrize("axis", [0, 1])
@pytest.mark.parametrize("cfl", [0.5, 1.7, 6.0])
def test_mixed_linv_matches_oracle(shape, axis, cfl):
    g = workloads.ellipse_grid(shape[1]) if shape[0] == "ellipse" else workloads.disk_grid(shape[1])
    s = _mixed(g, cfl, 2)
    alpha = oracle.beta_max(2) / (cfl * g.hx)
    v = workloads.random_field((g.ny, g.nx), 11 + axis) * g.mask
    got = s.linv(_dev(v), axis).cpu().numpy()
    ref = oracle.linv_axis_embed(v, axis, g, alpha)
    cond = np.linalg.norm(v - ref) / np.linalg.norm(ref)
    assert _rel(got, ref) <= _tol(g) + 16 * _mixed_unit(cfl, 2) * cond, _rel(got, ref)
    assert not got[~g.mask].any()
    s.close()


@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("cfl", [0.8, 3.0])
def test_mixed_F_matches_oracle(P, cfl):
    g = workloads.ellipse_grid(73)
    s = _mixed(g, cfl, P)
    u = workloads.gaussian_embedded(g, seed=1006 + P, width=0.3)
    got = s.apply_F(_dev(u)).cpu().numpy()
    ref = oracle.F_embed(u, g, oracle.beta_max(P) / (cfl * g.hx), P, oracle.beta_max(P))
    assert _rel(got, ref) <= _tol(g) + 16 * _mixed_unit(cfl, P) * 2 * P, _rel(got, ref)
    s.close()


def _step_tol(g, u0, nsteps, alpha, P, beta, cfl, ref):
    Fsum, a = 0.0, u0
    b = oracle.run_embed(u0, 1, g, alpha, P, beta)
    Fsum += np.linalg.norm(b - a) * 2                  # the start adds F(u0) / 2
    for _ in range(nsteps - 1):
        F = oracle.F_embed(b, g, alpha, P, beta)
        Fsum += np.linalg.norm(F)
        a, b = b, 2 * b - a + F
    return 10 * _tol(g) + 8 * _mixed_unit(cfl, P) * 2 * P * Fsum / np.linalg.norm(ref)


@pytest.mark.parametrize("nsteps", [1, 2, 3, 12])
def test_mixed_time_stepping_matches_oracle(nsteps):
    g = workloads.ellipse_grid(65)
    P, cfl = 2, 1.5
    s = _mixed(g, cfl, P)
    u0 = workloads.gaussian_embedded(g, seed=1006, width=0.25)
    up = _dev(u0)
    uc = s.start(up)
    s.step(up, uc, nsteps - 1)
    beta = oracle.beta_max(P)
    alpha = beta / (cfl * g.hx)
    ref_cur = oracle.run_embed(u0, nsteps, g, alpha, P, beta)
    assert _rel(uc.cpu().numpy(), ref_cur) <= _step_tol(g, u0, nsteps, alpha, P, beta, cfl, ref_cur)
    if nsteps > 1:
        ref_prev = oracle.run_embed(u0, nsteps - 1, g, alpha, P, beta)
        assert _rel(up.cpu().numpy(), ref_prev) <= _step_tol(g, u0, nsteps - 1, alpha, P, beta, cfl, ref_prev)
    s.close()


def test_mixed_solve_host_matches_oracle_on_a_large_ellipse():
    g = workloads.ellipse_grid(801)
    P, cfl = 2, 2.0
    s = _mixed(g, cfl, P)
    u0 = workloads.gaussian_embedded(g, seed=1006, width=0.15)
    got = s.solve_host(u0, 3)
    beta = oracle.beta_max(P)
    alpha = beta / (cfl * g.hx)
    ref = oracle.run_embed(u0, 3, g, alpha, P, beta)
    assert _rel(got, ref) <= _step_tol(g, u0, 3, alpha, P, beta, cfl, ref)
    s.close()


def test_mixed_longest_line_object():
    g = workloads.disk_grid(2249, radius=1.0, half=1.1)
    s = _mixed(g, 1.0, 1)
    v = workloads.random_field((g.ny, g.nx), 5) * g.mask
    alpha = oracle.beta_max(1) / g.hx
    for axis in (0, 1):
        got = s.linv(_dev(v), axis).cpu().numpy()
        ref = oracle.linv_axis_embed(v, axis, g, alpha)
        cond = np.linalg.norm(v - ref) / np.linalg.norm(ref)
        assert _rel(got, ref) <= _tol(g) + 16 * _mixed_unit(1.0, 1) * cond
    s.close()


@pytest.mark.parametrize("P", [1, 2])
def test_mixed_disk_standing_mode_matches_fp64_error(P):
    """The float32 sweeps leave the discretisation error of the float64 path
    unchanged (to 1 %) on the converging disk mode."""
    special = pytest.importorskip("scipy.special")
    k = special.jn_zeros(0, 1)[0]
    T = 0.5
    g = workloads.disk_grid(177)
    x, y = g.coords()
    r = np.hypot(*np.meshgrid(x, y))
    ns = int(round(T / g.hx))
    u0 = np.where(g.mask, special.j0(k * r), 0.0)
    ex = np.where(g.mask, special.j0(k * r) * np.cos(k * T), 0.0)
    errs = []
    for make in (_solver, _mixed):
        s = make(g, T / ns / g.hx, P)
        u = s.solve_host(u0, ns)
        s.close()
        errs.append(np.sqrt(g.hx * g.hy * np.sum((u - ex) ** 2)))
    assert abs(errs[1] - errs[0]) <= 0.01 * errs[0], errs


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_ellipse_matches_oracle(prec):
    """The timed workload itself: the ellipse on the 2048^2 grid (1,359,906
    interior nodes, lines of up to 903), P = 2, CFL 1, three steps from host
    memory in the launch configuration the benchmark uses."""
    g = workloads.ellipse_grid(2048)
    P, cfl = 2, 1.0
    s = molt_solver(g, cfl, P, prec)
    u0 = workloads.gaussian_embedded(g, seed=1006, width=0.15)
    got = s.solve_host(u0, 3)
    beta = oracle.beta_max(P)
    alpha = beta / (cfl * g.hx)
    ref = oracle.run_embed(u0, 3, g, alpha, P, beta)
    tol = 10 * _tol(g) if prec == "fp64" else _step_tol(g, u0, 3, alpha, P, beta, cfl, ref)
    assert _rel(got, ref) <= tol, (_rel(got, ref), tol)
    assert not got[~g.mask].any()
    s.close()


def molt_solver(g, cfl, P, prec):
    return _solver(g, cfl, P) if prec == "fp64" else _mixed(g, cfl, P)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_domains(prec):
    """A disk around one grid node (every line object has m = 1) and a disk
    between the nodes (no interior node: no line, nothing to do)."""
    from paper_1308_3214_gb300 import molt
    g = workloads.disk_grid(11, radius=0.15, half=1.1)
    assert g.mask.sum() == 1
    P, cfl = 2, 1.0
    beta = oracle.beta_max(P)
    alpha = beta / (cfl * g.hx)
    s = molt.EmbedSolver(g, dt=cfl * g.hx, P=P, prec=prec)
    u0 = np.where(g.mask, 0.7, 0.0)
    for axis in (0, 1):
        got = s.linv(_dev(u0), axis).cpu().numpy()
        ref = oracle.linv_axis_embed(u0, axis, g, alpha)
        assert abs(got - ref).max() <= (1e-12 if prec == "fp64" else 1e-6)
    got = s.solve_host(u0, 5)
    ref = oracle.run_embed(u0, 5, g, alpha, P, beta)
    assert abs(got - ref).max() <= (1e-12 if prec == "fp64" else 1e-6)
    s.close()
    g = workloads.disk_grid(10, radius=0.05, half=1.1)
    assert not g.mask.any()
    s = molt.EmbedSolver(g, dt=cfl * g.hx, P=P, prec=prec)
    z = np.zeros((g.ny, g.nx))
    assert not s.solve_host(z, 3).any()
    assert not s.apply_F(_dev(z)).cpu().numpy().any()
    s.close()
