"""mol_solve_source: the source terms of Sec. 4.1 (P = 1, 2) on the GPU.

float64: fields equal the oracle's (oracle.run_source) on the point-source
example and on a rectangle; the manufactured solution sin(pi x) sin(pi y)
cos(w t) is reached at order 2 (P = 1) and 4 (P = 2); the point-source
example's fourth-order wave is closer to the exact 2D point-source solution
than the second-order one, as on the oracle.  Mixed: the fourth-order rate at
coarse steps.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt

pytestmark = pytest.mark.gpu

import test_oracle_source as src


def gpu_source(shape, lo, hi, dt, P, prec, g, f, M, u0=None):
    s = molt.Solver(shape, dt=dt, P=P, bc="dirichlet", prec=prec, lo=lo, hi=hi)
    u0 = np.zeros(shape) if u0 is None else u0
    out = s.solve_source(torch.from_numpy(u0).cuda(), M, torch.from_numpy(g).cuda(), f).cpu().numpy()
    nu = s.nu
    s.close()
    return out, nu


@pytest.mark.parametrize("P", [1, 2])
def test_point_source_matches_oracle(P):
    n = 81
    g, f, nu, beta, dt, M, h = src.point_source_problem(n, P)
    got, nug = gpu_source((n, n), [-1.0, -1.0], [1.0, 1.0], dt, P, "fp64", g, f, M)
    ref = oracle.run_source(np.zeros((n, n)), M, nug, P, beta, dt ** 2, g, f)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_rectangle_with_initial_field_matches_oracle():
    shape, P, M, dt = (65, 97), 2, 9, 0.012
    rng = np.random.default_rng(5)
    y = np.linspace(0, 1, shape[0])[:, None]
    x = np.linspace(0, 1, shape[1])[None, :]
    u0 = np.sin(np.pi * x) * np.sin(2 * np.pi * y)
    g = rng.normal(size=shape)
    g[0, :] = g[-1, :] = g[:, 0] = g[:, -1] = 0.0
    f = np.cos(3.0 * dt * np.arange(M + 1))
    got, nu = gpu_source(shape, [0.0, 0.0], [1.0, 1.0], dt, P, "fp64", g, f, M, u0)
    ref = oracle.run_source(u0, M, nu, P, oracle.beta_max(P), dt ** 2, g, f)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def manufactured_error(n, P, M, prec):
    T, w = src.TW, src.W
    dt = T / M
    g = (2 * np.pi ** 2 - w ** 2) * src.mode(n)
    f = np.cos(w * dt * np.arange(M + 1))
    u, _ = gpu_source((n, n), [0.0, 0.0], [1.0, 1.0], dt, P, prec, g, f, M, src.mode(n))
    h = 1.0 / (n - 1)
    return np.sqrt(h * h * np.sum((u - src.mode(n) * np.cos(w * T)) ** 2))


@pytest.mark.parametrize("P,expect", [(1, 2), (2, 4)])
def test_fp64_manufactured_solution_converges(P, expect):
    e1, e2 = manufactured_error(321, P, 20, "fp64"), manufactured_error(321, P, 40, "fp64")
    rate = np.log2(e1 / e2)
    assert expect - 0.5 <= rate <= expect + 0.5, (P, e1, e2, rate)


def test_mixed_fourth_order_rate():
    e1, e2 = manufactured_error(321, 2, 10, "mixed"), manufactured_error(321, 2, 20, "mixed")
    assert e2 > 1e-5
    rate = np.log2(e1 / e2)
    assert 3.0 <= rate <= 4.5, (e1, e2, rate)


def test_point_source_fourth_order_is_closer_to_the_exact_wave():
    n = 161
    errs = {}
    for P in (1, 2):
        g, f, nu, beta, dt, M, h = src.point_source_problem(n, P)
        u, _ = gpu_source((n, n), [-1.0, -1.0], [1.0, 1.0], dt, P, "fp64", g, f, M)
        errs[P] = src.ray_errors(u, h, dt * M)
    assert all(e2 < 0.3 * e1 for e1, e2 in zip(errs[1], errs[2])), errs


def test_higher_orders_are_refused():
    s = molt.Solver((33, 33), dt=0.01, P=3, bc="dirichlet", prec="fp64")
    z = torch.zeros((33, 33), dtype=torch.float64, device="cuda")
    with pytest.raises(molt.MolError):
        s.solve_source(z, 2, z, np.zeros(3))


EPS32 = 2.0 ** -24


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_point_source_matches_oracle(prec):
    """The timed source workload: [-1, 1]^2 on 2048 x 2048 nodes, P = 2,
    CFL 2, the discrete delta 1/h^2 at the centre node times
    f(t) = sin(4 pi t)(1 - exp(-(t/0.2)^2)), four steps from rest.  Mixed:
    the stepping error model, 8 eps32 (1 + 1/(1 - d)) 2P sum_k |delta_k| /
    |u_M| with delta_k the oracle's own increment of step k (F plus the
    source terms; twice the first, half of which the start applies)."""
    n, P, M = 2048, 2, 4
    h = 2.0 / (n - 1)
    dt = 2.0 * h
    t = dt * np.arange(M + 1)
    g = np.zeros((n, n))
    g[n // 2, n // 2] = 1.0 / h ** 2
    f = np.sin(4 * np.pi * t) * (1.0 - np.exp(-(t / 0.2) ** 2))
    got, nu = gpu_source((n, n), [-1.0, -1.0], [1.0, 1.0], dt, P, prec, g, f, M)
    beta = oracle.beta_max(P)
    traj = [np.zeros((n, n))] + [oracle.run_source(np.zeros((n, n)), m, nu, P, beta, dt ** 2, g, f[:m + 1])
                                 for m in range(1, M + 1)]
    ref = traj[M]
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    if prec == "fp64":
        assert err <= 1e-12
    else:
        d = np.exp(-max(nu))
        inc = 2 * np.linalg.norm(traj[1] - traj[0])
        inc += sum(np.linalg.norm(traj[k] - 2 * traj[k - 1] + traj[k - 2]) for k in range(2, M + 1))
        assert err <= 8 * EPS32 * (1 + 1 / (1 - d)) * 2 * P * inc / np.linalg.norm(ref), err
