"""mol_solve_dirichlet: 1D problems with time-dependent Dirichlet data
(Sec. 3.2) against the float64 oracle and an exact solution.

u = cos(k pi x) cos(k pi t) on [0, 1], c = 1, is an exact solution with zero
initial velocity and end data u_L(t) = cos(k pi t), u_R(t) = cos(k pi) u_L(t);
its time derivatives are (d_tt)^m u_side = (-(k pi)^2)^m u_side.  float64:
the fields equal the oracle's on the scale of the data (M steps of
recurrences with memory 1/(1-d): 4 eps64 M / (1-d) |u^0|); the errors
against the exact solution fall at order 2P.  Mixed: the same rates for the
low orders.  Zero data: the homogeneous stepping.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt

pytestmark = pytest.mark.gpu

K = 3
T = 7.0 / 6.0          # cos(3 pi T) = 0: the phase error shows at first order


def data_for(M, P, dt):
    t = dt * np.arange(M + 1)
    d = np.empty((M + 1, 2, P + 1))
    for m in range(P + 1):
        f = (-(K * np.pi) ** 2) ** m * np.cos(K * np.pi * t)
        d[:, 0, m] = f
        d[:, 1, m] = np.cos(K * np.pi) * f
    return d


def gpu_run(n, M, P, prec):
    dt = T / M
    s = molt.Solver((n,), dt=dt, P=P, bc="dirichlet", prec=prec, lo=[0.0], hi=[1.0])
    x = np.linspace(0, 1, n)
    out = s.solve_dirichlet(torch.from_numpy(np.cos(K * np.pi * x)).cuda(), M, data_for(M, P, dt)).cpu().numpy()
    alpha, nu = s.alpha, s.nu[0]
    s.close()
    return out, alpha, nu


def err(u, n):
    x = np.linspace(0, 1, n)
    h = 1.0 / (n - 1)
    return np.sqrt(h * np.sum((u - np.cos(K * np.pi * x) * np.cos(K * np.pi * T)) ** 2))


@pytest.mark.parametrize("P,M", [(1, 40), (2, 20), (3, 20)])
def test_fp64_matches_oracle(P, M):
    n = 2001
    g, alpha, nu = gpu_run(n, M, P, "fp64")
    d = data_for(M, P, T / M)
    gam = d / alpha ** (2 * np.arange(P + 1))
    x = np.linspace(0, 1, n)
    ref = oracle.run_bc(np.cos(K * np.pi * x), M, nu, P, oracle.beta_max(P), gam)
    scale = np.linalg.norm(np.cos(K * np.pi * x))
    assert np.linalg.norm(g - ref) <= 4 * 2.0 ** -52 * M / (1 - np.exp(-nu)) * scale
    assert g[0] == d[-1, 0, 0] and g[-1] == d[-1, 1, 0]


@pytest.mark.parametrize("P,M1,M2", [(1, 40, 80), (2, 40, 80), (3, 20, 40)])
def test_fp64_converges_at_order_2P(P, M1, M2):
    n = 4001
    e1, e2 = err(gpu_run(n, M1, P, "fp64")[0], n), err(gpu_run(n, M2, P, "fp64")[0], n)
    rate = np.log2(e1 / e2)
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, e1, e2, rate)


@pytest.mark.parametrize("P,M1,M2", [(1, 40, 80), (2, 40, 80)])
def test_mixed_converges(P, M1, M2):
    n = 4001
    e1, e2 = err(gpu_run(n, M1, P, "mixed")[0], n), err(gpu_run(n, M2, P, "mixed")[0], n)
    assert e2 > 1e-5
    rate = np.log2(e1 / e2)
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, e1, e2, rate)


def test_zero_data_is_the_homogeneous_stepping():
    n, P, M = 1001, 2, 12
    dt = 0.01
    x = np.linspace(0, 1, n)
    u0 = np.sin(np.pi * x) + 0.2 * np.sin(4 * np.pi * x)
    s = molt.Solver((n,), dt=dt, P=P, bc="dirichlet", prec="fp64", lo=[0.0], hi=[1.0])
    got = s.solve_dirichlet(torch.from_numpy(u0).cuda(), M, np.zeros((M + 1, 2, P + 1))).cpu().numpy()
    up = torch.from_numpy(u0).cuda()
    uc = s.start(up)
    s.step(up, uc, M - 1)
    ref = uc.cpu().numpy()
    assert np.abs(got - ref).max() <= 1e-14 * np.abs(u0).max()


def test_rejects_other_grids():
    s = molt.Solver((16, 16), dt=0.01, P=1, bc="dirichlet", prec="fp64")
    with pytest.raises(molt.MolError):
        s.solve_dirichlet(torch.zeros((16, 16), dtype=torch.float64, device="cuda"), 2, np.zeros((3, 2, 2)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_standing_wave_matches_oracle(prec):
    """The timed 1D workload: 10001 points, P = 3, CFL 2, the standing wave
    cos(3 pi x) cos(3 pi t) with its end data, 20 steps.  float64: the bound
    above.  Mixed: the stepping error model, 8 eps32 (1 + 1/(1 - d)) 2P
    sum_k |delta_k| / |u_M| with delta_k the oracle's own increment of step k
    (twice the first, half of which the start applies); the end values equal
    the data exactly in float64, to the float32 pairs' 48 bits in mixed."""
    n, P, M = 10001, 3, 20
    h = 1.0 / (n - 1)
    dt = 2.0 * h
    x = np.linspace(0, 1, n)
    u0 = np.cos(K * np.pi * x)
    d = data_for(M, P, dt)
    s = molt.Solver((n,), dt=dt, P=P, bc="dirichlet", prec=prec, lo=[0.0], hi=[1.0])
    got = s.solve_dirichlet(torch.from_numpy(u0).cuda(), M, d).cpu().numpy()
    alpha, nu = s.alpha, s.nu[0]
    s.close()
    gam = d / alpha ** (2 * np.arange(P + 1))
    beta = oracle.beta_max(P)
    traj = [u0] + [oracle.run_bc(u0, m, nu, P, beta, gam[:m + 1]) for m in range(1, M + 1)]
    ref = traj[M]
    if prec == "fp64":
        assert np.linalg.norm(got - ref) <= 4 * 2.0 ** -52 * M / (1 - np.exp(-nu)) * np.linalg.norm(u0)
    else:
        inc = 2 * np.linalg.norm(traj[1] - traj[0])
        inc += sum(np.linalg.norm(traj[k] - 2 * traj[k - 1] + traj[k - 2]) for k in range(2, M + 1))
        tol = 8 * 2.0 ** -24 * (1 + 1 / (1 - np.exp(-nu))) * 2 * P * inc / np.linalg.norm(ref)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= tol, (np.linalg.norm(got - ref) / np.linalg.norm(ref), tol)
    if prec == "fp64":
        assert got[0] == d[-1, 0, 0] and got[-1] == d[-1, 1, 0]
    else:                                   # levels held as float32 pairs: about 48 bits
        assert abs(got[0] - d[-1, 0, 0]) <= 2.0 ** -46 and abs(got[-1] - d[-1, 1, 0]) <= 2.0 ** -46
