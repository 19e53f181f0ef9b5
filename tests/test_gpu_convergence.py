"""The paper's 1D convergence example (Sec. 3.2 numerical results: standing
wave sin(2 pi x), u_t = 0, homogeneous Dirichlet, dx = 1e-4) on the GPU.

float64: every field equals the oracle's (lines of 10001 points run on the
shared-memory kernels with the d^j table in global memory), and the errors
against the exact solution sin(2 pi x) cos(2 pi t) fall at order 2P.  At
t = 1.25 the exact solution vanishes, so the fields are compared on the
scale of the data: M steps of recurrences with memory 1/(1 - d) add about
eps64 M / (1 - d) |u^0| of rounding (4x that is the bound).
Mixed precision: the same rates while the error stays far above the float32
level of the levels (low orders).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt

pytestmark = pytest.mark.gpu

N = 10001
X = np.linspace(0.0, 1.0, N)
H = 1.0 / (N - 1)


def run_gpu(T, M, P, prec):
    dt = T / M
    s = molt.Solver((N,), dt=dt, P=P, bc="dirichlet", prec=prec, lo=[0.0], hi=[1.0])
    u0 = torch.from_numpy(np.sin(2 * np.pi * X)).cuda()
    up = u0.clone()
    uc = s.start(up)
    s.step(up, uc, M - 1)
    torch.cuda.synchronize()
    out = uc.cpu().numpy()
    s.close()
    return out


def run_oracle(T, M, P):
    beta = oracle.beta_max(P)
    nu = beta / (T / M) * H
    u0 = np.sin(2 * np.pi * X)
    _, uc = oracle.run(u0, oracle.start(u0, nu, P, beta, "dirichlet"), M - 1, nu, P, beta, "dirichlet")
    return uc


def err(u, T):
    return np.sqrt(H * np.sum((u - np.sin(2 * np.pi * X) * np.cos(2 * np.pi * T)) ** 2))


@pytest.mark.parametrize("P,M1,M2", [(1, 40, 80), (2, 40, 80), (3, 20, 40), (4, 20, 40), (5, 20, 40)])
def test_fp64_standing_wave_matches_oracle_and_converges(P, M1, M2):
    T = 1.25
    g1, g2 = run_gpu(T, M1, P, "fp64"), run_gpu(T, M2, P, "fp64")
    r1, r2 = run_oracle(T, M1, P), run_oracle(T, M2, P)
    scale = np.linalg.norm(np.sin(2 * np.pi * X))
    for g, r, M in ((g1, r1, M1), (g2, r2, M2)):
        d = np.exp(-oracle.beta_max(P) / (T / M) * H)
        assert np.linalg.norm(g - r) <= 4 * 2.0 ** -52 * M / (1 - d) * scale, (M, np.linalg.norm(g - r))
    rate = np.log2(err(g1, T) / err(g2, T))
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, rate)


@pytest.mark.parametrize("P,M1,M2", [(1, 40, 80), (2, 40, 80)])
def test_mixed_standing_wave_converges(P, M1, M2):
    T = 1.25
    e1, e2 = err(run_gpu(T, M1, P, "mixed"), T), err(run_gpu(T, M2, P, "mixed"), T)
    assert e2 > 1e-5
    rate = np.log2(e1 / e2)
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, e1, e2, rate)
