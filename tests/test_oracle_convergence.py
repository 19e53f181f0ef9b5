"""Temporal convergence of the oracle's scheme on the paper's 1D example
(Sec. 3.2 numerical results: standing wave u(x, 0) = sin(2 pi x), u_t = 0,
x in [0, 1], homogeneous Dirichlet, dx = 1e-4, beta = beta_max(P)).

The exact solution sin(2 pi x) cos(2 pi t) pins the whole stepping chain
(constants, the operator, the coefficient expansion, the start value, the
three-level update) independently of the oracle: the L2 error at a fixed
time falls as dt^{2P} (the order of eq. update_P) until the spatial error of
the quadrature floors it (the paper sees that floor in its 10th-order scheme).
At t = 1.25, cos(2 pi t) = 0 and the phase error shows at first order; at
t = 1 the wave is at an extremum, the phase error shows squared and the rate
doubles to 4P.  Reading of the figure (its values are not printed): rates
within one order of 2P (4P) for step pairs whose errors stay two decades
above the spatial floor.
"""
import numpy as np
import pytest

import oracle

N = 10001
X = np.linspace(0.0, 1.0, N)
H = 1.0 / (N - 1)


def error_at(T, M, P):
    beta = oracle.beta_max(P)
    dt = T / M
    nu = beta / dt * H
    u0 = np.sin(2 * np.pi * X)
    u1 = oracle.start(u0, nu, P, beta, "dirichlet")
    _, uc = oracle.run(u0, u1, M - 1, nu, P, beta, "dirichlet")
    exact = np.sin(2 * np.pi * X) * np.cos(2 * np.pi * T)
    return np.sqrt(H * np.sum((uc - exact) ** 2))


# (P, coarse step count, fine step count) at t = 1.25, errors >= 1e-7
CASES = [(1, 40, 80), (2, 40, 80), (3, 20, 40), (4, 20, 40), (5, 20, 40)]


@pytest.mark.parametrize("P,M1,M2", CASES)
def test_standing_wave_converges_at_order_2P(P, M1, M2):
    e1, e2 = error_at(1.25, M1, P), error_at(1.25, M2, P)
    assert e2 > 1e-7
    rate = np.log2(e1 / e2)
    assert 2 * P - 1.0 <= rate <= 2 * P + 0.5, (P, e1, e2, rate)


@pytest.mark.parametrize("P", [1, 2])
def test_rate_doubles_at_the_extremum(P):
    """t = 1: the wave sits at its maximum, so the O(dt^{2P}) phase error
    shows only squared (rate 4P)."""
    e1, e2 = error_at(1.0, 32, P), error_at(1.0, 64, P)
    rate = np.log2(e1 / e2)
    assert 4 * P - 0.5 <= rate <= 4 * P + 0.5, (P, e1, e2, rate)


def test_spatial_floor_is_far_below_the_temporal_error():
    """At dx = 1e-4 the spatial error of the quadratic rule sits near 1e-9:
    the highest order reaches it, the lowest does not come near."""
    floor = error_at(1.25, 160, 5)
    assert floor < 2e-9
    assert error_at(1.25, 160, 1) > 1e5 * floor
