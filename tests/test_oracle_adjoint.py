"""Pins of the oracle's transposed operators and adjoint (no GPU).

The adjoint has no counterpart in the paper; what fixes it is linear algebra:
  * (L^{-1})^T on a line equals the transpose of the dense matrix whose
    columns are L^{-1} applied to unit vectors (built with the forward
    routine, so a wrong statement in the transposed program shows up);
  * <A v, w> = <v, A^T w> for D_gamma, F and the trace map u^0 -> t;
  * the periodic L^{-1} is a symmetric circulant, so periodic F^T = F;
  * for the quadratic loss J = |T u^0 - d|^2 / 2 the central difference
    (J(u+e s) - J(u-e s)) / (2e) equals <grad J, s> up to rounding.
"""
import numpy as np
import pytest

import oracle


def dot(a, b):
    return float(np.sum(np.asarray(a) * np.asarray(b)))


def rel_dot_err(lhs, rhs, scale):
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("quad", [1, 2])
@pytest.mark.parametrize("n", [3, 4, 7, 16, 33])
@pytest.mark.parametrize("nu", [0.05, 0.4, 1.3, 8.0])
def test_linv_line_T_is_the_dense_transpose(bc, quad, n, nu):
    eye = np.eye(n)
    M = np.stack([oracle.linv_line(eye[k], nu, bc, quad) for k in range(n)], axis=1)
    MT = np.stack([oracle.linv_line_T(eye[k], nu, bc, quad) for k in range(n)], axis=1)
    assert np.abs(M.T - MT).max() <= 1e-14 * np.abs(M).max() * n


@pytest.mark.parametrize("quad", [1, 2])
@pytest.mark.parametrize("n", [5, 16, 33])
def test_periodic_linv_is_symmetric(quad, n):
    eye = np.eye(n)
    M = np.stack([oracle.linv_line(eye[k], 0.7, "periodic", quad) for k in range(n)], axis=1)
    assert np.abs(M - M.T).max() <= 1e-14


@pytest.mark.parametrize("shape", [(23, 17), (9, 11, 13)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_D_axis_T_dot_product(shape, bc):
    rng = np.random.default_rng(3)
    for axis in range(len(shape)):
        v, w = rng.normal(size=shape), rng.normal(size=shape)
        for power in (1, 2):
            lhs = dot(oracle.D_axis(v, axis, 0.9, bc, power=power), w)
            rhs = dot(v, oracle.D_axis_T(w, axis, 0.9, bc, power=power))
            assert rel_dot_err(lhs, rhs, np.linalg.norm(v) * np.linalg.norm(w)) <= 1e-14


@pytest.mark.parametrize("shape", [(40,), (21, 18), (8, 10, 12)])
@pytest.mark.parametrize("P", [1, 2, 3])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_FT_dot_product(shape, P, bc):
    rng = np.random.default_rng(4 + P)
    beta = oracle.beta_max(P)
    nu = [0.6 + 0.3 * a for a in range(len(shape))]
    u, w = rng.normal(size=shape), rng.normal(size=shape)
    lhs = dot(oracle.F(u, nu, P, beta, bc), w)
    rhs = dot(u, oracle.FT(w, nu, P, beta, bc))
    assert rel_dot_err(lhs, rhs, np.linalg.norm(u) * np.linalg.norm(w)) <= 1e-13


@pytest.mark.parametrize("shape", [(30,), (14, 17)])
def test_periodic_FT_equals_F(shape):
    rng = np.random.default_rng(9)
    u = rng.normal(size=shape)
    nu = [0.8, 1.1][: len(shape)]
    a = oracle.F(u, nu, 2, oracle.beta_max(2), "periodic")
    b = oracle.FT(u, nu, 2, oracle.beta_max(2), "periodic")
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def _problem(shape, seed, nrec=5):
    rng = np.random.default_rng(seed)
    u0 = rng.normal(size=shape)
    u0[..., 0] = u0[..., -1] = 0.0
    if len(shape) == 2:
        u0[0, :] = u0[-1, :] = 0.0
    size = int(np.prod(shape))
    rec = rng.choice(size, size=nrec, replace=False)
    return u0, rec


@pytest.mark.parametrize("shape,P,bc", [((24,), 1, "dirichlet"), ((30,), 3, "periodic"),
                                        ((13, 16), 2, "dirichlet"), ((12, 10), 1, "periodic")])
def test_traces_adjoint_dot_product(shape, P, bc):
    """<T s, r> = <s, T^T r> for the linear trace map of the time stepping."""
    nsteps = 9
    beta = oracle.beta_max(P)
    nu = [1.2, 0.9][: len(shape)]
    s, rec = _problem(shape, 21)
    r = np.random.default_rng(22).normal(size=(nsteps, rec.size))
    Ts = oracle.traces(s, nsteps, rec, nu, P, beta, bc)
    TTr = oracle.adjoint(r, shape, rec, nu, P, beta, bc)
    lhs, rhs = dot(Ts, r), dot(s, TTr)
    assert rel_dot_err(lhs, rhs, np.linalg.norm(Ts) * np.linalg.norm(r)) <= 1e-12


def test_traces_are_the_forward_run():
    shape, P, bc, nsteps = (11, 14), 2, "dirichlet", 6
    beta = oracle.beta_max(P)
    u0, rec = _problem(shape, 30)
    t = oracle.traces(u0, nsteps, rec, 1.0, P, beta, bc)
    a, b = u0, oracle.start(u0, 1.0, P, beta, bc)
    for n in range(1, nsteps + 1):
        assert np.array_equal(t[n - 1], b.reshape(-1)[rec])
        a, b = b, oracle.step(a, b, 1.0, P, beta, bc)


@pytest.mark.parametrize("shape,P,bc", [((20,), 2, "dirichlet"), ((11, 12), 3, "dirichlet"),
                                        ((10, 9), 2, "periodic")])
def test_adjoint_gradient_matches_central_difference(shape, P, bc):
    nsteps = 8
    beta = oracle.beta_max(P)
    nu = [1.4, 0.7][: len(shape)]
    u0, rec = _problem(shape, 40)
    d = np.random.default_rng(41).normal(size=(nsteps, rec.size))

    def J(u):
        return 0.5 * float(np.sum((oracle.traces(u, nsteps, rec, nu, P, beta, bc) - d) ** 2))

    grad = oracle.adjoint(oracle.traces(u0, nsteps, rec, nu, P, beta, bc) - d, shape, rec, nu, P, beta, bc)
    rng = np.random.default_rng(42)
    for _ in range(3):
        s = rng.normal(size=shape)
        eps = 1e-3
        fd = (J(u0 + eps * s) - J(u0 - eps * s)) / (2 * eps)
        assert abs(fd - dot(grad, s)) <= 1e-9 * max(abs(fd), np.linalg.norm(grad) * np.linalg.norm(s))


def test_single_step_adjoint_is_start_transpose():
    """nsteps = 1: the gradient is S^T R^T r with S = 1 + F/2."""
    shape, P, bc = (9, 10), 2, "dirichlet"
    beta = oracle.beta_max(P)
    _, rec = _problem(shape, 50)
    r = np.random.default_rng(51).normal(size=(1, rec.size))
    g = np.zeros(int(np.prod(shape)))
    np.add.at(g, rec, r[0])
    g = g.reshape(shape)
    expect = g + 0.5 * oracle.FT(g, 0.8, P, beta, bc)
    got = oracle.adjoint(r, shape, rec, 0.8, P, beta, bc)
    assert np.abs(got - expect).max() <= 1e-14 * np.abs(expect).max()
