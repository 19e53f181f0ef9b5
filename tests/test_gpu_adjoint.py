"""Adjoint path (mol_batch_apply_FT / mol_batch_traces / mol_batch_adjoint and
the autograd function) against the float64 oracle.

Tolerances: float64 1e-12 (relative L2; traces and gradients of a 2-level
recursion accumulate no more than the forward steps do).  Mixed: every step
adds the float32 error of one F (or F^T) application, 16 eps32 (1 + 1/(1-d))
2P relative to that application, and the recursion neither amplifies nor
damps it (A-stability), so the error of step N is at most
8 eps32 (1 + 1/(1-d)) 2P sum_n |F v^n| (the forward-stepping model of
test_gpu_parity) with v^n the oracle's own states; a trace value's error is
bounded by the field error in L2.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -52

SHAPES = [(64, 64), (65, 67), (5, 130), (100, 129), (250, 257), (33, 1021), (1024, 40)]
CFLS = [0.5, 2.0, 4.0, 1.3, 0.8, 3.3, 1.0]


def spec(i, shape):
    P = 1 + i % 3
    ny, nx = shape
    hx, hy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    dt = CFLS[i % len(CFLS)] * min(hx, hy)
    beta = oracle.beta_max(P)
    return P, dt, beta, (beta / dt * hx, beta / dt * hy)


def model(nu, P):
    dmax = max(math.exp(-v) for v in nu)
    return 8 * EPS32 * (1.0 + 1.0 / (1.0 - dmax)) * 2 * P


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def make(shapes, prec):
    specs = [spec(i, s) for i, s in enumerate(shapes)]
    return molt.BatchSolver(shapes, dt=[s[1] for s in specs], P=[s[0] for s in specs], prec=prec), specs


def receivers(shapes, offsets, per, seed):
    rng = np.random.default_rng(seed)
    rec, local = [], []
    for i, (ny, nx) in enumerate(shapes):
        iy = rng.integers(1, ny - 1, size=per)
        ix = rng.integers(1, nx - 1, size=per)
        loc = iy * nx + ix
        local.append(loc)
        rec.extend(offsets[i] + loc)
    return np.array(rec, dtype=np.int64), local


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("long_rows", ["split", "warp"])
def test_FT_matches_oracle(prec, long_rows):
    shapes = SHAPES + [(6, 513), (4, 529), (5, 1024), (7, 800)]
    b, specs = make(shapes, prec)
    b.set_tuning((4, 0 if long_rows == "split" else 4), 0)
    rng = np.random.default_rng(1)
    ws = [rng.normal(size=s) for s in shapes]
    got = b.unpack(b.apply_FT(b.pack(ws)))
    torch.cuda.synchronize()
    for i, (w, g, (P, dt, beta, nu)) in enumerate(zip(ws, got, specs)):
        ref = oracle.FT(w, nu, P, beta, "dirichlet")
        cond = np.linalg.norm(w) / max(np.linalg.norm(ref), 1e-300)
        tol = max(1e-12, 64 * EPS64 * cond) if prec == "fp64" else 2 * model(nu, P) * max(cond, 1.0)
        assert rel_l2(g.cpu().numpy(), ref) <= tol, (i, shapes[i])


def test_FT_is_the_transpose_of_F_on_the_gpu():
    """<F u, w> = <u, F^T w> with both sides from the GPU (float64), at the
    size of the adjoint workload."""
    shapes = [(1024, 1024), (77, 300)]
    b, _ = make(shapes, "fp64")
    rng = np.random.default_rng(2)
    u = b.pack([rng.normal(size=s) for s in shapes])
    w = b.pack([rng.normal(size=s) for s in shapes])
    Fu, FTw = b.apply_F(u), b.apply_FT(w)
    for i in range(len(shapes)):
        sl = slice(b.offsets[i], b.offsets[i + 1])
        lhs = float(torch.dot(Fu[sl], w[sl]))
        rhs = float(torch.dot(u[sl], FTw[sl]))
        scale = float(torch.linalg.norm(u[sl]) * torch.linalg.norm(w[sl]))
        assert abs(lhs - rhs) <= 1e-13 * scale


STEP_SHAPES = [(64, 64), (65, 67), (100, 129), (40, 250), (130, 9)]


def oracle_states(u0, nsteps, nu, P, beta):
    """Forward states u^1..u^N of the oracle and sum_n |F u^n|."""
    a, c = u0, oracle.start(u0, nu, P, beta, "dirichlet")
    Fsum = np.linalg.norm(oracle.F(u0, nu, P, beta, "dirichlet")) * 0.5
    for _ in range(nsteps - 1):
        F = oracle.F(c, nu, P, beta, "dirichlet")
        Fsum += np.linalg.norm(F)
        a, c = c, 2 * c - a + F
    return Fsum


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_traces_match_oracle(prec):
    nsteps = 9
    b, specs = make(STEP_SHAPES, prec)
    rng = np.random.default_rng(3)
    u0s = []
    for s in STEP_SHAPES:
        u = rng.normal(size=s)
        u[0, :] = u[-1, :] = 0
        u[:, 0] = u[:, -1] = 0
        u0s.append(u)
    rec, local = receivers(STEP_SHAPES, b.offsets, 4, 4)
    t = b.traces(b.pack(u0s), rec, nsteps).cpu().numpy()
    for i, (P, dt, beta, nu) in enumerate(specs):
        ref = oracle.traces(u0s[i], nsteps, local[i], nu, P, beta, "dirichlet")
        got = t[:, 4 * i:4 * (i + 1)]
        if prec == "fp64":
            assert rel_l2(got, ref) <= 1e-12, i
        else:
            bound = model(nu, P) * oracle_states(u0s[i], nsteps, nu, P, beta)
            assert np.abs(got - ref).max() <= bound, i


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_matches_oracle(prec):
    nsteps = 9
    b, specs = make(STEP_SHAPES, prec)
    rec, local = receivers(STEP_SHAPES, b.offsets, 4, 5)
    tg = np.random.default_rng(6).normal(size=(nsteps, rec.size))
    grad = b.unpack(b.adjoint(rec, torch.from_numpy(tg)))
    for i, (P, dt, beta, nu) in enumerate(specs):
        shape = STEP_SHAPES[i]
        tgi = tg[:, 4 * i:4 * (i + 1)]
        ref = oracle.adjoint(tgi, shape, local[i], nu, P, beta, "dirichlet")
        got = grad[i].cpu().numpy()
        if prec == "fp64":
            assert rel_l2(got, ref) <= 1e-12, i
        else:
            # sum_n |F^T mu^n| along the oracle's adjoint recursion
            size = int(np.prod(shape))
            g = np.zeros((nsteps, size))
            for n in range(nsteps):
                np.add.at(g[n], local[i], tgi[n])
            m2, m1 = np.zeros(shape), g[-1].reshape(shape)
            Fsum = 0.0
            for n in range(nsteps - 1, 0, -1):
                F = oracle.FT(m1, nu, P, beta, "dirichlet")
                Fsum += np.linalg.norm(F)
                m2, m1 = m1, 2 * m1 - m2 + F + g[n - 1].reshape(shape)
            Fsum += 0.5 * np.linalg.norm(oracle.FT(m1, nu, P, beta, "dirichlet"))
            assert np.linalg.norm(got - ref) <= model(nu, P) * Fsum, i


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_adjoint_with_receivers_sharing_nodes(prec):
    """Receivers listed in no particular order, several on one node (within
    a problem), some nodes once: the injection sums each node's receivers."""
    nsteps = 7
    shapes = STEP_SHAPES[:3]
    b, specs = make(shapes, prec)
    rng = np.random.default_rng(17)
    rec, local = [], []
    for i, (ny, nx) in enumerate(shapes):
        nodes = (rng.integers(1, ny - 1, size=3) * nx + rng.integers(1, nx - 1, size=3)).tolist()
        loc = np.array(nodes + [nodes[0], nodes[0], nodes[2]])[rng.permutation(6)]
        local.append(loc)
        rec.extend(b.offsets[i] + loc)
    rec = np.array(rec, dtype=np.int64)
    tg = rng.normal(size=(nsteps, rec.size))
    grad = b.unpack(b.adjoint(rec, torch.from_numpy(tg)))
    for i, (P, dt, beta, nu) in enumerate(specs):
        ref = oracle.adjoint(tg[:, 6 * i:6 * (i + 1)], shapes[i], local[i], nu, P, beta, "dirichlet")
        tol = 1e-12 if prec == "fp64" else 1e-4
        assert rel_l2(grad[i].cpu().numpy(), ref) <= tol, i


def test_gradient_matches_central_difference_on_gpu():
    """J(u0) = |T u0 - d|^2 / 2 is quadratic: the central difference along s
    equals <grad J, s> up to rounding (float64 path)."""
    shapes = [(96, 80), (51, 130)]
    nsteps = 12
    b, _ = make(shapes, "fp64")
    rng = np.random.default_rng(7)
    u0 = b.pack([rng.normal(size=s) for s in shapes])
    rec, _ = receivers(shapes, b.offsets, 6, 8)
    d = torch.from_numpy(rng.normal(size=(nsteps, rec.size))).cuda()

    def J(u):
        return 0.5 * float(((b.traces(u, rec, nsteps) - d) ** 2).sum())

    grad = b.adjoint(rec, b.traces(u0, rec, nsteps) - d)
    for _ in range(3):
        s = b.pack([rng.normal(size=sh) for sh in shapes])
        eps = 1e-3
        fd = (J(u0 + eps * s) - J(u0 - eps * s)) / (2 * eps)
        an = float(torch.dot(grad, s))
        assert abs(fd - an) <= 1e-9 * max(abs(fd), float(torch.linalg.norm(grad) * torch.linalg.norm(s)))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_autograd_function_runs_the_adjoint(prec):
    shapes = [(70, 90)]
    nsteps = 10
    b, _ = make(shapes, prec)
    rng = np.random.default_rng(9)
    u0 = b.pack([rng.normal(size=shapes[0])]).requires_grad_(True)
    rec, _ = receivers(shapes, b.offsets, 8, 10)
    d = torch.from_numpy(rng.normal(size=(nsteps, rec.size))).cuda()
    tr = molt.receiver_traces(u0, b, rec, nsteps)
    loss = 0.5 * ((tr - d) ** 2).sum()
    loss.backward()
    expect = b.adjoint(rec, (tr - d).detach())
    assert torch.equal(u0.grad, expect)


@pytest.mark.slow
def test_adjoint_workload_dot_product_and_mixed_error():
    """The adjoint workload: 1024^2 Dirichlet, P = 2, CFL 2, 400 steps, 64
    receivers.  Float64: <T s, r> = <s, T^T r>; mixed gradient within the
    accumulated float32 bound of the float64 one."""
    from paper_1308_3214_gb300 import workloads
    n, P, nsteps = 1024, 2, 400
    dt = 2.0 / (n - 1)
    rec = np.array([iy * n + ix for iy, ix in workloads.receivers_2d(n, 64, seed=1005)], dtype=np.int64)
    rng = np.random.default_rng(11)
    grads = {}
    for prec in ("fp64", "mixed"):
        b = molt.BatchSolver([(n, n)], dt=dt, P=P, prec=prec)
        s = b.pack([rng.normal(size=(n, n))]) if prec == "fp64" else s
        r = torch.from_numpy(np.random.default_rng(12).normal(size=(nsteps, rec.size))).cuda()
        grads[prec] = b.adjoint(rec, r)
        if prec == "fp64":
            Ts = b.traces(s, rec, nsteps)
            lhs, rhs = float((Ts * r).sum()), float(torch.dot(s, grads[prec]))
            assert abs(lhs - rhs) <= 1e-10 * float(torch.linalg.norm(Ts) * torch.linalg.norm(r))
        b.close()
    nu = oracle.beta_max(P) / 2.0
    err = float(torch.linalg.norm(grads["mixed"] - grads["fp64"]) / torch.linalg.norm(grads["fp64"]))
    assert err <= model((nu, nu), P) * nsteps * 4


# ---------------------------------------------------------------------------
# checkpoint-and-recompute adjoint of a general history loss
# ---------------------------------------------------------------------------
def _history_setup(prec="fp64"):
    shapes = [(48, 56), (33, 70)]
    b, specs = make(shapes, prec)
    rng = np.random.default_rng(20)
    u0s = [rng.normal(size=s) for s in shapes]
    for u in u0s:
        u[0, :] = u[-1, :] = 0
        u[:, 0] = u[:, -1] = 0
    w = b.pack([rng.uniform(0.5, 1.5, size=s) for s in shapes])
    return shapes, b, specs, u0s, w


def test_history_gradient_of_trace_loss_equals_trace_adjoint():
    """With g^n = R^T (trace residual) the checkpointed driver reproduces the
    dedicated trace adjoint, for every checkpoint interval."""
    shapes, b, specs, u0s, _ = _history_setup()
    nsteps = 11
    rec, _ = receivers(shapes, b.offsets, 5, 21)
    u0 = b.pack(u0s)
    d = torch.from_numpy(np.random.default_rng(22).normal(size=(nsteps, rec.size))).cuda()
    res = b.traces(u0, rec, nsteps) - d
    ref = b.adjoint(rec, res)
    rec_t = torch.from_numpy(rec).cuda()

    def g(n, u):
        if n == 0:
            return None
        out = torch.zeros_like(u)
        out.index_put_((rec_t,), res[n - 1], accumulate=True)
        return out

    outs = [molt.history_gradient(b, u0, nsteps, g, checkpoint_every=K) for K in (1, 4, nsteps)]
    for o in outs:
        assert float(torch.linalg.norm(o - ref) / torch.linalg.norm(ref)) <= 1e-12
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])


def test_history_gradient_of_quartic_loss_matches_oracle_adjoint():
    """J = sum_n sum_i w_i (u^n_i)^4 / 4: g^n = w (u^n)^3 needs every forward
    state; float64 GPU against the oracle's forward states and F^T."""
    shapes, b, specs, u0s, w = _history_setup()
    nsteps = 9
    u0 = b.pack(u0s)
    got = molt.history_gradient(b, u0, nsteps, lambda n, u: w * u ** 3, checkpoint_every=4)
    got_p = b.unpack(got)
    w_p = [t.cpu().numpy() for t in b.unpack(w)]
    for i, (P, dt, beta, nu) in enumerate(specs):
        states = [u0s[i], oracle.start(u0s[i], nu, P, beta, "dirichlet")]
        for _ in range(nsteps - 1):
            states.append(oracle.step(states[-2], states[-1], nu, P, beta, "dirichlet"))
        g = [w_p[i] * s ** 3 for s in states]
        m1 = np.zeros(shapes[i])
        m2 = np.zeros(shapes[i])
        for n in range(nsteps, 0, -1):
            m1, m2 = 2 * m1 - m2 + oracle.FT(m1, nu, P, beta, "dirichlet") + g[n], m1
        ref = m1 + 0.5 * oracle.FT(m1, nu, P, beta, "dirichlet") - m2 + g[0]
        assert rel_l2(got_p[i].cpu().numpy(), ref) <= 1e-12, i


def test_history_gradient_matches_central_difference():
    shapes, b, specs, u0s, w = _history_setup()
    nsteps = 7
    u0 = b.pack(u0s)

    def J(u):
        up = u.clone()
        uc = b.start(up)
        tot = float((w * u ** 4).sum()) / 4 + float((w * uc ** 4).sum()) / 4
        for _ in range(nsteps - 1):
            b.step(up, uc, 1)
            tot += float((w * uc ** 4).sum()) / 4
        return tot

    grad = molt.history_gradient(b, u0, nsteps, lambda n, u: w * u ** 3, checkpoint_every=3)
    s = b.pack([np.random.default_rng(23).normal(size=sh) for sh in shapes])
    eps = 1e-5
    fd = (J(u0 + eps * s) - J(u0 - eps * s)) / (2 * eps)
    an = float(torch.dot(grad, s))
    assert abs(fd - an) <= 1e-6 * abs(an)


def adjoint_bound(tg, shape, rec, nu, P, beta):
    """Mixed-precision error model of the adjoint recursion: 8 eps32
    (1 + 1/(1-d)) 2P times sum_n |F^T mu^n| over the oracle's own states."""
    nsteps = tg.shape[0]
    size = int(np.prod(shape))
    g = np.zeros((nsteps, size))
    for n in range(nsteps):
        np.add.at(g[n], rec, tg[n])
    m2, m1 = np.zeros(shape), g[-1].reshape(shape)
    Fsum = 0.0
    for n in range(nsteps - 1, 0, -1):
        F = oracle.FT(m1, nu, P, beta, "dirichlet")
        Fsum += np.linalg.norm(F)
        m2, m1 = m1, 2 * m1 - m2 + F + g[n - 1].reshape(shape)
    Fsum += 0.5 * np.linalg.norm(oracle.FT(m1, nu, P, beta, "dirichlet"))
    return model(nu, P) * Fsum


@pytest.mark.parametrize("shape", [(128, 1024), (192, 2048), (256, 1024)])
@pytest.mark.parametrize("strided_nb", [1, 0])
def test_single_path_adjoint_mixed_matches_oracle(shape, strided_nb):
    """Mixed-precision handles whose rows split over warps and whose columns
    split into strided segments run F^T, traces and the adjoint on the
    register kernels' transposed modes (not a one-problem batch: the
    handle's own pass timers see the passes); the transposed y pass with one
    neighbour exchange per sweep (strided_nb 1) or the full carries (0)."""
    P, nsteps = 2, 6
    ny, nx = shape
    dt = 2.0 / (max(shape) - 1)
    s = molt.Solver(shape, dt=dt, P=P, bc="dirichlet", prec="mixed")
    cur = s.tuning()
    s.set_tuning(cur["res_warps"], cur["strided_rpt"], cur["strided_warps"], cur["rows_warps"], strided_nb=strided_nb)
    nu, beta = s.nu, s.beta
    rng = np.random.default_rng(41)
    w = rng.normal(size=shape)
    s.set_pass_timing(True)
    got = s.apply_FT(torch.from_numpy(w).cuda()).cpu().numpy()
    t = s.pass_times()
    s.set_pass_timing(False)
    assert t[0][1] == 1 and t[1][1] == 1, t
    ref = oracle.FT(w, nu, P, beta, "dirichlet")
    cond = np.linalg.norm(w) / np.linalg.norm(ref)
    assert rel_l2(got, ref) <= 2 * model(nu, P) * max(cond, 1.0)
    u0 = rng.normal(size=shape)
    u0[0, :] = u0[-1, :] = 0
    u0[:, 0] = u0[:, -1] = 0
    rec = np.concatenate([rng.choice(ny * nx, size=7, replace=False), [5 * nx + 9, 5 * nx + 9]])
    tr = s.traces(torch.from_numpy(u0).cuda(), rec, nsteps).cpu().numpy()
    tref = oracle.traces(u0, nsteps, rec, nu, P, beta, "dirichlet")
    assert np.abs(tr - tref).max() <= model(nu, P) * oracle_states(u0, nsteps, nu, P, beta)
    tg = rng.normal(size=(nsteps, rec.size))
    g = s.adjoint(rec, torch.from_numpy(tg)).cpu().numpy()
    gref = oracle.adjoint(tg, shape, rec, nu, P, beta, "dirichlet")
    assert np.linalg.norm(g - gref) <= adjoint_bound(tg, shape, rec, nu, P, beta)


@pytest.mark.parametrize("rpt,warps", [(32, 4), (32, 8), (0, 4)])
def test_transposed_y_pass_over_clusters_matches_oracle(rpt, warps):
    """F^T of a mixed handle whose 1024-point columns span a cluster of CTAs
    (8, 4 or 4 CTAs per column group), the transposed y pass with one
    neighbour exchange per sweep and with the full carries."""
    shape, P = (1024, 512), 2
    s = molt.Solver(shape, dt=2.0 / 1023, P=P, bc="dirichlet", prec="mixed")
    rng = np.random.default_rng(43)
    w = rng.normal(size=shape)
    ref = oracle.FT(w, s.nu, P, s.beta, "dirichlet")
    cond = np.linalg.norm(w) / np.linalg.norm(ref)
    wd = torch.from_numpy(w).cuda()
    for nb in (1, 0):
        s.set_tuning(res_warps=2, strided_rpt=rpt, strided_warps=warps, rows_warps=0, strided_nb=nb)
        got = s.apply_FT(wd).cpu().numpy()
        assert rel_l2(got, ref) <= 2 * model(s.nu, P) * max(cond, 1.0), (nb, rel_l2(got, ref))
    s.close()


def test_single_path_FT_is_the_transpose_of_F():
    """<F u, w> = <u, F^T w> with both sides from the mixed single path on the
    adjoint workload's grid."""
    shape = (1024, 1024)
    s = molt.Solver(shape, dt=2.0 / 1023, P=2, bc="dirichlet", prec="mixed")
    rng = np.random.default_rng(42)
    u = torch.from_numpy(rng.normal(size=shape)).cuda()
    w = torch.from_numpy(rng.normal(size=shape)).cuda()
    lhs = float(torch.sum(s.apply_F(u) * w))
    rhs = float(torch.sum(u * s.apply_FT(w)))
    scale = float(torch.linalg.norm(u) * torch.linalg.norm(w))
    assert abs(lhs - rhs) <= 1e-5 * scale


@pytest.mark.parametrize("shape", [(128, 256), (100, 129)])
def test_single_handle_adjoint_matches_oracle(shape):
    """mol_apply_FT / mol_traces / mol_adjoint on a mol_create handle (a
    register-path grid and a ragged one), float64 against the oracle, and the
    autograd function on the same handle."""
    P, nsteps = 2, 8
    ny, nx = shape
    dt = 2.0 / (max(shape) - 1)
    s = molt.Solver(shape, dt=dt, P=P, bc="dirichlet", prec="fp64")
    nu = s.nu
    rng = np.random.default_rng(31)
    w = rng.normal(size=shape)
    got = s.apply_FT(torch.from_numpy(w).cuda()).cpu().numpy()
    assert rel_l2(got, oracle.FT(w, nu, P, s.beta, "dirichlet")) <= 1e-12
    u0 = rng.normal(size=shape)
    u0[0, :] = u0[-1, :] = 0
    u0[:, 0] = u0[:, -1] = 0
    rec = rng.choice(ny * nx, size=6, replace=False)
    tr = s.traces(torch.from_numpy(u0).cuda(), rec, nsteps).cpu().numpy()
    assert rel_l2(tr, oracle.traces(u0, nsteps, rec, nu, P, s.beta, "dirichlet")) <= 1e-12
    tg = rng.normal(size=(nsteps, rec.size))
    g = s.adjoint(rec, torch.from_numpy(tg)).cpu().numpy()
    assert rel_l2(g, oracle.adjoint(tg, shape, rec, nu, P, s.beta, "dirichlet")) <= 1e-12
    u = torch.from_numpy(u0).cuda().requires_grad_(True)
    t = molt.receiver_traces(u, s, rec, nsteps)
    (0.5 * (t ** 2).sum()).backward()
    assert torch.equal(u.grad, s.adjoint(rec, t.detach()))


# ---------------------------------------------------------------------------
# history gradient through mol_adjoint_history on single-problem handles
# ---------------------------------------------------------------------------
def test_single_handle_history_gradient_matches_oracle():
    """float64 handle (its adjoint runs on a one-problem batch): J = sum_n
    sum_i w_i (u^n_i)^4 / 4 against the oracle's forward states and F^T."""
    shape, P, nsteps = (96, 128), 2, 7
    dt = 2.0 / (max(shape) - 1)
    s = molt.Solver(shape, dt=dt, P=P, bc="dirichlet", prec="fp64")
    nu, beta = s.nu, s.beta
    rng = np.random.default_rng(51)
    u0 = rng.normal(size=shape)
    u0[0, :] = u0[-1, :] = 0
    u0[:, 0] = u0[:, -1] = 0
    w = rng.uniform(0.5, 1.5, size=shape)
    wd = torch.from_numpy(w).cuda()
    got = molt.history_gradient(s, torch.from_numpy(u0).cuda(), nsteps, lambda n, u: wd * u ** 3,
                                checkpoint_every=3).cpu().numpy()
    states = [u0, oracle.start(u0, nu, P, beta, "dirichlet")]
    for _ in range(nsteps - 1):
        states.append(oracle.step(states[-2], states[-1], nu, P, beta, "dirichlet"))
    g = [w * st ** 3 for st in states]
    m1, m2 = np.zeros(shape), np.zeros(shape)
    for n in range(nsteps, 0, -1):
        m1, m2 = 2 * m1 - m2 + oracle.FT(m1, nu, P, beta, "dirichlet") + g[n], m1
    ref = m1 + 0.5 * oracle.FT(m1, nu, P, beta, "dirichlet") - m2 + g[0]
    assert rel_l2(got, ref) <= 1e-12
    s.close()


def test_single_path_history_gradient_equals_trace_adjoint():
    """Mixed handle on the register kernels' transposed modes: with
    g^n = R^T (trace residual) the checkpointed driver reproduces mol_adjoint
    (to float32 rounding of the injection) and is bitwise the same for every
    checkpoint interval."""
    shape, P, nsteps = (128, 1024), 2, 10
    s = molt.Solver(shape, dt=2.0 / 1023, P=P, bc="dirichlet", prec="mixed")
    rng = np.random.default_rng(52)
    u0 = rng.normal(size=shape)
    u0[0, :] = u0[-1, :] = 0
    u0[:, 0] = u0[:, -1] = 0
    u0 = torch.from_numpy(u0).cuda()
    rec = rng.choice(shape[0] * shape[1], size=9, replace=False)
    d = torch.from_numpy(rng.normal(size=(nsteps, rec.size))).cuda()
    res = s.traces(u0, rec, nsteps) - d
    ref = s.adjoint(rec, res)
    rec_t = torch.from_numpy(rec).cuda()

    def g(n, u):
        if n == 0:
            return None
        out = torch.zeros(u.numel(), dtype=torch.float64, device="cuda")
        out.index_put_((rec_t,), res[n - 1], accumulate=True)
        return out.view(shape)

    outs = [molt.history_gradient(s, u0, nsteps, g, checkpoint_every=K) for K in (1, 4, nsteps)]
    for o in outs:
        assert float(torch.linalg.norm(o - ref) / torch.linalg.norm(ref)) <= 1e-6
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[1], outs[2])
    s.close()


def test_history_gradient_callback_errors_surface():
    shape = (64, 64)
    s = molt.Solver(shape, dt=2.0 / 63, P=1, bc="dirichlet", prec="fp64")
    u0 = torch.zeros(shape, dtype=torch.float64, device="cuda")

    def bad(n, u):
        raise ValueError("boom")

    with pytest.raises(ValueError, match="boom"):
        molt.history_gradient(s, u0, 3, bad, checkpoint_every=2)
    # the handle keeps working
    assert torch.isfinite(s.apply_F(u0)).all()
    s.close()
