"""Batches of 2D Dirichlet problems of uneven size (mol_batch_*), problem by
problem against the float64 oracle.

The shapes cover every segment length of both passes (x: 4..32 points per
lane; y: 4..64 rows per warp), lines whose last point falls anywhere in a
segment (n = 3 .. 1024, odd and even, one past and one short of a power of
two), rectangles in both orientations, and P = 1..3 with CFL 0.5..4.
Tolerances as in test_gpu_parity: float64 1e-12 (or the oracle's own
cancellation floor); mixed 16 eps32 (1 + 1/(1 - d)) 2P for F and the
accumulated model 8 eps32 (1 + 1/(1 - d)) 2P sum|F_k| / |u_n| for steps.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt, workloads

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24
EPS64 = 2.0 ** -52

SHAPES = [(64, 64), (65, 67), (3, 3), (5, 130), (100, 129), (250, 257), (17, 300), (300, 17), (511, 513),
          (700, 1000), (1024, 1024), (33, 1021), (129, 4), (40, 512), (512, 40), (1023, 7)]
CFLS = [0.5, 4.0, 1.3, 2.0, 0.8, 3.3, 1.0]


def spec(i, shape):
    P = 1 + i % 3
    cfl = CFLS[i % len(CFLS)]
    ny, nx = shape
    hx, hy = 1.0 / (nx - 1), 1.0 / (ny - 1)
    dt = cfl * min(hx, hy)
    beta = oracle.beta_max(P)
    alpha = beta / dt
    nu = (alpha * hx, alpha * hy)           # x first, as the oracle takes it
    return P, dt, beta, nu


def rough_field(shape, seed):
    u = workloads.random_field(shape, seed)
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    return u


def smooth_field(shape, seed):
    rng = np.random.default_rng(seed)
    y = np.linspace(0, 1, shape[0])[:, None]
    x = np.linspace(0, 1, shape[1])[None, :]
    u = np.zeros(shape)
    for _ in range(3):
        kx, ky = rng.integers(1, 4, size=2)
        u += rng.normal() * np.sin(np.pi * kx * x) * np.sin(np.pi * ky * y)
    return u


def rel_l2(a, b):
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def make_batch(shapes, prec, **kw):
    specs = [spec(i, s) for i, s in enumerate(shapes)]
    b = molt.BatchSolver(shapes, dt=[s[1] for s in specs], P=[s[0] for s in specs], prec=prec, **kw)
    return b, specs


def mixed_tol(nu, p):
    dmax = max(math.exp(-v) for v in nu)
    return 16 * EPS32 * (1.0 + 1.0 / (1.0 - dmax)) * p


# rows of 513..1024 points with the last point at the first, a middle and the
# last point of a 16-point segment of the split x pass, and in either warp
LONG_SHAPES = [(6, 513), (5, 528), (4, 529), (7, 545), (3, 1023), (8, 1024), (9, 777)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("long_rows", ["split", "warp"])
def test_batch_F_matches_oracle(prec, long_rows):
    shapes = SHAPES + LONG_SHAPES
    b, specs = make_batch(shapes, prec)
    b.set_tuning((4, 0 if long_rows == "split" else 4), 0)
    assert b.tuning()["x_warps"][1] == (0 if long_rows == "split" else 4)
    us = [rough_field(s, 300 + i) for i, s in enumerate(shapes)]
    got = b.unpack(b.apply_F(b.pack(us)))
    torch.cuda.synchronize()
    for i, (u, g, (P, dt, beta, nu)) in enumerate(zip(us, got, specs)):
        ref = oracle.F(u, nu, P, beta, "dirichlet")
        cond = np.linalg.norm(u) / max(np.linalg.norm(ref), 1e-300)
        tol = max(1e-12, 64 * EPS64 * cond) if prec == "fp64" else mixed_tol(nu, 2 * P)
        err = rel_l2(g.cpu().numpy(), ref)
        assert err <= tol, (i, shapes[i], P, err, tol)


STEP_SHAPES = [(64, 64), (65, 67), (5, 130), (100, 129), (250, 257), (300, 17), (129, 4), (40, 512), (33, 1021)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batch_start_and_steps_match_oracle(prec):
    nsteps = 7
    b, specs = make_batch(STEP_SHAPES, prec)
    u0s = [smooth_field(s, 400 + i) + 0.05 * rough_field(s, 500 + i) for i, s in enumerate(STEP_SHAPES)]
    u1 = b.start(b.pack(u0s))
    up, uc = b.pack(u0s), u1.clone()
    b.step(up, uc, nsteps)
    torch.cuda.synchronize()
    g1, gp, gc = b.unpack(u1), b.unpack(up), b.unpack(uc)
    for i, (u0, (P, dt, beta, nu)) in enumerate(zip(u0s, specs)):
        r1 = oracle.start(u0, nu, P, beta, "dirichlet")
        rp, rc = oracle.run(u0, r1, nsteps, nu, P, beta, "dirichlet")
        if prec == "fp64":
            tol1 = tol = 1e-12
        else:
            F0 = oracle.F(u0, nu, P, beta, "dirichlet")
            tol1 = mixed_tol(nu, 2 * P) * 0.5 * np.linalg.norm(F0) / np.linalg.norm(r1)
            Fsum, a, c = 0.0, u0, r1
            for _ in range(nsteps):
                F = oracle.F(c, nu, P, beta, "dirichlet")
                Fsum += np.linalg.norm(F)
                a, c = c, 2 * c - a + F
            dmax = max(math.exp(-v) for v in nu)
            tol = 8 * EPS32 * (1 + 1 / (1 - dmax)) * 2 * P * Fsum / np.linalg.norm(rc)
        assert rel_l2(g1[i].cpu().numpy(), r1) <= tol1, (i, "start")
        assert rel_l2(gc[i].cpu().numpy(), rc) <= tol, (i, "u_cur")
        assert rel_l2(gp[i].cpu().numpy(), rp) <= tol, (i, "u_prev")


# square problems of every size class: each class's y launch (cluster size)
# and x launch (row group) cover the same problems, so the graph runs the
# classes as independent chains
CHAIN_SHAPES = [(64, 64), (200, 200), (130, 130), (300, 300), (450, 450), (600, 600), (1000, 1000)]


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
@pytest.mark.parametrize("nsteps", [3, 7])
def test_batch_chained_graph_agrees_bitwise(prec, nsteps):
    outs = []
    for graphs, chains in ((True, True), (True, False), (False, True)):
        b, _ = make_batch(CHAIN_SHAPES, prec, use_graphs=graphs, chains=chains)
        u0s = [smooth_field(s, 650 + i) for i, s in enumerate(CHAIN_SHAPES)]
        up = b.pack(u0s)
        uc = b.start(up)
        b.step(up, uc, nsteps)
        b.step(up, uc, nsteps)             # a second call replays the graph
        torch.cuda.synchronize()
        outs.append((up.cpu().numpy(), uc.cpu().numpy()))
        b.close()
    for o in outs[1:]:
        assert np.array_equal(outs[0][0], o[0]) and np.array_equal(outs[0][1], o[1])


def test_batch_graph_and_direct_agree_bitwise():
    shapes = SHAPES[:8]
    outs = []
    for graphs in (True, False):
        b, _ = make_batch(shapes, "mixed", use_graphs=graphs)
        u0s = [smooth_field(s, 600 + i) for i, s in enumerate(shapes)]
        up = b.pack(u0s)
        uc = b.start(up)
        b.step(up, uc, 6)
        torch.cuda.synchronize()
        outs.append(uc.cpu().numpy())
        b.close()
    assert np.array_equal(outs[0], outs[1])


def test_batch_launches_and_pass_times():
    b, _ = make_batch(SHAPES, "mixed")
    u = b.pack([smooth_field(s, 700 + i) for i, s in enumerate(SHAPES)])
    v = b.start(u)
    n0 = b.launches
    b.step(u, v, 3)
    b.sync()
    # two level conversions in, two out; per step the y pass (one launch per
    # cluster size present: columns of <= 256 points on one 4-warp CTA,
    # 257..512 on two, longer on four) and the x pass (one launch per length
    # class present: rows of <= 256 points, 257..512, longer rows)
    y_launches = (int(any(s[0] <= 256 for s in SHAPES)) + int(any(256 < s[0] <= 512 for s in SHAPES))
                  + int(any(s[0] > 512 for s in SHAPES)))
    x_launches = (int(any(s[1] <= 256 for s in SHAPES)) + int(any(256 < s[1] <= 512 for s in SHAPES))
                  + int(any(s[1] > 512 for s in SHAPES)))
    assert b.launches - n0 == 4 + 3 * (y_launches + x_launches)
    b.set_pass_timing(True)
    b.step(u, v, 2)
    t = b.pass_times()
    assert set(t) == {0, 1} and t[0][1] == 2 and t[1][1] == 2 and t[0][0] > 0 and t[1][0] > 0


def test_batch_rejects_bad_pointers():
    b, _ = make_batch(SHAPES[:3], "fp64")
    u = b.empty()
    with pytest.raises(molt.MolError):
        b.apply_F(u, u)
    host = np.zeros(b.size)
    st = b.lib.mol_batch_apply_F(b.h, host.ctypes.data_as(molt.ctypes.c_void_p), molt.ctypes.c_void_p(u.data_ptr()),
                                 None)
    assert st == molt.MOL_EINVAL


@pytest.mark.slow
def test_batch_full_size_512_problems_sampled():
    """The 512-problem workload (n log-uniform in [64, 1024], P in 1..3, CFL
    in [0.5, 4]): float64 F of every problem against mixed F, and 10
    sampled problems against the oracle."""
    probs = workloads.batch_problems()
    shapes = [(p.n, p.n) for p in probs]
    dts = [p.cfl / (p.n - 1) for p in probs]
    Ps = [p.P for p in probs]
    us = [p.u0 for p in probs]
    res = {}
    for prec in ("fp64", "mixed"):
        b = molt.BatchSolver(shapes, dt=dts, P=Ps, prec=prec)
        res[prec] = [t.cpu().numpy() for t in b.unpack(b.apply_F(b.pack(us)))]
        b.close()
    rng = np.random.default_rng(11)
    for i in rng.choice(len(probs), size=10, replace=False):
        p = probs[i]
        beta = oracle.beta_max(p.P)
        nu = beta / dts[i] / (p.n - 1)
        ref = oracle.F(us[i], (nu, nu), p.P, beta, "dirichlet")
        assert rel_l2(res["fp64"][i], ref) <= 1e-12, i
    for i, p in enumerate(probs):
        nu = oracle.beta_max(p.P) / dts[i] / (p.n - 1)
        assert rel_l2(res["mixed"][i], res["fp64"][i]) <= mixed_tol((nu, nu), 2 * p.P), i


# The y pass with one neighbour exchange per sweep: columns whose last point
# falls at every kind of place in its segment (kl = 0, where the segment
# before the last is ragged too; kl = 1; kl = RPT - 1; in between), every
# segment length 4..64, decays on both sides of the exchange's limit
# d^(RPT-1) <= 2^-30 (where it does not hold the column takes the full
# carries), against the oracle with the exchange on (y rule 0, 1) and off
# (2, 3).
NB_SHAPES = [(577, 40), (578, 33), (640, 64), (1024, 20), (600, 70), (520, 36), (257, 50), (258, 40),
             (300, 64), (512, 31), (129, 45), (130, 64), (200, 17), (256, 40), (65, 40), (100, 64),
             (33, 40), (64, 64)]
NB_CFL = [0.4, 0.9, 0.3, 1.5, 3.5]


def rpt_y(ny, rule):
    r = 4
    while 16 * r < ny:
        r *= 2
    return min(64, 2 * r) if (rule & 1) and r < 64 else r


@pytest.mark.parametrize("rule", [0, 1, 2, 3])
def test_batch_y_neighbour_exchange_matches_oracle(rule):
    shapes = NB_SHAPES
    Ps = [1 + i % 3 for i in range(len(shapes))]
    cfls = [NB_CFL[i % len(NB_CFL)] for i in range(len(shapes))]
    dts, specs = [], []
    for (ny, nx), P, cfl in zip(shapes, Ps, cfls):
        hy = 1.0 / (ny - 1)
        dt = cfl * hy
        beta = oracle.beta_max(P)
        nu = (beta / dt / (nx - 1), beta / dt / (ny - 1))
        dts.append(dt)
        specs.append((P, dt, beta, nu))
    b = molt.BatchSolver(shapes, dt=dts, P=Ps, prec="mixed")
    b.set_tuning((4, 0), rule)
    assert b.tuning()["y_rule"] == rule
    # the exchange applies to a good share of the problems, ragged ends of
    # every kind among them
    nb = [math.exp(-nu[1]) ** (rpt_y(ny, rule) - 1) <= 2.0 ** -30 and (ny + rpt_y(ny, rule) - 1) // rpt_y(ny, rule) > 2
          for (ny, nx), (P, dt, beta, nu) in zip(shapes, specs)]
    kls = {(ny - 1) % rpt_y(ny, rule) for (ny, nx), on in zip(shapes, nb) if on}
    assert sum(nb) >= 8 and 0 in kls and any(0 < k < 8 for k in kls)
    us = [rough_field(s, 700 + i) for i, s in enumerate(shapes)]
    got = b.unpack(b.apply_F(b.pack(us)))
    for i, (u, g, (P, dt, beta, nu)) in enumerate(zip(us, got, specs)):
        ref = oracle.F(u, nu, P, beta, "dirichlet")
        err = rel_l2(g.cpu().numpy(), ref)
        assert err <= mixed_tol(nu, 2 * P), (i, shapes[i], P, nb[i], err)
    b.close()


def test_batch_set_tuning_rejects_bad_choices():
    b, _ = make_batch(SHAPES[:3], "mixed")
    for bad in (((3, 8), 0), ((8, 1), 0), ((8, 8), 4), ((8, 8), -1), ((0, 8), 0)):
        with pytest.raises(molt.MolError):
            b.set_tuning(*bad)


def test_batch_autotune_choice_keeps_parity():
    b, specs = make_batch(SHAPES, "mixed")
    tun = b.autotune()
    assert tun["x_warps"][0] in (2, 4, 8) and tun["x_warps"][1] in (0, 2, 4, 8) and tun["y_rule"] in (0, 1, 2)
    assert tun["x_ms"] > 0 and tun["y_ms"] > 0
    us = [rough_field(s, 900 + i) for i, s in enumerate(SHAPES)]
    got = b.unpack(b.apply_F(b.pack(us)))
    for i, (u, g, (P, dt, beta, nu)) in enumerate(zip(us, got, specs)):
        ref = oracle.F(u, nu, P, beta, "dirichlet")
        assert rel_l2(g.cpu().numpy(), ref) <= mixed_tol(nu, 2 * P), i
