"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (relative L2 over the whole field):
  * FP64 path: 1e-12, or the oracle's own cancellation floor where that is
    larger: the oracle forms D v = v - L^{-1} v, which loses about
    eps64 * |v| / |D v| (relevant only at extreme decay, nu > 20).
  * Mixed path, one operator: float32 sweeps.  A recurrence with decay d sums
    about 1/(1 - d) terms that matter, so one application of D carries a
    relative error of order eps32 * (1 + 1/(1 - d)); a power D^p compounds p
    of them and F (2P sweeps) 2P.  Bound: 16 * eps32 * (1 + 1/(1 - d)) * p
    (measured ratios to the unscaled estimate stay below 1.1).
  * Mixed path, n steps: every step adds the float32 error of F to the level,
    so the bound is 8 * eps32 * (1 + 1/(1 - d)) * 2P * sum_k |F_k| / |u_n|,
    with the F_k of the oracle's own run (measured ratios stay below 1.3).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from paper_1308_3214_gb300 import molt, workloads

pytestmark = pytest.mark.gpu

EPS32 = 2.0 ** -24


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


EPS64 = 2.0 ** -52


def mixed_tol(d_max, p=1):
    return 16 * EPS32 * (1.0 + 1.0 / (1.0 - d_max)) * p


def tol_for(prec, solver, p=1, cond=1.0):
    """cond = |input| / |output| of the oracle's last cancellation."""
    if prec == "fp64":
        return max(1e-12, 64 * EPS64 * cond)
    return mixed_tol(max(solver.d), p)


def cond_of(v, ref):
    return float(np.linalg.norm(v) / max(np.linalg.norm(ref), 1e-300))


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def field(shape, seed, bc):
    u = workloads.random_field(shape, seed)
    if bc == "dirichlet":
        for ax in range(u.ndim):
            sl = [slice(None)] * u.ndim
            sl[ax] = 0
            u[tuple(sl)] = 0
            sl[ax] = -1
            u[tuple(sl)] = 0
    return u


def smooth_field(shape, seed, bc):
    """A band-limited field (a few low modes), so that D u << u."""
    rng = np.random.default_rng(seed)
    grids = np.meshgrid(*[np.linspace(0, 1, s) for s in shape], indexing="ij")
    u = np.zeros(shape)
    for _ in range(4):
        k = rng.integers(1, 4, size=len(shape))
        term = rng.normal()
        for g, kk in zip(grids, k):
            term = term * np.sin(np.pi * kk * g) if bc == "dirichlet" else term * np.cos(2 * np.pi * kk * g)
        u += term
    return u


def make(shape, dt, P, bc, prec, quad=2, **kw):
    lo = [0.0] * len(shape)
    hi = [1.0] * len(shape)
    return molt.Solver(shape, dt=dt, P=P, bc=bc, prec=prec, lo=lo, hi=hi, quad_order=quad, **kw)


def spacing(n, bc):
    return 1.0 / (n - 1) if bc == "dirichlet" else 1.0 / n


# ---------------------------------------------------------------------------
# one application of D_gamma^p
# ---------------------------------------------------------------------------
CASES_D = [
    ((257,), 0.004), ((3,), 0.3), ((33,), 0.02), ((64,), 0.01), ((1000,), 0.0005),
    ((37, 70), 0.01), ((130, 5), 0.02), ((9, 13, 21), 0.03), ((16, 3, 40), 0.05),
]


@pytest.mark.parametrize("shape, dt", CASES_D)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("quad", [2, 1])
def test_apply_D_matches_oracle(shape, dt, bc, prec, quad):
    s = make(shape, dt, 2, bc, prec, quad)
    v = field(shape, 11, bc)
    vd = dev(v)
    for axis in range(len(shape)):
        for power in (1, 2, 3):
            got = s.apply_D(vd, axis, power).cpu().numpy()
            ref = oracle.D_axis(v, axis, s.nu[axis], bc, quad, power=power)
            err = rel_l2(got, ref)
            assert err <= tol_for(prec, s, power, cond_of(v, ref)), (axis, power, err)


@pytest.mark.parametrize("cfl", [0.05, 0.5, 2.0, 10.0, 100.0])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
def test_apply_D_extreme_decay(cfl, bc):
    """nu = beta/CFL from 24 (d ~ 1e-11) down to 0.012 (d ~ 0.99)."""
    n = 300
    h = spacing(n, bc)
    dt = cfl * h
    for prec in ("fp64", "mixed"):
        s = make((n,), dt, 1, bc, prec)
        v = smooth_field((n,), 3, bc) + 0.1 * field((n,), 4, bc)
        got = s.apply_D(dev(v), 0, 1).cpu().numpy()
        ref = oracle.D_axis(v, 0, s.nu[0], bc, 2)
        assert rel_l2(got, ref) <= tol_for(prec, s, cond=cond_of(v, ref)), (prec, rel_l2(got, ref))


def test_apply_D_longest_line():
    n = int(molt.load_library().mol_max_line(0))
    for prec in ("fp64", "mixed"):
        s = make((n,), 0.5 / n, 1, "dirichlet", prec)
        v = field((n,), 5, "dirichlet")
        got = s.apply_D(dev(v), 0, 1).cpu().numpy()
        ref = oracle.D_axis(v, 0, s.nu[0], "dirichlet", 2)
        assert rel_l2(got, ref) <= tol_for(prec, s)


# ---------------------------------------------------------------------------
# the full spatial operator F, the start value and time stepping
# ---------------------------------------------------------------------------
CASES_F = [((301,), 1, 0.004), ((256,), 3, 0.01), ((70, 41), 1, 0.02), ((48, 66), 3, 0.015),
           ((33, 35), 2, 0.05), ((11, 14, 17), 1, 0.06), ((12, 10, 19), 2, 0.04)]


@pytest.mark.parametrize("shape, P, dt", CASES_F)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_apply_F_matches_oracle(shape, P, dt, bc, prec):
    s = make(shape, dt, P, bc, prec)
    u = field(shape, 21, bc)
    got = s.apply_F(dev(u)).cpu().numpy()
    ref = oracle.F(u, s.nu, P, s.beta, bc)
    assert rel_l2(got, ref) <= tol_for(prec, s, 2 * P), rel_l2(got, ref)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_start_matches_oracle(prec):
    shape, P, bc = (40, 52), 2, "dirichlet"
    s = make(shape, 0.03, P, bc, prec)
    u0 = smooth_field(shape, 2, bc)
    got = s.start(dev(u0)).cpu().numpy()
    ref = oracle.start(u0, s.nu, P, s.beta, bc)
    F = oracle.F(u0, s.nu, P, s.beta, bc)
    tol = 1e-12 if prec == "fp64" else tol_for(prec, s, 2 * P) * 0.5 * np.linalg.norm(F) / np.linalg.norm(ref)
    assert rel_l2(got, ref) <= tol


STEP_CASES = [((256,), 1, "periodic", 200, 0.036816), ((130,), 5, "dirichlet", 60, 0.02),
              ((96, 130), 3, "dirichlet", 30, 0.0157), ((64, 64), 2, "periodic", 25, 0.03),
              ((20, 24, 28), 2, "periodic", 10, 0.05), ((18, 22, 15), 1, "dirichlet", 12, 0.07)]


@pytest.mark.parametrize("shape, P, bc, nsteps, dt", STEP_CASES)
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_time_stepping_matches_oracle(shape, P, bc, nsteps, dt, prec):
    s = make(shape, dt, P, bc, prec)
    u0 = smooth_field(shape, 7, bc) + 0.05 * field(shape, 8, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    tol = 1e-12
    if prec == "mixed":
        Fsum, a, b = 0.0, u0, u1
        for _ in range(nsteps):
            F = oracle.F(b, s.nu, P, s.beta, bc)
            Fsum += np.linalg.norm(F)
            a, b = b, 2 * b - a + F
        tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol
    assert rel_l2(up.cpu().numpy(), rp) <= tol


@pytest.mark.parametrize("nsteps", [1, 2, 3, 4, 9, 17, 20])
def test_graph_and_direct_launches_agree_bitwise(nsteps):
    """The time loop through its graphs (9, 3, then 1 or 2 steps) and through
    direct launches give the same bits, both levels."""
    shape, P = (40, 50), 3
    u0 = smooth_field(shape, 9, "dirichlet")
    outs = []
    for graphs in (True, False):
        s = make(shape, 0.02, P, "dirichlet", "mixed", use_graphs=graphs)
        up, uc = dev(u0), s.start(dev(u0))
        s.step(up, uc, nsteps)
        s.step(up, uc, nsteps)             # a second call reuses the graphs
        outs.append((up.cpu().numpy(), uc.cpu().numpy()))
    assert np.array_equal(outs[0][0], outs[1][0]) and np.array_equal(outs[0][1], outs[1][1])


def test_launch_count_reports_kernels():
    # a small Dirichlet grid runs as a batch of one: 2 conversions in (one
    # per level), 2 passes per step, 2 conversions out
    s = make((32, 40), 0.02, 2, "dirichlet", "mixed")
    u = dev(field((32, 40), 1, "dirichlet"))
    before = s.launches
    s.step(u.clone(), u.clone(), 6)
    assert s.launches - before == 2 + 2 * 6 + 2
    # the single-problem kernels: one conversion launch in for both levels,
    # 2 passes per step, one out
    s = make((32, 64), 0.02, 2, "periodic", "mixed")
    u = dev(field((32, 64), 1, "periodic"))
    before = s.launches
    s.step(u.clone(), u.clone(), 6)
    assert s.launches - before == 1 + 2 * 6 + 1


def test_solve_host_matches_device_path():
    shape, P = (48, 40), 2
    u0 = smooth_field(shape, 12, "dirichlet")
    s = make(shape, 0.02, P, "dirichlet", "fp64")
    host = s.solve_host(u0, 9)
    up = dev(u0)
    uc = s.start(up)
    s.step(up, uc, 8)
    assert np.array_equal(host, uc.cpu().numpy())


def test_bad_pointer_rejected():
    s = make((16, 16), 0.02, 1, "dirichlet", "fp64")
    import ctypes
    host = np.zeros((16, 16))
    st = s.lib.mol_apply_F(s.h, ctypes.c_void_p(host.ctypes.data), ctypes.c_void_p(host.ctypes.data), None)
    assert st == molt.MOL_EINVAL


# ---------------------------------------------------------------------------
# full-size workloads, in the launch configuration the benchmark times
# ---------------------------------------------------------------------------
_FULL2D = {}


def _full2d_reference(s, P):
    """u0, u1 and the oracle's u3 of the 2048^2 workload (computed once)."""
    if not _FULL2D:
        n = 2048
        u0 = workloads.gaussian_2d(n, seed=1002)
        u1 = oracle.start(u0, s.nu, P, s.beta, "dirichlet")
        _, rc = oracle.run(u0, u1, 2, s.nu, P, s.beta, "dirichlet")
        _FULL2D.update(u0=u0, u1=u1, rc=rc)
    return _FULL2D["u0"], _FULL2D["u1"], _FULL2D["rc"]


# tunings: the handle's defaults, the autotuner's own pick, and each launch
# variant the autotuner has kept on this grid (rows of the x pass over 2 or 4
# warps; 64-row float32 strided segments over 4 warps per CTA, so each
# 2048-row column runs in a cluster of 8 CTAs)
TUNINGS_2D = [None, "auto", dict(res_warps=4, strided_rpt=0, strided_warps=4, rows_warps=4),
              dict(res_warps=4, strided_rpt=0, strided_warps=4, rows_warps=2),
              dict(res_warps=2, strided_rpt=32, strided_warps=8, rows_warps=8)]


@pytest.mark.slow
@pytest.mark.parametrize("tuning", TUNINGS_2D, ids=["default", "auto", "rows4-cl8", "rows2-cl8", "rows8-rpt32"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_full_size_2d_gaussian_two_steps(prec, tuning):
    """The benchmark's 2048^2 workload, two steps, in every launch
    configuration the benchmark may time."""
    n, P, cfl = 2048, 3, 2.0
    h = 1.0 / (n - 1)
    dt = cfl * h
    s = make((n, n), dt, P, "dirichlet", prec)
    if tuning == "auto":
        s.autotune()
    elif tuning is not None:
        if prec == "fp64" and tuning["rows_warps"]:
            pytest.skip("the row split is a float32 kernel")
        s.set_tuning(**tuning)
        assert s.tuning()["strided_warps"] == tuning["strided_warps"]
    u0, u1, rc = _full2d_reference(s, P)
    up, uc = dev(u0), dev(u1)
    s.step(up, uc, 2)
    err = rel_l2(uc.cpu().numpy(), rc)
    assert err <= (1e-12 if prec == "fp64" else 1e-8), (err, s.tuning())
    s.close()


@pytest.mark.slow
@pytest.mark.parametrize("rpt,warps", [(0, 4), (0, 8), (32, 8)])
def test_full_size_2d_strided_powers(rpt, warps):
    """D_y^p, p = 1..3, on the 2048^2 grid with the float32 strided pass in
    each segmenting the tuner offers (64-row segments over 4 warps: clusters
    of 8 CTAs per 2048-row column; over 8 warps: clusters of 4; 32-row
    segments over 8 warps: clusters of 8)."""
    n = 2048
    s = make((n, n), 2.0 / (n - 1), 3, "dirichlet", "mixed")
    s.set_tuning(res_warps=4, strided_rpt=rpt, strided_warps=warps, rows_warps=4)
    v = field((n, n), 61, "dirichlet")
    vd = dev(v)
    for power in (1, 2, 3):
        got = s.apply_D(vd, 1, power).cpu().numpy()
        ref = oracle.D_axis(v, 1, s.nu[1], "dirichlet", 2, power=power)
        assert rel_l2(got, ref) <= tol_for("mixed", s, power), (power, rel_l2(got, ref))
    s.close()


TUNINGS_3D = [None, "auto", dict(res_warps=2, strided_rpt=32, strided_warps=8, rows_warps=0, strided_nb=2),
              dict(res_warps=2, strided_rpt=0, strided_warps=4, rows_warps=0, strided_nb=1, strided_stage=0),
              dict(res_warps=2, strided_rpt=0, strided_warps=8, rows_warps=0, strided_nb=0)]


@pytest.mark.slow
def test_full_size_3d_fourier_one_step():
    n, P, cfl = 256, 2, 1.5
    h = 2 * np.pi / n
    dt = cfl * h
    u0, _ = workloads.fourier_3d(n, seed=1003)
    box = dict(lo=[0.0] * 3, hi=[2 * np.pi] * 3)
    s64 = molt.Solver((n, n, n), dt=dt, P=P, bc="periodic", prec="fp64", **box)
    ref = oracle.F(u0, s64.nu, P, s64.beta, "periodic")
    got = s64.apply_F(dev(u0)).cpu().numpy()
    assert rel_l2(got, ref) <= 1e-12, rel_l2(got, ref)
    s64.close()
    smx = molt.Solver((n, n, n), dt=dt, P=P, bc="periodic", prec="mixed", **box)
    ud = dev(u0)
    for tuning in TUNINGS_3D:
        # every launch configuration the 3D benchmark may time: the default,
        # the tuner's pick, the neighbour-exchange y Horner pass with and
        # without its fields staged in shared memory, the full-carry passes
        if tuning == "auto":
            smx.autotune()
        elif tuning is not None:
            smx.set_tuning(**tuning)
        got = smx.apply_F(ud).cpu().numpy()
        assert rel_l2(got, ref) <= tol_for("mixed", smx, 2 * P), (tuning, rel_l2(got, ref))
    smx.close()


# ---------------------------------------------------------------------------
# shapes whose lines are whole multiples of the register segment length, so
# the register-resident kernels run (x: 32*RPT >= n with RPT | n; strided
# axes: 64 | n for float32, 32 | n for float64; 2048-point strided lines are
# split over a 4-CTA (float32) or 8-CTA (float64) cluster)
# ---------------------------------------------------------------------------
REG_SHAPES = [(64,), (512,), (2048,), (128, 256), (2048, 64), (256, 512), (64, 64, 128), (128, 64, 32)]


@pytest.mark.parametrize("shape", REG_SHAPES)
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_register_kernels_apply_D(shape, bc, prec):
    if prec == "fp64" and shape[-1] > 1024:
        pytest.skip("float64 contiguous lines longer than 1024 use the shared-memory kernels")
    dt = 1.5 / max(shape)
    s = make(shape, dt, 3, bc, prec)
    v = field(shape, 31, bc)
    vd = dev(v)
    for axis in range(len(shape)):
        for power in (1, 3):
            got = s.apply_D(vd, axis, power).cpu().numpy()
            ref = oracle.D_axis(v, axis, s.nu[axis], bc, 2, power=power)
            err = rel_l2(got, ref)
            assert err <= tol_for(prec, s, power, cond_of(v, ref)), (axis, power, err)


@pytest.mark.parametrize("shape, P", [((2048,), 3), ((128, 256), 3), ((2048, 64), 2), ((256, 512), 1),
                                      ((64, 64, 128), 2), ((128, 64, 32), 3)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_register_kernels_F_and_steps(shape, P, bc, prec):
    if prec == "fp64" and shape[-1] > 1024:
        pytest.skip("float64 contiguous lines longer than 1024 use the shared-memory kernels")
    dt = 2.0 / max(shape)
    s = make(shape, dt, P, bc, prec)
    u = field(shape, 41, bc)
    got = s.apply_F(dev(u)).cpu().numpy()
    ref = oracle.F(u, s.nu, P, s.beta, bc)
    assert rel_l2(got, ref) <= tol_for(prec, s, 2 * P), rel_l2(got, ref)
    u0 = smooth_field(shape, 42, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    nsteps = 6
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    tol = 1e-12
    if prec == "mixed":
        Fsum, a, b = 0.0, u0, u1
        for _ in range(nsteps):
            F = oracle.F(b, s.nu, P, s.beta, bc)
            Fsum += np.linalg.norm(F)
            a, b = b, 2 * b - a + F
        tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol


@pytest.mark.parametrize("shape, P, bc", [((256, 2048), 3, "dirichlet"), ((64, 128, 96), 2, "periodic"),
                                          ((512, 256), 2, "periodic")])
def test_programmatic_dependent_launch_is_bitwise_neutral(shape, P, bc):
    """The passes launched as programmatic dependents of the kernel before
    them (each waits for its predecessor before touching memory) give the
    same bits as ordinary stream order, through graphs and direct launches;
    and they match the oracle."""
    s = make(shape, 1.5 * spacing(shape[1], bc), P, bc, "mixed")
    u0 = smooth_field(shape, 61, bc) + 0.05 * field(shape, 62, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    out = {}
    for pdl in (1, 0):
        s.set_tuning(res_warps=2, strided_rpt=0, strided_warps=8, rows_warps=0, pdl=pdl)
        assert s.tuning()["pdl"] == pdl
        up, uc = dev(u0), dev(u1)
        s.step(up, uc, 7)
        out[pdl] = (up.clone(), uc.clone(), s.apply_F(dev(u0)))
    for a, b in zip(out[1], out[0]):
        assert torch.equal(a, b)
    ref = oracle.F(u0, s.nu, P, s.beta, bc)
    assert rel_l2(out[1][2].cpu().numpy(), ref) <= tol_for("mixed", s, 2 * P)
    s.close()


# A single contiguous line of >= 1024 points whose length no register kernel
# takes is swept by the whole CTA (512 segments, carries over lanes and warps):
# powers, F and steps against the oracle, both boundary conditions, lengths
# that leave the last segments partly or wholly empty.
@pytest.mark.parametrize("n", [1024, 1500, 3001, 5119])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_single_long_line_cta_sweep_matches_oracle(n, bc, prec):
    P = 3
    s = make((n,), 1.3 * spacing(n, bc), P, bc, prec)
    v = field((n,), 95, bc)
    vd = dev(v)
    for power in (1, 2, 3):
        got = s.apply_D(vd, 0, power).cpu().numpy()
        ref = oracle.D_axis(v, 0, s.nu[0], bc, 2, power=power)
        assert rel_l2(got, ref) <= tol_for(prec, s, power, cond_of(v, ref)), (power, rel_l2(got, ref))
    got = s.apply_F(vd).cpu().numpy()
    ref = oracle.F(v, s.nu, P, s.beta, bc)
    assert rel_l2(got, ref) <= tol_for(prec, s, 2 * P), rel_l2(got, ref)
    u0 = smooth_field((n,), 96, bc) + 0.05 * field((n,), 97, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    nsteps = 8
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    tol = 1e-12
    if prec == "mixed":
        Fsum, a, b = 0.0, u0, u1
        for _ in range(nsteps):
            F = oracle.F(b, s.nu, P, s.beta, bc)
            Fsum += np.linalg.norm(F)
            a, b = b, 2 * b - a + F
        tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol
    s.close()


# ---------------------------------------------------------------------------
# autotuner
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_autotune_choice_keeps_parity(prec):
    shape, P, bc, nsteps, dt = (256, 512), 3, "dirichlet", 6, 0.004
    s = make(shape, dt, P, bc, prec)
    tun = s.autotune()
    assert tun["res_warps"] in (1, 2, 4) and tun["strided_warps"] in (4, 8) and tun["strided_rpt"] in (0, 32)
    assert tun["rows_warps"] in (0, 2, 4, 8)
    assert tun["ms_per_step"] > 0
    u0 = smooth_field(shape, 7, bc) + 0.05 * field(shape, 8, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    tol = 1e-12
    if prec == "mixed":
        Fsum, a, b = 0.0, u0, u1
        for _ in range(nsteps):
            F = oracle.F(b, s.nu, P, s.beta, bc)
            Fsum += np.linalg.norm(F)
            a, b = b, 2 * b - a + F
        tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol


@pytest.mark.parametrize("rpt,warps", [(0, 8), (0, 4), (32, 8), (32, 4)])
def test_every_strided_choice_matches_oracle(rpt, warps):
    """Each strided segmenting the tuner may pick (segment length, segments
    per CTA, hence the cluster size) applies D_y^2 correctly."""
    shape, bc = (1024, 96), "dirichlet"
    s = make(shape, 0.002, 2, bc, "mixed")
    s.set_tuning(res_warps=2, strided_rpt=rpt, strided_warps=warps)
    v = field(shape, 40, bc)
    ref = oracle.D_axis(v, 1, s.nu[1], bc, 2, power=2)
    got = s.apply_D(dev(v), 1, 2).cpu().numpy()
    assert rel_l2(got, ref) <= tol_for("mixed", s, 2)



@pytest.mark.parametrize("shape, W", [((48, 2048), 2), ((40, 2048), 4), ((64, 1024), 2), ((36, 2048), 8),
                                      ((20, 4096), 8)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("P", [1, 3])
def test_rows_split_over_warps_match_oracle(shape, W, bc, P):
    """The x pass with each row split over W warps (carries and halos through
    shared memory): F and a few steps against the oracle."""
    dt = 2.0 / max(shape)
    s = make(shape, dt, P, bc, "mixed")
    s.set_tuning(rows_warps=W)
    assert s.tuning()["rows_warps"] == W
    u = field(shape, 50 + W, bc)
    ref = oracle.F(u, s.nu, P, s.beta, bc)
    assert rel_l2(s.apply_F(dev(u)).cpu().numpy(), ref) <= tol_for("mixed", s, 2 * P)
    u0 = smooth_field(shape, 51, bc) + 0.05 * field(shape, 52, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    nsteps = 5
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    Fsum, a, b = 0.0, u0, u1
    for _ in range(nsteps):
        F = oracle.F(b, s.nu, P, s.beta, bc)
        Fsum += np.linalg.norm(F)
        a, b = b, 2 * b - a + F
    tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol


# ---------------------------------------------------------------------------
# float32 strided powers with one neighbour exchange per sweep: used where
# the decay over one segment, d^(RPT-1), is below 2^-30; the full-carry
# kernel elsewhere.  Both choices against the oracle, over decays on either
# side of that limit.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape", [(2048, 96), (256, 64), (128, 160)])
@pytest.mark.parametrize("cfl", [0.5, 2.0, 3.5, 8.0])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("rpt,warps", [(0, 4), (0, 8), (32, 8)])
def test_strided_neighbour_exchange_matches_oracle(shape, cfl, bc, rpt, warps):
    n = shape[0]
    h = spacing(n, bc)
    s = make(shape, cfl * h, 3, bc, "mixed")
    v = field(shape, 70, bc)
    vd = dev(v)
    refs = [oracle.D_axis(v, 1, s.nu[1], bc, 2, power=p) for p in (1, 2, 3)]
    for nb in (1, 0):
        s.set_tuning(res_warps=2, strided_rpt=rpt, strided_warps=warps, rows_warps=0, strided_nb=nb)
        assert s.tuning()["strided_nb"] == nb
        for p, ref in zip((1, 2, 3), refs):
            got = s.apply_D(vd, 1, p).cpu().numpy()
            assert rel_l2(got, ref) <= tol_for("mixed", s, p), (nb, p, rel_l2(got, ref))
    s.close()


@pytest.mark.parametrize("shape", [(2048, 96), (256, 64), (128, 32, 64)])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("stage", [1, 2, 3])
@pytest.mark.parametrize("rpt,warps", [(0, 4), (0, 8), (32, 8)])
def test_strided_tma_staging_matches_oracle(shape, bc, stage, rpt, warps):
    """The neighbour-exchange strided pass with its tiles moved by TMA
    (tensor loads of the pair level, tensor stores of the powers, or both)
    equals the oracle's D^p, and mol_sync reports no timed-out wait."""
    n = shape[0]                         # the strided axis: y in 2D, z in 3D
    h = spacing(n, bc)
    s = make(shape, 1.5 * h, 3, bc, "mixed")
    v = field(shape, 80, bc)
    vd = dev(v)
    axis = 1 if len(shape) == 2 else 2
    s.set_tuning(res_warps=2, strided_rpt=rpt, strided_warps=warps, rows_warps=0, strided_nb=1, strided_stage=stage)
    assert s.tuning()["strided_stage"] == stage
    for p in (1, 2, 3):
        got = s.apply_D(vd, axis, p).cpu().numpy()
        ref = oracle.D_axis(v, axis, s.nu[axis], bc, 2, power=p)
        assert rel_l2(got, ref) <= tol_for("mixed", s, p), (p, rel_l2(got, ref))
    s.sync()
    s.close()


# The 3D y pass (Horner in D_y with P+1 outputs) with one neighbour exchange
# per sweep, its fields read from global memory (strided_nb 1) or staged in
# shared memory (2), against the oracle's F and steps; decays on either side
# of the exchange's limit (where it does not hold the full-carry pass runs),
# lines in one CTA and over a 2-CTA cluster, x extents that are not a multiple
# of the 32-line group.
@pytest.mark.parametrize("shape", [(64, 128, 64), (40, 256, 32), (96, 64, 48)])
@pytest.mark.parametrize("cfl", [0.5, 3.0])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("P", [1, 3])
@pytest.mark.parametrize("rpt,warps", [(0, 8), (32, 8), (32, 4)])
def test_strided_horner_neighbour_exchange_matches_oracle(shape, cfl, bc, P, rpt, warps):
    s = make(shape, cfl * spacing(shape[1], bc), P, bc, "mixed")
    u = field(shape, 90, bc)
    ud = dev(u)
    ref = oracle.F(u, s.nu, P, s.beta, bc)
    for nb in (2, 1, 0):
        s.set_tuning(res_warps=2, strided_rpt=rpt, strided_warps=warps, rows_warps=0, strided_nb=nb)
        assert s.tuning()["strided_nb"] == nb
        got = s.apply_F(ud).cpu().numpy()
        assert rel_l2(got, ref) <= tol_for("mixed", s, 2 * P), (nb, rel_l2(got, ref))
    s.sync()
    s.close()


def test_strided_horner_neighbour_exchange_steps():
    """Six steps of a 3D Dirichlet problem with the staged neighbour-exchange
    y pass follow the oracle's time stepping."""
    shape, P, bc, nsteps = (64, 128, 64), 2, "dirichlet", 6
    s = make(shape, 1.0 * spacing(shape[1], bc), P, bc, "mixed")
    s.set_tuning(res_warps=2, strided_rpt=32, strided_warps=8, rows_warps=0, strided_nb=2)
    u0 = smooth_field(shape, 91, bc) + 0.05 * field(shape, 92, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    Fsum, a, b = 0.0, u0, u1
    for _ in range(nsteps):
        F = oracle.F(b, s.nu, P, s.beta, bc)
        Fsum += np.linalg.norm(F)
        a, b = b, 2 * b - a + F
    tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol
    s.close()


@pytest.mark.parametrize("shape,W", [((40, 2048), 2), ((24, 1024), 2), ((40, 2048), 4), ((16, 4096), 4)])
@pytest.mark.parametrize("cfl", [0.5, 2.0, 3.0])
@pytest.mark.parametrize("bc", ["dirichlet", "periodic"])
@pytest.mark.parametrize("P", [1, 3])
@pytest.mark.parametrize("rows_nb", [1, 0])
def test_rows_neighbour_exchange_matches_oracle(shape, W, cfl, bc, P, rows_nb):
    """The x pass over W warps per row with one neighbour exchange per sweep
    (two warps: the neighbours, where d^(RPT-1) <= 2^-27; four warps: two on
    each side, where d^(2 RPT - 1) <= 2^-27; the full carries otherwise): F
    and a few steps against the oracle."""
    nx = shape[1]
    dt = cfl * spacing(nx, bc)
    s = make(shape, dt, P, bc, "mixed")
    s.set_tuning(res_warps=2, strided_rpt=0, strided_warps=8, rows_warps=W, rows_nb=rows_nb)
    assert s.tuning()["rows_nb"] == rows_nb
    u = field(shape, 90, bc)
    ref = oracle.F(u, s.nu, P, s.beta, bc)
    assert rel_l2(s.apply_F(dev(u)).cpu().numpy(), ref) <= tol_for("mixed", s, 2 * P)
    u0 = smooth_field(shape, 91, bc) + 0.05 * field(shape, 92, bc)
    u1 = oracle.start(u0, s.nu, P, s.beta, bc)
    up, uc = dev(u0), dev(u1)
    nsteps = 5
    s.step(up, uc, nsteps)
    rp, rc = oracle.run(u0, u1, nsteps, s.nu, P, s.beta, bc)
    Fsum, a, b = 0.0, u0, u1
    for _ in range(nsteps):
        F = oracle.F(b, s.nu, P, s.beta, bc)
        Fsum += np.linalg.norm(F)
        a, b = b, 2 * b - a + F
    tol = 8 * EPS32 * (1 + 1 / (1 - max(s.d))) * 2 * P * Fsum / np.linalg.norm(rc)
    assert rel_l2(uc.cpu().numpy(), rc) <= tol
    s.close()
