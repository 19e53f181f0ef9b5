"""Robustness paths of the library, exercised without faulting the GPU:
the bounded device wait (a wait that cannot succeed gives up and reports
MOL_ETIMEOUT), injected allocation failures (MOL_ENOMEM with nothing left
allocated), the instability check (MOL_EUNSTABLE), checkpoint files and the
field norm."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1308_3214_gb300 import molt, workloads

pytestmark = pytest.mark.gpu


def lib():
    return molt.load_library()


def test_wait_selftest_gives_up_and_the_context_survives():
    st = lib().mol_wait_selftest(2_000_000, None)          # about 1 ms of SM cycles
    assert st == molt.MOL_ETIMEOUT, molt.STATUS_NAMES.get(st)
    # the flag was taken: a solver afterwards syncs cleanly and computes
    shape = (256, 128)
    with molt.Solver(shape, dt=2.0 / 255, P=2, bc="dirichlet", prec="mixed") as s:
        u = torch.from_numpy(workloads.random_field(shape, 3)).cuda()
        F = s.apply_F(u)
        s.sync()
        assert torch.isfinite(F).all()


@pytest.mark.parametrize("limit", [0, -5, 1 << 41])
def test_wait_selftest_rejects_bad_limits(limit):
    assert lib().mol_wait_selftest(limit, None) == molt.MOL_EINVAL


def _free_bytes():
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _creators():
    shape = (256, 256)
    yield "single", lambda: molt.Solver(shape, dt=2.0 / 255, P=3, bc="dirichlet", prec="mixed")
    yield "batch", lambda: molt.BatchSolver([(64, 64), (96, 128)], dt=[0.02, 0.01], P=[1, 2])
    g = workloads.disk_grid(65)
    yield "embedded", lambda: molt.EmbedSolver(g, dt=0.02, P=2, prec="mixed")


@pytest.mark.parametrize("which", ["single", "batch", "embedded"])
def test_injected_allocation_failure(which):
    make = dict(_creators())[which]
    make().close()                                          # warm up library state outside the count
    base = _free_bytes()
    try:
        failures = 0
        for after in range(0, 64):
            lib().mol_debug_fail_alloc(after)
            try:
                obj = make()
            except molt.MolError as e:
                assert "MOL_ENOMEM" in str(e) and "injected" in str(e), str(e)
                failures += 1
                continue
            lib().mol_debug_fail_alloc(-1)
            obj.close()
            break
        else:
            pytest.fail("creation never succeeded within 64 allocations")
        assert failures >= 1
    finally:
        lib().mol_debug_fail_alloc(-1)
    # everything a failed creation allocated was freed again
    assert abs(_free_bytes() - base) < (8 << 20)


def test_field_norm_matches_numpy():
    shape = (200, 300)
    with molt.Solver(shape, dt=1.0 / 299, P=1, bc="periodic", prec="fp64", lo=[0, 0], hi=[2.0, 3.0]) as s:
        u = workloads.random_field(shape, 9)
        got = s.norm(torch.from_numpy(u).cuda())
        hx, hy = 3.0 / 300, 2.0 / 200
        assert got == pytest.approx(np.sqrt(hx * hy * np.sum(u * u)), rel=1e-12)


def test_step_checked_passes_a_stable_run_and_flags_non_finite_fields():
    n = 256
    with molt.Solver((n, n), dt=2.0 / (n - 1), P=3, bc="dirichlet", prec="mixed") as s:
        u0 = torch.from_numpy(workloads.gaussian_2d(n, width=0.05)).cuda()
        up, uc = u0.clone(), s.start(u0)
        s.step_checked(up, uc, 50)                          # A-stable at beta_max: bounded
        uc[n // 2, n // 2] = float("nan")
        with pytest.raises(molt.MolError, match="MOL_EUNSTABLE"):
            s.step_checked(up, uc, 3)


def test_step_checked_flags_growth_above_beta_max():
    n, P = 128, 1
    lib().mol_debug_allow_unstable(1)
    try:
        s = molt.Solver((n, n), dt=4.0 / (n - 1), P=P, bc="periodic", prec="fp64",
                        beta=1.6 * molt.beta_max(P))
    finally:
        lib().mol_debug_allow_unstable(0)
    with s:
        u = torch.from_numpy(workloads.random_field((n, n), 4)).cuda()
        up, uc = u.clone(), u.clone()
        with pytest.raises(molt.MolError, match="MOL_EUNSTABLE"):
            for _ in range(40):
                s.step_checked(up, uc, 25, growth_limit=1e3)
    with pytest.raises(molt.MolError, match="MOL_EUNSTABLE"):
        molt.Solver((n, n), dt=4.0 / (n - 1), P=P, bc="periodic", prec="fp64", beta=1.6 * molt.beta_max(P))


def test_checkpoint_round_trip_and_refusals(tmp_path):
    shape = (128, 256)
    mk = lambda **kw: molt.Solver(shape, dt=kw.get("dt", 2.0 / 255), P=kw.get("P", 2), bc="dirichlet", prec="mixed")
    with mk() as s:
        u0 = torch.from_numpy(workloads.gaussian_2d(256, ny=128, width=0.08)).cuda()
        up, uc = u0.clone(), s.start(u0)
        s.step(up, uc, 7)
        path = tmp_path / "run.ckp"
        s.checkpoint_write(path, up, uc, 8)
        # continuing directly and continuing from the file agree bitwise
        a_prev, a_cur = up.clone(), uc.clone()
        s.step(a_prev, a_cur, 5)
        b_prev, b_cur = torch.zeros_like(up), torch.zeros_like(uc)
        assert s.checkpoint_read(path, b_prev, b_cur) == 8
        assert torch.equal(b_prev, up) and torch.equal(b_cur, uc)
        s.step(b_prev, b_cur, 5)
        assert torch.equal(a_cur, b_cur)
        # corrupted data, truncated file
        raw = bytearray(path.read_bytes())
        raw[len(raw) // 2] ^= 0x40
        bad = tmp_path / "bad.ckp"
        bad.write_bytes(bytes(raw))
        with pytest.raises(molt.MolError, match="checksum"):
            s.checkpoint_read(bad, b_prev, b_cur)
        short = tmp_path / "short.ckp"
        short.write_bytes(path.read_bytes()[:1000])
        with pytest.raises(molt.MolError, match="truncated"):
            s.checkpoint_read(short, b_prev, b_cur)
    with mk(P=3) as other:                                   # another problem
        with pytest.raises(molt.MolError, match="another problem"):
            other.checkpoint_read(path, torch.zeros_like(up), torch.zeros_like(uc))


@pytest.mark.parametrize("d", [0.05, 0.5395, 0.9])
def test_toeplitz_experiment_variants_agree(d):
    """The tensor-core Toeplitz product and the scan give the same chunk
    recurrence (three TF32 products keep float32 accuracy)."""
    t_scan, t_tc, diff = molt.toeplitz_experiment(256, 512, d, reps=3)
    assert t_scan > 0 and t_tc > 0
    assert diff <= 2e-6, diff


def test_toeplitz_experiment_rejects_bad_sizes():
    assert lib().mol_toeplitz_experiment(100, 64, 0.5, 1, (ctypes.c_double * 2)(), ctypes.byref(ctypes.c_double()),
                                         None) == molt.MOL_EINVAL
