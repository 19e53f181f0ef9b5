"""The C-ABI library loads and exports every symbol include/molt.h declares;
host-only logic (argument validation, beta_max) works without a GPU."""
import ctypes
import re
from pathlib import Path

import numpy as np

import pytest

import oracle
from paper_1308_3214_gb300 import molt
from paper_1308_3214_gb300.build import build

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    build()
    return molt.load_library()


def _declared_functions():
    text = (ROOT / "include" / "molt.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mol_[A-Za-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert _declared_functions() == sorted(molt.EXPORTS)


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_beta_max_matches_oracle(lib):
    for P in range(1, 6):
        assert lib.mol_beta_max(P) == pytest.approx(oracle.beta_max(P), abs=1e-10)
    assert lib.mol_beta_max(0) == -1.0 and lib.mol_beta_max(6) == -1.0


def test_default_options(lib):
    o = molt.mol_options()
    lib.mol_default_options(ctypes.byref(o))
    assert (o.quad_order, o.lines_per_block, o.use_graphs) == (2, 0, 1)
    assert lib.mol_max_line(0) >= 2048


def _create(lib, ndim=2, n=(64, 64, 1), c=1.0, dt=0.01, beta=0.0, P=2, bc=1, prec=1, opt=None):
    g = molt.mol_grid()
    g.ndim = ndim
    for a in range(3):
        g.n[a] = n[a]
        g.lo[a] = 0.0
        g.hi[a] = 1.0
    h = ctypes.c_void_p()
    st = lib.mol_create(ctypes.byref(g), c, dt, beta, P, bc, prec,
                        ctypes.byref(opt) if opt is not None else None, ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("kw, status", [
    (dict(ndim=0), molt.MOL_EINVAL),
    (dict(ndim=4), molt.MOL_EINVAL),
    (dict(P=0), molt.MOL_EINVAL),
    (dict(P=6), molt.MOL_EINVAL),
    (dict(c=0.0), molt.MOL_EINVAL),
    (dict(dt=-1.0), molt.MOL_EINVAL),
    (dict(bc=7), molt.MOL_EINVAL),
    (dict(prec=9), molt.MOL_EINVAL),
    (dict(n=(2, 64, 1)), molt.MOL_EINVAL),
    (dict(n=(64, 10**6, 1)), molt.MOL_EINVAL),
    (dict(P=2, beta=1.49), molt.MOL_EUNSTABLE),
    (dict(P=1, beta=2.0001), molt.MOL_EUNSTABLE),
])
def test_create_rejects_bad_arguments_on_the_host(lib, kw, status):
    st, h = _create(lib, **kw)
    assert st == status
    assert not h.value
    assert len(lib.mol_last_error(None)) > 0


def test_create_rejects_bad_options(lib):
    opt = molt.mol_options(3, 0, 1)
    st, _ = _create(lib, opt=opt)
    assert st == molt.MOL_EINVAL
    opt = molt.mol_options(2, 3, 1)
    st, _ = _create(lib, opt=opt)
    assert st == molt.MOL_EINVAL


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.mol_step(None, None, None, 1, None) == molt.MOL_EINVAL
    assert lib.mol_destroy(None) == molt.MOL_EINVAL
    assert lib.mol_launch_count(None) == 0


# --------------------------------------------------------------------------
# embedded-boundary handles: the geometry is checked on the host, before any
# device work
# --------------------------------------------------------------------------
def _embed_create(lib, g, P=2, beta=0.0, prec=0):
    i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    arrs = [i64(g.r0), i64(g.r1), f64(g.ra), f64(g.rb), i64(g.c0), i64(g.c1), f64(g.ca), f64(g.cb)]
    geom = molt.mol_embed_geom(g.nx, g.ny, g.hx, g.hy, *[a.ctypes.data for a in arrs])
    h = ctypes.c_void_p()
    st = lib.mol_embed_create(ctypes.byref(geom), 1.0, 0.01, beta, P, prec, ctypes.byref(h))
    return st, h


def test_embed_create_rejects_bad_geometry_on_the_host(lib):
    from paper_1308_3214_gb300 import workloads
    g = workloads.ellipse_grid(41)
    bad = workloads.ellipse_grid(41)
    bad.ra = bad.ra.copy()
    bad.ra[20] = 0.0                                     # a boundary point on the first interior node
    assert _embed_create(lib, bad)[0] == molt.MOL_EINVAL
    bad = workloads.ellipse_grid(41)
    bad.r1 = bad.r1.copy()
    bad.r1[20] += 1                                      # the row claims a node its column does not
    st, h = _embed_create(lib, bad)
    assert st == molt.MOL_EINVAL and not h.value
    assert b"disagree" in lib.mol_last_error(None)
    bad = workloads.ellipse_grid(41)
    bad.c1 = bad.c1.copy()
    bad.c1[20] = 41                                      # past the grid
    assert _embed_create(lib, bad)[0] == molt.MOL_EINVAL
    assert _embed_create(lib, g, P=0)[0] == molt.MOL_EINVAL
    assert _embed_create(lib, g, P=2, beta=1.49)[0] == molt.MOL_EUNSTABLE
    assert _embed_create(lib, g, prec=7)[0] == molt.MOL_EINVAL
    big = workloads.disk_grid(2301, radius=1.0, half=1.1)   # the middle row holds more than 2046 nodes
    st, _ = _embed_create(lib, big)
    assert st == molt.MOL_EINVAL and b"2046" in lib.mol_last_error(None)


def test_embed_null_handle_calls_fail_cleanly(lib):
    assert lib.mol_embed_step(None, None, None, 1, None) == molt.MOL_EINVAL
    assert lib.mol_embed_destroy(None) == molt.MOL_OK
    assert lib.mol_embed_launch_count(None) == 0


def test_robustness_calls_refuse_bad_arguments_on_the_host(lib):
    """Host-side checks of the robustness entry points (no GPU needed)."""
    assert lib.mol_field_norm(None, None, None, None) == molt.MOL_EINVAL
    assert lib.mol_step_checked(None, None, None, 1, 10.0, None) == molt.MOL_EINVAL
    assert lib.mol_checkpoint_write(None, b"x", None, None, 0, None) == molt.MOL_EINVAL
    assert lib.mol_checkpoint_read(None, b"x", None, None, None, None) == molt.MOL_EINVAL
    for limit in (0, -1, 1 << 41):
        assert lib.mol_wait_selftest(limit, None) == molt.MOL_EINVAL
    lib.mol_debug_fail_alloc(-1)          # the hooks are plain host switches
    lib.mol_debug_allow_unstable(0)
