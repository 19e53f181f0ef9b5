"""mol_apply_F_noalloc: F[u] in float64 with every buffer in the library's
static scratch, against mol_apply_F on a float64 handle.

The file sorts last so that its GPU tests also run after every other test
of the suite in the same process (the scratch is shared and reused).  Two
calls in a row, on different inputs, must each match; nothing in the
scratch may depend on an earlier call.  The two paths run the same pass
kernels; they differ only in where the tables d^j come from (device exp
here, host exp in mol_create), a relative difference of a few units of
float64 rounding, so the bar is the float64 parity bar, 1e-12.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1308_3214_gb300 import molt, workloads

SCRATCH_BYTES = 32 << 20


def need_bytes(shape, P):
    """Scratch the entry point needs, as its header comment states."""
    r32 = lambda x: (x + 31) // 32 * 32
    nd = len(shape)
    planes = {1: 0, 2: P, 3: 2 * P + 1}[nd]
    N = int(np.prod(shape))
    return 8 * (512 + sum(r32(n + 1) for n in shape) + planes * r32(N))


def call_raw(shape, P, bc="dirichlet", dt=None, beta=0.0, quad=2, u=None, F=None):
    lib = molt.load_library()
    g = molt.make_grid(shape)
    dt = dt if dt is not None else 2.0 / max(shape)
    return lib.mol_apply_F_noalloc(ctypes.byref(g), 1.0, float(dt), float(beta), int(P), molt.BC[bc], int(quad),
                                   u, F, None)


# ---------------------------------------------------------------------------
# host-side checks (no GPU: every one fails before the first CUDA call)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("shape,P", [((2048, 2048), 3), ((64, 64, 512), 2), ((1184, 1184), 3)])
def test_oversize_rejected(shape, P):
    assert need_bytes(shape, P) > SCRATCH_BYTES
    st = call_raw(shape, P)
    assert st == molt.MOL_EINVAL
    msg = molt.load_library().mol_last_error(None).decode()
    assert "static scratch" in msg and str(SCRATCH_BYTES) in msg and str(need_bytes(shape, P)) in msg


@pytest.mark.parametrize("kw,status", [
    (dict(P=0), molt.MOL_EINVAL),
    (dict(P=6), molt.MOL_EINVAL),
    (dict(quad=3), molt.MOL_EINVAL),
    (dict(beta=5.0), molt.MOL_EUNSTABLE),
    (dict(shape=(2, 64)), molt.MOL_EINVAL),
    (dict(shape=(8193,)), molt.MOL_EINVAL),
])
def test_bad_arguments(kw, status):
    args = dict(shape=(64, 64), P=2)
    args.update(kw)
    shape, P = args.pop("shape"), args.pop("P")
    assert call_raw(shape, P, **args) == status


def test_null_grid():
    lib = molt.load_library()
    st = lib.mol_apply_F_noalloc(None, 1.0, 0.01, 0.0, 2, 0, 2, None, None, None)
    assert st == molt.MOL_EINVAL


# ---------------------------------------------------------------------------
# GPU: two calls in a row against mol_apply_F
# ---------------------------------------------------------------------------
CASES = [
    ((1000,), 4, "periodic"),
    ((256, 192), 3, "dirichlet"),        # register kernels on both axes
    ((250, 300), 2, "periodic"),         # ragged lines: shared-memory kernels
    ((250, 300), 2, "dirichlet"),        # ragged Dirichlet: shared-memory kernels here, the handle runs
                                         # the same F as a batch of one
    ((32, 36, 40), 2, "periodic"),
    ((64, 64, 64), 3, "dirichlet"),
    ((1024, 1280), 3, "dirichlet"),      # 2D close to the scratch limit
]


def rel(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0), np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.gpu
@pytest.mark.parametrize("shape,P,bc", CASES)
def test_matches_apply_F_two_calls(shape, P, bc):
    assert need_bytes(shape, P) <= SCRATCH_BYTES
    dt = 2.0 / max(shape)
    us = [torch.from_numpy(workloads.random_field(shape, 7100 + k)).cuda() for k in range(2)]
    with molt.Solver(shape, dt=dt, P=P, bc=bc, prec="fp64") as s:
        refs = [s.apply_F(u) for u in us]
        s.sync()
    outs = [torch.full(shape, float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    for u, o in zip(us, outs):                 # two calls in a row, no synchronisation between them
        molt.apply_F_noalloc(u, o, dt=dt, P=P, bc=bc)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        l2, mx = rel(o, r)
        assert l2 <= 1e-12 and mx <= 1e-12, (l2, mx)


@pytest.mark.gpu
def test_reuse_across_shapes():
    """Calls on different grids back to back (tables and planes of the
    previous call still in the scratch) match their own references."""
    seq = [CASES[4], CASES[1], CASES[0], CASES[4]]
    outs, refs = [], []
    for k, (shape, P, bc) in enumerate(seq):
        dt = 1.5 / max(shape)
        u = torch.from_numpy(workloads.random_field(shape, 7200 + k)).cuda()
        with molt.Solver(shape, dt=dt, P=P, bc=bc, prec="fp64") as s:
            refs.append(s.apply_F(u))
            s.sync()
        o = torch.empty(shape, dtype=torch.float64, device="cuda")
        molt.apply_F_noalloc(u, o, dt=dt, P=P, bc=bc)
        outs.append(o)
    torch.cuda.synchronize()
    for o, r in zip(outs, refs):
        l2, mx = rel(o, r)
        assert l2 <= 1e-12 and mx <= 1e-12, (l2, mx)


def test_fields_on_different_devices_rejected_before_the_library():
    """The binding refuses fields on two devices before it loads or calls
    the library (a launch on the wrong device would read another GPU's
    memory)."""
    u = torch.zeros((8, 8), dtype=torch.float64)
    o = torch.empty((8, 8), dtype=torch.float64, device="meta")
    with pytest.raises(ValueError, match="same CUDA device"):
        molt.apply_F_noalloc(u, o, dt=0.1, P=1)


@pytest.mark.gpu
@pytest.mark.skipif(not torch.cuda.is_available() or torch.cuda.device_count() < 2, reason="needs two GPUs")
def test_field_on_another_device_rejected():
    """Through the C ABI: a field on device 1 while device 0 is current."""
    torch.cuda.set_device(0)
    u = torch.zeros((64, 64), dtype=torch.float64, device="cuda:1")
    o = torch.empty((64, 64), dtype=torch.float64, device="cuda:0")
    st = call_raw((64, 64), 2, u=ctypes.c_void_p(u.data_ptr()), F=ctypes.c_void_p(o.data_ptr()))
    assert st == molt.MOL_EINVAL
    assert "current device" in molt.load_library().mol_last_error(None).decode()


@pytest.mark.gpu
def test_overlapping_fields_rejected():
    """F starting inside u (not the same pointer) is refused."""
    buf = torch.zeros(64 * 64 + 64, dtype=torch.float64, device="cuda")
    st = call_raw((64, 64), 2, u=ctypes.c_void_p(buf.data_ptr()), F=ctypes.c_void_p(buf.data_ptr() + 8 * 64))
    assert st == molt.MOL_EINVAL
    assert "overlap" in molt.load_library().mol_last_error(None).decode()


@pytest.mark.gpu
def test_rejects_host_pointer():
    u = np.zeros((64, 64))
    o = torch.empty((64, 64), dtype=torch.float64, device="cuda")
    st = call_raw((64, 64), 2, u=u.ctypes.data_as(ctypes.c_void_p), F=ctypes.c_void_p(o.data_ptr()))
    assert st == molt.MOL_EINVAL
