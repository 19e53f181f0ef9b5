"""ctypes binding of libmolt (include/molt.h): argument marshalling only.

Every operation runs in the CUDA library; torch is used for device memory
and streams.  Importing this module does not need a GPU; creating a
``Solver`` does, and fails loudly if the library or the GPU is missing.

Fields are torch float64 tensors on the GPU, C-contiguous with shape
``(nx,)``, ``(ny, nx)`` or ``(nz, ny, nx)`` (x fastest), matching the
library's ``index = x + nx*(y + ny*z)``.
"""
from __future__ import annotations

import ctypes
from pathlib import Path
from typing import Sequence

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "_build" / "libmolt.so"

MOL_OK, MOL_EINVAL, MOL_ENOMEM, MOL_ECUDA, MOL_EUNSTABLE, MOL_ETIMEOUT = range(6)
STATUS_NAMES = {0: "MOL_OK", 1: "MOL_EINVAL", 2: "MOL_ENOMEM", 3: "MOL_ECUDA", 4: "MOL_EUNSTABLE",
                5: "MOL_ETIMEOUT"}
BC = {"periodic": 0, "dirichlet": 1}
PREC = {"fp64": 0, "mixed": 1}

# Every symbol include/molt.h declares.
EXPORTS = ["mol_default_options", "mol_create", "mol_destroy", "mol_last_error", "mol_beta_max",
           "mol_max_line", "mol_get_params", "mol_apply_D", "mol_apply_F", "mol_start", "mol_step",
           "mol_solve_host", "mol_sync", "mol_launch_count", "mol_set_pass_timing", "mol_pass_times",
           "mol_apply_F_noalloc", "mol_batch_create", "mol_batch_destroy", "mol_batch_last_error",
           "mol_batch_offsets", "mol_batch_apply_F", "mol_batch_start", "mol_batch_step", "mol_batch_solve_host", "mol_batch_sync",
           "mol_batch_launch_count", "mol_batch_set_pass_timing", "mol_batch_pass_times", "mol_batch_apply_FT",
           "mol_batch_traces", "mol_batch_adjoint", "mol_batch_update", "mol_autotune", "mol_get_tuning", "mol_set_tuning",
           "mol_get_tuning_ex", "mol_set_tuning_ex",
           "mol_batch_autotune", "mol_batch_get_tuning", "mol_batch_set_tuning", "mol_solve_dirichlet", "mol_solve_source", "mol_apply_FT", "mol_traces", "mol_adjoint",
           "mol_embed_create", "mol_embed_destroy", "mol_embed_last_error", "mol_embed_linv", "mol_embed_apply_F",
           "mol_embed_start", "mol_embed_step", "mol_embed_solve_host", "mol_embed_sync", "mol_embed_launch_count",
           "mol_embed_set_pass_timing", "mol_embed_pass_times", "mol_field_norm", "mol_step_checked",
           "mol_checkpoint_write", "mol_checkpoint_read", "mol_wait_selftest", "mol_debug_fail_alloc",
           "mol_debug_allow_unstable", "mol_adjoint_history", "mol_batch_adjoint_history",
           "mol_toeplitz_experiment", "mol_pair_split", "mol_pair_join"]


class MolError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class mol_grid(ctypes.Structure):
    _fields_ = [("ndim", ctypes.c_int), ("n", ctypes.c_int64 * 3), ("lo", ctypes.c_double * 3),
                ("hi", ctypes.c_double * 3)]


class mol_embed_geom(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int64), ("ny", ctypes.c_int64), ("hx", ctypes.c_double), ("hy", ctypes.c_double),
                ("row_lo", ctypes.c_void_p), ("row_hi", ctypes.c_void_p), ("row_gap_lo", ctypes.c_void_p),
                ("row_gap_hi", ctypes.c_void_p), ("col_lo", ctypes.c_void_p), ("col_hi", ctypes.c_void_p),
                ("col_gap_lo", ctypes.c_void_p), ("col_gap_hi", ctypes.c_void_p)]


class mol_options(ctypes.Structure):
    _fields_ = [("quad_order", ctypes.c_int), ("lines_per_block", ctypes.c_int), ("use_graphs", ctypes.c_int)]


_lib = None


def load_library(path: Path | None = None):
    """Load libmolt.so (building it first if it is missing)."""
    global _lib
    if _lib is not None:
        return _lib
    p = Path(path) if path else LIB_PATH
    if not p.exists():
        from . import build as _build
        _build.build()
    if not p.exists():
        raise RuntimeError(f"libmolt.so not found at {p}; run `python -m paper_1308_3214_gb300.build`")
    lib = ctypes.CDLL(str(p))
    vp, dp, i64 = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64
    I, D = ctypes.c_int, ctypes.c_double
    lib.mol_default_options.argtypes = [ctypes.POINTER(mol_options)]
    lib.mol_create.argtypes = [ctypes.POINTER(mol_grid), D, D, D, I, I, I, ctypes.POINTER(mol_options),
                               ctypes.POINTER(vp)]
    lib.mol_destroy.argtypes = [vp]
    lib.mol_last_error.argtypes = [vp]
    lib.mol_last_error.restype = ctypes.c_char_p
    lib.mol_beta_max.argtypes = [I]
    lib.mol_beta_max.restype = D
    lib.mol_max_line.argtypes = [I]
    lib.mol_max_line.restype = i64
    lib.mol_get_params.argtypes = [vp, dp]
    lib.mol_apply_D.argtypes = [vp, vp, vp, I, I, vp]
    lib.mol_apply_F.argtypes = [vp, vp, vp, vp]
    lib.mol_start.argtypes = [vp, vp, vp, vp]
    lib.mol_step.argtypes = [vp, vp, vp, i64, vp]
    lib.mol_solve_host.argtypes = [vp, dp, dp, i64, vp]
    lib.mol_sync.argtypes = [vp, vp]
    lib.mol_set_pass_timing.argtypes = [vp, I]
    lib.mol_pass_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
    lib.mol_launch_count.argtypes = [vp]
    lib.mol_apply_F_noalloc.argtypes = [ctypes.POINTER(mol_grid), D, D, D, I, I, I, vp, vp, vp]
    lib.mol_batch_create.argtypes = [I, ctypes.POINTER(mol_grid), dp, dp, dp, ctypes.POINTER(I), I, I,
                                     ctypes.POINTER(mol_options), ctypes.POINTER(vp)]
    lib.mol_batch_destroy.argtypes = [vp]
    lib.mol_batch_last_error.argtypes = [vp]
    lib.mol_batch_last_error.restype = ctypes.c_char_p
    lib.mol_batch_offsets.argtypes = [vp, ctypes.POINTER(i64)]
    lib.mol_batch_apply_F.argtypes = [vp, vp, vp, vp]
    lib.mol_batch_start.argtypes = [vp, vp, vp, vp]
    lib.mol_batch_step.argtypes = [vp, vp, vp, i64, vp]
    lib.mol_batch_solve_host.argtypes = [vp, dp, dp, i64, vp]
    lib.mol_batch_sync.argtypes = [vp, vp]
    lib.mol_batch_launch_count.argtypes = [vp]
    lib.mol_batch_launch_count.restype = i64
    lib.mol_batch_set_pass_timing.argtypes = [vp, I]
    lib.mol_batch_pass_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
    lib.mol_batch_apply_FT.argtypes = [vp, vp, vp, vp]
    lib.mol_batch_traces.argtypes = [vp, vp, I, ctypes.POINTER(i64), i64, vp, vp]
    lib.mol_batch_adjoint.argtypes = [vp, I, ctypes.POINTER(i64), i64, vp, vp, vp]
    lib.mol_batch_update.argtypes = [vp, vp, vp, vp, D, D, D, I, vp, vp]
    lib.mol_autotune.argtypes = [vp, vp]
    lib.mol_get_tuning.argtypes = [vp, ctypes.POINTER(I), dp]
    lib.mol_set_tuning.argtypes = [vp, I, I, I, I]
    lib.mol_get_tuning_ex.argtypes = [vp, ctypes.POINTER(I), I, dp]
    lib.mol_set_tuning_ex.argtypes = [vp, ctypes.POINTER(I), I]
    lib.mol_batch_autotune.argtypes = [vp, vp]
    lib.mol_apply_FT.argtypes = [vp, vp, vp, vp]
    lib.mol_traces.argtypes = [vp, vp, I, ctypes.POINTER(i64), i64, vp, vp]
    lib.mol_adjoint.argtypes = [vp, I, ctypes.POINTER(i64), i64, vp, vp, vp]
    lib.mol_batch_get_tuning.argtypes = [vp, ctypes.POINTER(I), dp]
    lib.mol_batch_set_tuning.argtypes = [vp, I, I, I]
    lib.mol_solve_dirichlet.argtypes = [vp, vp, i64, dp, vp, vp]
    lib.mol_solve_source.argtypes = [vp, vp, i64, vp, dp, vp, vp]
    lib.mol_embed_create.argtypes = [ctypes.POINTER(mol_embed_geom), D, D, D, I, I, ctypes.POINTER(vp)]
    lib.mol_embed_destroy.argtypes = [vp]
    lib.mol_embed_last_error.argtypes = [vp]
    lib.mol_embed_last_error.restype = ctypes.c_char_p
    lib.mol_embed_linv.argtypes = [vp, vp, vp, I, vp]
    lib.mol_embed_apply_F.argtypes = [vp, vp, vp, vp]
    lib.mol_embed_start.argtypes = [vp, vp, vp, vp]
    lib.mol_embed_step.argtypes = [vp, vp, vp, i64, vp]
    lib.mol_embed_solve_host.argtypes = [vp, dp, dp, i64, vp]
    lib.mol_embed_sync.argtypes = [vp, vp]
    lib.mol_embed_launch_count.argtypes = [vp]
    lib.mol_embed_launch_count.restype = i64
    lib.mol_embed_set_pass_timing.argtypes = [vp, I]
    lib.mol_embed_pass_times.argtypes = [vp, dp, ctypes.POINTER(i64)]
    lib.mol_launch_count.restype = i64
    lib.mol_field_norm.argtypes = [vp, vp, dp, vp]
    lib.mol_pair_split.argtypes = [vp, vp, vp, i64, vp]
    lib.mol_pair_join.argtypes = [vp, vp, vp, i64, vp]
    lib.mol_step_checked.argtypes = [vp, vp, vp, i64, D, vp]
    lib.mol_checkpoint_write.argtypes = [vp, ctypes.c_char_p, vp, vp, i64, vp]
    lib.mol_checkpoint_read.argtypes = [vp, ctypes.c_char_p, vp, vp, ctypes.POINTER(i64), vp]
    lib.mol_wait_selftest.argtypes = [i64, vp]
    lib.mol_debug_fail_alloc.argtypes = [i64]
    lib.mol_debug_fail_alloc.restype = None
    lib.mol_debug_allow_unstable.argtypes = [I]
    lib.mol_debug_allow_unstable.restype = None
    lib.mol_adjoint_history.argtypes = [vp, vp, i64, i64, GRAD_FN, vp, vp, vp]
    lib.mol_toeplitz_experiment.argtypes = [I, I, D, I, dp, dp, vp]
    lib.mol_batch_adjoint_history.argtypes = [vp, vp, i64, i64, GRAD_FN, vp, vp, vp]
    for name in EXPORTS:
        if name not in ("mol_default_options", "mol_last_error", "mol_beta_max", "mol_max_line",
                        "mol_launch_count", "mol_batch_last_error", "mol_batch_launch_count",
                        "mol_embed_last_error", "mol_embed_launch_count", "mol_debug_fail_alloc",
                        "mol_debug_allow_unstable"):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def beta_max(P: int) -> float:
    return load_library().mol_beta_max(int(P))


def make_grid(shape: Sequence[int], lo: Sequence[float] | None = None,
              hi: Sequence[float] | None = None) -> mol_grid:
    """mol_grid of an array shape (nz, ny, nx); lo / hi in the same order
    (default [0, 1] on every axis)."""
    shape = tuple(int(s) for s in shape)
    nd = len(shape)
    lo = [0.0] * nd if lo is None else lo
    hi = [1.0] * nd if hi is None else hi
    g = mol_grid()
    g.ndim = nd
    for a in range(3):
        g.n[a] = shape[nd - 1 - a] if a < nd else 1
        g.lo[a] = float(lo[nd - 1 - a]) if a < nd else 0.0
        g.hi[a] = float(hi[nd - 1 - a]) if a < nd else 1.0
    return g


def apply_F_noalloc(u, out, dt: float, P: int, bc: str = "dirichlet", c: float = 1.0, beta: float = 0.0,
                    lo: Sequence[float] | None = None, hi: Sequence[float] | None = None,
                    quad_order: int = 2, stream=None):
    """F[u] in float64 through mol_apply_F_noalloc: no handle and no device
    allocation.  u and out: contiguous CUDA float64 tensors of one shape
    (nz, ny, nx); the library's static scratch bounds the grid size."""
    import torch
    for t, name in ((u, "u"), (out, "out")):
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
    if u.device != out.device:
        raise ValueError(f"u ({u.device}) and out ({out.device}) must be on the same CUDA device")
    for t, name in ((u, "u"), (out, "out")):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    if tuple(u.shape) != tuple(out.shape):
        raise ValueError("u and out must have the same shape")
    lib = load_library()
    g = make_grid(u.shape, lo, hi)
    with torch.cuda.device(u.device):           # the library launches on the current device
        if stream is not None and stream.device != u.device:
            raise ValueError(f"stream is on {stream.device}, the fields on {u.device}")
        st = lib.mol_apply_F_noalloc(ctypes.byref(g), float(c), float(dt), float(beta), int(P), BC[bc],
                                     int(quad_order), ctypes.c_void_p(u.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream)))
    if st != MOL_OK:
        raise MolError(st, lib.mol_last_error(None).decode())
    return out


def _pair_args(x, hi, lo):
    import torch
    for t, name, dt in ((x, "x", torch.float64), (hi, "hi", torch.float32), (lo, "lo", torch.float32)):
        if not isinstance(t, torch.Tensor) or t.dtype != dt or not t.is_cuda or not t.is_contiguous():
            raise TypeError(f"{name} must be a contiguous CUDA {dt} tensor")
    if not (x.numel() == hi.numel() == lo.numel()) or not (x.device == hi.device == lo.device):
        raise ValueError("x, hi and lo must have the same size and device")


def pair_split(x, hi=None, lo=None, stream=None):
    """(hi, lo) float32 planes with hi = x rounded to float32 and lo = x - hi
    rounded (mol_pair_split: the mixed path's level conversion)."""
    import torch
    hi = torch.empty(x.shape, dtype=torch.float32, device=x.device) if hi is None else hi
    lo = torch.empty(x.shape, dtype=torch.float32, device=x.device) if lo is None else lo
    _pair_args(x, hi, lo)
    lib = load_library()
    with torch.cuda.device(x.device):
        st = lib.mol_pair_split(ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(hi.data_ptr()),
                                ctypes.c_void_p(lo.data_ptr()), x.numel(), ctypes.c_void_p(_stream_ptr(stream)))
    if st != MOL_OK:
        raise MolError(st, lib.mol_last_error(None).decode())
    return hi, lo


def pair_join(hi, lo, out=None, stream=None):
    """x = hi + lo in float64 (mol_pair_join)."""
    import torch
    out = torch.empty(hi.shape, dtype=torch.float64, device=hi.device) if out is None else out
    _pair_args(out, hi, lo)
    lib = load_library()
    with torch.cuda.device(hi.device):
        st = lib.mol_pair_join(ctypes.c_void_p(hi.data_ptr()), ctypes.c_void_p(lo.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), hi.numel(), ctypes.c_void_p(_stream_ptr(stream)))
    if st != MOL_OK:
        raise MolError(st, lib.mol_last_error(None).decode())
    return out


def _stream_ptr(stream) -> int:
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Solver:
    """One MOL^T problem: grid, c, dt, beta, P, boundary condition, precision.

    ``shape`` is given in array order (nz, ny, nx) like the fields; ``lo`` and
    ``hi`` likewise.  ``beta <= 0`` selects beta_max(P)."""

    def __init__(self, shape: Sequence[int], dt: float, P: int, bc: str = "dirichlet",
                 prec: str = "mixed", c: float = 1.0, beta: float = 0.0,
                 lo: Sequence[float] | None = None, hi: Sequence[float] | None = None,
                 quad_order: int = 2, lines_per_block: int = 0, use_graphs: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmolt needs a CUDA GPU")
        self.lib = load_library()
        self.shape = tuple(int(s) for s in shape)
        nd = len(self.shape)
        g = make_grid(self.shape, lo, hi)
        opt = mol_options(int(quad_order), int(lines_per_block), 1 if use_graphs else 0)
        h = ctypes.c_void_p()
        torch.cuda.init()
        st = self.lib.mol_create(ctypes.byref(g), float(c), float(dt), float(beta), int(P), BC[bc],
                                 PREC[prec], ctypes.byref(opt), ctypes.byref(h))
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_last_error(None).decode())
        self.h = h
        self.P, self.bc, self.prec, self.dt, self.c = int(P), bc, prec, float(dt), float(c)
        prm = (ctypes.c_double * 8)()
        self._check(self.lib.mol_get_params(self.h, prm))
        self.alpha, self.beta = prm[0], prm[1]
        self.nu = tuple(prm[2 + a] for a in range(nd))      # x first
        self.d = tuple(prm[5 + a] for a in range(nd))

    # ------------------------------------------------------------------
    def _check(self, st: int):
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_last_error(self.h).decode())

    def _field(self, t, name):
        import torch
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda:
            raise TypeError(f"{name} must be a CUDA float64 tensor")
        if tuple(t.shape) != self.shape or not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous with shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    # ------------------------------------------------------------------
    def apply_D(self, v, axis: int, power: int = 1, out=None, stream=None):
        """D_axis^power v; axis 0 is x (the last array dimension)."""
        out = self.empty() if out is None else out
        self._check(self.lib.mol_apply_D(self.h, self._field(v, "v"), self._field(out, "out"), int(axis),
                                         int(power), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def apply_F(self, u, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_apply_F(self.h, self._field(u, "u"), self._field(out, "F"),
                                         ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def start(self, u0, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_start(self.h, self._field(u0, "u0"), self._field(out, "u1"),
                                       ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def step(self, u_prev, u_cur, nsteps: int, stream=None):
        """Advance (u_prev, u_cur) in place by nsteps."""
        self._check(self.lib.mol_step(self.h, self._field(u_prev, "u_prev"), self._field(u_cur, "u_cur"),
                                      int(nsteps), ctypes.c_void_p(_stream_ptr(stream))))
        return u_prev, u_cur

    def solve_host(self, u0: np.ndarray, nsteps: int, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """u^{nsteps} from host u0 (zero initial velocity), host result."""
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        if u0.shape != self.shape:
            raise ValueError(f"u0 must have shape {self.shape}")
        out = np.empty_like(u0) if out is None else out
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.mol_solve_host(self.h, u0.ctypes.data_as(dp), out.ctypes.data_as(dp), int(nsteps),
                                            ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def apply_FT(self, w, out=None, stream=None):
        """F^T w (2D Dirichlet grids of at most 1024 points per axis)."""
        out = self.empty() if out is None else out
        self._check(self.lib.mol_apply_FT(self.h, self._field(w, "w"), self._field(out, "out"),
                                          ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def traces(self, u0, rec, nsteps: int, stream=None):
        """(nsteps, nrec): u^n at the flat indices rec (y nx + x), n = 1..nsteps."""
        import torch
        rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int64).reshape(-1))
        out = torch.empty((int(nsteps), rec.size), dtype=torch.float64, device="cuda")
        self._check(self.lib.mol_traces(self.h, self._field(u0, "u0"), rec.size,
                                        rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), int(nsteps),
                                        ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def adjoint(self, rec, tgrad, stream=None):
        """dJ/du^0 from tgrad[n-1, r] = dJ/d(u^n at rec[r])."""
        import torch
        rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int64).reshape(-1))
        tg = tgrad.to(dtype=torch.float64, device="cuda").contiguous()
        if tg.dim() != 2 or tg.shape[1] != rec.size:
            raise ValueError("tgrad must be (nsteps, nrec)")
        out = self.empty()
        self._check(self.lib.mol_adjoint(self.h, rec.size, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                         int(tg.shape[0]), ctypes.c_void_p(tg.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def solve_dirichlet(self, u0, nsteps: int, data, stream=None):
        """u^nsteps of a 1D Dirichlet problem with time-dependent end data:
        data[k, side, m] = (d_tt / c^2)^m u_side(t_k), k = 0..nsteps,
        m = 0..P (host float64), zero initial velocity."""
        d = np.ascontiguousarray(np.asarray(data, dtype=np.float64).reshape(int(nsteps) + 1, 2, self.P + 1))
        out = self.empty()
        self._check(self.lib.mol_solve_dirichlet(self.h, self._field(u0, "u0"), int(nsteps),
                                                 d.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                                 self._field(out, "u_out"), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def solve_source(self, u0, nsteps: int, g, f, stream=None):
        """u^nsteps with the source S = g(x) f(t) (P = 1 or 2), zero initial
        velocity: g a CUDA float64 field, f[k] = f(k dt), k = 0..nsteps."""
        ff = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1))
        if ff.size < int(nsteps) + 1:
            raise ValueError("f needs nsteps + 1 values")
        out = self.empty()
        self._check(self.lib.mol_solve_source(self.h, self._field(u0, "u0"), int(nsteps), self._field(g, "g"),
                                              ff.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                              self._field(out, "u_out"), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def autotune(self, stream=None) -> dict:
        """Time the launch variants on this grid and keep the fastest."""
        self._check(self.lib.mol_autotune(self.h, ctypes.c_void_p(_stream_ptr(stream))))
        return self.tuning()

    TUNING_KEYS = ("res_warps", "strided_rpt", "strided_warps", "rows_warps", "rows_persist", "strided_nb",
                   "strided_stage", "rows_nb", "pdl")

    def set_tuning(self, res_warps: int = 2, strided_rpt: int = 0, strided_warps: int = 8, rows_warps: int = 0,
                   rows_persist: int | None = None, strided_nb: int | None = None,
                   strided_stage: int | None = None, rows_nb: int | None = None, pdl: int | None = None):
        """Launch choices by hand (mol_set_tuning_ex); rows_persist,
        strided_nb, strided_stage, rows_nb and pdl None keep the handle's
        settings."""
        cur = self.tuning()
        vals = [int(res_warps), int(strided_rpt), int(strided_warps), int(rows_warps),
                int(cur["rows_persist"] if rows_persist is None else rows_persist),
                int(cur["strided_nb"] if strided_nb is None else strided_nb),
                int(cur["strided_stage"] if strided_stage is None else strided_stage),
                int(cur["rows_nb"] if rows_nb is None else rows_nb),
                int(cur["pdl"] if pdl is None else pdl)]
        arr = (ctypes.c_int * len(vals))(*vals)
        self._check(self.lib.mol_set_tuning_ex(self.h, arr, len(vals)))

    def tuning(self) -> dict:
        n = len(self.TUNING_KEYS)
        out = (ctypes.c_int * n)()
        ms = ctypes.c_double()
        self._check(self.lib.mol_get_tuning_ex(self.h, out, n, ctypes.byref(ms)))
        d = {k: out[i] for i, k in enumerate(self.TUNING_KEYS)}
        d["ms_per_step"] = ms.value
        return d

    def sync(self, stream=None):
        self._check(self.lib.mol_sync(self.h, ctypes.c_void_p(_stream_ptr(stream))))

    def norm(self, u, stream=None) -> float:
        """Discrete L2 norm of a field of this grid (synchronous)."""
        out = ctypes.c_double()
        self._check(self.lib.mol_field_norm(self.h, self._field(u, "u"), ctypes.byref(out),
                                            ctypes.c_void_p(_stream_ptr(stream))))
        return out.value

    def step_checked(self, u_prev, u_cur, nsteps: int, growth_limit: float = 1e3, stream=None):
        """step() that raises MolError(MOL_EUNSTABLE) if the field stops being
        finite or its norm grows by more than growth_limit times."""
        self._check(self.lib.mol_step_checked(self.h, self._field(u_prev, "u_prev"), self._field(u_cur, "u_cur"),
                                              int(nsteps), float(growth_limit), ctypes.c_void_p(_stream_ptr(stream))))

    def checkpoint_write(self, path, u_prev, u_cur, step: int, stream=None):
        """Save (u^{n-1}, u^n, n) with a header naming this problem."""
        self._check(self.lib.mol_checkpoint_write(self.h, str(path).encode(), self._field(u_prev, "u_prev"),
                                                  self._field(u_cur, "u_cur"), int(step),
                                                  ctypes.c_void_p(_stream_ptr(stream))))

    def checkpoint_read(self, path, u_prev, u_cur, stream=None) -> int:
        """Restore the levels from a checkpoint of this problem; returns n."""
        step = ctypes.c_int64()
        self._check(self.lib.mol_checkpoint_read(self.h, str(path).encode(), self._field(u_prev, "u_prev"),
                                                 self._field(u_cur, "u_cur"), ctypes.byref(step),
                                                 ctypes.c_void_p(_stream_ptr(stream))))
        return step.value

    def set_pass_timing(self, enable: bool = True):
        self._check(self.lib.mol_set_pass_timing(self.h, 1 if enable else 0))

    def pass_times(self):
        """{axis: (total_ms, launches)} of the passes timed since enabling."""
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        self._check(self.lib.mol_pass_times(self.h, ms, cnt))
        return {a: (ms[a], int(cnt[a])) for a in range(3) if cnt[a] > 0}

    @property
    def launches(self) -> int:
        return int(self.lib.mol_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mol_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class BatchSolver:
    """Many independent 2D Dirichlet problems stepped together (one launch
    per pass for all of them).

    ``shapes``: one (ny, nx) per problem; ``dt``, ``P``, ``c``, ``beta``: one
    value per problem or a scalar for all; ``lo`` / ``hi``: per-problem
    (y, x) pairs or None for the unit square.  Fields are PACKED: one flat
    CUDA float64 tensor holding every problem's (ny, nx) array in turn;
    ``pack`` / ``unpack`` convert.  ``chains``: in the graph time loop,
    run the launches of each size class as an independent chain where the
    classes' y and x launches cover the same problems (False: join every
    pass of all problems at every step)."""

    def __init__(self, shapes, dt, P, c=1.0, beta=0.0, prec: str = "mixed", lo=None, hi=None,
                 quad_order: int = 2, use_graphs: bool = True, chains: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmolt needs a CUDA GPU")
        self.lib = load_library()
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        n = len(self.shapes)

        def per(v, cast):
            arr = np.broadcast_to(np.asarray(v), (n,)) if np.ndim(v) == 0 else np.asarray(v)
            if len(arr) != n:
                raise ValueError("per-problem arrays need one entry per shape")
            return [cast(x) for x in arr]

        grids = (mol_grid * n)()
        for i, shp in enumerate(self.shapes):
            if len(shp) != 2:
                raise ValueError("batched problems are 2D")
            grids[i] = make_grid(shp, None if lo is None else lo[i], None if hi is None else hi[i])
        self.dt, self.P, self.c = per(dt, float), per(P, int), per(c, float)
        betas = per(beta, float)
        dts = (ctypes.c_double * n)(*self.dt)
        cs = (ctypes.c_double * n)(*self.c)
        bs = (ctypes.c_double * n)(*betas)
        Ps = (ctypes.c_int * n)(*self.P)
        opt = mol_options(int(quad_order), 0, (1 if chains else 2) if use_graphs else 0)
        h = ctypes.c_void_p()
        torch.cuda.init()
        st = self.lib.mol_batch_create(n, grids, cs, dts, bs, Ps, BC["dirichlet"], PREC[prec], ctypes.byref(opt),
                                       ctypes.byref(h))
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_last_error(None).decode())
        self.h = h
        self.prec = prec
        offs = (ctypes.c_int64 * (n + 1))()
        self._check(self.lib.mol_batch_offsets(self.h, offs))
        self.offsets = [int(v) for v in offs]
        self.size = self.offsets[-1]

    def _check(self, st: int):
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_batch_last_error(self.h).decode())

    def _flat(self, t, name):
        import torch
        if (not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda or t.dim() != 1
                or t.numel() != self.size or not t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor of {self.size} elements")
        return ctypes.c_void_p(t.data_ptr())

    def empty(self):
        import torch
        return torch.empty(self.size, dtype=torch.float64, device="cuda")

    def pack(self, fields):
        """Packed device tensor from one (ny, nx) array per problem."""
        import torch
        parts = [torch.as_tensor(np.ascontiguousarray(f) if isinstance(f, np.ndarray) else f,
                                 dtype=torch.float64).reshape(-1) for f in fields]
        return torch.cat([p.cpu() for p in parts]).cuda()

    def unpack(self, flat):
        """Per-problem (ny, nx) views of a packed tensor."""
        return [flat[self.offsets[i]:self.offsets[i + 1]].view(*self.shapes[i]) for i in range(len(self.shapes))]

    def apply_F(self, u, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_batch_apply_F(self.h, self._flat(u, "u"), self._flat(out, "F"),
                                               ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def start(self, u0, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_batch_start(self.h, self._flat(u0, "u0"), self._flat(out, "u1"),
                                             ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def step(self, u_prev, u_cur, nsteps: int, stream=None):
        self._check(self.lib.mol_batch_step(self.h, self._flat(u_prev, "u_prev"), self._flat(u_cur, "u_cur"),
                                            int(nsteps), ctypes.c_void_p(_stream_ptr(stream))))
        return u_prev, u_cur

    def apply_FT(self, w, out=None, stream=None):
        """F^T w for every problem (packed)."""
        out = self.empty() if out is None else out
        self._check(self.lib.mol_batch_apply_FT(self.h, self._flat(w, "w"), self._flat(out, "out"),
                                                ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def update(self, u, up, ea: float, eb: float, ec: float, transpose: bool = False, add=None, out=None,
               stream=None):
        """ea u + eb up + ec Op(u) + add with Op = F or F^T (packed fields)."""
        out = self.empty() if out is None else out
        upp = self._flat(up, "up") if eb != 0.0 else None
        addp = self._flat(add, "add") if add is not None else None
        self._check(self.lib.mol_batch_update(self.h, self._flat(u, "u"), upp, self._flat(out, "out"), float(ea),
                                              float(eb), float(ec), 1 if transpose else 0, addp,
                                              ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def _rec(self, rec):
        rec = np.ascontiguousarray(np.asarray(rec, dtype=np.int64).reshape(-1))
        return rec, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))

    def traces(self, u0, rec, nsteps: int, stream=None):
        """(nsteps, nrec) CUDA float64: u^n at the packed indices rec, n = 1..nsteps."""
        import torch
        rec, rp = self._rec(rec)
        out = torch.empty((int(nsteps), rec.size), dtype=torch.float64, device="cuda")
        self._check(self.lib.mol_batch_traces(self.h, self._flat(u0, "u0"), rec.size, rp, int(nsteps),
                                              ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def adjoint(self, rec, tgrad, stream=None):
        """dJ/du^0 (packed) from tgrad[n-1, r] = dJ/d(u^n at rec[r])."""
        import torch
        rec, rp = self._rec(rec)
        tg = tgrad.to(dtype=torch.float64, device="cuda").contiguous()
        if tg.dim() != 2 or tg.shape[1] != rec.size:
            raise ValueError("tgrad must be (nsteps, nrec)")
        out = self.empty()
        self._check(self.lib.mol_batch_adjoint(self.h, rec.size, rp, int(tg.shape[0]), ctypes.c_void_p(tg.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def solve_host(self, u0: np.ndarray, nsteps: int, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        """Packed host u0 -> packed host u^{nsteps} (zero initial velocity)."""
        u0 = np.ascontiguousarray(u0, dtype=np.float64).reshape(-1)
        if u0.size != self.size:
            raise ValueError(f"u0 must hold {self.size} values")
        out = np.empty_like(u0) if out is None else out
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.mol_batch_solve_host(self.h, u0.ctypes.data_as(dp), out.ctypes.data_as(dp), int(nsteps),
                                                  ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def autotune(self, stream=None) -> dict:
        """Time the launch variants on this batch and keep the fastest."""
        self._check(self.lib.mol_batch_autotune(self.h, ctypes.c_void_p(_stream_ptr(stream))))
        return self.tuning()

    def set_tuning(self, x_warps=(8, 8), y_rule: int = 0):
        """Launch variants by hand: x_warps = (short rows, long rows; 0 = long
        rows split over two warps of one CTA), y_rule 0..3 (bit 0: doubled
        y segments; bit 1: full carries even where the y pass's neighbour
        exchange is exact)."""
        self._check(self.lib.mol_batch_set_tuning(self.h, int(x_warps[0]), int(x_warps[1]), int(y_rule)))

    def tuning(self) -> dict:
        out = (ctypes.c_int * 3)()
        ms = (ctypes.c_double * 2)()
        self._check(self.lib.mol_batch_get_tuning(self.h, out, ms))
        return {"x_warps": [out[0], out[1]], "y_rule": out[2], "x_ms": ms[0], "y_ms": ms[1]}

    def sync(self, stream=None):
        self._check(self.lib.mol_batch_sync(self.h, ctypes.c_void_p(_stream_ptr(stream))))

    def set_pass_timing(self, enable: bool = True):
        self._check(self.lib.mol_batch_set_pass_timing(self.h, 1 if enable else 0))

    def pass_times(self):
        ms = (ctypes.c_double * 3)()
        cnt = (ctypes.c_int64 * 3)()
        self._check(self.lib.mol_batch_pass_times(self.h, ms, cnt))
        return {a: (ms[a], int(cnt[a])) for a in range(3) if cnt[a] > 0}

    @property
    def launches(self) -> int:
        return int(self.lib.mol_batch_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mol_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class EmbedSolver:
    """The 2D scheme on a domain embedded in a grid (Sec. 4.3).

    ``geom`` describes the line objects: any object with the attributes nx,
    ny, hx, hy, r0, r1, ra, rb (rows: first / last interior x index, gaps
    before / after them) and c0, c1, ca, cb (columns), as
    ``workloads.EmbeddedGrid`` has.  Fields are contiguous CUDA float64
    tensors of shape (ny, nx) that vanish outside the domain.  ``prec`` is
    "fp64" (float64 sweeps) or "mixed" (float32 sweeps of the difference
    form of D, time levels kept as float32 pairs inside the library)."""

    def __init__(self, geom, dt: float, P: int, c: float = 1.0, beta: float = 0.0, prec: str = "fp64"):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("libmolt needs a CUDA GPU")
        self.lib = load_library()
        self.shape = (int(geom.ny), int(geom.nx))
        i64 = lambda a: np.ascontiguousarray(a, dtype=np.int64)
        f64 = lambda a: np.ascontiguousarray(a, dtype=np.float64)
        arrs = [i64(geom.r0), i64(geom.r1), f64(geom.ra), f64(geom.rb),
                i64(geom.c0), i64(geom.c1), f64(geom.ca), f64(geom.cb)]
        g = mol_embed_geom(int(geom.nx), int(geom.ny), float(geom.hx), float(geom.hy),
                           *[a.ctypes.data for a in arrs])
        h = ctypes.c_void_p()
        torch.cuda.init()
        st = self.lib.mol_embed_create(ctypes.byref(g), float(c), float(dt), float(beta), int(P), PREC[prec],
                                       ctypes.byref(h))
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_last_error(None).decode())
        self.h = h
        self.P, self.dt, self.c, self.prec = int(P), float(dt), float(c), prec

    def _check(self, st: int):
        if st != MOL_OK:
            raise MolError(st, self.lib.mol_embed_last_error(self.h).decode())

    def _field(self, t, name):
        import torch
        if (not isinstance(t, torch.Tensor) or t.dtype != torch.float64 or not t.is_cuda
                or tuple(t.shape) != self.shape or not t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous CUDA float64 tensor of shape {self.shape}")
        return ctypes.c_void_p(t.data_ptr())

    def empty(self):
        import torch
        return torch.empty(self.shape, dtype=torch.float64, device="cuda")

    def linv(self, v, axis: int, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_embed_linv(self.h, self._field(v, "v"), self._field(out, "w"), int(axis),
                                            ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def apply_F(self, u, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_embed_apply_F(self.h, self._field(u, "u"), self._field(out, "F"),
                                               ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def start(self, u0, out=None, stream=None):
        out = self.empty() if out is None else out
        self._check(self.lib.mol_embed_start(self.h, self._field(u0, "u0"), self._field(out, "u1"),
                                             ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def step(self, u_prev, u_cur, nsteps: int, stream=None):
        self._check(self.lib.mol_embed_step(self.h, self._field(u_prev, "u_prev"), self._field(u_cur, "u_cur"),
                                            int(nsteps), ctypes.c_void_p(_stream_ptr(stream))))

    def solve_host(self, u0: np.ndarray, nsteps: int, out: np.ndarray | None = None, stream=None) -> np.ndarray:
        u0 = np.ascontiguousarray(u0, dtype=np.float64)
        if u0.shape != self.shape:
            raise ValueError(f"u0 must have shape {self.shape}")
        out = np.empty_like(u0) if out is None else out
        dp = ctypes.POINTER(ctypes.c_double)
        self._check(self.lib.mol_embed_solve_host(self.h, u0.ctypes.data_as(dp), out.ctypes.data_as(dp),
                                                  int(nsteps), ctypes.c_void_p(_stream_ptr(stream))))
        return out

    def sync(self, stream=None):
        self._check(self.lib.mol_embed_sync(self.h, ctypes.c_void_p(_stream_ptr(stream))))

    def set_pass_timing(self, enable: bool = True):
        self._check(self.lib.mol_embed_set_pass_timing(self.h, 1 if enable else 0))

    def pass_times(self):
        """{kind: (total ms, launches)} since the last call: x_sweep, y_sweep,
        combine."""
        ms = (ctypes.c_double * 3)()
        n = (ctypes.c_int64 * 3)()
        self._check(self.lib.mol_embed_pass_times(self.h, ms, n))
        names = ("x_sweep", "y_sweep", "combine")
        return {names[k]: (float(ms[k]), int(n[k])) for k in range(3)}

    @property
    def launches(self) -> int:
        return int(self.lib.mol_embed_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.mol_embed_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _traces_function():
    import torch

    class ReceiverTraces(torch.autograd.Function):
        """traces = T(u0): the receiver values u^n[rec], n = 1..nsteps, of the
        forward run from u0 (zero initial velocity).  T is linear, so the
        backward pass is the adjoint run on the trace gradients alone."""

        @staticmethod
        def forward(ctx, u0, solver, rec, nsteps):
            ctx.solver, ctx.rec = solver, np.asarray(rec, dtype=np.int64)
            return solver.traces(u0.detach().contiguous(), ctx.rec, int(nsteps))

        @staticmethod
        def backward(ctx, grad_traces):
            return ctx.solver.adjoint(ctx.rec, grad_traces), None, None, None

    return ReceiverTraces


_RT = None


def receiver_traces(u0, solver: "BatchSolver", rec, nsteps: int):
    """Differentiable receiver traces: a (nsteps, nrec) tensor whose gradient
    with respect to the packed initial field u0 runs the adjoint kernels."""
    global _RT
    if _RT is None:
        _RT = _traces_function()
    return _RT.apply(u0, solver, rec, nsteps)


GRAD_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                           ctypes.c_void_p)


class _DeviceView:
    """A float64 device buffer of the library, seen by torch without a copy."""

    def __init__(self, ptr: int, shape):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": "<f8", "data": (int(ptr), False),
                                         "version": 2, "strides": None}


def history_gradient(solver, u0, nsteps: int, grad_fn, checkpoint_every: int = 40, stream=None):
    """dJ/du^0 for J = sum_{n=0}^{nsteps} phi_n(u^n) over the forward run from
    u0 (zero initial velocity), given grad_fn(n, u_n) -> dphi_n/du^n (a tensor
    of u0's shape, or None where phi_n is absent).

    Runs mol_adjoint_history (Solver) or mol_batch_adjoint_history
    (BatchSolver, packed fields): the forward pass keeps (u^{c-1}, u^c) every
    K = checkpoint_every steps on the device, the backward pass recomputes one
    segment of at most K states at a time and runs the adjoint recursion
    mu^n = 2 mu^{n+1} - mu^{n+2} + F^T mu^{n+1} + g^n through it.  grad_fn is
    called for n = nsteps .. 0; u_n is the library's buffer (do not write it)."""
    import torch
    lib = load_library()
    if not isinstance(u0, torch.Tensor) or u0.dtype != torch.float64 or not u0.is_cuda or not u0.is_contiguous():
        raise TypeError("u0 must be a contiguous CUDA float64 tensor")
    shape = tuple(u0.shape)
    errors = []

    def cb(n, u_ptr, g_ptr, _stream, _user):
        try:
            u = torch.as_tensor(_DeviceView(u_ptr, shape), device=u0.device)
            g = grad_fn(int(n), u)
            if g is None:
                return 1
            torch.as_tensor(_DeviceView(g_ptr, shape), device=u0.device).copy_(g.reshape(shape))
            return 0
        except Exception as e:                     # reported after the call returns
            errors.append(e)
            return 2

    c_cb = GRAD_FN(cb)
    grad = torch.empty_like(u0)
    sp = ctypes.c_void_p(_stream_ptr(stream))
    if isinstance(solver, BatchSolver):
        st = lib.mol_batch_adjoint_history(solver.h, ctypes.c_void_p(u0.data_ptr()), int(nsteps),
                                           int(checkpoint_every), c_cb, None, ctypes.c_void_p(grad.data_ptr()), sp)
    else:
        st = lib.mol_adjoint_history(solver.h, ctypes.c_void_p(u0.data_ptr()), int(nsteps), int(checkpoint_every),
                                     c_cb, None, ctypes.c_void_p(grad.data_ptr()), sp)
    if errors:
        raise errors[0]
    solver._check(st)
    return grad


def toeplitz_experiment(nrows: int = 2048, ncols: int = 2048, d: float = 0.5395, reps: int = 50, stream=None):
    """mol_toeplitz_experiment: (scan ms, tensor-core ms, max relative difference)."""
    lib = load_library()
    ms = (ctypes.c_double * 2)()
    diff = ctypes.c_double()
    st = lib.mol_toeplitz_experiment(int(nrows), int(ncols), float(d), int(reps), ms, ctypes.byref(diff),
                                     ctypes.c_void_p(_stream_ptr(stream)))
    if st != MOL_OK:
        raise MolError(st, lib.mol_last_error(None).decode())
    return ms[0], ms[1], diff.value
