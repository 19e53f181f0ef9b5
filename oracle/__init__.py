"""FP64 CPU oracle for the MOL^T recursive-convolution wave solver.

TEST INFRASTRUCTURE ONLY: the reference the CUDA library is checked against.
Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The library never calls it and it shares no
code with the library.

The arithmetic lives in ``molt_oracle.c`` (plain C, double precision, the
paper's operators in the paper's order); this module compiles it with gcc and
wraps it for numpy arrays.  Fields are numpy arrays in C order with shape
``(nz, ny, nx)`` (or ``(ny, nx)`` / ``(nx,)``), i.e. x varies fastest.

Parity status of each function (see the pins in ``tests/test_oracle_*.py``):
every function here is pinned; none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "molt_oracle.c"
_BUILD = _HERE / "_build"
_LIB = _BUILD / "libmolt_oracle.so"

PERIODIC = 0
DIRICHLET = 1

_lib = None


def build(force: bool = False) -> Path:
    """Compile the C oracle (gcc, OpenMP over lines) into ``oracle/_build``."""
    _BUILD.mkdir(exist_ok=True)
    if force or not _LIB.exists() or _LIB.stat().st_mtime < _SRC.stat().st_mtime:
        tmp = _LIB.with_suffix(f".{os.getpid()}.tmp")
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", str(tmp), str(_SRC), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(str(build()))
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        L, I, D = ctypes.c_long, ctypes.c_int, ctypes.c_double
        lib.orc_weights.argtypes = [D, I, dp]
        lib.orc_linv_line.argtypes = [dp, L, dp, L, L, D, I, I]
        lib.orc_linv_axis.argtypes = [dp, dp, I, lp, I, D, I, I]
        lib.orc_D_axis.argtypes = [dp, dp, I, lp, I, D, I, I]
        lib.orc_Ap.argtypes = [I, D, dp]
        lib.orc_beta_max.argtypes = [I]
        lib.orc_beta_max.restype = D
        lib.orc_F.argtypes = [dp, dp, I, lp, dp, I, I, I, D, lp]
        lib.orc_step.argtypes = [dp, dp, dp, I, lp, dp, I, I, I, D]
        lib.orc_start.argtypes = [dp, dp, I, lp, dp, I, I, I, D]
        lib.orc_run.argtypes = [dp, dp, L, I, lp, dp, I, I, I, D]
        lib.orc_linv_line_T.argtypes = [dp, L, dp, L, L, D, I, I]
        lib.orc_linv_axis_T.argtypes = [dp, dp, I, lp, I, D, I, I]
        lib.orc_D_axis_T.argtypes = [dp, dp, I, lp, I, D, I, I]
        lib.orc_FT.argtypes = [dp, dp, I, lp, dp, I, I, I, D]
        lib.orc_traces.argtypes = [dp, L, I, lp, dp, I, lp, dp, I, I, I, D]
        lib.orc_adjoint.argtypes = [dp, L, I, lp, dp, I, lp, dp, I, I, I, D]
        lib.orc_linv_line_bc.argtypes = [dp, dp, L, D, I, D, D]
        lib.orc_D_line_bc.argtypes = [dp, dp, L, D, I, D, D]
        lib.orc_F_bc.argtypes = [dp, dp, L, D, I, I, D, dp]
        lib.orc_run_bc.argtypes = [dp, dp, L, L, D, I, I, D, dp]
        lib.orc_bc_values.argtypes = [dp, I, dp]
        lib.orc_C.argtypes = [dp, dp, I, lp, dp, I, I]
        lib.orc_run_source.argtypes = [dp, dp, L, I, lp, dp, I, I, I, D, D, dp, dp]
        lib.orc_linv_obj.argtypes = [dp, L, dp, L, L, D, D, D, D]
        geo = [L, L, D, D, lp, lp, dp, dp, lp, lp, dp, dp]
        lib.orc_linv_axis_embed.argtypes = [dp, dp, I] + geo + [D]
        lib.orc_F_embed.argtypes = [dp, dp] + geo + [D, I, D]
        lib.orc_run_embed.argtypes = [dp, dp, L] + geo + [D, I, D]
        lib.orc_num_threads.restype = I
        lib.orc_set_threads.argtypes = [I]
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _shape(a: np.ndarray):
    shp = (ctypes.c_long * 3)(*([1, 1, 1]))
    for i, s in enumerate(reversed(a.shape)):
        shp[i] = s
    return a.ndim, shp


def _nu_arr(nu, ndim):
    nu = np.broadcast_to(np.asarray(nu, dtype=np.float64), (ndim,)).copy()
    return np.concatenate([nu, np.ones(3 - ndim)])


def _bc(bc) -> int:
    if isinstance(bc, str):
        return {"periodic": PERIODIC, "dirichlet": DIRICHLET}[bc]
    return int(bc)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops from now on (timing only)."""
    _load().orc_set_threads(int(n))


def weights(nu: float, quad: int = 2):
    """(d, W0, W1, R) of one increment, Sec. 2 (R = 0 for the linear rule)."""
    out = np.zeros(4)
    _load().orc_weights(float(nu), int(quad), _dp(out))
    return tuple(out)


def linv_line(v, nu: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """L^{-1} of eq. (L_Inverse) on one line, with the boundary correction."""
    v = _f64(v)
    w = np.empty_like(v)
    _load().orc_linv_line(_dp(v), 1, _dp(w), 1, v.size, float(nu), int(quad), _bc(bc))
    return w


def linv_axis(v, axis: int, nu: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """L_gamma^{-1} along ``axis`` (0 = x, the fastest index) of a field."""
    v = _f64(v)
    w = np.empty_like(v)
    nd, shp = _shape(v)
    _load().orc_linv_axis(_dp(v), _dp(w), nd, shp, int(axis), float(nu), int(quad), _bc(bc))
    return w


def D_axis(v, axis: int, nu: float, bc="dirichlet", quad: int = 2, power: int = 1) -> np.ndarray:
    """D_gamma^power v with D_gamma = 1 - L_gamma^{-1} (eq. LD_gam)."""
    out = _f64(v)
    nd, shp = _shape(out)
    for _ in range(power):
        src = out
        out = np.empty_like(src)
        _load().orc_D_axis(_dp(src), _dp(out), nd, shp, int(axis), float(nu), int(quad), _bc(bc))
    return out


def linv_line_T(w, nu: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """(L^{-1})^T on one line: the program of linv_line transposed."""
    w = _f64(w)
    v = np.empty_like(w)
    _load().orc_linv_line_T(_dp(w), 1, _dp(v), 1, w.size, float(nu), int(quad), _bc(bc))
    return v


def D_axis_T(v, axis: int, nu: float, bc="dirichlet", quad: int = 2, power: int = 1) -> np.ndarray:
    """(D_gamma^T)^power v, D_gamma^T = 1 - (L_gamma^{-1})^T."""
    out = _f64(v)
    nd, shp = _shape(out)
    for _ in range(power):
        src = out
        out = np.empty_like(src)
        _load().orc_D_axis_T(_dp(src), _dp(out), nd, shp, int(axis), float(nu), int(quad), _bc(bc))
    return out


def FT(u, nu, P: int, beta: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """F^T: the transpose of F (every per-axis operator transposed)."""
    u = _f64(u)
    out = np.empty_like(u)
    nd, shp = _shape(u)
    _load().orc_FT(_dp(u), _dp(out), nd, shp, _dp(_nu_arr(nu, nd)), int(quad), _bc(bc), int(P), float(beta))
    return out


def _rec_arr(rec, size):
    rec = np.ascontiguousarray(rec, dtype=np.int64).reshape(-1)
    if rec.size and (rec.min() < 0 or rec.max() >= size):
        raise ValueError("receiver index out of range")
    return rec


def traces(u0, nsteps: int, rec, nu, P: int, beta: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """t[n-1, r] = u^n at flat index rec[r] (C order), n = 1..nsteps, from
    u^1 = u^0 + F[u^0]/2 and the time steps."""
    u0 = _f64(u0)
    nd, shp = _shape(u0)
    rec = _rec_arr(rec, u0.size)
    out = np.zeros((int(nsteps), rec.size))
    _load().orc_traces(_dp(u0), int(nsteps), rec.size, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                       _dp(out), nd, shp, _dp(_nu_arr(nu, nd)), int(quad), _bc(bc), int(P), float(beta))
    return out


def adjoint(tgrad, shape, rec, nu, P: int, beta: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """dJ/du^0 for a loss J of the traces, given tgrad[n-1, r] = dJ/dt^n_r."""
    tgrad = _f64(np.asarray(tgrad, dtype=np.float64))
    nsteps = tgrad.shape[0]
    grad = np.zeros(tuple(shape))
    nd, shp = _shape(grad)
    rec = _rec_arr(rec, grad.size)
    _load().orc_adjoint(_dp(tgrad), int(nsteps), rec.size, rec.ctypes.data_as(ctypes.POINTER(ctypes.c_long)),
                        _dp(grad), nd, shp, _dp(_nu_arr(nu, nd)), int(quad), _bc(bc), int(P), float(beta))
    return grad


def Ap(P: int, beta: float) -> np.ndarray:
    """A_p(beta), p = 1..P, of eq. (update_P)."""
    out = np.zeros(P)
    _load().orc_Ap(int(P), float(beta), _dp(out))
    return out


def beta_max(P: int) -> float:
    """First positive root of -sum_p A_p(beta) = 4 (eq. Stab_cond, Table 1)."""
    return _load().orc_beta_max(int(P))


def F(u, nu, P: int, beta: float, bc="dirichlet", quad: int = 2, return_nops: bool = False):
    """F[u] = sum_p sum_m c_pm C^m D^{p-m} u (eq. Full_2D; eq. update_P in 1D).

    ``nu`` is alpha*h per axis (scalar or one value per axis, x first)."""
    u = _f64(u)
    out = np.empty_like(u)
    nd, shp = _shape(u)
    nus = _nu_arr(nu, nd)
    nops = ctypes.c_long(0)
    _load().orc_F(_dp(u), _dp(out), nd, shp, _dp(nus), int(quad), _bc(bc), int(P),
                  float(beta), ctypes.byref(nops))
    return (out, nops.value) if return_nops else out


def step(uprev, ucur, nu, P: int, beta: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """u^{n+1} = 2u^n - u^{n-1} + F[u^n]."""
    uprev, ucur = _f64(uprev), _f64(ucur)
    out = np.empty_like(ucur)
    nd, shp = _shape(ucur)
    nus = _nu_arr(nu, nd)
    _load().orc_step(_dp(uprev), _dp(ucur), _dp(out), nd, shp, _dp(nus), int(quad), _bc(bc),
                     int(P), float(beta))
    return out


def start(u0, nu, P: int, beta: float, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """u^1 = u^0 + F[u^0]/2 (zero initial velocity, Sec. 3.2)."""
    u0 = _f64(u0)
    out = np.empty_like(u0)
    nd, shp = _shape(u0)
    nus = _nu_arr(nu, nd)
    _load().orc_start(_dp(u0), _dp(out), nd, shp, _dp(nus), int(quad), _bc(bc), int(P), float(beta))
    return out


def run(uprev, ucur, nsteps: int, nu, P: int, beta: float, bc="dirichlet", quad: int = 2):
    """Advance (u^{n-1}, u^n) by ``nsteps`` steps; returns new copies."""
    up, uc = _f64(uprev).copy(), _f64(ucur).copy()
    nd, shp = _shape(uc)
    nus = _nu_arr(nu, nd)
    _load().orc_run(_dp(up), _dp(uc), int(nsteps), nd, shp, _dp(nus), int(quad), _bc(bc),
                    int(P), float(beta))
    return up, uc


def C(v, nu, bc="dirichlet", quad: int = 2) -> np.ndarray:
    """C[v] (eq. C_def_ADI): sum_g (prod_{a != g} L_a^{-1}) D_g v."""
    v = _f64(v)
    out = np.empty_like(v)
    nd, shp = _shape(v)
    _load().orc_C(_dp(v), _dp(out), nd, shp, _dp(_nu_arr(nu, nd)), int(quad), _bc(bc))
    return out


def run_source(u0, nsteps: int, nu, P: int, beta: float, sc: float, g, f, bc="dirichlet",
               quad: int = 2) -> np.ndarray:
    """u^nsteps with the source S = g(x) f(t) (Sec. 4.1; P = 1 or 2), zero
    initial velocity; sc = (c dt)^2, f[k] = f(t_k), k = 0..nsteps."""
    u0, g = _f64(u0), _f64(g)
    ff = _f64(np.asarray(f, dtype=np.float64).reshape(-1))
    if ff.size < int(nsteps) + 1:
        raise ValueError("f needs nsteps + 1 values")
    out = np.empty_like(u0)
    nd, shp = _shape(u0)
    st = _load().orc_run_source(_dp(u0), _dp(out), int(nsteps), nd, shp, _dp(_nu_arr(nu, nd)), int(quad), _bc(bc),
                                int(P), float(beta), float(sc), _dp(g), _dp(ff))
    if st != 0:
        raise ValueError("source terms are defined for P = 1 and 2")
    return out


# ---------------------------------------------------------------------------
# time-dependent Dirichlet data on a 1D line (Sec. 3.2)
# ---------------------------------------------------------------------------
def linv_line_bc(v, nu, gL: float, gR: float, quad: int = 2) -> np.ndarray:
    """L^{-1} v corrected so that D v = v - L^{-1} v takes the values gL, gR
    at the end nodes."""
    v = _f64(v)
    out = np.empty_like(v)
    _load().orc_linv_line_bc(_dp(v), _dp(out), v.size, float(nu), int(quad), float(gL), float(gR))
    return out


def D_line_bc(v, nu, gL: float, gR: float, quad: int = 2) -> np.ndarray:
    """D v with the end values gL, gR."""
    v = _f64(v)
    out = np.empty_like(v)
    _load().orc_D_line_bc(_dp(v), _dp(out), v.size, float(nu), int(quad), float(gL), float(gR))
    return out


def F_bc(u, nu, P: int, beta: float, g, quad: int = 2) -> np.ndarray:
    """F[u] = sum_p A_p D^p u on a 1D line, D^p u taking the end values
    g[p] = (at a, at b), p = 1..P (g has P + 1 rows; row 0 is not used)."""
    u = _f64(u)
    gg = _f64(np.asarray(g, dtype=np.float64).reshape(P + 1, 2))
    out = np.empty_like(u)
    _load().orc_F_bc(_dp(u), _dp(out), u.size, float(nu), int(quad), int(P), float(beta), _dp(gg))
    return out


def bc_values(s, P: int) -> np.ndarray:
    """Boundary values g[p, side] of D^p u, p = 0..P (row 0: the data itself),
    from s[side, j] = (d_tt / (c alpha)^2)^j u_side, j = 0..P."""
    ss = _f64(np.asarray(s, dtype=np.float64).reshape(2, P + 1))
    g = np.empty((P + 1, 2))
    _load().orc_bc_values(_dp(ss), int(P), _dp(g))
    return g


def run_bc(u0, nsteps: int, nu, P: int, beta: float, gam, quad: int = 2) -> np.ndarray:
    """u^nsteps of a 1D line with Dirichlet data: gam[k, side, j] =
    (d_tt / (c alpha)^2)^j u_side(t_k), k = 0..nsteps, j = 0..P."""
    u0 = _f64(u0)
    g = _f64(np.asarray(gam, dtype=np.float64).reshape(int(nsteps) + 1, 2, P + 1))
    out = np.empty_like(u0)
    _load().orc_run_bc(_dp(u0), _dp(out), int(nsteps), u0.size, float(nu), int(quad), int(P), float(beta), _dp(g))
    return out


def grid_spacing(n: int, length: float, bc) -> float:
    """Dirichlet axes include both end nodes; periodic axes hold n points."""
    return length / (n - 1) if _bc(bc) == DIRICHLET else length / n


# --------------------------------------------------------------------------
# Embedded boundaries (Sec. 4.3): line objects and the 2D scheme on a domain
# cut out of a grid.  ``g`` is a ``workloads.EmbeddedGrid``; fields have shape
# (ny, nx) and vanish outside the domain.
# --------------------------------------------------------------------------
def linv_obj(v, h: float, da: float, db: float, alpha: float) -> np.ndarray:
    """L^{-1} on one line object: m interior values at spacing h, boundary
    points (zero data) at distance da before the first and db after the last."""
    v = _f64(v)
    w = np.empty_like(v)
    _load().orc_linv_obj(_dp(v), 1, _dp(w), 1, v.size, h, da, db, alpha)
    return w


def _geo(g):
    li = lambda a: np.ascontiguousarray(a, dtype=np.int64)
    ld = lambda a: np.ascontiguousarray(a, dtype=np.float64)
    keep = [li(g.r0), li(g.r1), ld(g.ra), ld(g.rb), li(g.c0), li(g.c1), ld(g.ca), ld(g.cb)]
    lp = ctypes.POINTER(ctypes.c_long)
    ptr = [a.ctypes.data_as(lp) if a.dtype == np.int64 else _dp(a) for a in keep]
    return keep, [g.nx, g.ny, g.hx, g.hy] + ptr


def _embedded_field(u, g):
    u = _f64(u)
    if u.shape != (g.ny, g.nx):
        raise ValueError("field shape must be (ny, nx) of the grid")
    return np.ascontiguousarray(np.where(g.mask, u, 0.0))


def linv_axis_embed(v, axis: int, g, alpha: float) -> np.ndarray:
    v = _embedded_field(v, g)
    w = np.empty_like(v)
    keep, args = _geo(g)
    _load().orc_linv_axis_embed(_dp(v), _dp(w), axis, *args, alpha)
    return w


def D_axis_embed(v, axis: int, g, alpha: float) -> np.ndarray:
    v = _embedded_field(v, g)
    return v - linv_axis_embed(v, axis, g, alpha)


def F_embed(u, g, alpha: float, P: int, beta: float) -> np.ndarray:
    """F[u] of eq. (Full_2D) on the embedded domain (terms in Table 3 order)."""
    u = _embedded_field(u, g)
    F = np.empty_like(u)
    keep, args = _geo(g)
    _load().orc_F_embed(_dp(u), _dp(F), *args, alpha, P, beta)
    return F


def run_embed(u0, nsteps: int, g, alpha: float, P: int, beta: float) -> np.ndarray:
    """u^{nsteps} from u^0 with zero initial velocity (start u^1 = u^0 + F/2)."""
    u0 = _embedded_field(u0, g)
    out = np.empty_like(u0)
    keep, args = _geo(g)
    _load().orc_run_embed(_dp(u0), _dp(out), nsteps, *args, alpha, P, beta)
    return out
