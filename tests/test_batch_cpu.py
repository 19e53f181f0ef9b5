"""Host-side checks of mol_batch_create: every argument error is reported
before any device work, so these run without a GPU."""
import ctypes

import pytest

from paper_1308_3214_gb300 import molt


def create(shapes, P=2, dt=0.01, beta=None, bc="dirichlet", prec="mixed", quad=2, nprob=None):
    lib = molt.load_library()
    n = len(shapes)
    grids = (molt.mol_grid * max(n, 1))()
    for i, s in enumerate(shapes):
        grids[i] = molt.make_grid(s)
    c = (ctypes.c_double * max(n, 1))(*([1.0] * n))
    dts = (ctypes.c_double * max(n, 1))(*([dt] * n))
    Ps = (ctypes.c_int * max(n, 1))(*([P] * n))
    bs = None if beta is None else (ctypes.c_double * n)(*([beta] * n))
    opt = molt.mol_options(quad, 0, 1)
    h = ctypes.c_void_p()
    st = lib.mol_batch_create(n if nprob is None else nprob, grids, c, dts, bs, Ps, molt.BC[bc], molt.PREC[prec],
                              ctypes.byref(opt), ctypes.byref(h))
    return st, lib.mol_last_error(None).decode()


@pytest.mark.parametrize("kw,status,text", [
    (dict(bc="periodic"), molt.MOL_EINVAL, "Dirichlet"),
    (dict(shapes=[(64, 64, 64)]), molt.MOL_EINVAL, "2D"),
    (dict(shapes=[(64,)]), molt.MOL_EINVAL, "2D"),
    (dict(shapes=[(64, 1025)]), molt.MOL_EINVAL, "1024"),
    (dict(shapes=[(2, 64)]), molt.MOL_EINVAL, "3 <= n"),
    (dict(P=0), molt.MOL_EINVAL, "P must"),
    (dict(P=6), molt.MOL_EINVAL, "P must"),
    (dict(dt=0.0), molt.MOL_EINVAL, "positive"),
    (dict(beta=3.0), molt.MOL_EUNSTABLE, "beta_max"),
    (dict(quad=3), molt.MOL_EINVAL, "quad_order"),
    (dict(nprob=0), molt.MOL_EINVAL, "nprob"),
])
def test_batch_create_rejects(kw, status, text):
    args = dict(shapes=[(64, 64), (100, 37)])
    args.update(kw)
    st, msg = create(**args)
    assert st == status
    assert text in msg


def test_batch_error_names_the_problem():
    st, msg = create([(64, 64), (64, 2000), (50, 50)])
    assert st == molt.MOL_EINVAL and msg.startswith("problem 1:")
