"""The C-ABI library builds, loads and exports every entry point include/enkf.h declares;
host-side argument checking works without a GPU (no compute call is made here)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2606_19224_gb300 as enkf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(enkf_\w+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    lib = enkf.load()
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in sorted(declared) if not hasattr(lib, n)]
    assert not missing, missing
    assert declared <= set(enkf.EXPORTS) | declared


def test_binding_lists_every_declared_symbol():
    assert _declared() == set(enkf.EXPORTS)


def test_config_default_and_layout():
    cfg = enkf.default_config(100, 50, 20)
    assert (cfg.n, cfg.m, cfg.N) == (100, 50, 20)
    assert cfg.precision == enkf.FP64 and cfg.tol == 1e-8 and cfg.max_iter == 1000
    assert ctypes.sizeof(enkf.Config) == 104
    assert enkf.load().enkf_config_default(None, 1, 1, 2) == 1


def _create(cfg, rowptr, col, w, r):
    h = ctypes.c_void_p()
    lib = enkf.load()
    st = lib.enkf_create(ctypes.byref(cfg), rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                         r.ctypes.data, None, ctypes.byref(h))
    return st, h, lib.enkf_last_error(None).decode()


@pytest.mark.parametrize("case", ["N1", "bad_col", "neg_r", "rowptr", "N_big", "tol", "reserved",
                                  "variant", "senkf_bf16", "senkf_warm", "warm_accept", "reduce_order"])
def test_create_rejects_bad_arguments_before_touching_the_gpu(case):
    n, m, N = 10, 4, 5
    rowptr = np.arange(m + 1, dtype=np.int32)
    col = np.arange(m, dtype=np.int32)
    w = np.ones(m)
    r = np.ones(m)
    cfg = enkf.default_config(n, m, N)
    expect = 1
    if case == "N1":
        cfg.N = 1
    elif case == "bad_col":
        col[2] = n
    elif case == "neg_r":
        r[1] = -1.0
    elif case == "rowptr":
        rowptr[2] = 5
        rowptr[3] = 1
    elif case == "N_big":
        cfg.N = 129
        expect = 8
    elif case == "tol":
        cfg.tol = 0.0
    elif case == "reserved":
        cfg.reserved[1] = 1
    elif case == "warm_accept":
        cfg.warm_accept = 2
    elif case == "reduce_order":
        cfg.reduce_order = 2
    elif case == "variant":
        cfg.variant = 3
        expect = 8
    elif case == "senkf_bf16":   # the sEnKF comparator is built for FP64 and FP32 only
        cfg.variant, cfg.precision = enkf.SENKF, enkf.BF16_REFINE
        expect = 8
    elif case == "senkf_warm":
        cfg.variant, cfg.precision, cfg.warm_start = enkf.SENKF, enkf.FP32, 1
        expect = 8
    st, h, msg = _create(cfg, rowptr, col, w, r)
    assert st == expect and not h.value and msg


def test_status_strings():
    lib = enkf.load()
    for s in range(9):
        assert lib.enkf_status_str(s)
    assert enkf.load().enkf_destroy(None) == 0


def test_selftest_rejects_bad_arguments_without_a_gpu():
    # argument checks come before any CUDA call
    lib = enkf.load()
    for which, ms in ((2, 50.0), (0, 0.0), (1, 2e4)):
        assert enkf.STATUS[lib.enkf_selftest_wait_timeout(which, ms, None)] == "invalid_arg"


@pytest.mark.parametrize("case", ["null_off", "indefinite", "plain_cg", "nonfinite"])
def test_create_tridiag_rejects_bad_arguments_before_touching_the_gpu(case):
    n, m, N = 10, 4, 5
    rowptr = np.arange(m + 1, dtype=np.int32)
    col = np.arange(m, dtype=np.int32)
    w = np.ones(m)
    r = np.ones(m)
    off = np.full(m - 1, 0.2)
    cfg = enkf.default_config(n, m, N, precondition=1)
    expect = 1
    if case == "null_off":
        off = None
    elif case == "indefinite":
        off[:] = 0.9          # eigenvalues 1 + 1.8 cos(k pi / 5): the smallest is negative
    elif case == "plain_cg":
        cfg.precondition = 0
        expect = 8
    elif case == "nonfinite":
        off[1] = np.nan
    h = ctypes.c_void_p()
    lib = enkf.load()
    st = lib.enkf_create_tridiag(ctypes.byref(cfg), rowptr.ctypes.data, col.ctypes.data, w.ctypes.data,
                                 r.ctypes.data, None if off is None else off.ctypes.data, None, ctypes.byref(h))
    assert st == expect and not h.value, (case, st, lib.enkf_last_error(None))
