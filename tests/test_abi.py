"""The C-ABI library loads on a CPU-only host, exports every entry point
declared in include/qpr.h, and rejects invalid input before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2003_04930_gb300 import qpr
from paper_2003_04930_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return qpr.load_library()


def declared_entry_points():
    names = []
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if h.endswith(".h"):
            src = open(os.path.join(ROOT, "include", h)).read()
            names += re.findall(r"QPR_API[^;(]*?\b(qpr_\w+)\s*\(", src)
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert len(names) >= 13
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(qpr.EXPORTED)


def test_status_strings(lib):
    assert lib.qpr_status_string(0) == b"QPR_OK"
    assert lib.qpr_status_string(2) == b"QPR_E_GRAPH"
    assert lib.qpr_status_string(99) == b"QPR_E_UNKNOWN"


def _create(lib, n, src, dst, w=None, alpha=0.85, omega=0.5, **optkw):
    opt = qpr.qpr_options()
    lib.qpr_default_options(ctypes.byref(opt))
    for k, v in optkw.items():
        setattr(opt, k, v)
    src = np.ascontiguousarray(src, dtype=np.int64)
    dst = np.ascontiguousarray(dst, dtype=np.int64)
    wp = None if w is None else np.ascontiguousarray(w, dtype=np.float64)
    h = ctypes.c_void_p()
    st = lib.qpr_create(ctypes.byref(h), n, src.shape[0], qpr._ptr(src), qpr._ptr(dst), qpr._ptr(wp),
                        alpha, omega, ctypes.byref(opt))
    return st, h


@pytest.mark.parametrize("case,expect", [
    (dict(n=1, src=[], dst=[]), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], alpha=1.5), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], alpha=float("nan")), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], omega=-0.1), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], h_diag=7), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], dangling=5), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], precision=9), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], sparse_form=6), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], sparse_form=4), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], test_fault=2), qpr.QPR_E_ARG),
    (dict(n=3, src=[0], dst=[1], row_splits=65), qpr.QPR_E_ARG),
    (dict(n=3, src=[0, 3], dst=[1, 0]), qpr.QPR_E_GRAPH),
    (dict(n=3, src=[0, -1], dst=[1, 0]), qpr.QPR_E_GRAPH),
    (dict(n=3, src=[0, 1], dst=[1, 0], w=[1.0, -2.0]), qpr.QPR_E_GRAPH),
    (dict(n=3, src=[0, 1], dst=[1, 0], w=[1.0, np.inf]), qpr.QPR_E_GRAPH),
])
def test_invalid_input_rejected_before_cuda(lib, case, expect):
    st, h = _create(lib, **case)
    assert st == expect
    assert not h.value
    assert len(lib.qpr_last_error(None)) > 0


def test_null_out_rejected(lib):
    assert lib.qpr_create(None, 3, 0, None, None, None, 0.85, 0.5, None) == qpr.QPR_E_ARG


def test_null_context_calls(lib):
    assert lib.qpr_evolve(None, None, 0.01, 1) == qpr.QPR_E_ARG
    assert lib.qpr_profile_chain(None, None, 0.01, 1, None) == qpr.QPR_E_ARG
    assert lib.qpr_n(None) == 0
    lib.qpr_destroy(None)


def test_batch_rejects_invalid_problem_before_cuda(lib):
    src = np.array([0, 5], dtype=np.int64)
    dst = np.array([1, 0], dtype=np.int64)
    rho = np.eye(3, dtype=np.complex128) / 3
    arr = (qpr.qpr_problem * 1)()
    arr[0].n, arr[0].m = 3, 2
    arr[0].src, arr[0].dst, arr[0].w = qpr._ptr(src), qpr._ptr(dst), None
    arr[0].omega = 0.5
    arr[0].rho = qpr._ptr(rho)
    st = lib.qpr_batch_steady_state(1, arr, 0.85, 0.01, 1e-8, 10, None, None)
    assert st == qpr.QPR_E_GRAPH
    assert b"problem 0" in lib.qpr_last_error(None)
    assert lib.qpr_batch_steady_state(0, arr, 0.85, 0.01, 1e-8, 10, None, None) == qpr.QPR_E_ARG


def test_injected_allocation_failure_is_reported(lib, monkeypatch):
    # the library's host-side fault injection: qpr_create fails with QPR_E_OOM,
    # leaves no context behind and says why
    monkeypatch.setenv("QPR_FAULT", "oom")
    st, h = _create(lib, n=4, src=[0, 1, 2], dst=[1, 2, 3], device=0)
    assert st == qpr.QPR_E_OOM
    assert not h.value
    assert b"injected allocation failure" in lib.qpr_last_error(None)
