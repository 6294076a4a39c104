"""The C-ABI library loads and exports every entry point include/tpcf.h declares;
argument validation that needs no GPU returns the documented statuses."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import _capi
    return _capi.lib()


def _declared():
    src = open(os.path.join(ROOT, "include", "tpcf.h")).read()
    return sorted(set(re.findall(r"\b(tpcf_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_what_binding_lists():
    from paper_2408_16847_gb300 import _capi
    assert _declared() == sorted(_capi.EXPORTS)


def test_flag_constants_match_the_header():
    from paper_2408_16847_gb300 import _capi
    src = open(os.path.join(ROOT, "include", "tpcf.h")).read()
    flags = dict((k, int(v)) for k, v in re.findall(r"#define TPCF_([A-Z0-9_]+) (\d+)u", src))
    for name in ("SELF_PAIRS_SUBTRACT", "CONTRACT_TC", "NORM_BIN_MEAN", "NORM_PIVOT_TOTAL"):
        assert getattr(_capi, name) == flags[name], name


def test_every_declared_symbol_is_exported(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_2408_16847_gb300 import _capi
    for code, name in _capi.STATUS.items():
        assert lib.tpcf_status_string(code).decode() == name


def test_invalid_arguments_need_no_gpu(lib):
    from paper_2408_16847_gb300 import _capi
    import numpy as np
    e = np.array([0.01, 0.02, 0.03])
    b = _capi.Bins(2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4, 0)
    h = ctypes.c_void_p()
    # NULL out pointer, bad nside, bad bins: rejected before any CUDA call
    assert lib.tpcf_plan_create_map(None, 8, ctypes.byref(b), None) == 1
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 0, ctypes.byref(b), None) == 1
    bad = np.array([0.02, 0.01, 0.03])
    b2 = _capi.Bins(2, bad.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4, 0)
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 8, ctypes.byref(b2), None) == 1
    b3 = _capi.Bins(2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 17, 0)
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 8, ctypes.byref(b3), None) == 1
    b4 = _capi.Bins(2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4, 1 << 7)
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 8, ctypes.byref(b4), None) == 1
    assert lib.tpcf_forward(None, None, None, 0, 0, None, None, None, None) == 1
    assert lib.tpcf_backward(None, None, None, 0, 0, None, None, None, None) == 1
    assert lib.tpcf_plan_npoints(None) == -1
    lib.tpcf_plan_destroy(None)
    assert lib.tpcf_batch_create(None, None, 1, None, None, None, None, None, None, None) == 1
    hb = ctypes.c_void_p()
    assert lib.tpcf_batch_create(ctypes.byref(hb), None, 0, None, None, None, None, None, None, None) == 1
    assert lib.tpcf_batch_launch(None, None) == 1
    assert lib.tpcf_batch_kernel_launches(None) == -1
    lib.tpcf_batch_destroy(None)
    # both per-pivot normalisations at once; a normalisation with self-pair subtraction
    b5 = _capi.Bins(2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4,
                    _capi.NORM_BIN_MEAN | _capi.NORM_PIVOT_TOTAL)
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 8, ctypes.byref(b5), None) == 1
    b6 = _capi.Bins(2, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), 4,
                    _capi.NORM_BIN_MEAN | _capi.SELF_PAIRS_SUBTRACT)
    assert lib.tpcf_plan_create_map(ctypes.byref(h), 8, ctypes.byref(b6), None) == 5
    one = ctypes.c_void_p(16)  # never dereferenced: validation fails first
    assert lib.tpcf_edge_correct(None, one, 1.0, 2, 2, one, None) == 1
    assert lib.tpcf_edge_correct(one, one, 1.0, 2, 17, one, None) == 1
    assert lib.tpcf_edge_correct(one, one, 0.0, 2, 2, one, None) == 1
    assert lib.tpcf_edge_correct(one, one, 1.0, 33, 2, one, None) == 1
    assert lib.tpcf_forward_grouped(None, one, one, 3, 0, 1, one, one, None, None) == 1
    assert h.value is None
