"""ctypes binding of libtpcf.so (argument marshalling only).

The names mirror include/tpcf.h.  Loading fails loudly if the library has not been
built: there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpcf.so")

TPCF_OK = 0
STATUS = {0: "TPCF_OK", 1: "TPCF_ERR_INVALID_ARG", 2: "TPCF_ERR_CUDA", 3: "TPCF_ERR_OOM",
          4: "TPCF_ERR_TIMEOUT", 5: "TPCF_ERR_UNSUPPORTED", 6: "TPCF_ERR_DEVICE"}
SELF_PAIRS_SUBTRACT = 1
CONTRACT_TC = 2
NORM_BIN_MEAN = 4
NORM_PIVOT_TOTAL = 8
MAX_BINS = 32
MAX_M = 16

# every exported entry point of include/tpcf.h
EXPORTS = ["tpcf_status_string", "tpcf_last_error", "tpcf_plan_create_map", "tpcf_plan_create_catalog",
           "tpcf_plan_npoints", "tpcf_plan_kernel_launches", "tpcf_forward", "tpcf_forward_noalloc", "tpcf_backward", "tpcf_count_pairs", "tpcf_run_host", "tpcf_batch_create",
           "tpcf_batch_launch", "tpcf_batch_kernel_launches", "tpcf_batch_destroy", "tpcf_forward_batched", "tpcf_plan_sync", "tpcf_normalize",
           "tpcf_plan_destroy", "tpcf_test_fail_allocation", "tpcf_test_live_allocations",
           "tpcf_plan_halo", "tpcf_plan_autotune", "tpcf_plan_launch_config", "tpcf_plan_set_launch_config",
           "tpcf_probe_fp32_peak", "tpcf_forward_multi", "tpcf_edge_correct", "tpcf_forward_grouped"]


class TpcfError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__("%s failed: %s%s" % (where, STATUS.get(status, status),
                                               (" (" + detail + ")") if detail else ""))


class Bins(ctypes.Structure):
    _fields_ = [("nbins", ctypes.c_int32), ("theta_edges_rad", ctypes.POINTER(ctypes.c_double)),
                ("m_max", ctypes.c_int32), ("flags", ctypes.c_uint32)]


_lib = None
_vp = ctypes.c_void_p
_i64 = ctypes.c_int64


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("libtpcf.so is not built (run paper_2408_16847_gb300.build.build() or "
                          "__graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    L.tpcf_status_string.restype = ctypes.c_char_p
    L.tpcf_status_string.argtypes = [ctypes.c_int]
    L.tpcf_last_error.restype = ctypes.c_char_p
    L.tpcf_last_error.argtypes = []
    L.tpcf_plan_create_map.restype = ctypes.c_int
    L.tpcf_plan_create_map.argtypes = [ctypes.POINTER(_vp), _i64, ctypes.POINTER(Bins), _vp]
    L.tpcf_plan_create_catalog.restype = ctypes.c_int
    L.tpcf_plan_create_catalog.argtypes = [ctypes.POINTER(_vp), _vp, _i64, ctypes.POINTER(Bins), _vp]
    L.tpcf_plan_npoints.restype = _i64
    L.tpcf_plan_npoints.argtypes = [_vp]
    L.tpcf_plan_kernel_launches.restype = _i64
    L.tpcf_plan_kernel_launches.argtypes = [_vp]
    L.tpcf_forward.restype = ctypes.c_int
    L.tpcf_forward.argtypes = [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]
    L.tpcf_forward_grouped.restype = ctypes.c_int
    L.tpcf_forward_grouped.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _i64, _i64, _vp, _vp, _vp, _vp]
    L.tpcf_forward_noalloc.restype = ctypes.c_int
    L.tpcf_forward_noalloc.argtypes = [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp]
    L.tpcf_backward.restype = ctypes.c_int
    L.tpcf_backward.argtypes = [_vp, _vp, _vp, _i64, _i64, _vp, _vp, _vp, _vp]
    L.tpcf_count_pairs.restype = ctypes.c_int
    L.tpcf_count_pairs.argtypes = [_vp, _vp, _i64, _i64, _vp, _vp]
    L.tpcf_run_host.restype = ctypes.c_int
    L.tpcf_run_host.argtypes = [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]
    L.tpcf_batch_create.restype = ctypes.c_int
    L.tpcf_batch_create.argtypes = [ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_int32,
                                    ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                    ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]
    L.tpcf_batch_launch.restype = ctypes.c_int
    L.tpcf_batch_launch.argtypes = [_vp, _vp]
    L.tpcf_batch_kernel_launches.restype = _i64
    L.tpcf_batch_kernel_launches.argtypes = [_vp]
    L.tpcf_batch_destroy.restype = None
    L.tpcf_batch_destroy.argtypes = [_vp]
    L.tpcf_forward_batched.restype = ctypes.c_int
    L.tpcf_forward_batched.argtypes = [ctypes.POINTER(_vp), ctypes.c_int32] + [ctypes.POINTER(_vp)] * 6 + [_vp]
    L.tpcf_normalize.restype = ctypes.c_int
    L.tpcf_normalize.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
    L.tpcf_edge_correct.restype = ctypes.c_int
    L.tpcf_edge_correct.argtypes = [_vp, _vp, ctypes.c_double, ctypes.c_int32, ctypes.c_int32, _vp, _vp]
    L.tpcf_plan_sync.restype = ctypes.c_int
    L.tpcf_plan_sync.argtypes = [_vp]
    L.tpcf_plan_destroy.restype = None
    L.tpcf_plan_destroy.argtypes = [_vp]
    L.tpcf_plan_autotune.restype = ctypes.c_int
    L.tpcf_plan_autotune.argtypes = [_vp, _vp, _vp, ctypes.c_int32, _vp]
    L.tpcf_plan_launch_config.restype = ctypes.c_int
    L.tpcf_plan_launch_config.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
    L.tpcf_plan_set_launch_config.restype = ctypes.c_int
    L.tpcf_plan_set_launch_config.argtypes = [_vp, ctypes.POINTER(ctypes.c_int32)]
    L.tpcf_forward_multi.restype = ctypes.c_int
    L.tpcf_forward_multi.argtypes = [_vp] + [_vp] * 6 + [_i64, _i64, _vp, _vp, _vp, _vp]
    L.tpcf_probe_fp32_peak.restype = ctypes.c_int
    L.tpcf_probe_fp32_peak.argtypes = [ctypes.POINTER(ctypes.c_double), _vp]
    L.tpcf_plan_halo.restype = ctypes.c_int
    L.tpcf_plan_halo.argtypes = [_vp, _i64, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]
    L.tpcf_test_fail_allocation.restype = None
    L.tpcf_test_fail_allocation.argtypes = [_i64]
    L.tpcf_test_live_allocations.restype = _i64
    L.tpcf_test_live_allocations.argtypes = []
    _lib = L
    return L


def check(status: int, where: str) -> None:
    if status != TPCF_OK:
        detail = lib().tpcf_last_error().decode(errors="replace")
        raise TpcfError(status, where, detail)
