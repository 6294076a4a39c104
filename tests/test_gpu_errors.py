"""Error paths of the C ABI on a GPU, made on the host: an injected device-allocation
failure (tpcf_test_fail_allocation) at every allocation of plan creation and of the
host-buffer call must return TPCF_ERR_OOM, leave nothing allocated and leave an
existing plan usable."""
import ctypes

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

OOM = 3  # TPCF_ERR_OOM


def _lib():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import _capi
    return _capi


def _bins(_capi, edges_deg, M):
    e = np.ascontiguousarray(np.deg2rad(edges_deg), dtype=np.float64)
    return _capi.Bins(len(e) - 1, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), M, 0), e


def test_injected_oom_map_plan_and_run_host(cuda_device):
    _capi = _lib()
    lib = _capi.lib()
    torch.cuda.synchronize()
    base = lib.tpcf_test_live_allocations()
    nside, M = 8, 4
    bins, _keep = _bins(_capi, [3.0, 7.0, 15.0], M)
    K = 2
    npix = 12 * nside * nside
    d = synth.bump_map(nside, 50, (3.0, 9.0), 0.5, 0.05, seed=synth.BASE_SEED + 61).astype(np.float32)
    w = np.ones(npix, np.float32)
    z_ok = None
    failed_create = failed_run = 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for n in range(1, 200):
        lib.tpcf_test_fail_allocation(n)
        h = ctypes.c_void_p()
        st = lib.tpcf_plan_create_map(ctypes.byref(h), nside, ctypes.byref(bins), stream)
        if st != 0:
            lib.tpcf_test_fail_allocation(0)
            assert st == OOM, _capi.STATUS.get(st, st)
            assert not h.value
            assert lib.tpcf_test_live_allocations() == base
            failed_create += 1
            continue
        z = np.zeros((M + 1, K, K, 2))
        nrm = np.zeros((K, K))
        st = lib.tpcf_run_host(h, d.ctypes.data, w.ctypes.data, None, z.ctypes.data, nrm.ctypes.data, None, stream)
        lib.tpcf_test_fail_allocation(0)
        if st != 0:
            assert st == OOM, _capi.STATUS.get(st, st)
            failed_run += 1
            # the plan is still usable after the failed call
            st2 = lib.tpcf_run_host(h, d.ctypes.data, w.ctypes.data, None, z.ctypes.data, nrm.ctypes.data, None,
                                    stream)
            assert st2 == 0
        if z_ok is None and st == 0:
            z_ok = z.copy()
        if z_ok is not None:
            np.testing.assert_array_equal(np.isfinite(z), True)
        lib.tpcf_plan_destroy(h)
        assert lib.tpcf_test_live_allocations() == base
        if st == 0:
            break
    assert failed_create > 5 and failed_run > 0


def test_injected_oom_catalogue_plan(cuda_device):
    _capi = _lib()
    lib = _capi.lib()
    xyz = torch.from_numpy(synth.uniform_sphere(3000, synth.rng(62))).to(cuda_device)
    torch.cuda.synchronize()
    base = lib.tpcf_test_live_allocations()
    bins, _keep = _bins(_capi, [1.0, 4.0, 9.0], 3)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    failed = 0
    for n in range(1, 200):
        lib.tpcf_test_fail_allocation(n)
        h = ctypes.c_void_p()
        st = lib.tpcf_plan_create_catalog(ctypes.byref(h), xyz.data_ptr(), 3000, ctypes.byref(bins), stream)
        lib.tpcf_test_fail_allocation(0)
        if st != 0:
            assert st == OOM, _capi.STATUS.get(st, st)
            assert not h.value
            assert lib.tpcf_test_live_allocations() == base
            failed += 1
            continue
        lib.tpcf_plan_destroy(h)
        assert lib.tpcf_test_live_allocations() == base
        break
    assert failed > 5
