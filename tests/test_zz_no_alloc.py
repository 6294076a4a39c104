"""tpcf_forward_noalloc: the map forward for callers that cannot allocate device
memory (pool allocators that own all memory, allocation-free hot loops).  It must
give the same zeta and norm as tpcf_forward, call after call, although every call
reuses the same fixed scratch array.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

import synth
from gpu_util import TOL, rel_err_per_m

pytestmark = pytest.mark.gpu


def test_noalloc_forward_matches_forward_twice(cuda_device):
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import _capi, tpcf

    nside, M = 32, 10
    edges = np.geomspace(0.9, 14.7, 9)
    plan = tpcf.Plan.map(nside, edges, M)
    npix = 12 * nside * nside
    K = len(edges) - 1
    stream = torch.cuda.current_stream()
    for call, seed in enumerate([synth.BASE_SEED + 900, synth.BASE_SEED + 901]):
        d = synth.bump_map(nside, 800, (1.0, 6.0), 0.5, 0.05, seed=seed).astype(np.float32)
        w = synth.rng(seed + 1).uniform(0.5, 1.5, npix).astype(np.float32)
        if call == 1:
            w[: npix // 3] = 0.0  # a different mask, so stale scratch would show
        dt = torch.from_numpy(d).to(cuda_device)
        wt = torch.from_numpy(w).to(cuda_device)
        zeta_ref, norm_ref = plan.forward(dt, wt)
        zeta = torch.full((M + 1, K, K, 2), np.nan, dtype=torch.float64, device=cuda_device)
        norm = torch.full((K, K), np.nan, dtype=torch.float64, device=cuda_device)
        st = _capi.lib().tpcf_forward_noalloc(plan.handle, dt.data_ptr(), wt.data_ptr(), 0, npix,
                                              zeta.data_ptr(), norm.data_ptr(),
                                              ctypes.c_void_p(stream.cuda_stream))
        _capi.check(st, "tpcf_forward_noalloc")
        torch.cuda.synchronize()
        plan.sync()
        zr = tpcf.as_complex(zeta_ref).cpu().numpy()
        zn = tpcf.as_complex(zeta).cpu().numpy()
        assert np.all(np.isfinite(zn)), "call %d left non-finite values" % call
        err = rel_err_per_m(zn, zr).max()
        assert err < TOL, "call %d: per-m relative error %.3g" % (call, err)
        # the sums of a call are summed in a run-dependent order (atomics), so the two
        # entry points agree to rounding
        np.testing.assert_allclose(norm.cpu().numpy(), norm_ref.cpu().numpy(), rtol=1e-6, atol=0)


def _noalloc(plan, dt, wt, zeta, norm, lo=0, hi=None):
    from paper_2408_16847_gb300 import _capi
    stream = torch.cuda.current_stream()
    return _capi.lib().tpcf_forward_noalloc(plan.handle, dt.data_ptr(), wt.data_ptr(), lo,
                                            plan.npoints if hi is None else hi, zeta.data_ptr(),
                                            norm.data_ptr(), ctypes.c_void_p(stream.cuda_stream))


def test_noalloc_many_bins_fewer_ctas(cuda_device):
    """24 bins and m_max 12: one CTA's partial sums take 65 KB, so the fixed array
    holds fewer slots than the plain forward runs CTAs and the call runs fewer CTAs.
    Same zeta as tpcf_forward on two calls in a row (different masks)."""
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import _capi, tpcf

    nside, M = 16, 12
    edges = np.linspace(0.5, 30.0, 25)
    K = len(edges) - 1
    plan = tpcf.Plan.map(nside, edges, M)
    npix = 12 * nside * nside
    for call in range(2):
        d = synth.bump_map(nside, 300, (2.0, 8.0), 0.5, 0.05, seed=synth.BASE_SEED + 910 + call).astype(np.float32)
        w = np.ones(npix, np.float32)
        if call == 1:
            w[npix // 2:] = 0.0
        dt = torch.from_numpy(d).to(cuda_device)
        wt = torch.from_numpy(w).to(cuda_device)
        zeta_ref, norm_ref = plan.forward(dt, wt)
        zeta = torch.full((M + 1, K, K, 2), np.nan, dtype=torch.float64, device=cuda_device)
        norm = torch.full((K, K), np.nan, dtype=torch.float64, device=cuda_device)
        _capi.check(_noalloc(plan, dt, wt, zeta, norm), "tpcf_forward_noalloc")
        torch.cuda.synchronize()
        plan.sync()
        zr = tpcf.as_complex(zeta_ref).cpu().numpy()
        zn = tpcf.as_complex(zeta).cpu().numpy()
        assert np.all(np.isfinite(zn))
        assert rel_err_per_m(zn, zr).max() < TOL
        np.testing.assert_allclose(norm.cpu().numpy(), norm_ref.cpu().numpy(), rtol=1e-6, atol=0)
    plan.close()


def test_noalloc_rejects_unsupported_plans(cuda_device):
    """Self-pair subtraction, the tensor-core contraction and catalogue plans are not
    served by the allocation-free call: TPCF_ERR_UNSUPPORTED, outputs untouched."""
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import _capi, tpcf

    nside, M = 8, 4
    edges = np.array([2.0, 5.0, 9.0])
    K = 2
    npix = 12 * nside * nside
    dt = torch.ones(npix, dtype=torch.float32, device=cuda_device)
    wt = torch.ones(npix, dtype=torch.float32, device=cuda_device)
    zeta = torch.full((M + 1, K, K, 2), 7.0, dtype=torch.float64, device=cuda_device)
    norm = torch.full((K, K), 7.0, dtype=torch.float64, device=cuda_device)
    for plan in (tpcf.Plan.map(nside, edges, M, self_pairs="subtract"), tpcf.Plan.map(nside, edges, M, contract="tc")):
        assert _noalloc(plan, dt, wt, zeta, norm) == 5  # TPCF_ERR_UNSUPPORTED
        plan.close()
    xyz = torch.from_numpy(synth.uniform_sphere(500, synth.rng(3))).to(cuda_device)
    cat = tpcf.Plan.catalog(xyz, edges, M)
    d5 = torch.ones(500, dtype=torch.float32, device=cuda_device)
    assert _noalloc(cat, d5, d5, zeta, norm) == 5  # TPCF_ERR_UNSUPPORTED
    cat.close()
    torch.cuda.synchronize()
    assert torch.all(zeta == 7.0) and torch.all(norm == 7.0)
