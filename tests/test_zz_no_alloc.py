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
