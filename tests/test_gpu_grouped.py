"""tpcf_forward_grouped (shared neighbour lists: runs of `group` ring pixels take the
moments of their middle pixel) against the oracle's zeta_grouped, per multipole; group 1
is the exact forward; the mode's deviation from the exact estimate shrinks with the run
length; unsupported plans are rejected."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu


def _tpcf():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _map(nside, seed, masked=False):
    npix = 12 * nside * nside
    d = synth.bump_map(nside, 40 * nside, (2.0, 8.0), 0.5, 0.05, seed=seed).astype(np.float32)
    w = synth.rng(seed + 1).uniform(0.5, 1.5, npix)
    if masked:
        w = w * synth.galactic_mask_weights(nside)
    return d, w.astype(np.float32)


@pytest.mark.parametrize("nside,edges,M,group,pivots,masked", [
    (8, [2.03, 10.3, 20.7], 4, 3, None, False),
    (16, list(np.geomspace(1.53, 25.1, 7)), 10, 5, None, True),
    (16, [1.7, 6.3, 13.9], 8, 64, None, False),
    (32, list(np.geomspace(0.8, 12.0, 9)), 8, 7, (5000, 5999), True),
])
def test_grouped_vs_oracle(cuda_device, nside, edges, M, group, pivots, masked):
    tpcf = _tpcf()
    d, w = _map(nside, synth.BASE_SEED + 1900 + nside + group, masked)
    plan = tpcf.Plan.map(nside, np.asarray(edges), M)
    zeta, norm, sums = plan.forward_grouped(to_dev(d), to_dev(w), group, pivots, want_sums=True)
    plan.sync()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta_grouped(nside, d.astype(np.float64), w.astype(np.float64), np.asarray(edges), M, group,
                              pivots=piv)
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(tpcf.as_complex(zeta).cpu().numpy(), ref["zeta"]).max() < TOL
    assert rel_err_per_m(tpcf.as_complex(sums).cpu().numpy(), ref["S"]).max() < TOL
    np.testing.assert_allclose(norm.cpu().numpy(), ref["D"], rtol=1e-6, atol=1e-6 * np.abs(ref["D"]).max())
    plan.close()


def test_group_one_is_the_forward_and_errors_shrink(cuda_device):
    tpcf = _tpcf()
    nside, M = 64, 8
    edges = np.geomspace(1.0, 10.0, 9)
    d, w = _map(nside, synth.BASE_SEED + 1950)
    dt, wt = to_dev(d), to_dev(w)
    plan = tpcf.Plan.map(nside, edges, M)
    z1, n1 = plan.forward(dt, wt)
    zg, ng = plan.forward_grouped(dt, wt, 1)
    torch.cuda.synchronize()
    exact = tpcf.as_complex(z1).cpu().numpy()
    assert rel_err_per_m(tpcf.as_complex(zg).cpu().numpy(), exact).max() < 1e-6
    errs = []
    for group in (3, 9, 27):
        z, _ = plan.forward_grouped(dt, wt, group)
        torch.cuda.synchronize()
        errs.append(rel_err_per_m(tpcf.as_complex(z).cpu().numpy(), exact).max())
    assert errs[0] < errs[1] < errs[2], errs
    plan.close()


def test_grouped_rejections(cuda_device):
    tpcf = _tpcf()
    from paper_2408_16847_gb300 import _capi
    nside, M = 8, 2
    edges = np.array([2.03, 10.3])
    npix = 12 * nside * nside
    one = torch.ones(npix, dtype=torch.float32, device="cuda:0")
    for kw in ({"self_pairs": "subtract"}, {"contract": "tc"}, {"norm": "bin_mean"}):
        p = tpcf.Plan.map(nside, edges, M, **kw)
        with pytest.raises(tpcf.TpcfError) as e:
            p.forward_grouped(one, one, 3)
        assert e.value.status == 5
        p.close()
    p = tpcf.Plan.map(nside, edges, M)
    for bad in (0, 4097):
        with pytest.raises(tpcf.TpcfError) as e:
            p.forward_grouped(one, one, bad)
        assert e.value.status == 1
    p.close()
