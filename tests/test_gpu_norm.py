"""Per-pivot normalisations of the moments (Sec. 3.1: the prefactor of eq. Xm.binned,
a_m^k(i) / sum_k W^k(i), and the per-bin average of the binning figure's caption,
a_m^k(i) / W^k(i)) on map and catalogue plans, against the oracle's contract(norm=
"R1" / "R2"), per multipole; the allocation-free entry point gives the same result;
the flag combinations without a kernel are rejected."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu

NORMS = {"bin_mean": "R2", "pivot_total": "R1"}


def _tpcf():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _compare(tpcf, zeta, norm, sums, ref):
    zg = tpcf.as_complex(zeta).cpu().numpy()
    sg = tpcf.as_complex(sums).cpu().numpy()
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(zg, ref["zeta"]).max() < TOL
    assert rel_err_per_m(sg, ref["S"]).max() < TOL
    np.testing.assert_allclose(norm.cpu().numpy(), ref["D"], rtol=1e-6)


@pytest.mark.parametrize("norm", ["bin_mean", "pivot_total"])
@pytest.mark.parametrize("nside,edges,M,pivots,masked", [
    (8, [2.03, 10.3, 20.7], 4, None, False),
    (16, list(np.geomspace(1.53, 25.1, 7)), 10, None, True),
    (32, list(np.geomspace(0.8, 12.0, 9)), 8, (5000, 5999), True),
])
def test_map_norms_vs_oracle(cuda_device, norm, nside, edges, M, pivots, masked):
    tpcf = _tpcf()
    npix = 12 * nside * nside
    seed = synth.BASE_SEED + 1500 + nside + M
    d = synth.bump_map(nside, 40 * nside, (2.0, 8.0), 0.5, 0.05, seed=seed).astype(np.float32)
    w = synth.rng(seed + 1).uniform(0.5, 1.5, npix)
    if masked:
        w = w * synth.galactic_mask_weights(nside)
    w = w.astype(np.float32)
    plan = tpcf.Plan.map(nside, np.asarray(edges), M, norm=norm)
    zeta, nrm, sums = plan.forward(to_dev(d), to_dev(w), pivots, want_sums=True)
    plan.sync()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta(oracle.pix2vec_ring(nside), d.astype(np.float64), w.astype(np.float64), np.asarray(edges), M,
                      pivots=piv, norm=NORMS[norm])
    _compare(tpcf, zeta, nrm, sums, ref)
    plan.close()


@pytest.mark.parametrize("norm", ["bin_mean", "pivot_total"])
def test_catalogue_norms_vs_oracle(cuda_device, norm):
    tpcf = _tpcf()
    xyz = synth.clustered_catalog(6000, 120, 0.8, synth.BASE_SEED + 1510)
    g = synth.rng(1511)
    d = (g.standard_normal(len(xyz)) + 0.3).astype(np.float32)
    w = g.uniform(0.5, 1.5, len(xyz)).astype(np.float32)
    edges = np.geomspace(0.4, 6.0, 8)
    xd = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float64)).to("cuda:0")
    plan = tpcf.Plan.catalog(xd, edges, 8, norm=norm)
    for pivots in (None, (1000, 2500)):
        zeta, nrm, sums = plan.forward(to_dev(d), to_dev(w), pivots, want_sums=True)
        plan.sync()
        piv = None if pivots is None else np.arange(pivots[0], pivots[1])
        ref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), edges, 8, pivots=piv, norm=NORMS[norm])
        _compare(tpcf, zeta, nrm, sums, ref)
    plan.close()


def test_noalloc_with_a_norm_matches_forward(cuda_device):
    tpcf = _tpcf()
    from paper_2408_16847_gb300 import _capi
    nside, M = 16, 6
    edges = np.geomspace(1.53, 25.1, 6)
    K = len(edges) - 1
    npix = 12 * nside * nside
    d = synth.bump_map(nside, 600, (2.0, 8.0), 0.5, 0.05, seed=synth.BASE_SEED + 1520).astype(np.float32)
    w = synth.rng(1521).uniform(0.5, 1.5, npix).astype(np.float32)
    dt, wt = to_dev(d), to_dev(w)
    plan = tpcf.Plan.map(nside, edges, M, norm="bin_mean")
    z1, n1 = plan.forward(dt, wt)
    zeta = torch.full((M + 1, K, K, 2), np.nan, dtype=torch.float64, device="cuda:0")
    nrm = torch.full((K, K), np.nan, dtype=torch.float64, device="cuda:0")
    st = _capi.lib().tpcf_forward_noalloc(plan.handle, dt.data_ptr(), wt.data_ptr(), 0, npix, zeta.data_ptr(),
                                          nrm.data_ptr(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    _capi.check(st, "tpcf_forward_noalloc")
    torch.cuda.synchronize()
    assert rel_err_per_m(tpcf.as_complex(zeta).cpu().numpy(), tpcf.as_complex(z1).cpu().numpy()).max() < 1e-6
    np.testing.assert_allclose(nrm.cpu().numpy(), n1.cpu().numpy(), rtol=1e-6)
    plan.close()


def test_norm_rejections(cuda_device):
    tpcf = _tpcf()
    nside, M = 8, 2
    edges = np.array([2.03, 10.3])
    npix = 12 * nside * nside
    one = torch.ones(npix, dtype=torch.float32, device="cuda:0")
    for kw in ({"self_pairs": "subtract"}, {"contract": "tc"}):
        with pytest.raises(tpcf.TpcfError) as e:
            tpcf.Plan.map(nside, edges, M, norm="bin_mean", **kw)
        assert e.value.status == 5
    p = tpcf.Plan.map(nside, edges, M, norm="pivot_total")
    z, n = p.forward(one, one)
    dl = torch.zeros_like(z)
    with pytest.raises(tpcf.TpcfError) as e:
        p.backward(one, one, n, dl)
    assert e.value.status == 5
    with pytest.raises(tpcf.TpcfError) as e:
        p.forward_multi([(one, one)] * 3)
    assert e.value.status == 5
    p.close()
