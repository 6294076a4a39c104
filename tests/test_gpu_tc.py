"""The split-precision tensor-core contraction (TPCF_CONTRACT_TC) vs the FP64 oracle
and vs the FP32 contraction."""
import numpy as np
import pytest

import oracle
import synth
from gpu_util import TOL, gpu_zeta, rel_err_per_m

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    from paper_2408_16847_gb300 import build
    build()


def _tpcf():
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _case(nside, seed, masked=False):
    d = synth.bump_map(nside, 60 * nside, (2.0, 8.0), 0.5, 0.05, seed=seed).astype(np.float32)
    w = synth.galactic_mask_weights(nside) if masked else synth.rng(seed + 1).uniform(0.5, 1.5, 12 * nside ** 2)
    return d, w.astype(np.float32)


@pytest.mark.parametrize("nside,edges,M,self_pairs", [
    (8, [2.03, 10.3, 20.7], 4, "keep"),
    (8, [1.03, 7.1, 20.3, 40.7, 60.9], 16, "keep"),
    (16, list(np.geomspace(1.53, 25.1, 7)), 10, "keep"),
    (16, list(np.geomspace(1.5, 20.0, 5)), 6, "subtract"),
    (8, list(np.linspace(3.3, 71.0, 33)), 2, "keep"),   # K = 32: two accumulator row blocks
    (16, [2.03, 30.7], 0, "keep"),
])
def test_tc_contraction_vs_oracle_and_fp32(nside, edges, M, self_pairs):
    tpcf = _tpcf()
    edges = np.asarray(edges)
    d, w = _case(nside, synth.BASE_SEED + 1100 + nside + M)
    ptc = tpcf.Plan.map(nside, edges, M, self_pairs=self_pairs, contract="tc")
    p32 = tpcf.Plan.map(nside, edges, M, self_pairs=self_pairs)
    ztc, ntc = gpu_zeta(ptc, d, w)
    z32, n32 = gpu_zeta(p32, d, w)
    ref = oracle.zeta(oracle.pix2vec_ring(nside), d.astype(np.float64), w.astype(np.float64), edges, M,
                      self_pairs=self_pairs)
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(ztc, ref["zeta"]).max() < TOL
    np.testing.assert_allclose(ntc, ref["D"], rtol=1e-6, atol=1e-6 * np.abs(ref["D"]).max())
    assert rel_err_per_m(ztc, z32).max() < TOL
    np.testing.assert_allclose(ntc, n32, rtol=1e-6, atol=1e-6 * np.abs(n32).max())


def test_tc_nside64_workload_and_pivot_ranges():
    tpcf = _tpcf()
    wl = synth.map_nside64()
    d = wl.delta().astype(np.float32)
    w = wl.weights().astype(np.float32)
    plan = tpcf.Plan.map(wl.nside, wl.bins.edges_deg, wl.bins.m_max, contract="tc")
    xyz = oracle.pix2vec_ring(wl.nside)
    zg, _ = gpu_zeta(plan, d, w)
    ref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), wl.bins.edges_deg, wl.bins.m_max)
    assert rel_err_per_m(zg, ref["zeta"]).max() < TOL
    for lo, hi in [(0, 1), (1000, 1037), (30000, 33333)]:
        zg, _ = gpu_zeta(plan, d, w, (lo, hi))
        ref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), wl.bins.edges_deg, wl.bins.m_max,
                          pivots=np.arange(lo, hi))
        assert rel_err_per_m(zg, ref["zeta"]).max() < TOL, (lo, hi)


def test_tc_flag_rejected_where_unsupported():
    tpcf = _tpcf()
    import torch
    xyz = torch.from_numpy(synth.uniform_sphere(100, synth.rng(1))).to("cuda:0")
    with pytest.raises(tpcf.TpcfError) as e:
        tpcf.Plan.catalog(xyz, [5.0, 10.0], 2, contract="tc")
    assert e.value.status == 5
