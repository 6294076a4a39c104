"""The multi-field forward (tpcf_forward_multi, three fields on one plan's points,
cyclic sum over the pivot field) against the oracle's zeta_multi, per multipole;
one field reduces to the single-field forward; unsupported plans are rejected."""
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


def _fields(nside, seed, masked=False):
    npix = 12 * nside * nside
    out = []
    for f in range(3):
        d = synth.bump_map(nside, 40 * nside, (2.0, 8.0), 0.5, 0.05, seed=seed + 10 * f).astype(np.float32)
        w = synth.rng(seed + 10 * f + 1).uniform(0.5, 1.5, npix)
        if masked and f == 1:
            w = w * synth.galactic_mask_weights(nside)
        out.append((d, w.astype(np.float32)))
    return out


@pytest.mark.parametrize("nside,edges,M,pivots,masked", [
    (8, [2.03, 10.3, 20.7], 4, None, False),
    (16, list(np.geomspace(1.53, 25.1, 7)), 10, None, True),
    (16, [1.7, 6.3, 13.9], 16, (700, 1733), False),
    (32, list(np.geomspace(0.8, 12.0, 9)), 8, (5000, 5999), True),
])
def test_multi_field_vs_oracle(cuda_device, nside, edges, M, pivots, masked):
    tpcf = _tpcf()
    fields = _fields(nside, synth.BASE_SEED + 1300 + nside + M, masked)
    plan = tpcf.Plan.map(nside, np.asarray(edges), M)
    dev = [(to_dev(d), to_dev(w)) for d, w in fields]
    zeta, norm, sums = plan.forward_multi(dev, pivots, want_sums=True)
    plan.sync()
    zg = tpcf.as_complex(zeta).cpu().numpy()
    sg = tpcf.as_complex(sums).cpu().numpy()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta_multi(oracle.pix2vec_ring(nside), [(d.astype(np.float64), w.astype(np.float64))
                                                          for d, w in fields], np.asarray(edges), M, pivots=piv)
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(zg, ref["zeta"]).max() < TOL
    assert rel_err_per_m(sg, ref["S"]).max() < TOL
    np.testing.assert_allclose(norm.cpu().numpy(), ref["D"], rtol=1e-6, atol=1e-6 * np.abs(ref["D"]).max())
    plan.close()


def test_one_field_equals_single_forward(cuda_device):
    tpcf = _tpcf()
    nside, M = 16, 8
    edges = np.geomspace(1.53, 25.1, 6)
    d, w = _fields(nside, synth.BASE_SEED + 1400)[0]
    dt, wt = to_dev(d), to_dev(w)
    plan = tpcf.Plan.map(nside, edges, M)
    zm, nm = plan.forward_multi([(dt, wt)] * 3)
    z1, n1 = plan.forward(dt, wt)
    torch.cuda.synchronize()
    assert rel_err_per_m(tpcf.as_complex(zm).cpu().numpy(), tpcf.as_complex(z1).cpu().numpy()).max() < 1e-6
    np.testing.assert_allclose(nm.cpu().numpy(), 3 * n1.cpu().numpy(), rtol=1e-6)
    plan.close()


def test_multi_rejects_unsupported_plans(cuda_device):
    tpcf = _tpcf()
    nside, M = 8, 2
    edges = np.array([2.03, 10.3])
    npix = 12 * nside * nside
    one = torch.ones(npix, dtype=torch.float32, device="cuda:0")
    for kw in ({"self_pairs": "subtract"}, {"contract": "tc"}):
        p = tpcf.Plan.map(nside, edges, M, **kw)
        with pytest.raises(tpcf.TpcfError) as e:
            p.forward_multi([(one, one)] * 3)
        assert e.value.status == 5
        p.close()


@pytest.mark.parametrize("n,edges,M,pivots", [
    (4000, [0.9, 2.1, 4.3, 7.7], 6, None),
    (12000, list(np.geomspace(0.4, 6.0, 7)), 10, (2500, 7100)),
])
def test_catalogue_multi_field_vs_oracle(cuda_device, n, edges, M, pivots):
    tpcf = _tpcf()
    xyz = synth.clustered_catalog(n, 150, 0.8, synth.BASE_SEED + 1360 + n)
    g = synth.rng(1361 + n)
    fields = [((g.standard_normal(n) + 0.3 * f).astype(np.float32), g.uniform(0.5, 1.5, n).astype(np.float32))
              for f in range(3)]
    plan = tpcf.Plan.catalog(torch.from_numpy(np.ascontiguousarray(xyz)).to("cuda:0"), np.asarray(edges), M)
    zeta, norm, sums = plan.forward_multi([(to_dev(d), to_dev(w)) for d, w in fields], pivots, want_sums=True)
    plan.sync()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta_multi(xyz, [(d.astype(np.float64), w.astype(np.float64)) for d, w in fields],
                            np.asarray(edges), M, pivots=piv)
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(tpcf.as_complex(zeta).cpu().numpy(), ref["zeta"]).max() < TOL
    assert rel_err_per_m(tpcf.as_complex(sums).cpu().numpy(), ref["S"]).max() < TOL
    np.testing.assert_allclose(norm.cpu().numpy(), ref["D"], rtol=1e-6, atol=1e-6 * np.abs(ref["D"]).max())
    # one field three times is the single-field catalogue forward
    d, w = fields[0]
    zm, nm = plan.forward_multi([(to_dev(d), to_dev(w))] * 3, pivots)
    z1, n1 = plan.forward(to_dev(d), to_dev(w), pivots)
    torch.cuda.synchronize()
    assert rel_err_per_m(tpcf.as_complex(zm).cpu().numpy(), tpcf.as_complex(z1).cpu().numpy()).max() < 1e-6
    np.testing.assert_allclose(nm.cpu().numpy(), 3 * n1.cpu().numpy(), rtol=1e-6)
    plan.close()
