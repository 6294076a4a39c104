"""Parity at the full workload sizes, in the configuration bench.py times.

The oracle cannot sweep 12.6M or 201M pivots, so these tests compare the GPU with
the oracle on pivot subsets (the C ABI's pivot range): the GPU runs the full-size
plan on the full map; the oracle gets every pixel within the outer bin edge of the
sampled pivots, which contains all of their neighbours.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu


def _tpcf():
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def ring_first(nside, r):
    """First pixel of 1-based RING ring r (test-side bookkeeping)."""
    n = nside
    if r > 4 * n - 1:
        return 12 * n * n
    if r < n:
        return 2 * r * (r - 1)
    if r <= 3 * n:
        return 2 * n * (n - 1) + 4 * n * (r - n)
    rr = 4 * n - r
    return 12 * n * n - 2 * rr * (rr + 1)


def band(nside, r0, r1, th_max_deg):
    """Pixel range of the rings within th_max (with margin) of rings [r0, r1].  Ring
    spacing in colatitude is below 1.15 pi / (4 nside) everywhere."""
    pad = int(math.ceil(math.radians(th_max_deg) / (math.pi / (4.0 * nside)) * 1.2)) + 3
    lo = max(1, r0 - pad)
    hi = min(4 * nside - 1, r1 + pad)
    return ring_first(nside, lo), ring_first(nside, hi + 1)


def oracle_on_band(nside, d, w, edges, M, piv_lo, piv_hi, r0, r1, grad_cot=None, targets=None):
    a, b = band(nside, r0, r1, edges[-1])
    idx = np.arange(a, b)
    xyz = oracle.pix2vec_ring(nside, idx)
    dd = d[a:b].astype(np.float64)
    ww = w[a:b].astype(np.float64)
    piv = np.arange(piv_lo - a, piv_hi - a)
    ref = oracle.zeta(xyz, dd, ww, edges, M, pivots=piv)
    g = None
    if grad_cot is not None:
        g = oracle.gradient(xyz, dd, ww, edges, M, grad_cot, pivots=piv, targets=np.asarray(targets) - a)
    return ref, g


def check_rings(plan, nside, d, w, edges, M, rings, npiv):
    """GPU forward on npiv pivots of each ring vs the oracle: per multipole m, the error
    relative to that m's largest |zeta| must stay below TOL."""
    tpcf = _tpcf()
    dt, wt = to_dev(d), to_dev(w)
    report = []
    for r in rings:
        lo = ring_first(nside, r)
        hi = min(lo + npiv, ring_first(nside, r + 1))
        zg, _ = plan.forward(dt, wt, (lo, hi))
        zg = tpcf.as_complex(zg).cpu().numpy()
        ref, _ = oracle_on_band(nside, d, w, edges, M, lo, hi, r, r)
        assert ref["min_margin"] > 1e-12
        if ref["pairs"] == 0:
            assert np.all(zg == 0)
            continue
        report.append((r, rel_err_per_m(zg, ref["zeta"])))
    bad = [(r, float(e.max()), int(np.argmax(e))) for r, e in report if e.max() >= TOL]
    assert not bad, "rings with per-m error above %g: %s" % (TOL, bad)
    return report


@pytest.fixture(scope="module")
def masked1024(cuda_device):
    from paper_2408_16847_gb300 import build
    build()
    wl = synth.masked_map_nside1024()
    d = wl.delta().astype(np.float32)
    w = wl.weights().astype(np.float32)
    plan = _tpcf().Plan.map(wl.nside, wl.bins.edges_deg, wl.bins.m_max)
    return wl, d, w, plan


def test_masked_nside1024_forward_subsets(masked1024):
    wl, d, w, plan = masked1024
    n = wl.nside
    b_edge = int(round((4.0 / 3.0 - math.sin(math.radians(20.0))) * 1.5 * n))
    # a belt ring at z = 1/2, the polar cap (near the pole and further out), the mask edge
    check_rings(plan, n, d, w, wl.bins.edges_deg, wl.bins.m_max, [(5 * n) // 4, 7, 40, b_edge, 4 * n - 3], 700)


def test_masked_nside1024_gradient_subset(masked1024):
    wl, d, w, plan = masked1024
    n = wl.nside
    M, K = wl.bins.m_max, wl.bins.nbins
    cot = wl.cotangent()
    r = (5 * n) // 4
    lo = ring_first(n, r) + 100
    hi = lo + 1500
    dt, wt = to_dev(d), to_dev(w)
    zeta, norm = plan.forward(dt, wt, (lo, hi))
    g = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dt.device)
    g[..., 0] = torch.from_numpy(cot).to(dt.device)
    grad = plan.backward(dt, wt, norm, g, (lo, hi)).cpu().numpy()
    rng = synth.rng(77)
    # targets: pivots of the range, and neighbours of the range on nearby rings
    tg = np.concatenate([rng.integers(lo, hi, 24), rng.integers(ring_first(n, r - 30), ring_first(n, r + 31), 40)])
    _, gref = oracle_on_band(n, d, w, wl.bins.edges_deg, M, lo, hi, r, r,
                             grad_cot=cot.astype(np.complex128), targets=tg)
    scale = np.abs(gref).max()
    assert scale > 0
    err = np.abs(grad[tg] - gref).max() / scale
    assert err < TOL, err
    # outside the reach of the pivots the gradient vanishes
    far = ring_first(n, r + 200)
    assert np.all(grad[far:far + 1000] == 0)


def test_fullsky_nside4096_sampled_pivots(cuda_device):
    from paper_2408_16847_gb300 import build
    build()
    tpcf = _tpcf()
    wl = synth.fullsky_nside4096()
    d = wl.delta().astype(np.float32)
    w = wl.weights().astype(np.float32)
    n, M = wl.nside, wl.bins.m_max
    plan = tpcf.Plan.map(n, wl.bins.edges_deg, M)
    # equator, z = 1/2, the cap edge, close to each pole
    check_rings(plan, n, d, w, wl.bins.edges_deg, M, [2 * n, (5 * n) // 4, n, 9, 4 * n - 20], 256)
    total, _, _ = plan.count_pairs(to_dev(w))
    assert abs(total / tpcf.pairs_hint(12 * n * n, 0.1, 2.0) - 1) < 1e-3
    plan.close()


def test_catalog_2e7_sampled_pivots(cuda_device):
    """The full catalogue workload (2e7 clustered points + 6e7 randoms): GPU raw sums S
    of the union on a range of data pivots and D of the randoms on a range of random
    pivots, against the oracle on the same pivots with neighbours from all points."""
    from paper_2408_16847_gb300 import build
    build()
    tpcf = _tpcf()
    wl = synth.catalog_2e7()
    xd, wd = wl.data()
    xr = wl.randoms()
    nd, nr = len(xd), len(xr)
    wd32 = wd.astype(np.float32)
    alpha = np.float32(float(wd32.astype(np.float64).sum()) / nr)
    xu = np.concatenate([xd, xr])
    du = np.concatenate([np.ones(nd, np.float32), np.full(nr, -alpha, np.float32)])
    wu = np.concatenate([wd32, np.ones(nr, np.float32)])
    edges, M = wl.bins.edges_deg, wl.bins.m_max
    pu = tpcf.Plan.catalog(torch.from_numpy(xu).to("cuda:0"), edges, M)
    lo, hi = 7_000_000, 7_000_400
    _, _, S = pu.forward(to_dev(du), to_dev(wu), (lo, hi), want_sums=True)
    sg = tpcf.as_complex(S).cpu().numpy()
    ref = oracle.zeta(xu, du.astype(np.float64), wu.astype(np.float64), edges, M, pivots=np.arange(lo, hi))
    assert ref["min_margin"] > 1e-12
    assert rel_err_per_m(sg, ref["S"]).max() < TOL
    pu.close()
    pr = tpcf.Plan.catalog(torch.from_numpy(np.ascontiguousarray(xr)).to("cuda:0"), edges, M)
    one = torch.ones(nr, dtype=torch.float32, device="cuda:0")
    rlo, rhi = 31_000_000, 31_000_300
    _, D = pr.forward(one, one, (rlo, rhi))
    refr = oracle.zeta(xr, np.ones(nr), np.ones(nr), edges, M, pivots=np.arange(rlo, rhi))
    np.testing.assert_allclose(D.cpu().numpy(), refr["D"], rtol=1e-6, atol=1e-6 * np.abs(refr["D"]).max())
    pr.close()
