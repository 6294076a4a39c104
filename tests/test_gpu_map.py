"""GPU map path vs the FP64 oracle (element by element, same seeded inputs).

The CUDA path reads float32 (delta, w); the oracle gets the same float32 values
promoted to float64, so the comparison measures the kernels, not input rounding.
"""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, gpu_zeta, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    from paper_2408_16847_gb300 import build
    build()


def _tpcf():
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _case(nside, nbumps, sig, seed, masked=False):
    d = synth.bump_map(nside, nbumps, sig, 0.5, 0.05, seed=seed).astype(np.float32)
    w = synth.galactic_mask_weights(nside) if masked else np.ones(12 * nside * nside)
    return d, w.astype(np.float32)


def _check_forward(nside, edges, M, d32, w32, pivots=None, self_pairs="keep", tol=TOL):
    tpcf = _tpcf()
    plan = tpcf.Plan.map(nside, edges, M, self_pairs=self_pairs)
    zg, ng = gpu_zeta(plan, d32, w32, pivots)
    xyz = oracle.pix2vec_ring(nside)
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta(xyz, d32.astype(np.float64), w32.astype(np.float64), edges, M, pivots=piv,
                      self_pairs=self_pairs)
    # the bin decision is exact on both sides; make sure no pair sits within rounding of an edge
    assert ref["min_margin"] > 1e-12
    np.testing.assert_allclose(ng, ref["D"], rtol=1e-6, atol=1e-6 * max(1.0, np.abs(ref["D"]).max()))
    e = rel_err_per_m(zg, ref["zeta"])
    assert e.max() < tol, "per-m relative error %s" % np.array2string(e, precision=2)
    return zg, ref


@pytest.mark.parametrize("nside,edges,M", [
    # edges avoid the exact pixel separations of coarse grids (ties would be rounding-decided)
    (1, [10.3, 50.7, 88.9], 4),
    (2, [5.3, 30.7, 60.9, 84.1], 6),
    (4, [3.1, 10.3, 25.7, 44.9], 8),
    (8, [1.03, 7.1, 20.3, 40.7, 60.9], 16),
    (8, [2.03, 30.7], 0),
    (16, list(np.geomspace(1.53, 25.1, 7)), 10),
])
def test_small_maps(nside, edges, M):
    d, w = _case(nside, 60 * nside, (3.0, 12.0), synth.BASE_SEED + 300 + nside)
    _check_forward(nside, np.asarray(edges), M, d, w)


def test_map_nside64_workload():
    """10 linear bins 0.5-10 deg, m <= 8, full forward (the oracle runs in ~1 s)."""
    wl = synth.map_nside64()
    d = wl.delta().astype(np.float32)
    w = wl.weights().astype(np.float32)
    zg, ref = _check_forward(wl.nside, wl.bins.edges_deg, wl.bins.m_max, d, w)
    assert ref["pairs"] > 1.8e7


def test_pivot_ranges_and_ragged_tiles():
    nside = 16
    edges = np.geomspace(1.0, 15.0, 5)
    d, w = _case(nside, 500, (2.0, 6.0), synth.BASE_SEED + 401)
    npix = 12 * nside * nside
    # ranges that start and end inside tiles, inside the polar cap, across the belt edge
    for lo, hi in [(0, 1), (3, 77), (400, 1100), (1500, 1537), (npix - 45, npix)]:
        _check_forward(nside, edges, 6, d, w, pivots=(lo, hi))


def test_empty_range_and_full_mask_give_zeros():
    tpcf = _tpcf()
    nside = 8
    edges = np.array([2.0, 10.0, 20.0])
    plan = tpcf.Plan.map(nside, edges, 3)
    d, w = _case(nside, 100, (3.0, 8.0), synth.BASE_SEED + 402)
    zg, ng = gpu_zeta(plan, d, w, (100, 100))
    assert np.all(zg == 0) and np.all(ng == 0)
    zg, ng = gpu_zeta(plan, d, np.zeros_like(w))
    assert np.all(zg == 0) and np.all(ng == 0)


def test_masked_map():
    nside = 32
    edges = np.geomspace(0.8, 12.0, 8)
    d, w = _case(nside, 1500, (1.0, 5.0), synth.BASE_SEED + 403, masked=True)
    _check_forward(nside, edges, 10, d, w)


def test_self_pair_subtraction():
    nside = 16
    edges = np.geomspace(1.5, 20.0, 6)
    d, w = _case(nside, 400, (2.0, 8.0), synth.BASE_SEED + 404)
    _check_forward(nside, edges, 8, d, w, self_pairs="subtract")


def test_weights_and_negative_values():
    nside = 16
    edges = np.linspace(2.0, 16.0, 6)
    d, _ = _case(nside, 400, (2.0, 8.0), synth.BASE_SEED + 405)
    w = synth.rng(406).uniform(0.0, 2.0, 12 * nside * nside).astype(np.float32)
    w[::7] = 0.0
    _check_forward(nside, edges, 7, d, w)


@pytest.mark.parametrize("nside,M", [(8, 5), (16, 8)])
def test_gradient_vs_oracle_and_fd(nside, M):
    tpcf = _tpcf()
    edges = np.geomspace(2.0, 24.0, 6)
    K = len(edges) - 1
    d, _ = _case(nside, 50 * nside, (3.0, 10.0), synth.BASE_SEED + 500 + nside)
    w = synth.rng(501).uniform(0.5, 1.5, 12 * nside * nside).astype(np.float32)
    g = synth.rng(502)
    cot = g.standard_normal((M + 1, K, K)) + 1j * g.standard_normal((M + 1, K, K))
    plan = tpcf.Plan.map(nside, edges, M)
    dt, wt = to_dev(d), to_dev(w)
    zeta, norm = plan.forward(dt, wt)
    gl = torch.from_numpy(np.stack([cot.real, cot.imag], axis=-1)).to("cuda:0")
    grad = plan.backward(dt, wt, norm, gl).cpu().numpy()
    plan.sync()
    xyz = oracle.pix2vec_ring(nside)
    gref = oracle.gradient(xyz, d.astype(np.float64), w.astype(np.float64), edges, M, cot)
    err = np.abs(grad - gref).max() / np.abs(gref).max()
    assert err < TOL, err
    # central differences of the GPU forward (exact in exact arithmetic for any step,
    # the loss being quadratic in each single delta_p)
    def L(dd):
        z, _ = plan.forward(to_dev(dd), wt)
        zc = tpcf.as_complex(z).cpu().numpy()
        return float(np.sum(cot.real * zc.real + cot.imag * zc.imag))
    for p in [0, 5, 12 * nside * nside // 2 + 3, 12 * nside * nside - 1]:
        h = 1.0
        dp = d.copy(); dp[p] += h
        dm = d.copy(); dm[p] -= h
        fd = (L(dp) - L(dm)) / (2 * h)
        assert abs(fd - grad[p]) <= 1e-3 * np.abs(gref).max(), (p, fd, grad[p])


def test_autograd_function():
    tpcf = _tpcf()
    nside, M = 8, 4
    edges = np.geomspace(3.1, 30.7, 4)
    d, w = _case(nside, 200, (3.0, 10.0), synth.BASE_SEED + 510)
    plan = tpcf.Plan.map(nside, edges, M)
    dt = to_dev(d).requires_grad_(True)
    z = tpcf.ZetaFn.apply(dt, to_dev(w), plan)
    c = torch.randn(z.shape, dtype=torch.float64, device=z.device, generator=torch.Generator("cuda").manual_seed(3))
    (z * c).sum().backward()
    zeta, norm = plan.forward(to_dev(d), to_dev(w))
    ref = plan.backward(to_dev(d), to_dev(w), norm, c)
    assert torch.allclose(dt.grad, ref)


def test_run_host_matches_device_path():
    tpcf = _tpcf()
    nside, M = 16, 6
    edges = np.geomspace(1.5, 20.0, 5)
    d, w = _case(nside, 300, (2.0, 8.0), synth.BASE_SEED + 520)
    K = len(edges) - 1
    cot = np.zeros((M + 1, K, K, 2))
    cot[..., 0] = synth.rng(521).standard_normal((M + 1, K, K))
    plan = tpcf.Plan.map(nside, edges, M)
    zh, nh, gh = plan.run_host(d, w, cot)
    zeta, norm = plan.forward(to_dev(d), to_dev(w))
    gd = plan.backward(to_dev(d), to_dev(w), norm, to_dev(cot, torch.float64))
    # the same kernels on the same inputs; summation order across warps and CTAs is
    # not fixed, so agreement is to rounding, not bitwise
    zd = zeta.cpu().numpy()
    assert np.abs(zh - zd).max() <= 1e-6 * np.abs(zd).max()
    assert np.allclose(nh, norm.cpu().numpy(), rtol=1e-12, atol=0)
    gdn = gd.cpu().numpy()
    assert np.abs(gh - gdn).max() <= 1e-5 * np.abs(gdn).max()


@pytest.mark.parametrize("nside,edges", [(16, np.geomspace(1.53, 25.1, 7)), (64, np.linspace(0.5, 10.0, 11))])
def test_pair_count_exact(nside, edges):
    tpcf = _tpcf()
    plan = tpcf.Plan.map(nside, edges, 2)
    w = synth.galactic_mask_weights(nside).astype(np.float32)
    total, sym, single = plan.count_pairs(to_dev(w))
    xyz = oracle.pix2vec_ring(nside)
    live = np.nonzero(w)[0]
    ref = int(oracle.pair_counts(xyz, edges, pivots=live).sum())
    assert total == ref and sym + single == total
    lo, hi = 1000, 1500
    t2, _, _ = plan.count_pairs(to_dev(np.ones_like(w)), (lo, hi))
    assert t2 == int(oracle.pair_counts(xyz, edges, pivots=np.arange(lo, hi)).sum())


@pytest.mark.parametrize("nside,M", [(8, 4), (16, 8)])
def test_gradient_with_self_pair_subtraction(nside, M):
    """The adjoint of the self-pair-subtracted estimator: the a-part plus the
    derivative of the subtracted diagonal (pivot and neighbour legs)."""
    tpcf = _tpcf()
    edges = np.geomspace(2.0, 24.0, 6)
    K = len(edges) - 1
    d, _ = _case(nside, 50 * nside, (3.0, 10.0), synth.BASE_SEED + 530 + nside)
    w = synth.rng(531).uniform(0.5, 1.5, 12 * nside * nside).astype(np.float32)
    g = synth.rng(532)
    cot = g.standard_normal((M + 1, K, K)) + 1j * g.standard_normal((M + 1, K, K))
    plan = tpcf.Plan.map(nside, edges, M, self_pairs="subtract")
    dt, wt = to_dev(d), to_dev(w)
    zeta, norm = plan.forward(dt, wt)
    gl = torch.from_numpy(np.stack([cot.real, cot.imag], axis=-1)).to("cuda:0")
    grad = plan.backward(dt, wt, norm, gl).cpu().numpy()
    plan.sync()
    xyz = oracle.pix2vec_ring(nside)
    gref = oracle.gradient(xyz, d.astype(np.float64), w.astype(np.float64), edges, M, cot, self_pairs="subtract")
    err = np.abs(grad - gref).max() / np.abs(gref).max()
    assert err < TOL, err

    def L(dd):
        z, _ = plan.forward(to_dev(dd), wt)
        zc = tpcf.as_complex(z).cpu().numpy()
        return float(np.sum(cot.real * zc.real + cot.imag * zc.imag))
    for p in [3, 12 * nside * nside // 3, 12 * nside * nside - 2]:
        dp = d.copy(); dp[p] += 1.0
        dm = d.copy(); dm[p] -= 1.0
        fd = (L(dp) - L(dm)) / 2.0
        assert abs(fd - grad[p]) <= 1e-3 * np.abs(gref).max(), (p, fd, grad[p])


def test_halo_makes_the_adjoint_slice_exact(cuda_device):
    """tpcf_plan_halo: the pivots of the halo of a pixel slice hold every pivot with a
    neighbour in the slice (checked by brute force on the pixel centres), and the
    adjoint over the halo pivots equals the full adjoint on the slice."""
    tpcf = _tpcf()
    nside, M = 16, 6
    edges = list(np.geomspace(1.53, 12.1, 5))
    K = len(edges) - 1
    d32, w32 = _case(nside, 400, (2.0, 8.0), synth.BASE_SEED + 71)
    plan = tpcf.Plan.map(nside, edges, M)
    npix = 12 * nside * nside
    xyz = oracle.pix2vec_ring(nside)
    c = 2 * np.sin(np.deg2rad(edges[-1]) / 2)
    dt, wt = to_dev(d32), to_dev(w32)
    _, norm = plan.forward(dt, wt)
    cot = synth.rng(72).standard_normal((M + 1, K, K))
    g = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dt.device)
    g[..., 0] = torch.from_numpy(cot).to(dt.device)
    full = plan.backward(dt, wt, norm, g).cpu().numpy()
    for lo, hi in [(0, 300), (1000, 1700), (npix // 2 - 64, npix // 2 + 64), (npix - 500, npix)]:
        a, b = plan.halo(lo, hi)
        d2 = ((xyz[:, None, :] - xyz[None, lo:hi, :]) ** 2).sum(-1)
        near = np.nonzero((d2 < c * c).any(axis=1))[0]
        assert a <= near.min() and b >= near.max() + 1 and a <= lo and b >= hi
        part = plan.backward(dt, wt, norm, g, (a, b)).cpu().numpy()
        scale = np.abs(full[lo:hi]).max()
        assert np.abs(part[lo:hi] - full[lo:hi]).max() <= 1e-6 * scale
    assert plan.halo(5, 5) == (5, 5)
    plan.close()
