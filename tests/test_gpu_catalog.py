"""GPU catalogue path (device-built sphere grid) vs the FP64 oracle."""
import math

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import TOL, rel_err_per_m, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built(cuda_device):
    from paper_2408_16847_gb300 import build
    build()


def _tpcf():
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _xyz_dev(xyz):
    return torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.float64)).to("cuda:0")


def _field(n, seed):
    g = synth.rng(seed)
    d = (g.standard_normal(n) + 0.3).astype(np.float32)
    w = g.uniform(0.5, 1.5, n).astype(np.float32)
    return d, w


def _check(xyz, d, w, edges, M, pivots=None, self_pairs="keep", tol=TOL):
    tpcf = _tpcf()
    plan = tpcf.Plan.catalog(_xyz_dev(xyz), np.asarray(edges), M, self_pairs=self_pairs)
    zeta, norm, sums = plan.forward(to_dev(d), to_dev(w), pivots, want_sums=True)
    plan.sync()
    zg = tpcf.as_complex(zeta).cpu().numpy()
    sg = tpcf.as_complex(sums).cpu().numpy()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    ref = oracle.zeta(xyz, d.astype(np.float64), w.astype(np.float64), np.asarray(edges), M, pivots=piv,
                      self_pairs=self_pairs)
    assert ref["min_margin"] > 1e-12
    np.testing.assert_allclose(norm.cpu().numpy(), ref["D"], rtol=1e-6, atol=1e-6 * np.abs(ref["D"]).max())
    # the bar: per multipole, each m against its own largest entry
    e = rel_err_per_m(zg, ref["zeta"])
    assert e.max() < tol, "per-m relative error of zeta %s" % np.array2string(e, precision=2)
    e = rel_err_per_m(sg, ref["S"])
    assert e.max() < tol, "per-m relative error of S %s" % np.array2string(e, precision=2)
    plan.close()
    return zg, ref


@pytest.mark.parametrize("n,edges,M", [
    (3000, [3.1, 8.3, 15.7, 25.9], 6),
    (5000, list(np.geomspace(0.9, 12.3, 9)), 10),
    (800, [10.3, 40.7, 80.9], 16),
    (4000, [2.1, 7.7], 0),
])
def test_uniform_catalogues(n, edges, M):
    xyz = synth.uniform_sphere(n, synth.rng(900 + n))
    d, w = _field(n, 901 + n)
    _check(xyz, d, w, edges, M)


def test_clustered_catalogue_with_pivot_ranges():
    xyz = synth.clustered_catalog(20000, 300, 0.8, synth.BASE_SEED + 910)
    d, w = _field(len(xyz), 911)
    edges = np.linspace(0.2, 3.0, 9)
    _check(xyz, d, w, edges, 8)
    for lo, hi in [(0, 1), (77, 1290), (19950, 20000), (500, 500)]:
        if lo == hi:
            tpcf = _tpcf()
            plan = tpcf.Plan.catalog(_xyz_dev(xyz), edges, 8)
            z, n = plan.forward(to_dev(d), to_dev(w), (lo, hi))
            assert torch.all(z == 0) and torch.all(n == 0)
            continue
        _check(xyz, d, w, edges, 8, pivots=(lo, hi))


def test_poles_duplicates_and_masked_points():
    g = synth.rng(920)
    xyz = synth.uniform_sphere(3000, g)
    # points exactly on both poles, a duplicated point, masked points near a pole
    xyz[0] = [0.0, 0.0, 1.0]
    xyz[1] = [0.0, 0.0, -1.0]
    xyz[2] = xyz[3]
    t = np.radians(np.array([0.5, 1.3, 2.7]))
    xyz[4:7] = np.stack([np.sin(t), np.zeros(3), np.cos(t)], axis=1)
    d, w = _field(len(xyz), 921)
    w[5] = 0.0
    _check(xyz, d, w, [1.1, 4.3, 9.7, 20.9], 8)


def test_self_pair_subtraction():
    xyz = synth.uniform_sphere(4000, synth.rng(930))
    d, w = _field(len(xyz), 931)
    _check(xyz, d, w, list(np.geomspace(1.3, 17.0, 6)), 8, self_pairs="subtract")


def test_catalogue_path_equals_map_path_on_pixel_centres():
    """The same field on the HEALPix pixel centres through both neighbour searches."""
    tpcf = _tpcf()
    nside = 16
    edges = np.geomspace(1.53, 25.1, 7)
    d = synth.bump_map(nside, 800, (2.0, 6.0), 0.5, 0.05, seed=synth.BASE_SEED + 940).astype(np.float32)
    w = synth.rng(941).uniform(0.5, 1.5, 12 * nside * nside).astype(np.float32)
    pm = tpcf.Plan.map(nside, edges, 10)
    zm, nm = pm.forward(to_dev(d), to_dev(w))
    pc = tpcf.Plan.catalog(_xyz_dev(oracle.pix2vec_ring(nside)), edges, 10)
    zc, nc = pc.forward(to_dev(d), to_dev(w))
    zm = tpcf.as_complex(zm).cpu().numpy()
    zc = tpcf.as_complex(zc).cpu().numpy()
    assert rel_err_per_m(zc, zm).max() < TOL
    np.testing.assert_allclose(nc.cpu().numpy(), nm.cpu().numpy(), rtol=1e-6)


def test_edge_corrected_data_minus_randoms():
    """zeta = S(data with 1, randoms with -alpha) / (alpha^3 D_randoms)."""
    tpcf = _tpcf()
    xd = synth.clustered_catalog(3000, 60, 1.0, synth.BASE_SEED + 950)
    wd = synth.rng(951).uniform(0.5, 1.5, len(xd))
    xr = synth.uniform_sphere(9000, synth.rng(952))
    edges = np.linspace(0.5, 6.0, 7)
    M = 10
    nd, nr = len(xd), len(xr)
    alpha = float(wd.astype(np.float32).astype(np.float64).sum()) / nr
    xu = np.concatenate([xd, xr])
    du = np.concatenate([np.ones(nd), np.full(nr, -alpha)]).astype(np.float32)
    wu = np.concatenate([wd, np.ones(nr)]).astype(np.float32)
    pu = tpcf.Plan.catalog(_xyz_dev(xu), edges, M)
    pr = tpcf.Plan.catalog(_xyz_dev(xr), edges, M)
    _, _, S = pu.forward(to_dev(du), to_dev(wu), want_sums=True)
    _, DR = pr.forward(to_dev(np.ones(nr, np.float32)), to_dev(np.ones(nr, np.float32)))
    zeta = tpcf.normalize(S, DR, (float(np.float32(-du[-1]))) ** 3)
    zg = tpcf.as_complex(zeta).cpu().numpy()
    ref = oracle.catalog_zeta(xd, wu[:nd].astype(np.float64), xr, edges, M)
    # the oracle's alpha is computed from the float32 weights it is given; the GPU
    # reads delta = -alpha as float32, so compare with the oracle fed those values
    u = oracle.zeta(xu, du.astype(np.float64), wu.astype(np.float64), edges, M)
    r = oracle.zeta(xr, np.ones(nr), np.ones(nr), edges, M)
    a32 = float(np.float32(-du[-1]))
    zo = u["S"] / ((a32 ** 3) * r["D"])[None]
    assert rel_err_per_m(zg, zo).max() < TOL
    # and the oracle's own D-R composition (alpha in fp64) agrees with that up to the
    # float32 rounding of alpha, amplified by the D-R cancellation
    assert rel_err_per_m(zo, ref["zeta"]).max() < 1e-4


def test_catalogue_pair_count_exact():
    tpcf = _tpcf()
    xyz = synth.clustered_catalog(15000, 200, 0.7, synth.BASE_SEED + 970)
    w = synth.rng(971).uniform(0.5, 1.5, len(xyz)).astype(np.float32)
    w[::5] = 0.0
    edges = np.linspace(0.3, 3.1, 8)
    plan = tpcf.Plan.catalog(_xyz_dev(xyz), edges, 4)
    total, sym, single = plan.count_pairs(to_dev(w))
    live = np.nonzero(w)[0]
    assert total == int(oracle.pair_counts(xyz, edges, pivots=live).sum())
    assert sym == 0 and single == total
    t2, _, _ = plan.count_pairs(to_dev(np.ones_like(w)), (1000, 4000))
    assert t2 == int(oracle.pair_counts(xyz, edges, pivots=np.arange(1000, 4000)).sum())


@pytest.mark.parametrize("n,edges,M,pivots", [
    (3000, [3.1, 8.3, 15.7, 25.9], 6, None),
    (6000, list(np.geomspace(1.1, 12.3, 6)), 10, (500, 2300)),
])
def test_catalogue_gradient_vs_oracle_and_fd(n, edges, M, pivots):
    tpcf = _tpcf()
    xyz = synth.clustered_catalog(n, 80, 2.0, synth.BASE_SEED + 980 + n)
    d, w = _field(n, 981 + n)
    K = len(edges) - 1
    g = synth.rng(982)
    cot = g.standard_normal((M + 1, K, K)) + 1j * g.standard_normal((M + 1, K, K))
    plan = tpcf.Plan.catalog(_xyz_dev(xyz), np.asarray(edges), M)
    dt, wt = to_dev(d), to_dev(w)
    zeta, norm = plan.forward(dt, wt, pivots)
    gl = torch.from_numpy(np.stack([cot.real, cot.imag], axis=-1)).to("cuda:0")
    grad = plan.backward(dt, wt, norm, gl, pivots).cpu().numpy()
    plan.sync()
    piv = None if pivots is None else np.arange(pivots[0], pivots[1])
    gref = oracle.gradient(xyz, d.astype(np.float64), w.astype(np.float64), np.asarray(edges), M, cot, pivots=piv)
    scale = np.abs(gref).max()
    assert scale > 0
    assert np.abs(grad - gref).max() < TOL * scale

    def L(dd):
        z, _ = plan.forward(to_dev(dd), wt, pivots)
        zc = tpcf.as_complex(z).cpu().numpy()
        return float(np.sum(cot.real * zc.real + cot.imag * zc.imag))
    for p in [1, n // 2, n - 3]:
        dp = d.copy(); dp[p] += 1.0
        dm = d.copy(); dm[p] -= 1.0
        assert abs((L(dp) - L(dm)) / 2.0 - grad[p]) <= 1e-3 * scale, p
