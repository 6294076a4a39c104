"""Pins for the oracle's shared-neighbour-list estimator (zeta_grouped: the pivots of a
run of `group` consecutive ring pixels take the moments of the run's middle pixel).

* group = 1 is the exact estimator;
* the runs tile every ring and each run's representative is one of its own pixels;
* a constant field c gives zeta_0 = c^3 exactly whatever the grouping (S_0 = c^3 D);
* brute force on a small map: the triplet sum written out with each pivot moved to its
  representative, haversine separations and initial bearings;
* pivot ranges: the sums are additive over disjoint pivot ranges.
"""
import math

import numpy as np
import pytest

import oracle
import synth


def _map(nside, seed):
    npix = 12 * nside * nside
    d = synth.bump_map(nside, 40 * nside, (2.0, 8.0), 0.5, 0.05, seed=seed)
    w = synth.rng(seed + 1).uniform(0.5, 1.5, npix)
    return d, w


def test_group_one_is_the_exact_estimator():
    nside, M = 8, 4
    edges = np.array([3.1, 8.3, 15.7])
    d, w = _map(nside, synth.BASE_SEED + 1800)
    g = oracle.zeta_grouped(nside, d, w, edges, M, 1)
    e = oracle.zeta(oracle.pix2vec_ring(nside), d, w, edges, M)
    np.testing.assert_allclose(g["S"], e["S"], rtol=1e-12, atol=1e-12 * np.abs(e["S"]).max())
    np.testing.assert_allclose(g["D"], e["D"], rtol=1e-12)


@pytest.mark.parametrize("nside,group", [(4, 3), (8, 5), (16, 7), (16, 64)])
def test_runs_tile_the_rings(nside, group):
    reps, members = oracle.pivot_groups(nside, group)
    allpix = np.concatenate(members)
    assert np.array_equal(np.sort(allpix), np.arange(12 * nside * nside))
    for r, m in zip(reps, members):
        assert r in m and len(m) <= group
        assert r == m[(len(m) - 1) // 2]
    # the ring table agrees with the pixel centres: one z per ring, decreasing
    rings = oracle.ring_pixels(nside)
    z = oracle.pix2vec_ring(nside)[:, 2]
    zr = [z[f:f + n] for f, n in rings]
    assert all(np.ptp(x) < 1e-12 for x in zr)
    assert np.all(np.diff([x[0] for x in zr]) < 0)
    # every run stays within one ring
    first = np.array([f for f, _ in rings])
    for m in members:
        assert np.searchsorted(first, m[0], side="right") == np.searchsorted(first, m[-1], side="right")


def test_constant_field_gives_c_cubed():
    nside, M, c = 8, 3, 1.3
    edges = np.array([4.1, 9.3, 18.7])
    w = synth.rng(1810).uniform(0.5, 1.5, 12 * nside * nside)
    g = oracle.zeta_grouped(nside, np.full(len(w), c), w, edges, M, 5)
    np.testing.assert_allclose(g["zeta"][0].real, c ** 3, rtol=1e-12)


def _brute(nside, d, w, edges_deg, M, group):
    xyz = oracle.pix2vec_ring(nside)
    lat = np.arcsin(np.clip(xyz[:, 2], -1, 1))
    lon = np.arctan2(xyz[:, 1], xyz[:, 0])
    th_e = np.deg2rad(edges_deg)
    K = len(th_e) - 1
    S = np.zeros((M + 1, K, K), dtype=complex)
    D = np.zeros((K, K))
    reps, members = oracle.pivot_groups(nside, group)
    for rho, mem in zip(reps, members):
        dlat = lat - lat[rho]
        dlon = lon - lon[rho]
        hav = np.sin(dlat / 2) ** 2 + math.cos(lat[rho]) * np.cos(lat) * np.sin(dlon / 2) ** 2
        th = 2 * np.arcsin(np.sqrt(np.clip(hav, 0, 1)))
        k = np.searchsorted(th_e, th, side="right") - 1
        sel = (k >= 0) & (k < K)
        beta = np.arctan2(np.sin(dlon[sel]) * np.cos(lat[sel]),
                          math.cos(lat[rho]) * np.sin(lat[sel]) - math.sin(lat[rho]) * np.cos(lat[sel]) * np.cos(dlon[sel]))
        onehot = np.zeros((int(sel.sum()), K))
        onehot[np.arange(int(sel.sum())), k[sel]] = 1.0
        v = (w * d)[sel]
        for i in mem:  # every pivot of the run, at its representative's place
            for m in range(M + 1):
                a = onehot.T @ (v * np.exp(-1j * m * beta))
                S[m] += w[i] * d[i] * np.outer(a, np.conj(a))
            Wk = onehot.T @ w[sel]
            D += w[i] * np.outer(Wk, Wk)
    return S, D


def test_brute_force_triplets_with_moved_pivots():
    nside, M, group = 4, 3, 3
    edges = np.array([9.1, 21.3, 37.9])
    d, w = _map(nside, synth.BASE_SEED + 1820)
    g = oracle.zeta_grouped(nside, d, w, edges, M, group)
    assert g["min_margin"] > 1e-9
    Sb, Db = _brute(nside, d, w, edges, M, group)
    assert np.abs(g["S"] - Sb).max() < 1e-11 * np.abs(Sb).max()
    assert np.abs(g["D"] - Db).max() < 1e-11 * np.abs(Db).max()
    # and it is not the exact estimator
    e = oracle.zeta(oracle.pix2vec_ring(nside), d, w, edges, M)
    assert np.abs(g["S"] - e["S"]).max() > 1e-6 * np.abs(e["S"]).max()


def test_sums_are_additive_over_pivot_ranges():
    nside, M, group = 8, 4, 5
    edges = np.array([3.1, 8.3, 15.7])
    d, w = _map(nside, synth.BASE_SEED + 1830)
    npix = 12 * nside * nside
    full = oracle.zeta_grouped(nside, d, w, edges, M, group)
    a = oracle.zeta_grouped(nside, d, w, edges, M, group, pivots=np.arange(0, 301))
    b = oracle.zeta_grouped(nside, d, w, edges, M, group, pivots=np.arange(301, npix))
    np.testing.assert_allclose(a["S"] + b["S"], full["S"], rtol=1e-12, atol=1e-12 * np.abs(full["S"]).max())
    np.testing.assert_allclose(a["D"] + b["D"], full["D"], rtol=1e-12)
