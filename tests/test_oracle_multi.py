"""Pins for the oracle's multi-field estimator zeta^{ABC} (end of section 2: a pivot
field, two neighbour fields, summed over the cyclic permutations of {A, B, C}).

* brute force: the triplet sum written directly, with the haversine separation and
  the initial-bearing position angle, for three different fields and weights;
* one field: zeta^{AAA} equals the single-field estimator (S and D are three times
  the single-field sums);
* the cyclic sum does not depend on which field is named first, and exchanging the
  two neighbour fields gives the Hermitian transpose;
* S^{ABC} is linear in each field.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from test_oracle_estimator import _cap_points, _latlon


def brute_force_multi(xyz, fields, edges_deg, M):
    """S^{ABC}_m(k1,k2) = sum over cyclic (P, X, Y) of
    sum_i w^P_i P_i sum_{j,l != i} w^X_j X_j w^Y_l Y_l Theta_k1(ij) Theta_k2(il)
    exp(-i m (beta_ij - beta_il)), and D the same with every field set to 1, m = 0."""
    lat, lon = _latlon(xyz)
    th_e = np.deg2rad(np.asarray(edges_deg))
    K = len(th_e) - 1
    S = np.zeros((M + 1, K, K), dtype=complex)
    D = np.zeros((K, K))
    for i in range(len(xyz)):
        dlat = lat - lat[i]
        dlon = lon - lon[i]
        hav = np.sin(dlat / 2) ** 2 + np.cos(lat[i]) * np.cos(lat) * np.sin(dlon / 2) ** 2
        th = 2 * np.arcsin(np.sqrt(np.clip(hav, 0, 1)))
        k = np.searchsorted(th_e, th, side="right") - 1
        sel = (k >= 0) & (k < K)
        sel[i] = False
        if not np.any(sel):
            continue
        kk = k[sel]
        beta = np.arctan2(np.sin(dlon[sel]) * np.cos(lat[sel]),
                          math.cos(lat[i]) * np.sin(lat[sel]) - math.sin(lat[i]) * np.cos(lat[sel]) * np.cos(dlon[sel]))
        onehot = np.zeros((len(kk), K))
        onehot[np.arange(len(kk)), kk] = 1.0
        E1 = np.exp(-1j * (beta[:, None] - beta[None, :]))
        for P, X, Y in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
            dP, wP = fields[P]
            dX, wX = fields[X]
            dY, wY = fields[Y]
            T = np.outer(wX[sel] * dX[sel], wY[sel] * dY[sel]).astype(complex)
            for m in range(M + 1):
                if m:
                    T = T * E1
                S[m] += wP[i] * dP[i] * (onehot.T @ T @ onehot)
            D += wP[i] * (onehot.T @ np.outer(wX[sel], wY[sel]) @ onehot)
    return S, D


@pytest.fixture(scope="module")
def multi_case():
    xyz = _cap_points(500, 8.0, seed=41)
    g = synth.rng(42)
    fields = tuple((g.standard_normal(len(xyz)) + 0.2 * c, g.uniform(0.5, 1.5, len(xyz))) for c in range(3))
    edges = np.array([0.7, 1.3, 2.0, 2.9])
    return xyz, fields, edges, 4


def test_multi_brute_force(multi_case):
    xyz, fields, edges, M = multi_case
    res = oracle.zeta_multi(xyz, fields, edges, M)
    assert res["min_margin"] > 1e-9
    Sb, Db = brute_force_multi(xyz, fields, edges, M)
    assert np.abs(res["S"] - Sb).max() < 1e-11 * np.abs(Sb).max()
    assert np.abs(res["D"] - Db).max() < 1e-11 * np.abs(Db).max()
    # the three fields really differ: zeta^{ABC} is not Hermitian
    z = res["zeta"]
    assert np.abs(z - np.conj(np.transpose(z, (0, 2, 1)))).max() > 1e-3 * np.abs(z).max()


def test_one_field_reduces_to_the_single_field_estimator(multi_case):
    xyz, fields, edges, M = multi_case
    d, w = fields[0]
    multi = oracle.zeta_multi(xyz, (fields[0],) * 3, edges, M)
    single = oracle.zeta(xyz, d, w, edges, M)
    np.testing.assert_allclose(multi["S"], 3 * single["S"], rtol=1e-12, atol=1e-12 * np.abs(single["S"]).max())
    np.testing.assert_allclose(multi["D"], 3 * single["D"], rtol=1e-12)
    np.testing.assert_allclose(multi["zeta"], single["zeta"], rtol=1e-11, atol=1e-12 * np.abs(single["zeta"]).max())


def test_cyclic_invariance_and_neighbour_swap(multi_case):
    xyz, (A, B, C), edges, M = multi_case
    abc = oracle.zeta_multi(xyz, (A, B, C), edges, M)["zeta"]
    bca = oracle.zeta_multi(xyz, (B, C, A), edges, M)["zeta"]
    acb = oracle.zeta_multi(xyz, (A, C, B), edges, M)["zeta"]
    scale = np.abs(abc).max()
    assert np.abs(bca - abc).max() < 1e-12 * scale
    assert np.abs(acb - np.conj(np.transpose(abc, (0, 2, 1)))).max() < 1e-12 * scale


def test_linear_in_each_field(multi_case):
    xyz, (A, B, C), edges, M = multi_case
    A2 = (synth.rng(43).standard_normal(len(xyz)), A[1])
    c = -0.7
    Amix = (A[0] + c * A2[0], A[1])
    s1 = oracle.zeta_multi(xyz, (A, B, C), edges, M)["S"]
    s2 = oracle.zeta_multi(xyz, (A2, B, C), edges, M)["S"]
    sm = oracle.zeta_multi(xyz, (Amix, B, C), edges, M)["S"]
    assert np.abs(sm - (s1 + c * s2)).max() < 1e-11 * np.abs(sm).max()
