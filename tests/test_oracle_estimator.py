"""Pins for the oracle's estimator (arXiv:2408.16847 section 3.1).

Each test checks the oracle against something it does not compute itself:

* brute force: the O(N N_p^2) triplet sum of eq. zeta/zetahom written with
  navigation trigonometry (haversine separation, initial-bearing position angle),
  with the j = k self term kept (the paper's estimator, section 3.4) or removed;
* a hand-worked three-point example that fixes the orientation and conjugation
  convention (phi from north through east, a_m = sum w d e^{-i m phi});
* m = 0 reduces to products of weighted pair counts, taken from scipy's k-d tree;
* closed forms for a constant field;
* the invariances the paper states: per-pivot reference direction (after eq.
  zetamEst2), rotation of the catalogue, reflection flips Im zeta (end of 3.1),
  Hermitian symmetry, Im zeta_m(theta, theta) = 0 on the diagonal (section 3.4);
* the adjoint: exact central differences (the loss is quadratic in each single
  d_p because a point is never its own neighbour) and Euler's identity for the
  homogeneous cubic, sum_p d_p dL/dd_p = 3 L;
* the catalogue D-R composition: data placed on the randoms' positions with a
  constant weight cancel the randoms exactly (S = 0), and the d = 1 data-only
  normalisation equals alpha^3 D_R.
"""
import math

import numpy as np
import pytest
from scipy.spatial import cKDTree

import oracle
import synth


def _cap_points(n, radius_deg, seed, centre=(0.3, -0.5, 0.81)):
    g = synth.rng(seed)
    c = np.asarray(centre, dtype=float)
    c /= np.linalg.norm(c)
    zc = g.uniform(math.cos(math.radians(radius_deg)), 1.0, n)
    ph = g.uniform(0, 2 * math.pi, n)
    s = np.sqrt(1 - zc * zc)
    local = np.stack([s * np.cos(ph), s * np.sin(ph), zc], axis=1)
    # rotate +z onto c
    zax = np.array([0.0, 0.0, 1.0])
    v = np.cross(zax, c)
    sv = np.linalg.norm(v)
    cv = float(zax @ c)
    vx = np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])
    R = np.eye(3) + vx + vx @ vx * ((1 - cv) / (sv * sv))
    return local @ R.T


def _latlon(xyz):
    return np.arcsin(np.clip(xyz[:, 2], -1, 1)), np.arctan2(xyz[:, 1], xyz[:, 0])


def brute_force_S(xyz, delta, w, edges_deg, M, keep_self=True):
    """Triplet sum  S_m(k1,k2) = sum_i w_i d_i sum_{j,l} w_j d_j w_l d_l
    Theta_k1(ij) Theta_k2(il) exp(-i m (beta_ij - beta_il)),  beta = initial bearing.
    The phase matrix of each pivot is raised to the m-th power elementwise."""
    lat, lon = _latlon(xyz)
    th_e = np.deg2rad(np.asarray(edges_deg))
    K = len(th_e) - 1
    S = np.zeros((M + 1, K, K), dtype=complex)
    wd = w * delta
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
                          math.cos(lat[i]) * np.sin(lat[sel])
                          - math.sin(lat[i]) * np.cos(lat[sel]) * np.cos(dlon[sel]))
        x = wd[sel]
        onehot = np.zeros((len(kk), K))
        onehot[np.arange(len(kk)), kk] = 1.0
        E1 = np.exp(-1j * (beta[:, None] - beta[None, :]))
        T = (x[:, None] * x[None, :]).astype(complex)
        if not keep_self:
            np.fill_diagonal(T, 0.0)
        for m in range(M + 1):
            if m:
                T = T * E1
            S[m] += wd[i] * (onehot.T @ T @ onehot)
    return S


@pytest.fixture(scope="module")
def brute_case():
    """About 2000 points in a 10 deg cap, ~170 neighbours per pivot in 4 bins."""
    xyz = _cap_points(2000, 10.0, seed=11)
    g = synth.rng(12)
    delta = g.standard_normal(len(xyz))
    w = g.uniform(0.5, 1.5, len(xyz))
    edges = np.array([0.6, 1.1, 1.7, 2.4, 3.2])
    return xyz, delta, w, edges, 5


@pytest.fixture(scope="module")
def cap_case():
    xyz = _cap_points(700, 12.0, seed=11)
    g = synth.rng(12)
    delta = g.standard_normal(len(xyz))
    w = g.uniform(0.5, 1.5, len(xyz))
    edges = np.array([1.0, 1.7, 2.9, 4.6, 7.0])
    return xyz, delta, w, edges, 5


@pytest.mark.parametrize("keep", [True, False])
def test_brute_force_triplets(brute_case, keep):
    xyz, delta, w, edges, M = brute_case
    res = oracle.zeta(xyz, delta, w, edges, M, self_pairs="keep" if keep else "subtract")
    assert res["min_margin"] > 1e-9  # no pair sits on a bin edge: both bin the same way
    Sb = brute_force_S(xyz, delta, w, edges, M, keep_self=keep)
    scale = np.abs(Sb).max()
    assert np.abs(res["S"] - Sb).max() < 1e-11 * scale


def test_hand_worked_orientation():
    """Pivot P on the equator at longitude 0, A at angle d due north of P, B at 1.5 d
    due east.  Bins [0.5d,1.2d) and [1.2d,1.6d); |AB| = 1.80 d is outside every bin.
    d_P = 1, d_A = 2, d_B = 3, unit weights.  By hand:
      a^0(P) = 2, a^1_m(P) = 3 e^{-i m pi/2};  A sees P due south (phi = pi),
      B sees P due west (phi = -pi/2);  so
      zeta_m(0,1) = S_m(0,1)/D(0,1) = 1 * 2 * conj(3 (-i)^m) / 1 = 6 i^m,
      S_m(0,0) = 1*4 + 2*1 = 6,  S_m(1,1) = 1*9 + 3*1 = 12,  D(0,0) = 1+2... (w = 1)."""
    d = math.radians(2.0)
    P = np.array([1.0, 0.0, 0.0])
    A = np.array([math.cos(d), 0.0, math.sin(d)])
    B = np.array([math.cos(1.5 * d), math.sin(1.5 * d), 0.0])
    xyz = np.stack([P, A, B])
    delta = np.array([1.0, 2.0, 3.0])
    w = np.ones(3)
    edges = np.rad2deg(np.array([0.5 * d, 1.2 * d, 1.6 * d]))
    res = oracle.zeta(xyz, delta, w, edges, 4)
    S, D, z = res["S"], res["D"], res["zeta"]
    for m in range(5):
        np.testing.assert_allclose(z[m, 0, 1], 6 * (1j ** m), atol=1e-12)
        np.testing.assert_allclose(z[m, 1, 0], np.conj(6 * (1j ** m)), atol=1e-12)
        # S(0,0): P (wd 1) * |2|^2 + A (wd 2) * |(-1)^m|^2
        np.testing.assert_allclose(S[m, 0, 0], 4 + 2, atol=1e-12)
        # S(1,1): P * |3|^2 + B (wd 3) * |i^m|^2
        np.testing.assert_allclose(S[m, 1, 1], 9 + 3, atol=1e-12)
    # D: P has W = (1,1); A has W = (1,0); B has W = (0,1)
    np.testing.assert_allclose(D, [[2, 1], [1, 2]], atol=1e-12)
    assert res["pairs"] == 4


def test_m0_is_pair_counts(cap_case):
    xyz, delta, w, edges, M = cap_case
    res = oracle.zeta(xyz, delta, w, edges, 0)
    ce = 2 * np.sin(np.deg2rad(edges) / 2)
    tree = cKDTree(xyz)
    wd = w * delta
    K = len(edges) - 1
    P = np.zeros((len(xyz), K))
    Wc = np.zeros((len(xyz), K))
    for e in range(K + 1):
        # weighted counts strictly inside chord ce[e], excluding the point itself
        lists = tree.query_ball_point(xyz, ce[e] * (1 - 1e-12))
        cum = np.array([wd[l].sum() - wd[i] for i, l in enumerate(lists)])
        cumw = np.array([w[l].sum() - w[i] for i, l in enumerate(lists)])
        if e > 0:
            P[:, e - 1] += cum
            Wc[:, e - 1] += cumw
        if e < K:
            P[:, e] -= cum
            Wc[:, e] -= cumw
    S0 = np.einsum("i,ik,il->kl", wd, P, P)
    D = np.einsum("i,ik,il->kl", w, Wc, Wc)
    np.testing.assert_allclose(res["S"][0].real, S0, rtol=1e-11, atol=1e-9)
    np.testing.assert_allclose(res["D"], D, rtol=1e-11, atol=1e-9)
    assert np.abs(res["S"][0].imag).max() < 1e-12


def test_constant_field_closed_form(cap_case):
    xyz, _, w, edges, M = cap_case
    c = 1.7
    r1 = oracle.zeta(xyz, np.ones(len(xyz)), w, edges, M)
    rc = oracle.zeta(xyz, np.full(len(xyz), c), w, edges, M)
    np.testing.assert_allclose(rc["S"], c ** 3 * r1["S"], rtol=1e-12, atol=1e-12)
    D = r1["D"]
    np.testing.assert_allclose(rc["zeta"][0].real[D > 0], c ** 3, rtol=1e-12)
    # R2 of a constant field: every per-bin average is the constant itself
    r2 = oracle.zeta(xyz, np.full(len(xyz), c), w, edges, M, norm="R2")
    W = r2["moments"]["W"]
    full = np.all(W > 0, axis=0)
    if full.any():
        frac = np.einsum("i,ik,il->kl", w, (W > 0).astype(float), (W > 0).astype(float)) / w.sum()
        np.testing.assert_allclose(r2["zeta"][0].real, c ** 3 * frac, rtol=1e-12)


def _rotation(seed):
    q = synth.rng(seed).standard_normal(4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([[a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
                     [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
                     [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d]])


def test_invariances(cap_case):
    xyz, delta, w, edges, M = cap_case
    base = oracle.zeta(xyz, delta, w, edges, M)
    z0 = base["zeta"]
    scale = np.abs(z0).max()
    # rotation of the whole catalogue
    R = _rotation(5)
    rot = oracle.zeta(xyz @ R.T, delta, w, edges, M)
    assert np.abs(rot["zeta"] - z0).max() < 1e-10 * scale
    # per-pivot reference direction
    psi = synth.rng(6).uniform(0, 2 * math.pi, len(xyz))
    ps = oracle.zeta(xyz, delta, w, edges, M, psi=psi)
    assert np.abs(ps["zeta"] - z0).max() < 1e-10 * scale
    # mirror reflection: Re unchanged, Im flips
    mir = oracle.zeta(xyz * np.array([1.0, -1.0, 1.0]), delta, w, edges, M)
    assert np.abs(mir["zeta"].real - z0.real).max() < 1e-10 * scale
    assert np.abs(mir["zeta"].imag + z0.imag).max() < 1e-10 * scale
    assert np.abs(z0[1:].imag).max() > 1e-6 * scale  # the flip is not vacuous
    # Hermitian, Im zeta_0 = 0, diagonal Im = 0
    assert np.abs(z0 - np.conj(np.transpose(z0, (0, 2, 1)))).max() < 1e-13 * scale
    assert np.abs(z0[0].imag).max() < 1e-13 * scale
    K = z0.shape[1]
    assert np.abs(z0[:, np.arange(K), np.arange(K)].imag).max() < 1e-13 * scale


@pytest.mark.parametrize("self_pairs", ["keep", "subtract"])
def test_gradient_exact_fd_and_euler(cap_case, self_pairs):
    xyz, delta, w, edges, M = cap_case
    K = len(edges) - 1
    g = synth.rng(21)
    cot = g.standard_normal((M + 1, K, K)) + 1j * g.standard_normal((M + 1, K, K))

    def L(d):
        z = oracle.zeta(xyz, d, w, edges, M, self_pairs=self_pairs)["zeta"]
        return float(np.sum(cot.real * z.real + cot.imag * z.imag))

    grad = oracle.gradient(xyz, delta, w, edges, M, cot, self_pairs=self_pairs)
    L0 = L(delta)
    # Euler's identity for a homogeneous cubic
    assert abs(np.dot(delta, grad) - 3 * L0) < 1e-10 * max(1.0, abs(L0))
    # central differences are exact (quadratic in each single d_p)
    for p in [0, 17, 301, 650]:
        h = 0.75
        dp = delta.copy()
        dm = delta.copy()
        dp[p] += h
        dm[p] -= h
        fd = (L(dp) - L(dm)) / (2 * h)
        assert abs(fd - grad[p]) < 1e-9 * max(1.0, abs(grad[p]))


def test_gradient_pivot_subset(cap_case):
    """Restricting the pivots restricts the loss; targets may lie outside the pivots."""
    xyz, delta, w, edges, M = cap_case
    K = len(edges) - 1
    cot = synth.rng(22).standard_normal((M + 1, K, K))
    piv = np.arange(100, 400)

    def L(d):
        z = oracle.zeta(xyz, d, w, edges, M, pivots=piv)["zeta"]
        return float(np.sum(cot * z.real))

    tg = np.array([5, 150, 399, 600])
    grad = oracle.gradient(xyz, delta, w, edges, M, cot, pivots=piv, targets=tg)
    for t, p in enumerate(tg):
        dp = delta.copy()
        dm = delta.copy()
        dp[p] += 0.5
        dm[p] -= 0.5
        fd = (L(dp) - L(dm)) / 1.0
        assert abs(fd - grad[t]) < 1e-9 * max(1.0, abs(grad[t]))


def test_map_is_catalogue_of_centres():
    """A map is the estimator on its pixel centres: the pair count of Nside 16 with
    one bin [pixel-scale, 8 deg) agrees with scipy's k-d tree."""
    n = 16
    xyz = oracle.pix2vec_ring(n)
    edges = np.array([0.5, 8.0])
    cnt = oracle.pair_counts(xyz, edges)
    tree = cKDTree(xyz)
    ce = 2 * np.sin(np.deg2rad(edges) / 2)
    hi = np.array([len(l) for l in tree.query_ball_point(xyz, ce[1] * (1 - 1e-12))])
    lo = np.array([len(l) for l in tree.query_ball_point(xyz, ce[0] * (1 - 1e-12))])
    np.testing.assert_array_equal(cnt, hi - lo)


def test_r1_normalisation_of_a_constant_field(cap_case):
    """R1 (eq. Xm.binned's prefactor: each pivot's moments over the weight of all its
    neighbours, then eq. zetamEst's 1/sum w) for delta = c: zeta_0(k1,k2) =
    c^3 sum_i w_i W^k1(i) W^k2(i) / Wtot(i)^2 / sum_i w_i, with the per-pivot bin weights
    taken from cKDTree counts (independent of the oracle's neighbour search)."""
    xyz, _, w, edges, M = cap_case
    c = -0.8
    r1 = oracle.zeta(xyz, np.full(len(xyz), c), w, edges, M, norm="R1")
    ce = 2 * np.sin(np.deg2rad(edges) / 2)
    tree = cKDTree(xyz)
    K = len(edges) - 1
    Wc = np.zeros((len(xyz), K))
    for e in range(K + 1):
        lists = tree.query_ball_point(xyz, ce[e] * (1 - 1e-12))
        cumw = np.array([w[l].sum() - w[i] for i, l in enumerate(lists)])
        if e > 0:
            Wc[:, e - 1] += cumw
        if e < K:
            Wc[:, e] -= cumw
    tot = Wc.sum(axis=1)
    live = tot > 0
    ref = c ** 3 * np.einsum("i,ik,il->kl", w[live], Wc[live] / tot[live, None], Wc[live] / tot[live, None]) / w.sum()
    np.testing.assert_allclose(r1["zeta"][0].real, ref, rtol=1e-11, atol=1e-14)
    assert np.abs(r1["zeta"][0].imag).max() < 1e-14


def test_catalog_zeta_randoms_cancel_data():
    """D-R composition, data at the randoms' positions with a constant weight c: then
    alpha = sum w_D / n_R = c, and every position carries w d = c (data) and -alpha
    (random), so every union moment a_m^k vanishes and S = 0 up to rounding.  A wrong
    alpha or a sign slip on the randoms leaves S of the order of the data-only S."""
    xyz = _cap_points(2000, 10.0, seed=31)
    edges = np.array([0.6, 1.1, 1.7, 2.4, 3.2])
    M = 4
    for c in (1.0, 1.3):
        wd = np.full(len(xyz), c)
        res = oracle.catalog_zeta(xyz, wd, xyz, edges, M)
        assert res["alpha"] == pytest.approx(c, rel=1e-15)
        data_only = oracle.zeta(xyz, np.ones(len(xyz)), wd, edges, M)["S"]
        scale = np.abs(data_only).max()
        assert scale > 0
        assert np.abs(res["S"]).max() < 1e-12 * scale


def test_catalog_zeta_normalisation_is_alpha_cubed():
    """Same layout (data at the randoms' positions, weight c): the D-R denominator
    alpha^3 D_R must equal the d = 1 estimator run on the data alone, whose every
    weight is c, i.e. sum_i c (c W^k1)(c W^k2) = c^3 D_R.  alpha or alpha^2 in place of
    alpha^3 fails.  zeta is S over that denominator."""
    xyz = _cap_points(2000, 10.0, seed=32)
    edges = np.array([0.6, 1.1, 1.7, 2.4, 3.2])
    M = 3
    c = 1.7
    wd = np.full(len(xyz), c)
    res = oracle.catalog_zeta(xyz, wd, xyz, edges, M)
    Dd = oracle.zeta(xyz, np.ones(len(xyz)), wd, edges, M)["D"]
    np.testing.assert_allclose(res["D"], Dd, rtol=1e-12)
    DR = oracle.zeta(xyz, np.ones(len(xyz)), np.ones(len(xyz)), edges, M)["D"]
    assert np.abs(Dd - c ** 2 * DR).max() > 0.1 * np.abs(Dd).max()  # alpha^2 would be caught
    # ratio: data at other positions; zeta = S / (alpha^3 D_R) entry by entry
    xd = _cap_points(1500, 10.0, seed=33)
    wd2 = synth.rng(34).uniform(0.5, 1.5, len(xd))
    r2 = oracle.catalog_zeta(xd, wd2, xyz, edges, M)
    alpha = wd2.sum() / len(xyz)
    np.testing.assert_allclose(r2["D"], alpha ** 3 * DR, rtol=1e-12)
    live = DR > 0
    np.testing.assert_allclose(r2["zeta"][:, live], r2["S"][:, live] / (alpha ** 3 * DR[live])[None], rtol=1e-12)
