"""Pins for the oracle's m-coupling (edge) correction, edge_correct: the D - R estimate
of zeta(phi) = N(phi) / R(phi) in harmonic space, S_m = sum_m' z_m' R_{m-m'}.

* no coupling (R_n = 0 for n != 0): the correction is the plain ratio S / (scale R_0);
* a known zeta(phi) on a random triplet-angle density: S is summed directly from the
  angles (not from the convolution), and edge_correct recovers the z_m;
* data at the randoms' positions with a constant field c on an irregular patch: N(phi)
  = c^3 R(phi) exactly, so the corrected estimate is c^3 at m = 0 and 0 above, while the
  uncorrected ratio S_m / R_0 carries the patch's own multipoles.
"""
import numpy as np
import pytest

import oracle
import synth
from test_oracle_estimator import _cap_points


def test_no_coupling_is_the_plain_ratio():
    g = synth.rng(1600)
    M, K = 5, 3
    S = g.standard_normal((M + 1, K, K)) + 1j * g.standard_normal((M + 1, K, K))
    S[0] = S[0].real
    R = np.zeros((2 * M + 1, K, K), dtype=complex)
    R[0] = g.uniform(1.0, 2.0, (K, K))
    z = oracle.edge_correct(S, R, 0.37)
    np.testing.assert_allclose(z, S / (0.37 * R[0])[None], rtol=1e-13, atol=0)


def test_known_zeta_is_recovered_from_a_triplet_angle_density():
    g = synth.rng(1601)
    M, K = 4, 2
    S = np.zeros((M + 1, K, K), dtype=complex)
    R = np.zeros((2 * M + 1, K, K), dtype=complex)
    Z = np.zeros((M + 1, K, K), dtype=complex)
    for k1 in range(K):
        for k2 in range(K):
            # triplet angles phi_t with weights, clustered so that R(phi) is far from flat
            phi = np.concatenate([g.uniform(-np.pi, np.pi, 150), g.normal(0.7, 0.3, 100)])
            wt = g.uniform(0.2, 1.0, len(phi))
            z = g.standard_normal(M + 1) + 1j * g.standard_normal(M + 1)
            z[0] = z[0].real
            zeta_phi = z[0].real + 2 * sum((z[m] * np.exp(1j * m * phi)).real for m in range(1, M + 1))
            for n in range(2 * M + 1):
                R[n, k1, k2] = np.sum(wt * np.exp(-1j * n * phi))
            for m in range(M + 1):
                S[m, k1, k2] = np.sum(wt * zeta_phi * np.exp(-1j * m * phi))
            Z[:, k1, k2] = z
    got = oracle.edge_correct(S, R)
    np.testing.assert_allclose(got, Z, rtol=0, atol=1e-10 * np.abs(Z).max())
    # the uncorrected ratio is visibly biased by the clustered density
    assert np.abs(S / R[0][None] - Z).max() > 1e-2 * np.abs(Z).max()


@pytest.fixture(scope="module")
def patch():
    """An irregular patch: a 9-degree cap with an off-centre wedge cut out, so its
    triplet-angle density has odd and imaginary multipoles."""
    xyz = _cap_points(900, 9.0, seed=1602)
    lon = np.arctan2(xyz[:, 1], xyz[:, 0])
    keep = ~((lon > 0.3) & (lon < 1.6) & (xyz[:, 2] < np.cos(np.deg2rad(3.0))))
    return xyz[keep]


def test_constant_field_on_a_patch_is_corrected_to_a_constant(patch):
    xyz = patch
    n = len(xyz)
    c, M = 1.7, 4
    edges = np.array([0.8, 1.9, 3.1, 4.4])
    data = oracle.zeta(xyz, np.full(n, c), np.ones(n), edges, M)
    rand = oracle.zeta(xyz, np.ones(n), np.ones(n), edges, 2 * M)
    assert data["min_margin"] > 1e-9 and rand["min_margin"] > 1e-9
    R = rand["S"]
    # the patch couples multipoles: R_m off the diagonal is complex, |R_m| not small
    assert np.abs(R[1:].imag).max() > 1e-4 * np.abs(R[0]).max()
    z = oracle.edge_correct(data["S"], R, 1.0)
    scale = c ** 3
    np.testing.assert_allclose(z[0].real, scale, rtol=1e-9)
    assert np.abs(z[0].imag).max() < 1e-9 * scale
    assert np.abs(z[1:]).max() < 1e-9 * scale
    naive = data["S"] / R[0][None]
    assert np.abs(naive[1:]).max() > 1e-2 * scale


def test_coupled_catalogue_estimate_composes_the_pieces(patch):
    xyz_r = patch
    g = synth.rng(1603)
    xyz_d = xyz_r[g.choice(len(xyz_r), 300, replace=False)]
    w_d = g.uniform(0.5, 1.5, len(xyz_d))
    edges = np.array([0.8, 1.9, 3.1])
    M = 3
    res = oracle.catalog_zeta_coupled(xyz_d, w_d, xyz_r, edges, M)
    plain = oracle.catalog_zeta(xyz_d, w_d, xyz_r, edges, M)
    r = oracle.zeta(xyz_r, np.ones(len(xyz_r)), np.ones(len(xyz_r)), edges, 2 * M)
    np.testing.assert_allclose(res["S"], plain["S"])
    np.testing.assert_allclose(res["R"], r["S"])
    np.testing.assert_allclose(res["zeta"], oracle.edge_correct(plain["S"], r["S"], plain["alpha"] ** 3))
    # R_0 of the randoms is the plain estimate's D_R
    np.testing.assert_allclose(r["S"][0].real, plain["D"] / plain["alpha"] ** 3, rtol=1e-12)
