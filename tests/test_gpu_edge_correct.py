"""tpcf_edge_correct (the m-coupling correction of a D - R estimate) against the
oracle's edge_correct on the same seeded sums, and the whole coupled catalogue
estimate (union forward at m <= M, randoms' delta = 1 forward at m <= 2M, correction)
against the oracle's catalog_zeta_coupled on an irregular patch."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_util import rel_err_per_m, to_dev
from test_oracle_estimator import _cap_points

pytestmark = pytest.mark.gpu


def _tpcf():
    from paper_2408_16847_gb300 import build
    build()
    from paper_2408_16847_gb300 import tpcf
    return tpcf


def _pack(c):
    return torch.from_numpy(np.ascontiguousarray(np.stack([c.real, c.imag], axis=-1))).to("cuda:0")


def _hermitian_sums(g, n, K, pos_def=False):
    """n multipoles of a K x K bin-pair array whose m = 0 entry is real on the diagonal
    pairs; with pos_def, the Fourier sums of a positive density per pair."""
    if pos_def:
        out = np.zeros((n, K, K), dtype=complex)
        for k1 in range(K):
            for k2 in range(K):
                phi = np.concatenate([g.uniform(-np.pi, np.pi, 80), g.normal(g.uniform(-3, 3), 0.4, 60)])
                wt = g.uniform(0.2, 1.0, len(phi))
                out[:, k1, k2] = [np.sum(wt * np.exp(-1j * m * phi)) for m in range(n)]
        return out
    out = g.standard_normal((n, K, K)) + 1j * g.standard_normal((n, K, K))
    out[0] = out[0].real
    return out


@pytest.mark.parametrize("M,K,scale", [(0, 3, 1.0), (3, 5, 0.37), (8, 4, 2.5), (16, 2, 1.0)])
def test_edge_correct_matches_oracle(cuda_device, M, K, scale):
    tpcf = _tpcf()
    g = synth.rng(1700 + 10 * M + K)
    S = _hermitian_sums(g, M + 1, K)
    R = _hermitian_sums(g, 2 * M + 1, K, pos_def=True)
    R[:, 0, 1] = 0.0  # an empty bin pair: zeta = 0
    ref = oracle.edge_correct(S, R, scale)
    z = tpcf.edge_correct(_pack(S), _pack(R), scale)
    torch.cuda.synchronize()
    zc = tpcf.as_complex(z).cpu().numpy()
    assert np.all(zc[:, 0, 1] == 0)
    np.testing.assert_allclose(zc, ref, rtol=0, atol=1e-10 * np.abs(ref).max())


def test_no_coupling_equals_normalize(cuda_device):
    tpcf = _tpcf()
    g = synth.rng(1710)
    M, K = 5, 4
    S = _hermitian_sums(g, M + 1, K)
    R = np.zeros((2 * M + 1, K, K), dtype=complex)
    D = g.uniform(1.0, 3.0, (K, K))
    R[0] = D
    z = tpcf.edge_correct(_pack(S), _pack(R), 0.8)
    zn = tpcf.normalize(_pack(S), torch.from_numpy(D).to("cuda:0"), 0.8)
    torch.cuda.synchronize()
    np.testing.assert_allclose(z.cpu().numpy(), zn.cpu().numpy(), rtol=1e-14, atol=0)


def test_coupled_catalogue_estimate_vs_oracle(cuda_device):
    tpcf = _tpcf()
    xyz = _cap_points(6000, 9.0, seed=1720)
    lon = np.arctan2(xyz[:, 1], xyz[:, 0])
    xyz_r = xyz[~((lon > 0.3) & (lon < 1.6) & (xyz[:, 2] < np.cos(np.deg2rad(3.0))))]
    g = synth.rng(1721)
    xyz_d = xyz_r[g.choice(len(xyz_r), 1500, replace=False)] + 0.0
    w_d = g.uniform(0.5, 1.5, len(xyz_d))
    edges = np.array([0.5, 1.1, 1.9, 3.0])
    M = 3
    ref = oracle.catalog_zeta_coupled(xyz_d, w_d, xyz_r, edges, M)
    nd, nr = len(xyz_d), len(xyz_r)
    alpha = ref["alpha"]
    xyz_u = np.concatenate([xyz_d, xyz_r])
    du = np.concatenate([np.ones(nd), np.full(nr, -alpha)]).astype(np.float32)
    wu = np.concatenate([w_d, np.ones(nr)]).astype(np.float32)
    xu = torch.from_numpy(np.ascontiguousarray(xyz_u)).to("cuda:0")
    xr = torch.from_numpy(np.ascontiguousarray(xyz_r)).to("cuda:0")
    pu = tpcf.Plan.catalog(xu, edges, M)
    pr = tpcf.Plan.catalog(xr, edges, 2 * M)
    _, _, S = pu.forward(to_dev(du), to_dev(wu), want_sums=True)
    one = torch.ones(nr, dtype=torch.float32, device="cuda:0")
    _, _, R = pr.forward(one, one, want_sums=True)
    z = tpcf.edge_correct(S, R, alpha ** 3)
    torch.cuda.synchronize()
    zc = tpcf.as_complex(z).cpu().numpy()
    # the GPU sums carry fp32 rounding (1e-6 of the largest term); the solve amplifies it
    # by at most the condition number of the coupling matrix, which is small here
    assert rel_err_per_m(zc, ref["zeta"]).max() < 1e-4
    assert np.abs(zc[1:]).max() > 0
    pu.close()
    pr.close()
