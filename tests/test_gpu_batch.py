"""Batched, graph-captured execution of several map plans vs single calls and the oracle."""
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


# (nside, edges in degrees, m_max, self-pair mode): mixed sizes, bin counts and M,
# two plans sharing an M (one work queue), one with self-pair subtraction
CASES = [
    (8, [2.03, 10.3, 20.7], 4, "keep"),
    (16, list(np.geomspace(1.53, 25.1, 6)), 8, "keep"),
    (16, [1.7, 6.3, 13.9], 4, "keep"),
    (32, list(np.geomspace(0.8, 12.0, 8)), 10, "keep"),
    (4, [3.1, 10.3, 25.7, 44.9], 0, "keep"),
    (16, list(np.geomspace(1.5, 20.0, 5)), 6, "subtract"),
]


def _inputs(i, nside):
    d = synth.bump_map(nside, 40 * nside, (2.0, 8.0), 0.5, 0.05, seed=synth.BASE_SEED + 700 + i).astype(np.float32)
    w = synth.rng(720 + i).uniform(0.5, 1.5, 12 * nside * nside).astype(np.float32)
    return d, w


def _outs(plan):
    dev = "cuda:0"
    z = torch.zeros((plan.M + 1, plan.K, plan.K, 2), dtype=torch.float64, device=dev)
    n = torch.zeros((plan.K, plan.K), dtype=torch.float64, device=dev)
    return z, n


def test_batch_forward_matches_single_calls_and_oracle():
    tpcf = _tpcf()
    plans, ds, ws, zs, ns = [], [], [], [], []
    host = []
    for i, (nside, edges, M, sp) in enumerate(CASES):
        p = tpcf.Plan.map(nside, np.asarray(edges), M, self_pairs=sp)
        d, w = _inputs(i, nside)
        host.append((d, w))
        plans.append(p)
        ds.append(to_dev(d))
        ws.append(to_dev(w))
        z, n = _outs(p)
        zs.append(z)
        ns.append(n)
    b = tpcf.Batch(plans, ds, ws, zs, ns)
    # one persistent pair kernel for every plan: pack, zero, forward, reduce, finalize
    assert b.kernel_launches() == 5
    for replay in range(2):
        for z in zs:
            z.fill_(float("nan"))
        b.launch()
        torch.cuda.synchronize()
        for i, p in enumerate(plans):
            p.sync()
            z1, n1 = p.forward(ds[i], ws[i])
            torch.cuda.synchronize()
            zb = tpcf.as_complex(zs[i]).cpu().numpy()
            zo = tpcf.as_complex(z1).cpu().numpy()
            assert np.isfinite(zb).all()
            assert np.abs(zb - zo).max() <= 1e-6 * max(np.abs(zo).max(), 1e-300), (replay, i)
            # D is summed in fp32 within a tile (shared-memory atomics, unordered)
            np.testing.assert_allclose(ns[i].cpu().numpy(), n1.cpu().numpy(), rtol=1e-6, atol=0)
    for i, (nside, edges, M, sp) in enumerate(CASES):
        d, w = host[i]
        ref = oracle.zeta(oracle.pix2vec_ring(nside), d.astype(np.float64), w.astype(np.float64),
                          np.asarray(edges), M, self_pairs=sp)
        assert ref["min_margin"] > 1e-12
        zb = tpcf.as_complex(zs[i]).cpu().numpy()
        e = rel_err_per_m(zb, ref["zeta"])
        assert e.max() < TOL, (i, e)
    b.close()


def test_batch_adjoint_matches_single_calls():
    tpcf = _tpcf()
    cases = [c for c in CASES if c[3] == "keep"]
    plans, ds, ws, zs, ns, dls, gs = [], [], [], [], [], [], []
    for i, (nside, edges, M, sp) in enumerate(cases):
        p = tpcf.Plan.map(nside, np.asarray(edges), M)
        d, w = _inputs(i, nside)
        plans.append(p)
        ds.append(to_dev(d))
        ws.append(to_dev(w))
        z, n = _outs(p)
        zs.append(z)
        ns.append(n)
        g = torch.from_numpy(synth.rng(740 + i).standard_normal((M + 1, p.K, p.K, 2))).to("cuda:0")
        dls.append(g)
        gs.append(torch.full((12 * nside * nside,), float("nan"), dtype=torch.float32, device="cuda:0"))
    b = tpcf.Batch(plans, ds, ws, zs, ns, dls, gs)
    # pack, zero, forward, reduce, finalize, adjoint coefficients, adjoint
    assert b.kernel_launches() == 7
    b.launch()
    torch.cuda.synchronize()
    for i, p in enumerate(plans):
        p.sync()
        z1, n1 = p.forward(ds[i], ws[i])
        g1 = p.backward(ds[i], ws[i], n1, dls[i])
        torch.cuda.synchronize()
        gb, go = gs[i].cpu().numpy(), g1.cpu().numpy()
        assert np.isfinite(gb).all()
        assert np.abs(gb - go).max() <= 1e-5 * np.abs(go).max(), i
    # the gradient of one batch member against the oracle
    nside, edges, M, _ = cases[1]
    d, w = _inputs(1, nside)
    gref = oracle.gradient(oracle.pix2vec_ring(nside), d.astype(np.float64), w.astype(np.float64),
                           np.asarray(edges), M, tpcf.as_complex(dls[1]).cpu().numpy())
    assert np.abs(gs[1].cpu().numpy() - gref).max() < TOL * np.abs(gref).max()
    b.close()


def test_batch_rejects_bad_members():
    tpcf = _tpcf()
    p = tpcf.Plan.map(8, np.array([2.03, 10.3]), 2)
    d, w = _inputs(0, 8)
    z, n = _outs(p)
    dd, wd = to_dev(d), to_dev(w)
    with pytest.raises(tpcf.TpcfError) as e:
        tpcf.Batch([p, p], [dd, dd], [wd, wd], [z, z], [n, n])
    assert e.value.status == 1
    q = tpcf.Plan.map(8, np.array([2.03, 10.3]), 2, self_pairs="subtract")
    g = torch.zeros((3, 1, 1, 2), dtype=torch.float64, device="cuda:0")
    gr = torch.zeros(768, dtype=torch.float32, device="cuda:0")
    with pytest.raises(tpcf.TpcfError) as e:
        tpcf.Batch([q], [dd], [wd], [z], [n], [g], [gr])
    assert e.value.status == 5


def test_batch_members_of_the_mixed_nside_workload():
    """The first four maps of the 64-map batched workload (Nside 256, 512, 1024, 2048,
    their own bins and m_max) at full size, forward + adjoint in one graph replay:
    every zeta equals the single-call forward, the two smaller maps' gradients equal
    the single-call adjoint, and the Nside 2048 member matches the oracle on sampled
    pivots of the belt and of a polar cap."""
    import math
    tpcf = _tpcf()
    wls = synth.batched_maps(64)[:4]
    assert [wl.nside for wl in wls] == [256, 512, 1024, 2048]
    plans, ds, ws, zs, ns, dls, gs, host = [], [], [], [], [], [], [], []
    for wl in wls:
        K, M = wl.bins.nbins, wl.bins.m_max
        d = wl.delta().astype(np.float32)
        w = wl.weights().astype(np.float32)
        host.append((d, w))
        p = tpcf.Plan.map(wl.nside, wl.bins.edges_deg, M)
        plans.append(p)
        ds.append(to_dev(d))
        ws.append(to_dev(w))
        z, n = _outs(p)
        zs.append(z)
        ns.append(n)
        g = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device="cuda:0")
        g[..., 0] = torch.from_numpy(wl.cotangent()).to("cuda:0")
        dls.append(g)
        gs.append(torch.full((12 * wl.nside ** 2,), float("nan"), dtype=torch.float32, device="cuda:0"))
    b = tpcf.Batch(plans, ds, ws, zs, ns, dls, gs)
    b.launch()
    torch.cuda.synchronize()
    for i, p in enumerate(plans):
        p.sync()
        z1, n1 = p.forward(ds[i], ws[i])
        torch.cuda.synchronize()
        zb = tpcf.as_complex(zs[i]).cpu().numpy()
        zo = tpcf.as_complex(z1).cpu().numpy()
        assert np.isfinite(zb).all()
        assert rel_err_per_m(zb, zo).max() < 1e-6, i
        if i < 2:
            g1 = p.backward(ds[i], ws[i], n1, dls[i]).cpu().numpy()
            gb = gs[i].cpu().numpy()
            assert np.abs(gb - g1).max() <= 1e-5 * np.abs(g1).max(), i
    # Nside 2048 member: single calls on sampled pivots against the oracle
    wl, p = wls[3], plans[3]
    d, w = host[3]
    n = wl.nside
    from test_gpu_fullsize import oracle_on_band, ring_first
    for r in ((5 * n) // 4, 40):
        lo = ring_first(n, r)
        hi = lo + 160
        zg, _ = p.forward(ds[3], ws[3], (lo, hi))
        ref, _ = oracle_on_band(n, d, w, wl.bins.edges_deg, wl.bins.m_max, lo, hi, r, r)
        assert ref["min_margin"] > 1e-12
        assert rel_err_per_m(tpcf.as_complex(zg).cpu().numpy(), ref["zeta"]).max() < TOL, r
    b.close()
    for p in plans:
        p.close()
