"""Pivot sharding across ranks (paper_2408_16847_gb300.shard), on CPU ranks.

Two gloo processes each run the oracle over their pivot range behind a plan-like
adapter; shard.py's host logic (balanced ranges, all-reduce of S and D, all-reduce
of the partial gradients) must give the single-process oracle result.  No GPU: the
per-rank compute is the oracle, the transport is gloo.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth

NSIDE, M = 8, 6
EDGES = np.array([3.1, 9.3, 17.9, 30.7])


def _field():
    d = synth.bump_map(NSIDE, 300, (3.0, 10.0), 0.5, 0.05, seed=synth.BASE_SEED + 960)
    w = synth.galactic_mask_weights(NSIDE) * synth.rng(961).uniform(0.5, 1.5, 12 * NSIDE * NSIDE)
    return d, w


class OraclePlan:
    """Plan-like adapter over the oracle (test only): forward / backward on a pivot range."""

    def __init__(self, xyz):
        self.xyz = xyz

    def forward(self, delta, w, pivots, want_sums=False):
        lo, hi = pivots
        r = oracle.zeta(self.xyz, delta.numpy(), w.numpy(), EDGES, M, pivots=np.arange(lo, hi))
        S = torch.from_numpy(np.stack([r["S"].real, r["S"].imag], axis=-1).copy())
        D = torch.from_numpy(r["D"].copy())
        return None, D, S

    def backward(self, delta, w, norm, dL, pivots):
        lo, hi = pivots
        # the oracle's adjoint takes D from its own pivots; the shard passes the global
        # one, so rescale: for fixed D the adjoint is linear in dL / D
        r = oracle.zeta(self.xyz, delta.numpy(), w.numpy(), EDGES, M, pivots=np.arange(lo, hi))
        Dg = norm.numpy()
        with np.errstate(divide="ignore", invalid="ignore"):
            scale = np.where(Dg != 0, r["D"] / np.where(Dg == 0, 1.0, Dg), 0.0)
        c = (dL[..., 0].numpy() + 1j * dL[..., 1].numpy()) * scale[None]
        g = oracle.gradient(self.xyz, delta.numpy(), w.numpy(), EDGES, M, c, pivots=np.arange(lo, hi))
        return torch.from_numpy(g.astype(np.float64))


def _cpu_normalize(S, D):
    with np.errstate(divide="ignore", invalid="ignore"):
        d = D.numpy()
        z = np.where(d[None, ..., None] != 0, S.numpy() / np.where(d == 0, 1.0, d)[None, ..., None], 0.0)
    return torch.from_numpy(z)


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2408_16847_gb300 import shard
        d, w = _field()
        xyz = oracle.pix2vec_ring(NSIDE)
        plan = OraclePlan(xyz)
        dt, wt = torch.from_numpy(d), torch.from_numpy(w)
        zeta, D = shard.sharded_forward(plan, dt, wt, normalize=_cpu_normalize)
        K = len(EDGES) - 1
        cot = synth.rng(962).standard_normal((M + 1, K, K, 2))
        g = shard.sharded_backward(plan, dt, wt, D, torch.from_numpy(cot))
        np.save(os.path.join(out_dir, "zeta_%d.npy" % rank), zeta.numpy())
        np.save(os.path.join(out_dir, "grad_%d.npy" % rank), g.numpy())
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_balanced_ranges_cover_and_balance():
    from paper_2408_16847_gb300 import shard
    w = torch.from_numpy(synth.galactic_mask_weights(32))
    for world in (1, 2, 3, 4, 7):
        rs = shard.balanced_ranges(w, world)
        assert rs[0][0] == 0 and rs[-1][1] == w.numel()
        assert all(rs[i][1] == rs[i + 1][0] for i in range(world - 1))
        live = [int((w[a:b] != 0).sum()) for a, b in rs]
        assert max(live) - min(live) <= 1, live
    assert shard.balanced_ranges(torch.zeros(10), 3)[-1] == (6, 10)


def test_two_gloo_ranks_match_single_process(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    d, w = _field()
    xyz = oracle.pix2vec_ring(NSIDE)
    ref = oracle.zeta(xyz, d, w, EDGES, M)
    K = len(EDGES) - 1
    cot = synth.rng(962).standard_normal((M + 1, K, K, 2))
    gref = oracle.gradient(xyz, d, w, EDGES, M, cot[..., 0] + 1j * cot[..., 1])
    for r in range(world):
        z = np.load(tmp_path / ("zeta_%d.npy" % r))
        zc = z[..., 0] + 1j * z[..., 1]
        assert np.abs(zc - ref["zeta"]).max() <= 1e-12 * np.abs(ref["zeta"]).max()
        g = np.load(tmp_path / ("grad_%d.npy" % r))
        assert np.abs(g - gref).max() <= 1e-10 * np.abs(gref).max()
