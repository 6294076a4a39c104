"""Pivot sharding across ranks (paper_2408_16847_gb300.shard), on CPU ranks.

Two or three gloo processes each run the oracle over their pivot range behind a
plan-like adapter; shard.py's host logic (balanced ranges, all-reduce of S and D,
the adjoint over each gradient slice's halo and the gather of the slices) must give
the single-process oracle result.  A further case drops a rank between two steps:
the survivors learn of it through the store, form a new group and redo its pivots.
No GPU: the per-rank compute is the oracle, the transport is gloo.
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

    def halo(self, lo, hi):
        """Pivots with a neighbour in [lo, hi), by brute force over all pixel pairs
        (contiguous hull in RING order)."""
        if hi <= lo:
            return lo, lo
        c = 2 * np.sin(np.deg2rad(EDGES[-1]) / 2)
        d2 = ((self.xyz[:, None, :] - self.xyz[None, lo:hi, :]) ** 2).sum(-1)
        near = np.nonzero((d2 < c * c).any(axis=1))[0]
        return int(min(near.min(), lo)), int(max(near.max() + 1, hi))

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


def _step(plan, tag, rank, out_dir):
    from paper_2408_16847_gb300 import shard
    d, w = _field()
    dt, wt = torch.from_numpy(d), torch.from_numpy(w)
    zeta, D = shard.sharded_forward(plan, dt, wt, normalize=_cpu_normalize)
    K = len(EDGES) - 1
    cot = synth.rng(962).standard_normal((M + 1, K, K, 2))
    g = shard.sharded_backward(plan, dt, wt, D, torch.from_numpy(cot))
    np.save(os.path.join(out_dir, "zeta_%s_%d.npy" % (tag, rank)), zeta.numpy())
    np.save(os.path.join(out_dir, "grad_%s_%d.npy" % (tag, rank)), g.numpy())


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        _step(OraclePlan(oracle.pix2vec_ring(NSIDE)), "s1", rank, out_dir)
    finally:
        dist.destroy_process_group()


def _leave_worker(rank, world, ports, out_dir):
    """Step 1 on `world` ranks; the last rank leaves between the steps; the others
    re-form a group and run step 2 over all pivots."""
    from paper_2408_16847_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(ports[0])
    dist.init_process_group("gloo", rank=rank, world_size=world)
    store = dist.TCPStore("127.0.0.1", ports[1], world, rank == 0)
    plan = OraclePlan(oracle.pix2vec_ring(NSIDE))
    _step(plan, "s1", rank, out_dir)
    leaving = rank == world - 1
    alive = shard.continuing_ranks(store, rank, world, step=2, leaving=leaving, timeout_s=60.0)
    dist.destroy_process_group()
    if leaving:
        return
    assert alive == list(range(world - 1)), alive
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % ports[2], rank=alive.index(rank),
                            world_size=len(alive))
    try:
        _step(plan, "s2", rank, out_dir)
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


def _reference():
    d, w = _field()
    xyz = oracle.pix2vec_ring(NSIDE)
    ref = oracle.zeta(xyz, d, w, EDGES, M)
    K = len(EDGES) - 1
    cot = synth.rng(962).standard_normal((M + 1, K, K, 2))
    gref = oracle.gradient(xyz, d, w, EDGES, M, cot[..., 0] + 1j * cot[..., 1])
    return ref["zeta"], gref


def _check(tmp_path, tag, ranks):
    zref, gref = _reference()
    for r in ranks:
        z = np.load(tmp_path / ("zeta_%s_%d.npy" % (tag, r)))
        zc = z[..., 0] + 1j * z[..., 1]
        assert np.abs(zc - zref).max() <= 1e-12 * np.abs(zref).max()
        g = np.load(tmp_path / ("grad_%s_%d.npy" % (tag, r)))
        assert np.abs(g - gref).max() <= 1e-10 * np.abs(gref).max()


@pytest.mark.parametrize("world", [2, 3])
def test_gloo_ranks_match_single_process(tmp_path, world):
    """2 ranks, and 3 ranks whose balanced ranges differ in length (the mask and the
    pixel count split unevenly)."""
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    _check(tmp_path, "s1", range(world))


def test_rank_leaves_between_steps(tmp_path):
    world = 3
    ports = (_free_port(), _free_port(), _free_port())
    mp.spawn(_leave_worker, args=(world, ports, str(tmp_path)), nprocs=world, join=True)
    _check(tmp_path, "s1", range(world))
    _check(tmp_path, "s2", range(world - 1))
