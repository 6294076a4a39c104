"""Pivot sharding of one estimate across ranks (one process per GPU).

zeta_m = S_m / D with S_m and D sums over pivots (Sec. 3.1, eq. zetamEst2), so one
map or catalogue splits into contiguous pivot ranges, one per rank: every rank holds
the whole field (neighbours come from everywhere), runs the forward over its range,
and one FP64 all-reduce of (S, D) -- (m_max+1) K^2 complex plus K^2 real values --
gives every rank the full sums; the division runs on the device (tpcf_normalize).

The adjoint dL/d(delta_p) is a sum over the pivots i that have p as a neighbour
(plus p's own pivot term).  For a map, each rank owns one slice of the gradient
(its pivot range) and runs the adjoint over the halo of that slice
(tpcf_plan_halo: every pivot within the outer bin edge of the slice), which makes
its slice exact without any reduction over the N points; only the slices are
gathered if the caller wants the whole gradient.  Catalogue plans have no spatial
order in the caller's indexing, so there each rank's adjoint over its own pivot
range is a partial gradient over all points, summed by one all-reduce.

Ranges are balanced by the number of live pivots (w != 0), which tracks the pair
work on maps (every live pixel has the same neighbourhood size up to the mask).
When a rank leaves between steps, the survivors form a new group and call these
functions again: the ranges are recomputed over the new world size, so the departed
rank's pivots are redone by the others.
"""
from __future__ import annotations

from typing import Callable, Optional, Tuple

import torch
import torch.distributed as dist


def balanced_ranges(w: torch.Tensor, world: int) -> list:
    """Contiguous [lo, hi) pivot ranges, one per rank, holding equal numbers of live
    pivots (w != 0).  Ranges cover [0, len(w)) without gaps."""
    n = w.numel()
    live = torch.cumsum((w != 0).to(torch.int64), 0)
    total = int(live[-1]) if n else 0
    cuts = [0]
    for r in range(1, world):
        target = (total * r) // world
        # first index whose running live count exceeds the target
        cuts.append(int(torch.searchsorted(live, torch.tensor([target], dtype=live.dtype, device=live.device),
                                           right=True)[0]) if total else (n * r) // world)
    cuts.append(n)
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def _rank_world(group) -> Tuple[int, int]:
    return dist.get_rank(group), dist.get_world_size(group)


def sharded_forward(plan, delta: torch.Tensor, w: torch.Tensor, group=None,
                    normalize: Optional[Callable] = None):
    """(zeta, norm) of the whole field, computed over this rank's pivot range and
    all-reduced.  ``normalize(sums, norm)`` defaults to the library's device kernel."""
    if normalize is None:
        from .tpcf import normalize as _dev_normalize
        normalize = _dev_normalize
    rank, world = _rank_world(group)
    lo, hi = balanced_ranges(w, world)[rank]
    _, norm, sums = plan.forward(delta, w, (lo, hi), want_sums=True)
    ns = sums.numel()
    buf = torch.cat([sums.reshape(-1), norm.reshape(-1)]).to(torch.float64)
    dist.all_reduce(buf, op=dist.ReduceOp.SUM, group=group)
    S = buf[:ns].reshape(sums.shape).contiguous()
    D = buf[ns:].reshape(norm.shape).contiguous()
    return normalize(S, D), D


def _halo(plan, lo: int, hi: int):
    """The plan's halo of [lo, hi), or None where the plan has none (catalogues)."""
    try:
        return plan.halo(lo, hi)
    except Exception as e:  # the library's UNSUPPORTED status for catalogue plans
        if getattr(e, "status", None) == 5:
            return None
        raise


def sharded_backward(plan, delta: torch.Tensor, w: torch.Tensor, norm: torch.Tensor, dL_dzeta: torch.Tensor,
                     group=None, gather: bool = True):
    """dL/d(delta).  ``norm`` is the all-reduced D of sharded_forward.

    Map plans: this rank's slice [lo, hi) of the gradient from the adjoint over the
    slice's halo pivots; with ``gather`` the slices of all ranks are gathered into
    the full gradient (every rank gets it), else returns (slice, (lo, hi)).
    Catalogue plans: the adjoint over this rank's pivot range, all-reduced (full
    gradient on every rank)."""
    rank, world = _rank_world(group)
    ranges = balanced_ranges(w, world)
    lo, hi = ranges[rank]
    halo = _halo(plan, lo, hi)
    if halo is None:
        g = plan.backward(delta, w, norm, dL_dzeta, (lo, hi))
        dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
        return g if gather else (g[lo:hi].clone(), (lo, hi))
    g = plan.backward(delta, w, norm, dL_dzeta, halo)
    mine = g[lo:hi].contiguous()
    if not gather:
        return mine, (lo, hi)
    width = max(b - a for a, b in ranges)
    buf = torch.zeros(width, dtype=mine.dtype, device=mine.device)
    buf[: hi - lo] = mine
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf, group=group)
    return torch.cat([p[: b - a] for p, (a, b) in zip(parts, ranges)])


def continuing_ranks(store, rank: int, world: int, step: int, leaving: bool = False,
                     timeout_s: float = 30.0) -> list:
    """Between two steps, on the host: this rank announces in ``store`` (a
    torch.distributed Store shared by all ranks) whether it takes part in step
    ``step``, then waits for every other rank's announcement.  Returns the sorted
    ranks that continue; a rank that announced it is leaving, or that said nothing
    within ``timeout_s`` (it died), is left out.  The survivors then form a new
    process group over the returned ranks and call sharded_forward / sharded_backward
    again, which re-balances the pivot ranges over them."""
    import datetime
    store.set("tpcf/step%d/rank%d" % (step, rank), "left" if leaving else "on")
    if leaving:
        return []
    alive = []
    for r in range(world):
        key = "tpcf/step%d/rank%d" % (step, r)
        try:
            store.wait([key], datetime.timedelta(seconds=timeout_s))
        except Exception:  # no answer in time: the rank is gone
            continue
        if store.get(key) == b"on":
            alive.append(r)
    return alive
