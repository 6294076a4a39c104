"""Pivot sharding of one estimate across ranks (one process per GPU).

zeta_m = S_m / D with S_m and D sums over pivots (Sec. 3.1, eq. zetamEst2), so one
map or catalogue splits into contiguous pivot ranges, one per rank: every rank holds
the whole field (neighbours come from everywhere), runs the forward over its range,
and one FP64 all-reduce of (S, D) -- (m_max+1) K^2 complex plus K^2 real values --
gives every rank the full sums; the division runs on the device (tpcf_normalize).
The adjoint is a sum over pivots as well: each rank's adjoint over its range is a
partial dL/d(delta) over all points, and one all-reduce sums them.

Ranges are balanced by the number of live pivots (w != 0), which tracks the pair
work on maps (every live pixel has the same neighbourhood size up to the mask).
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


def sharded_backward(plan, delta: torch.Tensor, w: torch.Tensor, norm: torch.Tensor, dL_dzeta: torch.Tensor,
                     group=None) -> torch.Tensor:
    """dL/d(delta) over all points: this rank's adjoint over its pivot range, summed
    over ranks.  ``norm`` is the all-reduced D of sharded_forward."""
    rank, world = _rank_world(group)
    lo, hi = balanced_ranges(w, world)[rank]
    g = plan.backward(delta, w, norm, dL_dzeta, (lo, hi))
    dist.all_reduce(g, op=dist.ReduceOp.SUM, group=group)
    return g
