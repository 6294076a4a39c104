"""PyTorch-facing wrapper of the C ABI (device memory and streams only).

Every step of the estimator runs in libtpcf's CUDA kernels; this module allocates
output tensors, passes raw pointers and the current CUDA stream, and checks the
returned status.
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _capi
from ._capi import TpcfError, check, lib  # noqa: F401  (TpcfError re-exported)


def _stream_ptr(stream: Optional[torch.cuda.Stream] = None) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t: Optional[torch.Tensor]) -> Optional[int]:
    return None if t is None else t.data_ptr()


def _need(t: torch.Tensor, dtype, n: int, name: str) -> None:
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    if t.numel() != n:
        raise ValueError("%s has %d elements, expected %d" % (name, t.numel(), n))


class Plan:
    """A map or catalogue plan (owns its device tables; see include/tpcf.h)."""

    def __init__(self, handle: int, K: int, M: int, npoints: int, edges_rad: np.ndarray, flags: int):
        self._h = ctypes.c_void_p(handle)
        self.K = K
        self.M = M
        self.npoints = npoints
        self.edges_rad = edges_rad
        self.flags = flags

    # -- construction
    @staticmethod
    def _bins(edges_deg=None, edges_rad=None, m_max: int = 0, self_pairs: str = "keep", contract: str = "fp32",
              norm: str = "default"):
        if edges_rad is None:
            edges_rad = np.deg2rad(np.asarray(edges_deg, dtype=np.float64))
        e = np.ascontiguousarray(edges_rad, dtype=np.float64)
        flags = 0
        if self_pairs == "subtract":
            flags |= _capi.SELF_PAIRS_SUBTRACT
        elif self_pairs != "keep":
            raise ValueError(self_pairs)
        if contract == "tc":
            flags |= _capi.CONTRACT_TC
        if norm == "bin_mean":
            flags |= _capi.NORM_BIN_MEAN
        elif norm == "pivot_total":
            flags |= _capi.NORM_PIVOT_TOTAL
        elif norm != "default":
            raise ValueError(norm)
        b = _capi.Bins(len(e) - 1, e.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(m_max), flags)
        return b, e, flags

    @classmethod
    def map(cls, nside: int, edges_deg=None, m_max: int = 0, *, edges_rad=None, self_pairs: str = "keep",
            contract: str = "fp32", norm: str = "default", stream=None) -> "Plan":
        b, e, flags = cls._bins(edges_deg, edges_rad, m_max, self_pairs, contract, norm)
        h = ctypes.c_void_p()
        check(lib().tpcf_plan_create_map(ctypes.byref(h), int(nside), ctypes.byref(b), _stream_ptr(stream)),
              "tpcf_plan_create_map")
        return cls(h.value, len(e) - 1, int(m_max), 12 * nside * nside, e, flags)

    @classmethod
    def catalog(cls, xyz: torch.Tensor, edges_deg=None, m_max: int = 0, *, edges_rad=None,
                self_pairs: str = "keep", contract: str = "fp32", norm: str = "default", stream=None) -> "Plan":
        n = xyz.shape[0]
        _need(xyz, torch.float64, 3 * n, "xyz")
        b, e, flags = cls._bins(edges_deg, edges_rad, m_max, self_pairs, contract, norm)
        h = ctypes.c_void_p()
        check(lib().tpcf_plan_create_catalog(ctypes.byref(h), _ptr(xyz), n, ctypes.byref(b),
                                             _stream_ptr(stream)), "tpcf_plan_create_catalog")
        return cls(h.value, len(e) - 1, int(m_max), n, e, flags)

    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().tpcf_plan_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- calls
    def zeta_shape(self) -> Tuple[int, int, int, int]:
        return (self.M + 1, self.K, self.K, 2)

    def forward(self, delta: torch.Tensor, w: torch.Tensor, pivots: Optional[Tuple[int, int]] = None,
                want_sums: bool = False, stream=None):
        """Returns (zeta (M+1,K,K,2) float64 [re, im], norm (K,K) float64[, sums])."""
        n = self.npoints
        _need(delta, torch.float32, n, "delta")
        _need(w, torch.float32, n, "w")
        lo, hi = (0, n) if pivots is None else (int(pivots[0]), int(pivots[1]))
        dev = delta.device
        zeta = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev)
        norm = torch.empty((self.K, self.K), dtype=torch.float64, device=dev)
        sums = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev) if want_sums else None
        check(lib().tpcf_forward(self._h, _ptr(delta), _ptr(w), lo, hi, _ptr(zeta), _ptr(norm), _ptr(sums),
                                 _stream_ptr(stream)), "tpcf_forward")
        if want_sums:
            return zeta, norm, sums
        return zeta, norm

    def forward_grouped(self, delta: torch.Tensor, w: torch.Tensor, group: int,
                        pivots: Optional[Tuple[int, int]] = None, want_sums: bool = False, stream=None):
        """Shared-neighbour-list forward (tpcf_forward_grouped): runs of `group` ring pixels
        take the moments of their middle pixel.  Returns as forward()."""
        n = self.npoints
        _need(delta, torch.float32, n, "delta")
        _need(w, torch.float32, n, "w")
        lo, hi = (0, n) if pivots is None else (int(pivots[0]), int(pivots[1]))
        dev = delta.device
        zeta = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev)
        norm = torch.empty((self.K, self.K), dtype=torch.float64, device=dev)
        sums = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev) if want_sums else None
        check(lib().tpcf_forward_grouped(self._h, _ptr(delta), _ptr(w), int(group), lo, hi, _ptr(zeta), _ptr(norm),
                                         _ptr(sums), _stream_ptr(stream)), "tpcf_forward_grouped")
        if want_sums:
            return zeta, norm, sums
        return zeta, norm

    def forward_multi(self, fields, pivots: Optional[Tuple[int, int]] = None, want_sums: bool = False,
                      stream=None):
        """Three-field estimate zeta^{ABC} (tpcf_forward_multi): ``fields`` =
        ((delta_A, w_A), (delta_B, w_B), (delta_C, w_C)) float32 CUDA tensors.  Returns
        (zeta (M+1,K,K,2) float64, norm (K,K)[, sums]); full K x K matrices."""
        n = self.npoints
        ptrs = []
        for name, (d, w) in zip("ABC", fields):
            _need(d, torch.float32, n, "delta_" + name)
            _need(w, torch.float32, n, "w_" + name)
            ptrs += [_ptr(d), _ptr(w)]
        lo, hi = (0, n) if pivots is None else (int(pivots[0]), int(pivots[1]))
        dev = fields[0][0].device
        zeta = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev)
        norm = torch.empty((self.K, self.K), dtype=torch.float64, device=dev)
        sums = torch.empty(self.zeta_shape(), dtype=torch.float64, device=dev) if want_sums else None
        check(lib().tpcf_forward_multi(self._h, *ptrs, lo, hi, _ptr(zeta), _ptr(norm), _ptr(sums),
                                       _stream_ptr(stream)), "tpcf_forward_multi")
        if want_sums:
            return zeta, norm, sums
        return zeta, norm

    def backward(self, delta: torch.Tensor, w: torch.Tensor, norm: torch.Tensor, dL_dzeta: torch.Tensor,
                 pivots: Optional[Tuple[int, int]] = None, stream=None) -> torch.Tensor:
        """dL/d(delta) (float32, npoints) given dL/dzeta (M+1,K,K,2) float64 and the forward's norm."""
        n = self.npoints
        _need(delta, torch.float32, n, "delta")
        _need(w, torch.float32, n, "w")
        _need(norm, torch.float64, self.K * self.K, "norm")
        _need(dL_dzeta, torch.float64, (self.M + 1) * self.K * self.K * 2, "dL_dzeta")
        lo, hi = (0, n) if pivots is None else (int(pivots[0]), int(pivots[1]))
        grad = torch.empty(n, dtype=torch.float32, device=delta.device)
        check(lib().tpcf_backward(self._h, _ptr(delta), _ptr(w), lo, hi, _ptr(norm), _ptr(dL_dzeta),
                                  _ptr(grad), _stream_ptr(stream)), "tpcf_backward")
        return grad

    def count_pairs(self, w: torch.Tensor, pivots: Optional[Tuple[int, int]] = None, stream=None):
        """(total, mirror-pair, single) in-bin ordered pair counts of the live pivots."""
        n = self.npoints
        _need(w, torch.float32, n, "w")
        lo, hi = (0, n) if pivots is None else (int(pivots[0]), int(pivots[1]))
        out = torch.zeros(3, dtype=torch.int64, device=w.device)
        check(lib().tpcf_count_pairs(self._h, _ptr(w), lo, hi, _ptr(out), _stream_ptr(stream)),
              "tpcf_count_pairs")
        return tuple(int(v) for v in out.cpu())

    def autotune(self, delta: torch.Tensor, w: torch.Tensor, forward: bool = True, adjoint: bool = True,
                 stream=None) -> dict:
        """Pick the pair kernels' launch configuration on this device (tpcf_plan_autotune);
        returns it (see launch_config)."""
        _need(delta, torch.float32, self.npoints, "delta")
        _need(w, torch.float32, self.npoints, "w")
        passes = (1 if forward else 0) | (2 if adjoint else 0)
        check(lib().tpcf_plan_autotune(self._h, _ptr(delta), _ptr(w), passes, _stream_ptr(stream)),
              "tpcf_plan_autotune")
        return self.launch_config()

    def launch_config(self) -> dict:
        """forward: variant, ctas_per_sm, flush_rings, quarter_turn_tiles; adjoint: the first three."""
        c = (ctypes.c_int32 * 7)()
        check(lib().tpcf_plan_launch_config(self._h, c), "tpcf_plan_launch_config")
        return {"forward": {"variant": c[0], "ctas_per_sm": c[1], "flush_rings": c[2], "quarter_turn_tiles": c[3]},
                "adjoint": {"variant": c[4], "ctas_per_sm": c[5], "flush_rings": c[6]}}

    def set_launch_config(self, cfg: dict) -> None:
        f, b = cfg["forward"], cfg["adjoint"]
        c = (ctypes.c_int32 * 7)(f["variant"], f["ctas_per_sm"], f["flush_rings"], f.get("quarter_turn_tiles", 0),
                                 b["variant"], b["ctas_per_sm"], b["flush_rings"])
        check(lib().tpcf_plan_set_launch_config(self._h, c), "tpcf_plan_set_launch_config")

    def halo(self, begin: int, end: int) -> Tuple[int, int]:
        """Pixel range of the pivots that can have a neighbour in [begin, end) (map plans)."""
        a, b = ctypes.c_int64(), ctypes.c_int64()
        check(lib().tpcf_plan_halo(self._h, int(begin), int(end), ctypes.byref(a), ctypes.byref(b)),
              "tpcf_plan_halo")
        return int(a.value), int(b.value)

    def run_host(self, delta: np.ndarray, w: np.ndarray, dL_dzeta: Optional[np.ndarray] = None,
                 stream=None):
        """End-to-end on host (pinned or pageable) float32 arrays; returns numpy
        (zeta, norm[, grad]).  Synchronises."""
        delta = np.ascontiguousarray(delta, dtype=np.float32)
        w = np.ascontiguousarray(w, dtype=np.float32)
        return self.run_host_into(delta, w, dL_dzeta, stream=stream)

    def run_host_into(self, delta, w, dL_dzeta=None, out=None, stream=None):
        """Like run_host but accepts torch CPU tensors (e.g. pinned) or numpy arrays and
        optional preallocated outputs (zeta, norm, grad) as torch CPU tensors."""
        def hp(a):
            if isinstance(a, torch.Tensor):
                return a.data_ptr()
            return a.ctypes.data

        if out is None:
            zeta = np.empty(self.zeta_shape(), dtype=np.float64)
            norm = np.empty((self.K, self.K), dtype=np.float64)
            grad = np.empty(self.npoints, dtype=np.float32) if dL_dzeta is not None else None
        else:
            zeta, norm, grad = out
        dl = None
        if dL_dzeta is not None:
            dl = dL_dzeta if isinstance(dL_dzeta, torch.Tensor) else np.ascontiguousarray(dL_dzeta, np.float64)
        check(lib().tpcf_run_host(self._h, hp(delta), hp(w), None if dl is None else hp(dl), hp(zeta), hp(norm),
                                  None if grad is None else hp(grad), _stream_ptr(stream)), "tpcf_run_host")
        if dL_dzeta is not None:
            return zeta, norm, grad
        return zeta, norm

    def kernel_launches(self) -> int:
        return int(lib().tpcf_plan_kernel_launches(self._h))

    def sync(self) -> None:
        check(lib().tpcf_plan_sync(self._h), "tpcf_plan_sync")


def probe_fp32_peak(stream=None) -> Tuple[float, float]:
    """Measured FP32-pipe throughput of the current device in TFLOP/s: (scalar FMA,
    packed f32x2 FMA) (tpcf_probe_fp32_peak)."""
    out = (ctypes.c_double * 2)()
    check(lib().tpcf_probe_fp32_peak(out, _stream_ptr(stream)), "tpcf_probe_fp32_peak")
    return float(out[0]), float(out[1])


def as_complex(zeta: torch.Tensor) -> torch.Tensor:
    """(M+1,K,K,2) float64 -> (M+1,K,K) complex128 view."""
    return torch.view_as_complex(zeta)


def normalize(sums: torch.Tensor, norm: torch.Tensor, scale: float = 1.0, stream=None) -> torch.Tensor:
    """zeta = sums / (scale * norm) on the device (tpcf_normalize); sums (M+1,K,K,2)."""
    M1, K = sums.shape[0], sums.shape[1]
    _need(sums, torch.float64, M1 * K * K * 2, "sums")
    _need(norm, torch.float64, K * K, "norm")
    zeta = torch.empty_like(sums)
    check(lib().tpcf_normalize(_ptr(sums), _ptr(norm), float(scale), K, M1 - 1, _ptr(zeta), _stream_ptr(stream)),
          "tpcf_normalize")
    return zeta


def edge_correct(sums: torch.Tensor, rsums: torch.Tensor, scale: float = 1.0, stream=None) -> torch.Tensor:
    """m-coupling correction (tpcf_edge_correct): sums (M+1,K,K,2) of the D - R run,
    rsums (>= 2M+1,K,K,2) of the randoms' delta = 1 run; returns zeta (M+1,K,K,2)."""
    M1, K = sums.shape[0], sums.shape[1]
    _need(sums, torch.float64, M1 * K * K * 2, "sums")
    if rsums.shape[0] < 2 * M1 - 1 or rsums.shape[1:] != sums.shape[1:]:
        raise ValueError("rsums needs multipoles 0..2M with the same bins")
    _need(rsums, torch.float64, rsums.shape[0] * K * K * 2, "rsums")
    zeta = torch.empty_like(sums)
    check(lib().tpcf_edge_correct(_ptr(sums), _ptr(rsums), float(scale), K, M1 - 1, _ptr(zeta), _stream_ptr(stream)),
          "tpcf_edge_correct")
    return zeta


class ZetaFn(torch.autograd.Function):
    """zeta = ZetaFn.apply(delta, w, plan[, lo, hi]) with a hand-written adjoint.

    Output: (M+1, K, K, 2) float64 (re, im); the gradient flows to delta only."""

    @staticmethod
    def forward(ctx, delta, w, plan: Plan, lo: int = 0, hi: int = -1):
        hi = plan.npoints if hi < 0 else hi
        zeta, norm = plan.forward(delta.detach(), w.detach(), (lo, hi))
        ctx.plan = plan
        ctx.range = (lo, hi)
        ctx.save_for_backward(delta, w, norm)
        return zeta

    @staticmethod
    def backward(ctx, g):
        delta, w, norm = ctx.saved_tensors
        grad = ctx.plan.backward(delta.detach(), w.detach(), norm, g.contiguous(), ctx.range)
        return grad, None, None, None, None


class Batch:
    """A CUDA-graph-captured batch of map plans (tpcf_batch_*)."""

    def __init__(self, plans: Sequence[Plan], deltas, ws, zetas, norms, dLs=None, grads=None, stream=None):
        n = len(plans)
        arr = lambda xs: (ctypes.c_void_p * n)(*[ctypes.c_void_p(_ptr(x)) for x in xs])
        self._keep = (plans, deltas, ws, zetas, norms, dLs, grads)
        ph = (ctypes.c_void_p * n)(*[p.handle for p in plans])
        h = ctypes.c_void_p()
        check(lib().tpcf_batch_create(ctypes.byref(h), ph, n, arr(deltas), arr(ws), arr(zetas), arr(norms),
                                      arr(dLs) if dLs is not None else None,
                                      arr(grads) if grads is not None else None, _stream_ptr(stream)),
              "tpcf_batch_create")
        self._h = h

    def launch(self, stream=None) -> None:
        check(lib().tpcf_batch_launch(self._h, _stream_ptr(stream)), "tpcf_batch_launch")

    def kernel_launches(self) -> int:
        """Kernels in one replay of the batch's graph."""
        return int(lib().tpcf_batch_kernel_launches(self._h))

    def close(self) -> None:
        if self._h is not None and self._h.value:
            lib().tpcf_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def edges_from(lo_deg: float, hi_deg: float, k: int, log: bool) -> np.ndarray:
    """Bin edges in degrees: linear, or geometric theta_lo (theta_hi/theta_lo)^(j/k)."""
    if log:
        return lo_deg * (hi_deg / lo_deg) ** (np.arange(k + 1) / k)
    return np.linspace(lo_deg, hi_deg, k + 1)


def pairs_hint(npix: int, theta_lo_deg: float, theta_hi_deg: float) -> float:
    """Expected in-bin ordered pairs of a full unit-weight map (N^2 (cos lo - cos hi) / 2)."""
    return npix * npix * (math.cos(math.radians(theta_lo_deg)) - math.cos(math.radians(theta_hi_deg))) / 2
