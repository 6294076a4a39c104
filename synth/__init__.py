"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module only draws random numbers and paints input maps; it contains none of
the estimator's arithmetic (no neighbour search, binning, harmonics or
contraction).  Both the oracle tests and the GPU tests/bench take their inputs
from here, so the two sides see bit-identical values.

Random draws use numpy's counter-based Philox generator, whose stream is
identical on every platform.  Bumps are painted by ``paint.c`` (compiled on
first use); see that file for the profile definition.

Workloads mirror the configurations the estimator is evaluated on (the paper's
own maps, the ray-traced convergence fields of its section 3.3, are not
available, so Gaussian-bump maps with the same HEALPix shapes stand in).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None
_LOCK = threading.Lock()

BASE_SEED = 20240830


def build(force: bool = False) -> str:
    """Compile paint.c into _paint.so (in-tree).  Returns the library path."""
    src = os.path.join(_HERE, "paint.c")
    out = os.path.join(_HERE, "_paint.so")
    if force or not os.path.exists(out) or os.path.getmtime(out) < os.path.getmtime(src):
        tmp = out + ".%d.tmp" % os.getpid()
        cmd = ["gcc", "-O3", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
               src, "-o", tmp, "-lm"]
        subprocess.check_call(cmd)
        os.replace(tmp, out)
    return out


def _lib():
    global _LIB
    with _LOCK:
        if _LIB is None:
            lib = ctypes.CDLL(build())
            lib.synth_paint_bumps.restype = ctypes.c_int
            lib.synth_paint_bumps.argtypes = [
                ctypes.c_int64, ctypes.c_int64,
                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                ctypes.c_double, ctypes.c_void_p]
            _LIB = lib
    return _LIB


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


# --------------------------------------------------------------------------- maps

def bump_map(nside: int, n_bumps: int, sigma_deg=(1.0, 4.0), amp_sigma_ln: float = 0.5,
             noise_sigma: float = 0.05, seed: int = BASE_SEED, trunc: float = 3.0) -> np.ndarray:
    """Mean-subtracted sum of ``n_bumps`` Gaussian bumps plus white noise.

    Bump centres are uniform on the sphere, widths sigma ~ U(sigma_deg), amplitudes
    lognormal exp(amp_sigma_ln * N(0,1)); the profile is A exp(-c^2/2 sigma^2) in
    chord c, truncated at c = trunc * sigma.  White noise N(0, noise_sigma) is added
    per pixel, then the mean over all pixels is subtracted.  Returns float64 in
    HEALPix RING order, length 12 nside^2.
    """
    g = rng(seed)
    npix = 12 * nside * nside
    z = g.uniform(-1.0, 1.0, n_bumps)
    ph = g.uniform(0.0, 2.0 * math.pi, n_bumps)
    sg = np.deg2rad(g.uniform(sigma_deg[0], sigma_deg[1], n_bumps))
    amp = np.exp(amp_sigma_ln * g.standard_normal(n_bumps))
    th = np.arccos(np.clip(z, -1.0, 1.0))
    order = np.argsort(th, kind="stable")
    th, ph, sg, amp = (np.ascontiguousarray(a[order]) for a in (th, ph, sg, amp))
    m = np.zeros(npix, dtype=np.float64)
    rc = _lib().synth_paint_bumps(nside, n_bumps, th.ctypes.data, ph.ctypes.data,
                                  sg.ctypes.data, amp.ctypes.data, float(trunc), m.ctypes.data)
    if rc != 0:
        raise RuntimeError("synth_paint_bumps failed")
    if noise_sigma > 0:
        m += noise_sigma * g.standard_normal(npix)
    m -= m.mean()
    return m


def ring_z_of_pixels(nside: int) -> np.ndarray:
    """cos(colatitude) of every RING pixel (input-mask helper, float64)."""
    zs = []
    n = nside
    for r in range(1, 4 * n):
        if r < n:
            z, cnt = 1.0 - r * r / (3.0 * n * n), 4 * r
        elif r > 3 * n:
            rr = 4 * n - r
            z, cnt = -(1.0 - rr * rr / (3.0 * n * n)), 4 * rr
        else:
            z, cnt = 4.0 / 3.0 - 2.0 * r / (3.0 * n), 4 * n
        zs.append(np.full(cnt, z))
    return np.concatenate(zs)


def galactic_mask_weights(nside: int, b_cut_deg: float = 20.0) -> np.ndarray:
    """w = 0 for |b| < b_cut (map taken to be in galactic coordinates), else 1."""
    z = ring_z_of_pixels(nside)
    return (np.abs(z) >= math.sin(math.radians(b_cut_deg))).astype(np.float64)


# ----------------------------------------------------------------------- catalogues

def uniform_sphere(n: int, g: np.random.Generator) -> np.ndarray:
    z = g.uniform(-1.0, 1.0, n)
    ph = g.uniform(0.0, 2.0 * math.pi, n)
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    return np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)


def clustered_catalog(n_points: int, n_parents: int, offset_sigma_deg: float,
                      seed: int) -> np.ndarray:
    """Clustered Poisson process: each point picks a parent uniformly and is displaced
    by an isotropic Gaussian tangent-plane offset (sigma per axis), then projected
    back to the unit sphere.  Returns (n, 3) float64 unit vectors."""
    g = rng(seed)
    parents = uniform_sphere(n_parents, g)
    pick = g.integers(0, n_parents, n_points)
    p = parents[pick]
    # tangent basis at the parent (any orthonormal pair works for an isotropic offset)
    ref = np.where(np.abs(p[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    e1 = np.cross(ref, p)
    e1 /= np.linalg.norm(e1, axis=1, keepdims=True)
    e2 = np.cross(p, e1)
    sg = math.radians(offset_sigma_deg)
    u = g.standard_normal(n_points) * sg
    v = g.standard_normal(n_points) * sg
    q = p + u[:, None] * e1 + v[:, None] * e2
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


# ------------------------------------------------------------------------- workloads

@dataclass
class Bins:
    """Angular bins: edges in degrees (nbins+1, strictly increasing, > 0)."""
    edges_deg: np.ndarray
    m_max: int

    @property
    def nbins(self) -> int:
        return len(self.edges_deg) - 1


def lin_bins(lo: float, hi: float, k: int, m_max: int) -> Bins:
    return Bins(np.linspace(lo, hi, k + 1), m_max)


def log_bins(lo: float, hi: float, k: int, m_max: int) -> Bins:
    return Bins(lo * (hi / lo) ** (np.arange(k + 1) / k), m_max)


@dataclass
class MapWorkload:
    name: str
    nside: int
    bins: Bins
    n_bumps: int
    sigma_deg: tuple
    noise_sigma: float = 0.05
    masked: bool = False
    seed: int = BASE_SEED
    cot_seed: Optional[int] = None  # seed of the cotangent c ~ N(0,1) for L = sum c Re zeta

    def delta(self) -> np.ndarray:
        return bump_map(self.nside, self.n_bumps, self.sigma_deg, 0.5, self.noise_sigma, self.seed)

    def weights(self) -> np.ndarray:
        if self.masked:
            return galactic_mask_weights(self.nside)
        return np.ones(12 * self.nside * self.nside)

    def cotangent(self) -> np.ndarray:
        """c_m(k1,k2) ~ N(0,1) (float64, shape (M+1, K, K)) for L = sum c Re zeta."""
        g = rng(self.cot_seed if self.cot_seed is not None else self.seed + 7)
        K, M = self.bins.nbins, self.bins.m_max
        return g.standard_normal((M + 1, K, K))


def map_nside64() -> MapWorkload:
    """Plain forward, Nside 64, 2000 bumps of width 1-4 deg, 10 linear bins 0.5-10 deg, m<=8."""
    return MapWorkload("map_nside64", 64, lin_bins(0.5, 10.0, 10, 8), 2000, (1.0, 4.0),
                       seed=BASE_SEED + 1)


def masked_map_nside1024() -> MapWorkload:
    """Masked map with gradient: Nside 1024, 20000 bumps 0.2-2 deg, |b|<20 deg masked,
    20 log bins 0.2-3 deg, m<=10."""
    return MapWorkload("masked_map_nside1024", 1024, log_bins(0.2, 3.0, 20, 10), 20000, (0.2, 2.0),
                       masked=True, seed=BASE_SEED + 2, cot_seed=BASE_SEED + 102)


def fullsky_nside4096() -> MapWorkload:
    """Full sky: Nside 4096, 1e6 bumps 0.05-1 deg, 20 log bins 0.1-2 deg, m<=10."""
    return MapWorkload("fullsky_nside4096", 4096, log_bins(0.1, 2.0, 20, 10), 1_000_000, (0.05, 1.0),
                       seed=BASE_SEED + 5, cot_seed=BASE_SEED + 105)


def fullsky_nside4096_paper() -> MapWorkload:
    """The shape of the paper's own timing (Sec. 3.2): Nside 4096, 20 log bins over
    8-200 arcmin, m <= 8; the field is the full-sky bump recipe."""
    return MapWorkload("fullsky_nside4096_paper", 4096, log_bins(8.0 / 60.0, 200.0 / 60.0, 20, 8), 1_000_000,
                       (0.05, 1.0), seed=BASE_SEED + 5, cot_seed=BASE_SEED + 107)


def fullsky_nside2048() -> MapWorkload:
    """The full-sky recipe at Nside 2048 (bumps scaled by pixel count: 250,000): the
    case profiled with ncu at the full recipe's neighbour density per bin."""
    return MapWorkload("fullsky_nside2048", 2048, log_bins(0.1, 2.0, 20, 10), 250_000, (0.05, 1.0),
                       seed=BASE_SEED + 8, cot_seed=BASE_SEED + 108)


def fullsky_nside512() -> MapWorkload:
    """The full-sky recipe at Nside 512 (bumps scaled by pixel count: 15,625): the
    small case profiled in place of the Nside 4096 map."""
    return MapWorkload("fullsky_nside512", 512, log_bins(0.1, 2.0, 20, 10), 15_625, (0.05, 1.0),
                       seed=BASE_SEED + 6, cot_seed=BASE_SEED + 106)


def batched_maps(n_maps: int = 64, nsides=(256, 512, 1024, 2048)) -> List[MapWorkload]:
    """64 independent maps, 16 each at Nside 256/512/1024/2048; one bump per 629 pixels;
    K ~ U{8..24} bins over 0.2-4 deg, lin/log alternating; m_max ~ U{6..12}."""
    out = []
    g = rng(BASE_SEED + 4)
    for i in range(n_maps):
        ns = nsides[i % len(nsides)]
        k = int(g.integers(8, 25))
        m = int(g.integers(6, 13))
        b = lin_bins(0.2, 4.0, k, m) if i % 2 == 0 else log_bins(0.2, 4.0, k, m)
        out.append(MapWorkload("batched_%02d_nside%d" % (i, ns), ns, b,
                               max(1, (12 * ns * ns) // 629), (0.1, 1.0),
                               seed=BASE_SEED + 1000 + i, cot_seed=BASE_SEED + 2000 + i))
    return out


@dataclass
class CatalogWorkload:
    name: str
    n_points: int
    n_parents: int
    offset_sigma_deg: float
    n_randoms: int
    bins: Bins
    seed: int = BASE_SEED + 3

    def data(self):
        """(xyz (n,3) float64, w (n,) float64 ~ U(0.5,1.5))."""
        xyz = clustered_catalog(self.n_points, self.n_parents, self.offset_sigma_deg, self.seed)
        w = rng(self.seed + 11).uniform(0.5, 1.5, self.n_points)
        return xyz, w

    def randoms(self) -> np.ndarray:
        return uniform_sphere(self.n_randoms, rng(self.seed + 23))


def catalog_2e6() -> CatalogWorkload:
    """The catalogue recipe at a tenth of the size (2e6 clustered points, 1e4 parents,
    6e6 randoms): the case profiled in place of catalog_2e7."""
    return CatalogWorkload("catalog_2e6", 2_000_000, 10_000, 0.3, 6_000_000, lin_bins(0.1, 2.0, 16, 10))


def catalog_2e7() -> CatalogWorkload:
    """2e7 clustered points (1e5 parents, 0.3 deg offsets), 6e7 randoms, 16 lin bins 0.1-2 deg, m<=10."""
    return CatalogWorkload("catalog_2e7", 20_000_000, 100_000, 0.3, 60_000_000,
                           lin_bins(0.1, 2.0, 16, 10))
