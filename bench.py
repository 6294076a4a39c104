#!/usr/bin/env python
"""Throughput of the harmonic 3PCF estimator on GB300: neighbour pairs/s.

One step = one pass of the estimator over one batch of synthetic input:

  fullsky_nside4096 (default)  forward (neighbour search, binning, harmonics,
                               contraction, normalisation) over the whole HEALPix
                               Nside 4096 map (201,326,592 pixels), 20 log bins
                               0.1-2 deg, m <= 10.  The forward + adjoint dL/d(delta)
                               of L = sum c Re zeta is timed beside it over
                               --fb-steps full steps and reported under "parts".
  masked_map_nside1024         forward + adjoint of the masked Nside 1024 map
  fullsky_nside512, map_nside64  forward (+ adjoint part) on smaller maps
                               (fullsky_nside512 is the case profiled with ncu)
  catalog_2e7                  catalogue D-R estimate: forward over 2e7 clustered
                               points + 6e7 randoms, forward over the randoms,
                               normalisation (16 lin bins 0.1-2 deg, m <= 10)
  batched_maps                 64 maps of mixed Nside / bins / m_max, forward +
                               adjoint in one graph-captured launch sequence
                               (--batch-nsides scales the Nside set down)

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl gb300|reference]

Under torchrun the map workloads split ONE map across the ranks (strong scaling:
balanced pivot ranges, one FP64 all-reduce of (S, D) per forward, the adjoint by
halo with the gradient sliced per rank); the catalogue and batch workloads run an
independent input of the same size per GPU (weak scaling).  Rank 0 prints ONE JSON
line.
--impl reference times the FP64 CPU oracle on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "neighbour pairs/s; Nside=4096 ζ_m time fwd & fwd+bwd at stated err vs FP64"
FP32_LANES_PER_SM = 128
MAP_WORKLOADS = ("fullsky_nside4096", "masked_map_nside1024", "fullsky_nside512", "map_nside64",
                 "fullsky_nside4096_paper", "fullsky_nside2048")
# The paper's exact-path timing (Sec. 3.2): ~40 min for one Nside 4096 map, 20 log bins over
# 8-200 arcmin, m <= 8, forward only, one 128-thread CPU node; with the 3.42e13 in-bin
# pairs of that shape (N^2 (cos 8' - cos 200') / 2) that is 1.43e10 pairs/s.
PAPER_FWD_PAIRS_PER_S = {"fullsky_nside4096_paper": 3.42e13 / 2400.0}


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- workloads

def map_workload(name):
    import synth
    return getattr(synth, name)()


def map_inputs(wl, rank: int, same: bool = False):
    """float32 (delta, w) of the workload; unless ``same``, every rank > 0 gets an
    independent white-noise draw added."""
    import synth
    cache = "/dev/shm/tpcf_bench_%s_%d.npy" % (wl.name, wl.seed)
    if os.path.exists(cache):
        d = np.load(cache)
    else:
        d = wl.delta().astype(np.float32)
        if rank == 0:
            try:
                np.save(cache + ".tmp.npy", d)
                os.replace(cache + ".tmp.npy", cache)
            except OSError:
                pass
    if rank > 0 and not same:
        d = d + (0.05 * synth.rng(wl.seed + 9000 + rank).standard_normal(d.shape[0])).astype(np.float32)
    return np.ascontiguousarray(d, np.float32), wl.weights().astype(np.float32)


def catalog_inputs(rank: int, name: str = "catalog_2e7"):
    """Union (data then randoms) positions, delta, w; randoms positions; alpha."""
    import synth
    wl = getattr(synth, name)()
    xd, wd = wl.data()
    xr = wl.randoms()
    if rank > 0:  # an independent draw per rank
        g = synth.rng(wl.seed + 9000 + rank)
        xd = synth.clustered_catalog(wl.n_points, wl.n_parents, wl.offset_sigma_deg, wl.seed + 9100 + rank)
        xr = synth.uniform_sphere(wl.n_randoms, g)
    wd32 = wd.astype(np.float32)
    alpha = float(wd32.astype(np.float64).sum()) / len(xr)
    nd, nr = len(xd), len(xr)
    xu = np.concatenate([xd, xr])
    du = np.concatenate([np.ones(nd, np.float32), np.full(nr, -alpha, np.float32)])
    wu = np.concatenate([wd32, np.ones(nr, np.float32)])
    return wl, xu, du, wu, xr, float(np.float32(alpha))


# ------------------------------------------------------------- roofline model

def alg_flops_per_pair(M: int, adjoint: bool):
    """Algorithmic FP32 flops per in-bin pair: 24 for the geometry, chord, bin and
    position-angle normalisation, 10 per multipole m >= 1 (one complex multiply of the
    recurrence and one complex accumulate).  The adjoint recomputes the moments and
    then visits every pair again with the same per-m work (its neighbour legs), so it
    counts twice that."""
    f = 24 + 10 * M
    return 2 * f if adjoint else f


def flops_per_pair(M: int, adjoint: bool):
    """FP32 flops (FMA = 2) of the implemented per-pair arithmetic of the map kernels,
    for a pixel visited singly and for one visited as half of a mirror pair.  Counted
    from the pixel loop: position angle 29 (series for sin/cos of half the longitude
    offset, east/north components, normalisation), harmonics 2 recurrences + 2
    accumulations per m >= 2."""
    mm = max(M - 1, 0)
    if not adjoint:
        single = 29 + 1 + 1 + 2 + 2 + 1 + 6 * mm + 1          # ~ 37 + 6 (M - 1)
        mirror = (29 + 2 + 1 + 1 + 2 + 2 + 1 + 6 * mm + 2) / 2.0
    else:
        single = 29 + 2 + 1 + 1 + 8 * mm + 3
        mirror = (29 + 2 + 1 + 1 + 8 * mm + 6) / 2.0
    return single, mirror


def cat_flops_per_pair(M: int):
    """FP32 flops of the catalogue pair loop: chord from hi/lo differences 11, bin
    lookup 4, north/east components and normalisation 14, harmonics 6 per m >= 2
    plus 6 for m <= 1."""
    return 35 + 6 * max(M - 1, 0)


# DRAM bytes per pixel per launch of the map kernels, from the ncu capture of the
# Nside 512 case (profiles/map_kernels_fullsky_nside512.md: dram__bytes_read.sum +
# dram__bytes_write.sum / pixels), valid only for the kernel code it was taken on:
# the key is a hash of map_kernels.cuh with comments and blank lines removed.
TRAFFIC = {"map_bwd_kernel": (18.24, "b151b72319927b3f"), "map_fwd_kernel": (19.18, "263caf8e58838b4c")}


def kernel_code_hash(path):
    import hashlib
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.rstrip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def traffic_per_launch(kernel, npix):
    bpp, sha = TRAFFIC[kernel]
    src = os.path.join(ROOT, "paper_2408_16847_gb300", "csrc", "map_kernels.cuh")
    return bpp * npix if kernel_code_hash(src) == sha else None


def sm_count(dev=None):
    import torch
    return int(torch.cuda.get_device_properties(dev if dev is not None else torch.cuda.current_device())
               .multi_processor_count)


_PEAK = {}


def fp32_peak_tflops(clk, sms):
    """FP32-pipe peak: the larger of the two FMA throughputs measured on this GPU by the
    library's probe (scalar FMA, packed f32x2 FMA), if measured; else SMs x 128 lanes x 2
    flops x the maximum SM clock."""
    if _PEAK.get("measured"):
        return max(_PEAK["measured"])
    return fp32_peak_derived(clk, sms)


def fp32_peak_derived(clk, sms):
    return sms * FP32_LANES_PER_SM * 2 * (clk.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12


def measure_fp32_peak():
    from paper_2408_16847_gb300 import tpcf
    _PEAK["measured"] = tpcf.probe_fp32_peak()
    return _PEAK["measured"]


# --------------------------------------------------------------- GPU clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.p = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=10)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        load = [c for c in sm if c > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU baseline

def oracle_sample(wl, d32, w32, n_piv: int, adjoint: bool = True):
    """The FP64 oracle, as it stands, on a bounded sample of a map workload: n_piv
    consecutive pivots from the first pixel of the belt ring at z = 1/2 (outside the
    galactic mask), neighbours from every pixel within the outer bin edge.
    Returns timings, pair count, the pivot range and the oracle's zeta (for parity)."""
    import oracle
    nside = wl.nside
    ring = (5 * nside) // 4  # z = 1/2 (1-based ring number)
    first = 2 * nside * (nside - 1) + 4 * nside * (ring - nside)
    lo, hi = first, first + n_piv
    # rings within the outer edge plus a margin of two rings
    th_max = math.radians(wl.bins.edges_deg[-1])
    dz = math.sin(th_max) + 4.0 / (3.0 * nside)
    span = (n_piv + 4 * nside - 1) // (4 * nside)  # belt rings the pivots cover
    r_lo = max(nside, int(ring - dz * 3 * nside / 2) - 2)
    r_hi = min(3 * nside, int(ring + span - 1 + dz * 3 * nside / 2) + 2)
    a = 2 * nside * (nside - 1) + 4 * nside * (r_lo - nside)
    b = 2 * nside * (nside - 1) + 4 * nside * (r_hi - nside + 1)
    idx = np.arange(a, b)
    xyz = oracle.pix2vec_ring(nside, idx)
    d = d32[a:b].astype(np.float64)
    w = w32[a:b].astype(np.float64)
    piv = np.arange(lo - a, hi - a)
    M = wl.bins.m_max
    cot = wl.cotangent()
    t0 = time.perf_counter()
    ref = oracle.zeta(xyz, d, w, wl.bins.edges_deg, M, pivots=piv)
    t1 = time.perf_counter()
    if adjoint:
        oracle.gradient(xyz, d, w, wl.bins.edges_deg, M, cot.astype(np.complex128), pivots=piv, targets=piv)
    t2 = time.perf_counter()
    return dict(t_fwd=t1 - t0, t_bwd=t2 - t1, pairs=ref["pairs"], lo=lo, hi=hi, zeta=ref["zeta"],
                cores=int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), npts=len(idx),
                desc="%d pivots at z=0.5 of %s (neighbours from %d pixels)" % (n_piv, wl.name, len(idx)))


def oracle_sample_catalog(xu, du, wu, edges, M, n_piv: int):
    """The oracle's forward on n_piv union pivots (half data, half randoms) with
    neighbours from every point.  Returns timing, pairs, the pivot index range
    (data part) and the oracle's raw sums for those pivots."""
    import oracle
    nd = int(np.sum(du > 0))
    lo = min(1_000_000, nd // 2)
    hi = lo + n_piv
    t0 = time.perf_counter()
    ref = oracle.zeta(xu, du.astype(np.float64), wu.astype(np.float64), edges, M, pivots=np.arange(lo, hi))
    t1 = time.perf_counter()
    assert hi <= nd
    return dict(t_fwd=t1 - t0, t_bwd=0.0, pairs=ref["pairs"], lo=lo, hi=hi, S=ref["S"],
                cores=int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), npts=len(xu),
                desc="%d data pivots of catalog_2e7 (neighbours from all %d points), FP64 forward" %
                     (n_piv, len(xu)))


# ---------------------------------------------------------------- GPU arm

def autotune(args, plan, d_dev, w_dev):
    """The plan's launch configuration, picked by the library's autotuner on this GPU
    (set-up, outside the timed region; cached in TPCF_AUTOTUNE_CACHE when set)."""
    if not args.autotune or args.contract == "tc":
        # the tensor-core forward has a single configuration (3 CTAs per SM)
        return dict(plan.launch_config(), autotuned=False)
    t0 = time.time()
    cfg = plan.autotune(d_dev, w_dev)
    log("autotune: %s in %.1fs" % (cfg, time.time() - t0))
    return dict(cfg, autotuned=True, seconds=round(time.time() - t0, 2))


def setup_map(args, dev, rank):
    import torch
    from paper_2408_16847_gb300 import tpcf

    wl = map_workload(args.workload)
    t0 = time.time()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        # one map split across the ranks: rank 0 paints it once (cached in /dev/shm),
        # the other ranks read the cache
        import torch.distributed as dist
        if rank == 0:
            d32, w32 = map_inputs(wl, rank, same=True)
        dist.barrier()
        if rank != 0:
            d32, w32 = map_inputs(wl, rank, same=True)
    else:
        d32, w32 = map_inputs(wl, rank)
    log("[rank %d] inputs ready in %.1fs" % (rank, time.time() - t0))
    K, M = wl.bins.nbins, wl.bins.m_max
    plan = tpcf.Plan.map(wl.nside, wl.bins.edges_deg, M, contract=args.contract)
    d_dev = torch.from_numpy(d32).to(dev)
    w_dev = torch.from_numpy(w32).to(dev)
    cot = wl.cotangent()
    g_dev = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dev)
    g_dev[..., 0] = torch.from_numpy(cot).to(dev)
    piv = None
    if args.profile_band:
        # pivots of `profile_band` belt rings from z = 1/2: the full-resolution kernels on a
        # slice small enough for an ncu capture (not a bench number)
        n = wl.nside
        first = 2 * n * (n - 1) + 4 * n * ((5 * n) // 4 - n)
        piv = (first, first + 4 * n * args.profile_band)
    elif args.profile_cap:
        # pivots of the first `profile_cap` rings of the north polar cap (ring r holds 4r
        # pixels): the cap's kernels alone (not a bench number)
        r = min(args.profile_cap, wl.nside - 1)
        piv = (0, 2 * r * (r + 1))
    total, n_sym, n_single = plan.count_pairs(w_dev, piv)
    tune = autotune(args, plan, d_dev, w_dev)
    state = {}
    if world > 1:
        return setup_map_sharded(args, dev, rank, world, wl, plan, d32, w32, d_dev, w_dev, g_dev, total,
                                 n_sym, n_single, tune)
    # the masked map's configuration is the forward + backward pass; the full-sky maps
    # time the forward and report the forward + adjoint beside it
    headline_both = args.pass_ == "both" or (args.pass_ == "auto" and wl.name == "masked_map_nside1024")

    def step_fwd(ev=None):
        state["zeta"], state["norm"] = plan.forward(d_dev, w_dev, piv)
        if ev is not None:
            ev.record(torch.cuda.current_stream())

    def step_fb(ev=None):
        zeta, norm = plan.forward(d_dev, w_dev, piv)
        if ev is not None:
            ev.record(torch.cuda.current_stream())
        state["grad"] = plan.backward(d_dev, w_dev, norm, g_dev, piv)

    def warm_adjoint():
        # one adjoint over a slice of 8 belt rings: loads the adjoint kernel's module
        # and warms the tables before the timed forward + adjoint steps
        n = wl.nside
        first = 2 * n * (n - 1) + 4 * n * ((5 * n) // 4 - n)
        sl = (first, min(plan.npoints, first + 4 * n * 8))
        z, nn = plan.forward(d_dev, w_dev, sl)
        plan.backward(d_dev, w_dev, nn, g_dev, sl)

    # e2e: the public host-buffer call (tpcf_run_host), copies inside the timed region
    h_d = torch.from_numpy(d32).pin_memory()
    h_w = torch.from_numpy(w32).pin_memory()
    h_dl = torch.from_numpy(np.stack([cot, np.zeros_like(cot)], axis=-1).copy()).pin_memory()
    h_z = torch.empty((M + 1, K, K, 2), dtype=torch.float64).pin_memory()
    h_n = torch.empty((K, K), dtype=torch.float64).pin_memory()
    h_g = torch.empty(plan.npoints, dtype=torch.float32).pin_memory()

    def e2e_step():
        if headline_both:
            plan.run_host_into(h_d, h_w, h_dl, out=(h_z, h_n, h_g))
        else:
            plan.run_host_into(h_d, h_w, None, out=(h_z, h_n, None))

    in_bytes = h_d.numel() * 4 + h_w.numel() * 4 + (h_dl.numel() * 8 if headline_both else 0)
    out_bytes = h_z.numel() * 8 + h_n.numel() * 8 + (h_g.numel() * 4 if headline_both else 0)

    f_single, f_mirror = flops_per_pair(M, adjoint=False)
    a_single, a_mirror = flops_per_pair(M, adjoint=True)
    fwd_impl = n_single * f_single + n_sym * f_mirror
    adj_impl = n_single * a_single + n_sym * a_mirror
    fwd_alg = total * alg_flops_per_pair(M, False)
    fb_alg = total * (alg_flops_per_pair(M, False) + alg_flops_per_pair(M, True))

    def cpu_baseline(n_piv):
        s = oracle_sample(wl, d32, w32, n_piv, adjoint=headline_both)
        zs, _ = plan.forward(d_dev, w_dev, (s["lo"], s["hi"]))
        zg = tpcf.as_complex(zs).cpu().numpy()
        zo = s["zeta"]
        per_m = [float(np.abs(zg[m] - zo[m]).max() / max(np.abs(zo[m]).max(), 1e-300)) for m in range(M + 1)]
        glob = float(np.abs(zg - zo).max() / np.abs(zo).max())
        scale = [float(np.abs(zo[m]).max() / np.abs(zo).max()) for m in range(M + 1)]
        return s, {"pivots": s["hi"] - s["lo"], "max_rel_err_per_m": max(per_m),
                   "rel_err_per_m": per_m, "max_rel_err_vs_max_zeta": glob, "tolerance_per_m": 1e-5,
                   "max_abs_zeta_m_over_max_abs_zeta": scale}

    def roof_fwd(ms, clk, sms):
        # ms: the forward step (pack + pair kernel + two reductions; the pair kernel is
        # > 99.9% of it), so the achieved rate is a slight underestimate of the kernel's
        return {"bound": "alu", "kernel": "map_fwd_kernel",
                "achieved": fwd_alg / (ms * 1e-3) / 1e12, "peak": fp32_peak_tflops(clk, sms), "unit": "TFLOP/s",
                "flops_per_pair": alg_flops_per_pair(M, False),
                "achieved_implemented": fwd_impl / (ms * 1e-3) / 1e12,
                "implemented_note": "flops of the implemented loop (mirror pairs share one angle "
                                    "and one recurrence)",
                "peak_note": "measured FMA throughput (tpcf_probe_fp32_peak, the larger of scalar and f32x2)",
                "traffic": traffic_per_launch("map_fwd_kernel", 12 * wl.nside ** 2),
                "traffic_note": "DRAM bytes per launch scaled by pixels from the Nside 512 ncu capture "
                                "(null when the kernel changed since)"}

    def roof_fb(ms_total, ms_fwd, clk, sms):
        ms_adj = ms_total - ms_fwd
        return {"bound": "alu", "kernel": "map_bwd_kernel",
                "achieved": total * alg_flops_per_pair(M, True) / (ms_adj * 1e-3) / 1e12,
                "peak": fp32_peak_tflops(clk, sms), "unit": "TFLOP/s",
                "flops_per_pair": alg_flops_per_pair(M, True),
                "achieved_implemented": adj_impl / (ms_adj * 1e-3) / 1e12,
                "step_achieved": fb_alg / (ms_total * 1e-3) / 1e12,
                "traffic": traffic_per_launch("map_bwd_kernel", 12 * wl.nside ** 2)}

    config = {"workload": wl.name, "nside": wl.nside, "npix": 12 * wl.nside * wl.nside,
              "bins": "%d %s bins %.2f-%.2f deg" % (K, "lin" if wl.name == "map_nside64" else "log",
                                                    wl.bins.edges_deg[0], wl.bins.edges_deg[-1]),
              "m_max": M, "pass": "forward + adjoint" if headline_both else "forward",
              "pairs_per_step_per_gpu": total,
              "contraction": "tensor cores, TF32x3" if args.contract == "tc" else "FP32 pipe",
              "pivots": "all" if piv is None else ("profile band: %d rings from z = 1/2 (%d pivots)" % (
                  args.profile_band, piv[1] - piv[0]) if args.profile_band else
                  "profile cap: %d rings from the north pole (%d pivots)" % (args.profile_cap, piv[1] - piv[0])),
              "l2": "inputs larger than L2 (%.2f GB of (w d, w) per map)" % (8 * 12 * wl.nside ** 2 / 1e9)
              if 12 * wl.nside ** 2 * 8 > 129e6 else "L2 flushed between steps",
              "parallelism": "independent map per GPU", "launch_config": tune}
    W = dict(step=step_fb if headline_both else step_fwd,
             split=("forward", "adjoint") if headline_both else ("forward", None),
             pairs=total, e2e=e2e_step, e2e_bytes=(in_bytes, out_bytes),
             vs_baseline=PAPER_FWD_PAIRS_PER_S.get(wl.name) if (not headline_both and piv is None) else None,
             launches=plan.kernel_launches, config=config, cpu_baseline=cpu_baseline,
             small_l2=12 * wl.nside ** 2 * 8 <= 129e6, close=plan.close)
    if headline_both:
        W["roofline"] = lambda t1, t2, clk, sms: roof_fb(t1 + t2, t1, clk, sms)
    else:
        W["roofline"] = lambda t1, t2, clk, sms: roof_fwd(t1, clk, sms)
        if args.fb_steps > 0:
            W["part_fb"] = dict(name="forward_adjoint", step=step_fb, warm=warm_adjoint, steps=args.fb_steps,
                                roofline=lambda t1, t2, clk, sms: roof_fb(t1 + t2, t1, clk, sms))
        if args.grouped > 1:
            # shared neighbour lists (tpcf_forward_grouped): time and deviation from the
            # exact forward of the timed region
            def step_grouped(ev=None):
                state["zg"], _ = plan.forward_grouped(d_dev, w_dev, args.grouped, piv)
                if ev is not None:
                    ev.record(torch.cuda.current_stream())

            def deviation():
                zg = tpcf.as_complex(state["zg"]).cpu().numpy()
                ze = tpcf.as_complex(state["zeta"]).cpu().numpy()
                return [float(np.abs(zg[m] - ze[m]).max() / max(np.abs(ze[m]).max(), 1e-300)) for m in range(M + 1)]

            W["part_grouped"] = dict(group=args.grouped, step=step_grouped, steps=max(2, args.fb_steps),
                                     deviation=deviation)
    return W


def setup_map_sharded(args, dev, rank, world, wl, plan, d32, w32, d_dev, w_dev, g_dev, total, n_sym, n_single,
                      tune=None):
    """One map's estimate split across the ranks (strong scaling): each rank runs the
    forward over its balanced pivot range and one FP64 all-reduce of (S, D) gives
    every rank zeta (shard.sharded_forward); the adjoint gives each rank its slice of
    dL/d(delta) from the slice's halo pivots, with no reduction over the pixels
    (shard.sharded_backward, gather=False)."""
    import torch
    from paper_2408_16847_gb300 import shard

    K, M = wl.bins.nbins, wl.bins.m_max
    state = {}

    def step_fwd(ev=None):
        state["zeta"], state["norm"] = shard.sharded_forward(plan, d_dev, w_dev)
        if ev is not None:
            ev.record(torch.cuda.current_stream())

    def step_fb(ev=None):
        zeta, norm = shard.sharded_forward(plan, d_dev, w_dev)
        if ev is not None:
            ev.record(torch.cuda.current_stream())
        state["grad"] = shard.sharded_backward(plan, d_dev, w_dev, norm, g_dev, gather=False)

    def warm_adjoint():
        step_fb()

    h_d = torch.from_numpy(d32).pin_memory()
    h_w = torch.from_numpy(w32).pin_memory()
    h_z = torch.empty((M + 1, K, K, 2), dtype=torch.float64).pin_memory()

    def e2e_step():
        d = h_d.to(dev, non_blocking=True)
        w = h_w.to(dev, non_blocking=True)
        zeta, _ = shard.sharded_forward(plan, d, w)
        h_z.copy_(zeta, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    f_single, f_mirror = flops_per_pair(M, adjoint=False)
    fwd_alg = total * alg_flops_per_pair(M, False)

    def roof_fwd(ms, clk, sms):
        # whole-job flops over the slowest rank's time, against one GPU's peak x ranks
        return {"bound": "alu", "kernel": "map_fwd_kernel", "achieved": fwd_alg / (ms * 1e-3) / 1e12,
                "peak": fp32_peak_tflops(clk, sms) * world, "unit": "TFLOP/s",
                "flops_per_pair": alg_flops_per_pair(M, False), "peak_note": "per-GPU peak x %d GPUs" % world,
                "traffic": None}

    def roof_fb(ms_total, ms_fwd, clk, sms):
        ms_adj = ms_total - ms_fwd
        return {"bound": "alu", "kernel": "map_bwd_kernel",
                "achieved": total * alg_flops_per_pair(M, True) / (ms_adj * 1e-3) / 1e12,
                "peak": fp32_peak_tflops(clk, sms) * world, "unit": "TFLOP/s",
                "flops_per_pair": alg_flops_per_pair(M, True), "traffic": None}

    config = {"workload": wl.name, "nside": wl.nside, "npix": 12 * wl.nside * wl.nside,
              "bins": "%d log bins %.2f-%.2f deg" % (K, wl.bins.edges_deg[0], wl.bins.edges_deg[-1]),
              "m_max": M, "pass": "forward", "pairs_per_step": total, "contraction": "FP32 pipe",
              "pivots": "all", "l2": "inputs larger than L2",
              "parallelism": "pivot ranges over %d GPUs, FP64 all-reduce of (S, D); adjoint by halo, "
                             "gradient sliced per GPU" % world, "launch_config": tune}
    return dict(step=step_fwd, split=("forward", None), pairs=total, scaling="strong", e2e=e2e_step,
                e2e_bytes=(h_d.numel() * 4 + h_w.numel() * 4, h_z.numel() * 8),
                vs_baseline=None, launches=plan.kernel_launches, config=config, cpu_baseline=None,
                small_l2=False, close=plan.close,
                roofline=lambda t1, t2, clk, sms: roof_fwd(t1, clk, sms),
                part_fb=dict(name="forward_adjoint", step=step_fb, warm=warm_adjoint, steps=args.fb_steps,
                             roofline=lambda t1, t2, clk, sms: roof_fb(t1 + t2, t1, clk, sms))
                if args.fb_steps > 0 else None)


def setup_catalog(args, dev, rank):
    import torch
    from paper_2408_16847_gb300 import tpcf

    t0 = time.time()
    wl, xu, du, wu, xr, alpha32 = catalog_inputs(rank, args.workload)
    log("[rank %d] catalogue ready in %.1fs (%d + %d points)" % (rank, time.time() - t0, len(xu) - len(xr), len(xr)))
    K, M = wl.bins.nbins, wl.bins.m_max
    edges = wl.bins.edges_deg
    xu_dev = torch.from_numpy(xu).to(dev)
    pu = tpcf.Plan.catalog(xu_dev, edges, M)
    del xu_dev
    xr_dev = torch.from_numpy(np.ascontiguousarray(xr)).to(dev)
    pr = tpcf.Plan.catalog(xr_dev, edges, M)
    del xr_dev
    nr = len(xr)
    du_dev = torch.from_numpy(du).to(dev)
    wu_dev = torch.from_numpy(wu).to(dev)
    one_dev = torch.ones(nr, dtype=torch.float32, device=dev)
    cu, _, _ = pu.count_pairs(wu_dev)
    cr, _, _ = pr.count_pairs(one_dev)
    scale = alpha32 ** 3
    state = {}

    def step(ev=None):
        _, _, S = pu.forward(du_dev, wu_dev, want_sums=True)
        if ev is not None:
            ev.record(torch.cuda.current_stream())
        _, DR = pr.forward(one_dev, one_dev)
        state["zeta"] = tpcf.normalize(S, DR, scale)

    h_du = torch.from_numpy(du).pin_memory()
    h_wu = torch.from_numpy(wu).pin_memory()
    h_one = torch.ones(nr, dtype=torch.float32).pin_memory()
    h_z = torch.empty((M + 1, K, K, 2), dtype=torch.float64).pin_memory()

    def e2e_step():
        d = h_du.to(dev, non_blocking=True)
        w = h_wu.to(dev, non_blocking=True)
        o = h_one.to(dev, non_blocking=True)
        _, _, S = pu.forward(d, w, want_sums=True)
        _, DR = pr.forward(o, o)
        h_z.copy_(tpcf.normalize(S, DR, scale), non_blocking=True)
        torch.cuda.current_stream().synchronize()

    flops = (cu + cr) * cat_flops_per_pair(M)
    alg = (cu + cr) * alg_flops_per_pair(M, False)

    def cpu_baseline(n_piv):
        s = oracle_sample_catalog(xu, du, wu, edges, M, n_piv)
        _, _, S = pu.forward(du_dev, wu_dev, (s["lo"], s["hi"]), want_sums=True)
        sg = tpcf.as_complex(S).cpu().numpy()
        so = s["S"]
        per_m = [float(np.abs(sg[m] - so[m]).max() / max(np.abs(so[m]).max(), 1e-300)) for m in range(M + 1)]
        return s, {"pivots": s["hi"] - s["lo"], "quantity": "raw sums S", "max_rel_err_per_m": max(per_m),
                   "tolerance": 1e-5}

    config = {"workload": wl.name, "points": len(xu) - nr, "randoms": nr,
              "bins": "%d lin bins %.2f-%.2f deg" % (K, edges[0], edges[-1]), "m_max": M,
              "pass": "D-R forward (union) + randoms forward + normalisation",
              "pairs_per_step_per_gpu": cu + cr, "pairs_union": cu, "pairs_randoms": cr,
              "l2": "inputs larger than L2", "parallelism": "independent catalogue per GPU"}
    return dict(step=step, split=("union_forward", "randoms_forward"), pairs=cu + cr, e2e=e2e_step,
                e2e_bytes=(h_du.numel() * 4 + h_wu.numel() * 4 + h_one.numel() * 4, h_z.numel() * 8),
                launches=lambda: pu.kernel_launches() + pr.kernel_launches(), extra_launches_per_step=1,
                config=config,
                cpu_baseline=cpu_baseline,
                roofline=lambda t1, t2, clk, sms: {
                    "bound": "alu", "kernel": "cat_fwd_kernel",
                    "achieved": alg / ((t1 + t2) * 1e-3) / 1e12, "peak": fp32_peak_tflops(clk, sms),
                    "unit": "TFLOP/s", "flops_per_pair": alg_flops_per_pair(M, False),
                    "achieved_implemented": flops / ((t1 + t2) * 1e-3) / 1e12},
                small_l2=False, close=lambda: (pu.close(), pr.close()))


def setup_batch(args, dev, rank):
    import torch
    import synth
    from paper_2408_16847_gb300 import tpcf

    nsides = tuple(int(x) for x in args.batch_nsides.split(","))
    wls = synth.batched_maps(64, nsides)
    plans, ds, ws, zs, ns, dls, gs = [], [], [], [], [], [], []
    total = 0
    flops = 0.0
    alg = 0.0
    for wl in wls:
        K, M = wl.bins.nbins, wl.bins.m_max
        d32, w32 = map_inputs(wl, rank)
        p = tpcf.Plan.map(wl.nside, wl.bins.edges_deg, M)
        plans.append(p)
        ds.append(torch.from_numpy(d32).to(dev))
        ws.append(torch.from_numpy(w32).to(dev))
        if args.autotune:
            p.autotune(ds[-1], ws[-1])  # the batch takes each member's tuned flush length
        zs.append(torch.empty((M + 1, K, K, 2), dtype=torch.float64, device=dev))
        ns.append(torch.empty((K, K), dtype=torch.float64, device=dev))
        g = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dev)
        g[..., 0] = torch.from_numpy(wl.cotangent()).to(dev)
        dls.append(g)
        gs.append(torch.empty(12 * wl.nside ** 2, dtype=torch.float32, device=dev))
        t, sym, single = p.count_pairs(ws[-1])
        total += t
        fs, fm = flops_per_pair(M, False)
        as_, am = flops_per_pair(M, True)
        flops += single * (fs + as_) + sym * (fm + am)
        alg += t * (alg_flops_per_pair(M, False) + alg_flops_per_pair(M, True))
    batch = tpcf.Batch(plans, ds, ws, zs, ns, dls, gs)

    def step(ev=None):
        batch.launch()
        if ev is not None:
            ev.record(torch.cuda.current_stream())

    # e2e: every map's delta, w and dL/dzeta from pinned host memory into the batch's
    # device buffers, one graph replay, zeta, norm and the gradients back to the host
    h_in = [(x.cpu().pin_memory(), y.cpu().pin_memory(), z.cpu().pin_memory()) for x, y, z in zip(ds, ws, dls)]
    h_out = [(torch.empty_like(z, device="cpu").pin_memory(), torch.empty_like(n, device="cpu").pin_memory(),
              torch.empty_like(g, device="cpu").pin_memory()) for z, n, g in zip(zs, ns, gs)]

    def e2e_step():
        for (hd, hw, hl), d, w, l in zip(h_in, ds, ws, dls):
            d.copy_(hd, non_blocking=True)
            w.copy_(hw, non_blocking=True)
            l.copy_(hl, non_blocking=True)
        batch.launch()
        for (oz, on, og), z, n, g in zip(h_out, zs, ns, gs):
            oz.copy_(z, non_blocking=True)
            on.copy_(n, non_blocking=True)
            og.copy_(g, non_blocking=True)
        torch.cuda.current_stream().synchronize()

    e2e_in = sum(a.numel() * a.element_size() for t in h_in for a in t)
    e2e_out = sum(a.numel() * a.element_size() for t in h_out for a in t)

    config = {"workload": "batched_maps", "maps": len(wls), "nsides": list(nsides),
              "bins": "8-24 lin/log bins over 0.2-4 deg", "m_max": "6-12",
              "pass": "forward + adjoint, one graph replay", "pairs_per_step_per_gpu": total,
              "kernels_per_replay": batch.kernel_launches(),
              "l2": "inputs larger than L2" if sum(12 * n * n for n in (wl.nside for wl in wls)) * 8 > 129e6
              else "L2-resident inputs", "parallelism": "independent batch per GPU"}
    if nsides != (256, 512, 1024, 2048):
        config["scaled"] = "Nside set scaled down from 256/512/1024/2048"
    return dict(step=step, split=("batch", None), pairs=total, e2e=e2e_step, e2e_bytes=(e2e_in, e2e_out),
                launches=plans[0].kernel_launches, config=config, cpu_baseline=None,
                roofline=lambda t1, t2, clk, sms: {"bound": "alu", "kernel": "batch_bwd_kernel",
                                                   "achieved": alg / (t1 * 1e-3) / 1e12,
                                                   "peak": fp32_peak_tflops(clk, sms), "unit": "TFLOP/s",
                                                   "achieved_implemented": flops / (t1 * 1e-3) / 1e12},
                small_l2=False, close=lambda: (batch.close(), [p.close() for p in plans]))


def run_gpu(args):
    import torch
    import torch.distributed as dist

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", rank=rank, world_size=world, device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2408_16847_gb300 import build
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()

    if args.workload in MAP_WORKLOADS:
        W = setup_map(args, dev, rank)
    elif args.workload in ("catalog_2e7", "catalog_2e6"):
        W = setup_catalog(args, dev, rank)
    elif args.workload == "batched_maps":
        W = setup_batch(args, dev, rank)
    else:
        raise SystemExit("unknown workload " + args.workload)
    stream = torch.cuda.current_stream()
    sms = sm_count(dev)
    peak_meas = measure_fp32_peak()
    log("[rank %d] FP32 FMA throughput: %.1f TFLOP/s scalar, %.1f TFLOP/s f32x2" % (rank, *peak_meas))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev) if W["small_l2"] else None
    gpu_id = str(local)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass

    def timed(step, nsteps):
        """nsteps of `step` bracketed by barrier + synchronize, CUDA events on the
        launching stream; returns (total ms, first-part ms, second-part ms, clocks),
        max over ranks."""
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks = ClockSampler(gpu_id)
        ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(nsteps)]
        for k in range(nsteps):
            if flush is not None:
                flush.fill_(float(k))  # write a buffer larger than L2 between steps
            ev[k][0].record(stream)
            step(ev[k][1])
            ev[k][2].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clk = clocks.stop()
        t1 = sum(ev[k][0].elapsed_time(ev[k][1]) for k in range(nsteps))
        t2 = sum(ev[k][1].elapsed_time(ev[k][2]) for k in range(nsteps))
        tot = sum(ev[k][0].elapsed_time(ev[k][2]) for k in range(nsteps))
        t_max = torch.tensor([tot, t1, t2], dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
        tot, t1, t2 = (float(v) for v in t_max.cpu())
        return tot, t1, t2, clk

    t_setup = time.time()
    for _ in range(args.warmup):
        W["step"]()
    torch.cuda.synchronize()
    log("[rank %d] %d warm-up steps in %.1fs" % (rank, args.warmup, time.time() - t_setup))
    launches0 = W["launches"]()
    total_ms, ms1, ms2, clk = timed(W["step"], args.steps)
    launches = W["launches"]() - launches0 + W.get("extra_launches_per_step", 0) * args.steps
    ms_step = total_ms / args.steps
    strong = W.get("scaling") == "strong"
    units = W["pairs"] if strong else world * W["pairs"]  # pairs of the whole job per step
    value = units * args.steps / (total_ms * 1e-3)
    log("[rank %d] %d timed steps: %.1f ms/step" % (rank, args.steps, ms_step))

    e2e = None
    if W["e2e"] is not None and args.e2e and args.e2e_steps > 0:
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        e_start = torch.cuda.Event(enable_timing=True)
        e_end = torch.cuda.Event(enable_timing=True)
        e_start.record(stream)
        for _ in range(args.e2e_steps):
            W["e2e"]()
        e_end.record(stream)
        torch.cuda.synchronize()
        e2e_ms = torch.tensor([e_start.elapsed_time(e_end), (time.perf_counter() - t0) * 1e3],
                              dtype=torch.float64, device=dev)
        if world > 1:
            dist.all_reduce(e2e_ms, op=dist.ReduceOp.MAX)
        e2e_ms = float(e2e_ms.max().cpu())
        e2e = {"value": units * args.e2e_steps / (e2e_ms * 1e-3), "unit": "pairs/s",
               "h2d_bytes_per_step": W["e2e_bytes"][0], "d2h_bytes_per_step": W["e2e_bytes"][1],
               "steps": args.e2e_steps, "call": "tpcf_run_host (pinned host buffers)"}

    part = None
    if W.get("part_fb") is not None:
        P = W["part_fb"]
        P["warm"]()
        p_tot, p1, p2, p_clk = timed(P["step"], P["steps"])
        roof_p = P["roofline"](p1 / P["steps"], p2 / P["steps"], p_clk, sms)
        roof_p["frac"] = roof_p["achieved"] / roof_p["peak"]
        part = {"steps": P["steps"], "ms": p_tot / P["steps"], "forward_ms": p1 / P["steps"],
                "adjoint_ms": p2 / P["steps"],
                "value": units * P["steps"] / (p_tot * 1e-3), "unit": "pairs/s",
                "roofline": roof_p, "clocks": p_clk}
        log("[rank %d] forward + adjoint: %.1f ms/step" % (rank, p_tot / P["steps"]))

    gpart = None
    if W.get("part_grouped") is not None:
        G = W["part_grouped"]
        G["step"]()  # builds the run tile list and warms the kernel
        g_tot, _, _, g_clk = timed(G["step"], G["steps"])
        gpart = {"group": G["group"], "steps": G["steps"], "ms": g_tot / G["steps"],
                 "speedup_vs_forward": (ms1 / args.steps) / (g_tot / G["steps"]),
                 "deviation_from_exact_per_m": G["deviation"](), "clocks": g_clk}
        log("[rank %d] shared lists (group %d): %.1f ms/step" % (rank, G["group"], g_tot / G["steps"]))

    result = None
    if rank == 0:
        roof = W["roofline"](ms1 / args.steps, ms2 / args.steps, clk, sms)
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof.setdefault("traffic", None)
        cpu = None
        parity = None
        if world == 1 and args.cpu_baseline and W["cpu_baseline"] is not None:
            log("[rank 0] CPU oracle sample ...")
            s, parity = W["cpu_baseline"](args.cpu_pivots)
            cpu = {"value": s["pairs"] / (s["t_fwd"] + s["t_bwd"]), "unit": "pairs/s", "cores": s["cores"],
                   "kind": "oracle",
                   "sample": "%s; FP64 forward %.1fs%s; %d pairs" % (
                       s["desc"], s["t_fwd"], (" + adjoint %.1fs" % s["t_bwd"]) if s["t_bwd"] else "",
                       s["pairs"])}
        a, b = W["split"]
        parts = {a: {"ms": ms1 / args.steps}}
        if b is not None:
            parts[b] = {"ms": ms2 / args.steps}
        if part is not None:
            parts["forward_adjoint"] = part
        if gpart is not None:
            parts["forward_grouped"] = gpart
        result = {
            "metric": METRIC,
            "value": value,
            "unit": "pairs/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": W.get("scaling", "weak"),
            "vs_baseline": (value / W["vs_baseline"]) if W.get("vs_baseline") else None,
            "dtype": "f32",
            "data": "synthetic",
            "config": W["config"],
            "parts": parts,
            "roofline": roof,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk,
            "sm_count": sms,
            "fp32_peak": {"scalar_fma_tflops": peak_meas[0], "f32x2_fma_tflops": peak_meas[1],
                          "derived_tflops": fp32_peak_derived(clk, sms),
                          "note": "measured by tpcf_probe_fp32_peak on this GPU; roofline peaks use the larger"},
            "cpu_baseline": cpu,
            "parity": parity,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    W["close"]()
    return result


# ---------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    if args.workload in MAP_WORKLOADS:
        wl = map_workload(args.workload)
        d32, w32 = map_inputs(wl, 0)
        both = args.pass_ == "both" or (args.pass_ == "auto" and wl.name == "masked_map_nside1024")
        sample = lambda: oracle_sample(wl, d32, w32, args.ref_pivots, adjoint=both)
        cfg = {"workload": wl.name, "nside": wl.nside, "m_max": wl.bins.m_max,
               "pass": "forward + adjoint" if both else "forward", "sample_pivots": args.ref_pivots}
    elif args.workload in ("catalog_2e7", "catalog_2e6"):
        wl, xu, du, wu, xr, _ = catalog_inputs(0, args.workload)
        sample = lambda: oracle_sample_catalog(xu, du, wu, wl.bins.edges_deg, wl.bins.m_max, args.ref_pivots)
        cfg = {"workload": wl.name, "m_max": wl.bins.m_max, "pass": "D-R forward", "sample_pivots": args.ref_pivots}
    else:
        return {"impl": "reference", "unavailable": "the oracle arm covers the map and catalogue workloads"}
    vals = []
    s = None
    for k in range(args.warmup + args.steps):
        s = sample()
        if k >= args.warmup:
            vals.append((s["pairs"], s["t_fwd"] + s["t_bwd"]))
    pairs = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    value = pairs / secs
    cpu = {"value": value, "unit": "pairs/s", "cores": s["cores"], "kind": "oracle",
           "sample": "%s per step" % s["desc"]}
    return {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": cfg, "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="fullsky_nside4096")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-pivots", type=int, default=16384,
                    help="map workloads: pivots (one full belt ring at Nside 4096) in the CPU oracle sample")
    ap.add_argument("--ref-pivots", type=int, default=1024)
    ap.add_argument("--batch-nsides", default="256,512,1024,2048")
    ap.add_argument("--profile-band", type=int, default=0,
                    help="map workloads: restrict the pivots to this many belt rings from z = 1/2 "
                         "(for ncu captures of full-resolution kernels; not a bench configuration)")
    ap.add_argument("--profile-cap", type=int, default=0,
                    help="map workloads: restrict the pivots to this many rings from the north pole "
                         "(timing of the polar-cap kernels; not a bench configuration)")
    ap.add_argument("--pass", dest="pass_", default="auto", choices=["auto", "both", "forward"],
                    help="map workloads: the timed step is the forward (full-sky maps) or the forward + "
                         "adjoint (the masked map) by default")
    ap.add_argument("--grouped", type=int, default=0,
                    help="also time the shared-neighbour-list forward with runs of this many ring pixels "
                         "(map workloads, one GPU) and report its deviation from the exact forward")
    ap.add_argument("--fb-steps", type=int, default=2,
                    help="map workloads timed on the forward: full forward + adjoint steps reported in parts")
    ap.add_argument("--e2e-steps", type=int, default=1,
                    help="calls of the host-buffer entry point timed for e2e")
    ap.add_argument("--contract", default="fp32", choices=["fp32", "tc"],
                    help="contraction of the map forward: FP32 pipe or tensor cores (TF32x3)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch configuration instead of running the autotuner")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        log("note: fewer than 3 warm-up steps (%d)" % args.warmup)
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
