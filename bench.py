#!/usr/bin/env python
"""Throughput of the harmonic 3PCF estimator on GB300: neighbour pairs/s.

One step = one pass of the whole estimator over one full-sky map: the forward
(geometry tables are plan state; neighbour search, binning, harmonics, contraction,
normalisation) and the adjoint dL/d(delta) of L = sum c Re zeta.  Default workload:
HEALPix Nside 4096 (201,326,592 pixels), 20 log bins over 0.1-2 deg, m <= 10.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl gb300|reference]

Under torchrun each rank runs an independent map of the same size on its own GPU
(weak scaling, no data-path collective); rank 0 prints ONE JSON line.
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

METRIC = json.load(open(os.path.join(ROOT, "BASELINE.json")))["metric"]
SM_COUNT_NOMINAL = 152
FP32_LANES_PER_SM = 128


def log(*a):
    print(*a, file=sys.stderr, flush=True)


# ---------------------------------------------------------------- workloads

def workload(name):
    import synth
    table = {"fullsky_nside4096": synth.fullsky_nside4096, "masked_map_nside1024": synth.masked_map_nside1024,
             "map_nside64": synth.map_nside64}
    return table[name]()


def map_inputs(wl, rank: int):
    """float32 (delta, w) of the workload; every rank gets an independent white-noise draw."""
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
    if rank > 0:
        d = d + (0.05 * synth.rng(wl.seed + 9000 + rank).standard_normal(d.shape[0])).astype(np.float32)
    return np.ascontiguousarray(d, np.float32), wl.weights().astype(np.float32)


# ------------------------------------------------------------- roofline model

def flops_per_pair(M: int, adjoint: bool):
    """FP32 flops (FMA = 2) of the implemented per-pair arithmetic, for a pixel visited
    singly and for one visited as half of a mirror pair.  Counted from the pixel loop:
    position angle 29 (series for sin/cos of half the longitude offset, east/north
    components, normalisation), harmonics 2 recurrences + 2 accumulations per m >= 2."""
    mm = max(M - 1, 0)
    if not adjoint:
        single = 29 + 1 + 1 + 2 + 2 + 1 + 6 * mm + 1          # ~ 37 + 6 (M - 1)
        mirror = (29 + 2 + 1 + 1 + 2 + 2 + 1 + 6 * mm + 2) / 2.0
    else:
        single = 29 + 2 + 1 + 1 + 8 * mm + 3
        mirror = (29 + 2 + 1 + 1 + 8 * mm + 6) / 2.0
    return single, mirror


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

def oracle_sample(wl, d32, w32, n_piv: int):
    """The FP64 oracle, as it stands, on a bounded sample: n_piv consecutive pivots on
    the belt ring at z = 1/2 (outside the galactic mask), neighbours from every pixel
    within the outer bin edge.
    Returns timings, pair count, the pivot range and the oracle's zeta (for parity)."""
    import oracle
    nside = wl.nside
    npix = 12 * nside * nside
    ring = (5 * nside) // 4  # z = 1/2 (1-based ring number)
    first = 2 * nside * (nside - 1) + 4 * nside * (ring - nside)
    lo, hi = first, first + n_piv
    # rings within the outer edge plus a margin of two rings
    th_max = math.radians(wl.bins.edges_deg[-1])
    dz = math.sin(th_max) + 4.0 / (3.0 * nside)
    r_lo = max(nside, int(ring - dz * 3 * nside / 2) - 2)
    r_hi = min(3 * nside, int(ring + dz * 3 * nside / 2) + 2)
    a = 2 * nside * (nside - 1) + 4 * nside * (r_lo - nside)
    b = 2 * nside * (nside - 1) + 4 * nside * (r_hi - nside + 1)
    idx = np.arange(a, b)
    xyz = oracle.pix2vec_ring(nside, idx)
    d = d32[a:b].astype(np.float64)
    w = w32[a:b].astype(np.float64)
    piv = np.arange(lo - a, hi - a)
    K, M = wl.bins.nbins, wl.bins.m_max
    cot = wl.cotangent()
    t0 = time.perf_counter()
    ref = oracle.zeta(xyz, d, w, wl.bins.edges_deg, M, pivots=piv)
    t1 = time.perf_counter()
    oracle.gradient(xyz, d, w, wl.bins.edges_deg, M, cot.astype(np.complex128), pivots=piv, targets=piv)
    t2 = time.perf_counter()
    return dict(t_fwd=t1 - t0, t_bwd=t2 - t1, pairs=ref["pairs"], lo=lo, hi=hi, zeta=ref["zeta"],
                cores=int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1)), npts=len(idx))


# ---------------------------------------------------------------- GPU arm

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
    from paper_2408_16847_gb300 import tpcf

    wl = workload(args.workload)
    t0 = time.time()
    d32, w32 = map_inputs(wl, rank)
    log("[rank %d] inputs ready in %.1fs" % (rank, time.time() - t0))
    K, M = wl.bins.nbins, wl.bins.m_max
    plan = tpcf.Plan.map(wl.nside, wl.bins.edges_deg, M)
    d_dev = torch.from_numpy(d32).to(dev)
    w_dev = torch.from_numpy(w32).to(dev)
    cot = wl.cotangent()
    g_dev = torch.zeros((M + 1, K, K, 2), dtype=torch.float64, device=dev)
    g_dev[..., 0] = torch.from_numpy(cot).to(dev)
    total, n_sym, n_single = plan.count_pairs(w_dev)
    stream = torch.cuda.current_stream()

    def step():
        zeta, norm = plan.forward(d_dev, w_dev)
        grad = plan.backward(d_dev, w_dev, norm, g_dev)
        return zeta, grad

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    gpu_id = str(local)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(gpu_id)
    launches0 = plan.kernel_launches()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    start = torch.cuda.Event(enable_timing=True)
    end = torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        zeta, norm = plan.forward(d_dev, w_dev)
        ev[k][1].record(stream)
        grad = plan.backward(d_dev, w_dev, norm, g_dev)
        ev[k][2].record(stream)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = plan.kernel_launches() - launches0
    total_ms = start.elapsed_time(end)
    t_fwd = [ev[k][0].elapsed_time(ev[k][1]) for k in range(args.steps)]
    t_bwd = [ev[k][1].elapsed_time(ev[k][2]) for k in range(args.steps)]
    plan.sync()
    t_max = torch.tensor([total_ms, sum(t_fwd), sum(t_bwd)], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(t_max, op=dist.ReduceOp.MAX)
    total_ms, fwd_ms, bwd_ms = (float(v) for v in t_max.cpu())
    ms_step = total_ms / args.steps
    value = world * total * args.steps / (total_ms * 1e-3)

    # e2e: the public host-buffer call, with its copies inside the timed region
    h_d = torch.from_numpy(d32).pin_memory()
    h_w = torch.from_numpy(w32).pin_memory()
    h_dl = torch.from_numpy(np.stack([cot, np.zeros_like(cot)], axis=-1).copy()).pin_memory()
    h_z = torch.empty((M + 1, K, K, 2), dtype=torch.float64).pin_memory()
    h_n = torch.empty((K, K), dtype=torch.float64).pin_memory()
    h_g = torch.empty(plan.npoints, dtype=torch.float32).pin_memory()
    plan.run_host_into(h_d, h_w, h_dl, out=(h_z, h_n, h_g))
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(stream)
    for _ in range(args.steps):
        plan.run_host_into(h_d, h_w, h_dl, out=(h_z, h_n, h_g))
    e_end.record(stream)
    torch.cuda.synchronize()
    e2e_ms = torch.tensor([e_start.elapsed_time(e_end), (time.perf_counter() - t0) * 1e3], dtype=torch.float64,
                          device=dev)
    if world > 1:
        dist.all_reduce(e2e_ms, op=dist.ReduceOp.MAX)
    e2e_ms = float(e2e_ms.max().cpu())
    e2e_value = world * total * args.steps / (e2e_ms * 1e-3)
    h2d = h_d.numel() * 4 + h_w.numel() * 4 + h_dl.numel() * 8
    d2h = h_z.numel() * 8 + h_n.numel() * 8 + h_g.numel() * 4

    result = None
    if rank == 0:
        f_single, f_mirror = flops_per_pair(M, adjoint=False)
        a_single, a_mirror = flops_per_pair(M, adjoint=True)
        fwd_flops = n_single * f_single + n_sym * f_mirror
        adj_flops = n_single * a_single + n_sym * a_mirror
        bwd_s = bwd_ms * 1e-3 / args.steps
        fwd_s = fwd_ms * 1e-3 / args.steps
        peak = SM_COUNT_NOMINAL * FP32_LANES_PER_SM * 2 * (clk.get("sm_max_mhz") or 2070.0) * 1e6 / 1e12
        achieved = (fwd_flops + adj_flops) / bwd_s / 1e12  # adjoint kernel recomputes the forward
        cpu = None
        parity = None
        if world == 1 and args.cpu_baseline:
            log("[rank 0] CPU oracle sample ...")
            s = oracle_sample(wl, d32, w32, args.cpu_pivots)
            cpu = {"value": s["pairs"] / (s["t_fwd"] + s["t_bwd"]), "unit": "pairs/s", "cores": s["cores"],
                   "kind": "oracle",
                   "sample": "%d pivots at z=0.5 of %s (neighbours from %d pixels); FP64 forward %.1fs + "
                             "adjoint %.1fs; %d pairs" % (s["hi"] - s["lo"], wl.name, s["npts"], s["t_fwd"],
                                                          s["t_bwd"], s["pairs"])}
            zs, _ = plan.forward(d_dev, w_dev, (s["lo"], s["hi"]))
            zg = tpcf.as_complex(zs).cpu().numpy()
            zo = s["zeta"]
            per_m = [float(np.abs(zg[m] - zo[m]).max() / max(np.abs(zo[m]).max(), 1e-300)) for m in range(M + 1)]
            parity = {"pivots": s["hi"] - s["lo"], "max_rel_err_per_m": max(per_m), "tolerance": 1e-5}
        result = {
            "metric": METRIC,
            "value": value,
            "unit": "pairs/s",
            "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms_step,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": wl.name, "nside": wl.nside, "npix": 12 * wl.nside * wl.nside,
                       "bins": "%d %s bins %.2f-%.2f deg" % (K, "log" if wl.name != "map_nside64" else "lin",
                                                             wl.bins.edges_deg[0], wl.bins.edges_deg[-1]),
                       "m_max": M, "pass": "forward + adjoint", "pairs_per_step_per_gpu": total,
                       "l2": "inputs larger than L2 (%.2f GB of (w d, w) per map)" % (8 * 12 * wl.nside ** 2 / 1e9),
                       "parallelism": "independent map per GPU"},
            "forward": {"ms": fwd_ms / args.steps, "pairs_per_s": world * total / (fwd_ms * 1e-3 / args.steps)},
            "adjoint": {"ms": bwd_ms / args.steps},
            "roofline": {"bound": "alu", "kernel": "map_bwd_kernel", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                         "forward_kernel_frac": (fwd_flops / fwd_s / 1e12) / peak},
            "e2e": {"value": e2e_value, "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches,
            "clocks": clk,
            "cpu_baseline": cpu,
            "parity": parity,
        }
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    plan.close()
    return result


# ---------------------------------------------------------- reference arm

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    wl = workload(args.workload)
    d32, w32 = map_inputs(wl, 0)
    vals = []
    s = None
    for k in range(args.warmup + args.steps):
        s = oracle_sample(wl, d32, w32, args.ref_pivots)
        if k >= args.warmup:
            vals.append((s["pairs"], s["t_fwd"] + s["t_bwd"]))
    pairs = sum(v[0] for v in vals)
    secs = sum(v[1] for v in vals)
    value = pairs / secs
    cpu = {"value": value, "unit": "pairs/s", "cores": s["cores"], "kind": "oracle",
           "sample": "%d pivots at z=0.5 of %s per step (FP64 forward + adjoint)" % (args.ref_pivots, wl.name)}
    return {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "nside": wl.nside, "m_max": wl.bins.m_max, "pass": "forward + adjoint",
                       "sample_pivots": args.ref_pivots},
            "cpu_baseline": cpu,
            "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--workload", default="fullsky_nside4096")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--cpu-pivots", type=int, default=2048)
    ap.add_argument("--ref-pivots", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    args = ap.parse_args()
    if args.warmup < 3:
        log("warm-up raised to 3 steps")
        args.warmup = 3
    res = run_reference(args) if args.impl == "reference" else run_gpu(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
