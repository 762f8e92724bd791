#!/usr/bin/env python
"""Benchmark of the momentum power-spectrum estimator (one JSON line on stdout).

A step is one whole estimate (moments, BL assignment, four R2C FFTs, deconvolution,
shot noise and shell binning of P_dd, P_pp, P_tt, P_dt with and without the bulk
flow) of one synthetic catalogue already resident in HBM. Default workload: a
Zel'dovich catalogue of 256^3 particles in a 1000 Mpc/h box on a 256^3 FP32 grid
with 128 shells. Under torchrun every rank runs an independent replica on its own
GPU (the estimate of one catalogue does not shard); the slowest rank's time counts.

    python bench.py [--steps K] [--warmup W] [--workload NAME] [--impl reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particles/s & Mcells/s for 3 momentum spectra; batched p50/p99 latency vs plain"

WORKLOADS = {
    # name: (description, generator kwargs, grid, shells, precision)
    "zeldovich256_ng256": ("Zel'dovich 256^3 particles, L=1000 Mpc/h, 256^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow", dict(kind="zeldovich", n_side=256, L=1000.0, seed=1001),
                           256, 128, "f32"),
    "poisson32768_ng64_fp64": ("32768 Poisson particles, L=256 Mpc/h, sigma_v=300 km/s, 64^3 FP64 grid, BL3, "
                               "32 shells", dict(kind="poisson", n=32768, L=256.0, seed=1000), 64, 32, "f64"),
    "zeldovich256_ng512": ("Zel'dovich 256^3 particles, L=1000 Mpc/h, 512^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow (0.125 particle per cell)",
                           dict(kind="zeldovich", n_side=256, L=1000.0, seed=1001), 512, 128, "f32"),
    "zeldovich512_ng512": ("Zel'dovich 512^3 particles, L=1500 Mpc/h, 512^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow", dict(kind="zeldovich", n_side=512, L=1500.0, seed=1002),
                           512, 128, "f32"),
    "zeldovich512_ng1024": ("Zel'dovich 512^3 particles, L=1500 Mpc/h, 1024^3 FP32 grid, BL3, 128 shells, "
                            "with and without bulk flow", dict(kind="zeldovich", n_side=512, L=1500.0, seed=1002),
                            1024, 128, "f32"),
    "poisson830k_ng384": ("830,584 Poisson particles, L=900 Mpc/h, 384^3 FP32 grid, BL3, 128 shells (0.015 particle "
                          "per cell, as in the sparsest catalogues of the batch)",
                          dict(kind="poisson", n=830584, L=900.0, seed=5), 384, 128, "f32"),
}
DEFAULT = "zeldovich256_ng256"
# DRAM bytes (read + write) per launch of the dominant stage's kernels, from one ncu
# capture of the current kernels (profiles/kernels_zeldovich256_ng256.md); a stage
# whose kernels change drops its entry until it is captured again
MEASURED_TRAFFIC = {
    ("zeldovich256_ng256", "deposit"): ((619.302656 + 412.942592 + 458.1888 + 171.559168) * 1e6,
                                        "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_deposit_home and "
                                        "k_home_fixup, one launch each (profiles/kernels_zeldovich256_ng256.md)"),
}
# configs 4 and 5 run through their own drivers below
MULTI = {
    "batch64": "64 catalogues in one launch sequence: particle counts log-uniform in [1e5, 2e7], seeded "
               "Zel'dovich or Poisson (50/50), grids from {128, 256, 384}^3, L in [300, 1500] Mpc/h, "
               "FP32, 128 shells; lanes + CUDA graph + autotuned tiles",
    "serve": "Poisson arrivals (mean 20 requests/s) of estimation requests, particle counts log-uniform in "
             "[1e5, 1.3e8], grids from {128, 256, 512, 1024}^3, FP32, 128 shells, admitted by HBM footprint "
             "against 180 GB",
}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def make_catalog(spec, dtype):
    from paper_2005_06170_gb300 import catalogs
    if spec["kind"] == "zeldovich":
        return catalogs.zeldovich(spec["n_side"], spec["L"], seed=spec["seed"], dtype=dtype)
    return catalogs.poisson(spec["n"], spec["L"], sigma_v=300.0, seed=spec["seed"], dtype=dtype)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if gpu_id:
            cmd[1:1] = ["-i", gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                smax.append(float(r[1]))
            except ValueError:
                continue
            for name, flag in zip(names, r[4:8]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(cat, wl, steps=1, warmup=0, frac=None):
    """The oracle as it stands, on a bounded sample of the same workload: the first
    1/frac of the catalogue's particles on the full grid with the same shells."""
    from oracle import estimator as est
    desc, spec, ng, nbins, _ = WORKLOADS[wl]
    n = len(cat["pos"])
    if frac is None:
        frac = 4 if n >= 4_000_000 else 1
    m = n // frac
    pos, vel = cat["pos"][:m], cat["vel"][:m]
    est.estimate(pos[:1000], vel[:1000], L=spec["L"], ng=16, nbins=4)  # builds the C part
    for _ in range(warmup):
        est.estimate(pos, vel, L=spec["L"], ng=ng, nbins=nbins)
    t0 = time.perf_counter()
    for _ in range(steps):
        est.estimate(pos, vel, L=spec["L"], ng=ng, nbins=nbins)
    dt = (time.perf_counter() - t0) / steps
    sample = (f"the first 1/{frac} of the catalogue ({m} particles) on the full {ng}^3 grid with {nbins} shells"
              if frac > 1 else f"the whole catalogue ({m} particles), {ng}^3 grid, {nbins} shells")
    return {"value": m / dt, "unit": "particles/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": sample + "; FP64; C deposit single-threaded, scipy FFT on all cores",
            "seconds_per_step": dt}


def run_reference(args):
    """The reference arm: the oracle, timed on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = args.workload
    desc, spec, ng, nbins, prec = WORKLOADS[wl]
    cat = make_catalog(spec, np.float32 if prec == "f32" else np.float64)
    n = len(cat["pos"])
    frac = 16 if n >= 4_000_000 else 1
    cb = cpu_baseline(cat, wl, steps=args.steps, warmup=args.warmup, frac=frac)
    line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "particles/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": cb["seconds_per_step"] * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "parallelism": "replicas"}, "cpu_baseline": cb,
            "e2e": {"value": cb["value"], "unit": "particles/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def replica_throughput(elapsed_ms: float, units: int, steps: int, dist=None, device="cpu"):
    """Whole-job throughput of independent replicas: every rank processed `units` per
    step for `steps` steps, and the job took the slowest rank's time (a MAX all-reduce
    over the process group, on `device`: a CUDA device for NCCL, the CPU for gloo).
    Returns (that time in ms, units per second over all ranks)."""
    world = 1
    if dist is not None:
        import torch
        t = torch.tensor([float(elapsed_ms)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
        world = dist.get_world_size()
    return elapsed_ms, world * units * steps / (elapsed_ms * 1e-3)


def _clock_id(torch, dev):
    try:
        return "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        return None


def run_batch64(args):
    """Config 4: 64 uneven catalogues, batched (lanes + one CUDA graph + autotuner) vs
    the plain path (one catalogue after another through pkmom_estimate)."""
    import torch

    from paper_2005_06170_gb300 import catalogs, pkmom
    from paper_2005_06170_gb300.autotune import Autotuner
    from paper_2005_06170_gb300.batch import BatchRunner
    dev = torch.device("cuda", 0)
    counts = catalogs.log_uniform_counts(64, 1e5, 2e7, seed=1004)
    rng = np.random.Generator(np.random.PCG64(1005))
    kinds = rng.random(64) < 0.5
    grids = rng.choice([128, 256, 384], size=64)
    boxes = rng.uniform(300.0, 1500.0, size=64)
    cats, params = [], []
    for i in range(64):
        if kinds[i]:
            side = max(8, int(round(counts[i] ** (1.0 / 3.0))))
            c = catalogs.zeldovich_torch(side, float(boxes[i]), seed=2000 + i, device=dev)
        else:
            c = catalogs.poisson_torch(int(counts[i]), float(boxes[i]), seed=3000 + i, device=dev)
        cats.append(c)
        params.append(pkmom.params(float(boxes[i]), int(grids[i]), 128))
    torch.cuda.synchronize()
    n_total = sum(int(c["pos"].shape[0]) for c in cats)
    cells = sum(int(p.ng) ** 3 for p in params)
    runner = BatchRunner(cats, params, lanes=8, use_graph=True, tuner=Autotuner(repeats=2))
    l0 = runner.kernel_launches()
    runner.run()  # tuning, eager pass, capture
    launches = runner.kernel_launches() - l0
    origin = torch.cuda.current_stream(dev)
    for _ in range(max(3, args.warmup)):
        runner.run()
    torch.cuda.synchronize()
    clocks = ClockSampler(_clock_id(torch, dev))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(origin)
    for _ in range(args.steps):
        runner.run()
    e1.record(origin)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    runner.close()
    # plain: one catalogue at a time through pkmom_estimate on one stream
    ctx = pkmom.Context(0)
    outs = [torch.empty((pkmom.NROWS, p.nbins), dtype=torch.float64, device=dev) for p in params]
    for c, p, o in zip(cats, params, outs):
        ctx.estimate(c["pos"], c["vel"], p, out=o)
    torch.cuda.synchronize()
    e0.record(origin)
    for _ in range(max(1, args.steps // 2)):
        for c, p, o in zip(cats, params, outs):
            ctx.estimate(c["pos"], c["vel"], p, out=o)
    e1.record(origin)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1) / max(1, args.steps // 2)
    ctx.close()
    line = {"metric": METRIC, "value": n_total / (ms * 1e-3), "unit": "particles/s", "n_gpus": 1,
            "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": MULTI["batch64"], "n_particles": n_total, "cells": cells,
                       "l2": "inputs larger than L2, no flush"},
            "Mcells_per_s": cells / (ms * 1e-3) / 1e6, "plain_value": n_total / (ms_plain * 1e-3),
            "plain_ms_per_step": ms_plain, "batched_over_plain": ms_plain / ms,
            "gpu_launches": int(launches), "clocks": clk}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Config 5: a Poisson arrival stream served with continuous batching (4 lanes, one
    of them for large requests; admission by footprint against 180 GB) and, on the same
    trace, one request at a
    time (1 lane): throughput and p50/p99 latency of both."""
    import threading

    import torch

    from paper_2005_06170_gb300 import catalogs, pkmom
    from paper_2005_06170_gb300.serve import Request, Server, percentiles
    dev = torch.device("cuda", 0)
    nreq = args.requests
    rng = np.random.Generator(np.random.PCG64(1006))
    gaps = rng.exponential(1.0 / 20.0, size=nreq)
    t_arr = np.cumsum(gaps)
    counts = np.round(np.exp(rng.uniform(np.log(1e5), np.log(1.3e8), size=nreq))).astype(np.int64)
    grids = rng.choice([128, 256, 512, 1024], size=nreq)
    L = 1000.0
    pool = catalogs.poisson_torch(int(counts.max()), L, seed=1007, device=dev)
    params = [pkmom.params(L, int(g), 128) for g in grids]
    # warm plans and tables on every lane for every grid
    result = {}
    for name, lanes in (("served", 4), ("plain", 1)):
        srv = Server(lanes=lanes, budget_bytes=180e9)
        for ctx, s in zip(srv.ctxs, srv.streams):
            for g in (128, 256, 512, 1024):
                ctx.estimate(pool["pos"][:100000], pool["vel"][:100000], pkmom.params(L, g, 128), stream=s)
        torch.cuda.synchronize()
        clocks = ClockSampler(_clock_id(torch, dev)) if name == "served" else None
        futs = []
        t0 = time.perf_counter()

        def feeder():
            for i in range(nreq):
                wait = t0 + t_arr[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
                n = int(counts[i])
                r = Request(pool["pos"][:n], pool["vel"][:n], params[i], arrival=time.perf_counter())
                futs.append(srv.submit(r))

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        for f in futs:
            f.result(timeout=180)
        t1 = max(r.done for r in srv.completed)
        lat = srv.latencies()
        pc = percentiles(lat)
        result[name] = {"throughput_particles_per_s": float(counts.sum() / (t1 - t0)),
                        "p50_ms": pc["p50"] * 1e3, "p99_ms": pc["p99"] * 1e3,
                        "mean_ms": float(np.mean(lat) * 1e3), "wall_s": t1 - t0, "lanes": lanes}
        if clocks is not None:
            result["clocks"] = clocks.stop()
        srv.close()
    sv, pl = result["served"], result["plain"]
    line = {"metric": METRIC, "value": sv["throughput_particles_per_s"], "unit": "particles/s", "n_gpus": 1,
            "steps": nreq, "warmup": 1, "ms_per_step": sv["mean_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": MULTI["serve"], "requests": nreq, "n_particles": int(counts.sum())},
            "latency_ms": {"p50": sv["p50_ms"], "p99": sv["p99_ms"]},
            "plain": pl, "served": sv, "clocks": result.get("clocks")}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(MULTI))
    ap.add_argument("--requests", type=int, default=300, help="serve: number of requests")
    ap.add_argument("--tile", type=int, default=-1, help="deposit tile id (pkmom_set_tuning); -1 = automatic")
    ap.add_argument("--bl-radius", type=int, default=0,
                    help="0: exact BL kernel; 2..4: the BL function truncated to that many cells, deposited directly")
    ap.add_argument("--impl", default="pkmom", choices=["pkmom", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch64":
        return run_batch64(args)
    if args.workload == "serve":
        return run_serve(args)

    import torch

    from paper_2005_06170_gb300 import pkmom

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    desc, spec, ng, nbins, prec = WORKLOADS[args.workload]
    np_dtype = np.float32 if prec == "f32" else np.float64
    cat = make_catalog(spec, np_dtype)
    n = len(cat["pos"])
    L = spec["L"]
    pos = torch.from_numpy(cat["pos"]).to(dev)
    vel = torch.from_numpy(cat["vel"]).to(dev)
    p = pkmom.params(L, ng, nbins, precision=pkmom.F32 if prec == "f32" else pkmom.F64, bl_radius=args.bl_radius)
    ctx = pkmom.Context(local)
    if args.tile >= 0:
        ctx.set_tuning(args.tile, -1)
    stream = torch.cuda.Stream(device=dev)
    out = torch.empty((pkmom.NROWS, nbins), dtype=torch.float64, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            ctx.estimate(pos, vel, p, out=out, stream=stream)
        ctx.sync(stream)
        ctx.timing(True)
        ctx.timing_read()
        try:
            gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
        except Exception:
            gpu_id = None
        clocks = ClockSampler(gpu_id)
        time.sleep(0.3)
        launches0 = ctx.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            ctx.estimate(pos, vel, p, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        launches = ctx.kernel_launches() - launches0
        stages = ctx.timing_read()
        ctx.timing(False)
        ctx.sync(stream)
    elapsed_ms, value = replica_throughput(e0.elapsed_time(e1), n, args.steps, dist, dev)
    ms_step = elapsed_ms / args.steps
    cells_s = world * ng ** 3 * args.steps / (elapsed_ms * 1e-3)

    # roofline of the dominant own kernel, from the stage events of the timed region
    peak, peak_kind = load_peaks()
    stage_ms = {s: (ms / c if c else 0.0) for s, (ms, c) in stages.items()}
    own = {s: v for s, v in stage_ms.items() if s not in ("fft",)}
    dom = max(own, key=own.get)
    nh = ng // 2 + 1
    elem = 4 if prec == "f32" else 8
    umax2 = (ng / 2) ** 2
    nb_modes = None
    if dom == "bin":
        f = np.fft.fftfreq(ng, 1.0 / ng)
        n2 = f[:, None] ** 2 + f[None, :] ** 2
        nz = np.arange(nh) ** 2
        nb_modes = int(sum(np.count_nonzero((n2 + z <= umax2) & (n2 + z > 0)) for z in nz))
    alg_bytes = {
        "deposit": n * 8 * elem + 4 * elem * ng ** 3,
        "bin": (nb_modes or 0) * 4 * 2 * elem,
        "hist": n * 6 * elem + 4 * n,
        "scatter": n * (6 * elem + 4 + 8 * elem),
        "scan": 12 * ng ** 3,
        "final": 0,
    }[dom]
    achieved = alg_bytes / (stage_ms[dom] * 1e-3) / 1e9 if stage_ms[dom] > 0 else None
    home = prec == "f32" and ng % 16 == 0 and n >= ng ** 3 / 2  # the library's home-tile deposit
    home = home and not args.bl_radius
    deposit_kernels = "k_deposit_home + k_home_fixup" if home else ("k_deposit_fx" if prec == "f32" else "k_deposit")
    traffic = None if args.bl_radius else MEASURED_TRAFFIC.get((args.workload, dom))
    roof = {"kernel": {"deposit": deposit_kernels, "bin": "k_bin_shells + k_reduce_items", "hist": "k_hist",
                       "scatter": "k_scatter", "scan": "k_scan_*", "final": "k_finalize"}[dom],
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": traffic[0] if traffic else None,
            "traffic_source": traffic[1] if traffic else None,
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": stage_ms[dom]}

    line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": desc + (f"; BL function truncated to {args.bl_radius} cells, direct deposit"
                                           if args.bl_radius else ""),
                       "n_particles": n, "ng": ng, "nbins": nbins, "box_L": L,
                       "bulk": "with and without", "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2: catalogue {n * 6 * elem / 1e6:.0f} MB, grids "
                             f"{4 * ng * ng * (ng + 2) * elem / 1e6:.0f} MB, no flush"},
            "Mcells_per_s": cells_s / 1e6, "stages_ms_per_step": stage_ms, "roofline": roof,
            "gpu_launches": int(launches), "clocks": clk}

    if rank == 0 and not args.no_e2e:
        # end to end through the public host API with pinned host buffers: every step
        # copies its catalogue in and reads its spectra back. HostPipeline copies
        # catalogue i+1 while catalogue i is estimated (the link moves ~210 GB/s, about
        # the estimate's own pace at this size); pkmom_estimate_host (one call per step,
        # copies not overlapped) is reported beside it. The pipelined stream is 40
        # catalogues long: its timed region includes the first copy, which nothing
        # overlaps (about one step's time, spread over the stream).
        from paper_2005_06170_gb300.pipeline import HostPipeline
        hp = torch.from_numpy(cat["pos"]).pin_memory()
        hv = torch.from_numpy(cat["vel"]).pin_memory()
        hout = torch.empty((pkmom.NROWS, nbins), dtype=torch.float64).pin_memory()
        k_e = max(3, min(args.steps, 10))
        k_pipe = 40
        pipe = HostPipeline(n_max=n, nbins_max=nbins, precision=p.precision)
        pipe.submit(hp, hv, p).result()  # warm-up: plans, tables, buffers
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        prev = None
        for _ in range(k_pipe):
            cur = pipe.submit(hp, hv, p)
            if prev is not None:
                prev.result()
            prev = cur
        prev.result()
        dt = (time.perf_counter() - t0) / k_pipe
        pipe.close()
        hpn, hvn, hon = hp.numpy(), hv.numpy(), hout.numpy()
        ctx.estimate_host(hpn, hvn, p, out=hon, stream=stream)
        t1 = time.perf_counter()
        for _ in range(k_e):
            ctx.estimate_host(hpn, hvn, p, out=hon, stream=stream)
        dt1 = (time.perf_counter() - t1) / k_e
        line["e2e"] = {"value": n / dt, "unit": "particles/s", "h2d_bytes_per_step": int(hp.nbytes + hv.nbytes),
                       "d2h_bytes_per_step": int(hout.nbytes), "ms_per_step": dt * 1e3, "steps": k_pipe,
                       "api": "HostPipeline (copy of step i+1 overlaps the estimate of step i)",
                       "single_call": {"value": n / dt1, "ms_per_step": dt1 * 1e3, "steps": k_e,
                                       "api": "pkmom_estimate_host"}}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, args.workload)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
