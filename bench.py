#!/usr/bin/env python
"""Benchmark of the momentum power-spectrum estimator (one JSON line on stdout).

A step is one whole estimate (moments, BL assignment, four R2C FFTs, deconvolution,
shot noise and shell binning of P_dd, P_pp, P_tt, P_dt with and without the bulk
flow) of one synthetic catalogue already resident in HBM. Default workload: the
largest single-GPU configuration, a Zel'dovich catalogue of 512^3 particles in a
1500 Mpc/h box on a 512^3 FP32 grid with 128 shells. The same line carries, as extra
keys, the same catalogue on a 1024^3 grid, the resolution-pair aliasing report of
Sec. 2.4.3, the batched workload (64 uneven catalogues, batched against one at a
time) and the served workload (a Poisson arrival stream, p50/p99 latency served
against one at a time). Under torchrun every rank runs an independent replica on its
own GPU (the estimate of one catalogue does not shard); the slowest rank's time counts.

    python bench.py [--steps K] [--warmup W] [--workload NAME] [--impl reference]
"""
from __future__ import annotations

import argparse
import gc
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
    "zeldovich512_ng512": ("Zel'dovich 512^3 particles, L=1500 Mpc/h, 512^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow", dict(kind="zeldovich", n_side=512, L=1500.0, seed=1002),
                           512, 128, "f32"),
    "zeldovich512_ng1024": ("Zel'dovich 512^3 particles, L=1500 Mpc/h, 1024^3 FP32 grid, BL3, 128 shells, "
                            "with and without bulk flow", dict(kind="zeldovich", n_side=512, L=1500.0, seed=1002),
                            1024, 128, "f32"),
    "zeldovich256_ng256": ("Zel'dovich 256^3 particles, L=1000 Mpc/h, 256^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow", dict(kind="zeldovich", n_side=256, L=1000.0, seed=1001),
                           256, 128, "f32"),
    "poisson32768_ng64_fp64": ("32768 Poisson particles, L=256 Mpc/h, sigma_v=300 km/s, 64^3 FP64 grid, BL3, "
                               "32 shells", dict(kind="poisson", n=32768, L=256.0, seed=1000), 64, 32, "f64"),
    "zeldovich256_ng512": ("Zel'dovich 256^3 particles, L=1000 Mpc/h, 512^3 FP32 grid, BL3, 128 shells, "
                           "with and without bulk flow (0.125 particle per cell)",
                           dict(kind="zeldovich", n_side=256, L=1000.0, seed=1001), 512, 128, "f32"),
    "poisson830k_ng384": ("830,584 Poisson particles, L=900 Mpc/h, 384^3 FP32 grid, BL3, 128 shells (0.015 particle "
                          "per cell, as in the sparsest catalogues of the batch)",
                          dict(kind="poisson", n=830584, L=900.0, seed=5), 384, 128, "f32"),
}
DEFAULT = "zeldovich512_ng512"
# DRAM bytes (read + write) per launch of the dominant stage's kernels, from one ncu
# capture of the current kernels; a stage whose kernels change drops its entry until
# it is captured again
MEASURED_TRAFFIC = {
    ("zeldovich512_ng512", "deposit"): ((4981.8 + 3626.1 + 3716.0 + 1623.8) * 1e6,
                                        "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_deposit_home and "
                                        "k_home_fixup, mean of 5 launches of the 512^3 workload "
                                        "(profiles/launches_zeldovich512_ng512.md)"),
    # the same density (1/8 particle per cell) captured at 256^3 particles on 512^3 and
    # scaled by 8: the records read, the key rows read and the grid written all grow with
    # the particles and cells, which are both 8 times as many
    ("zeldovich512_ng1024", "deposit"): (8 * (1.27 + 2.11) * 1e9,
                                         "ncu dram__bytes_read.sum + dram__bytes_write.sum of one k_deposit_fx "
                                         "launch on 256^3 particles and a 512^3 grid "
                                         "(profiles/deposit_sparse_zeldovich256_ng512.md), times 8"),
}
# warp instructions per launch of the dominant kernel, from one ncu --set full capture of
# the current kernel on the 256^3 workload, scaled to other workloads by particle count
# (the same work per particle at one particle per cell)
MEASURED_INSTRUCTIONS = {
    "k_deposit_home": (596.13e6, 256 ** 3, "ncu smsp__inst_executed.sum of k_deposit_home on the 256^3 workload "
                                         "(profiles/kernels_zeldovich256_ng256.md), scaled by particles"),
}
# configs 4 and 5 run through their own drivers below
MULTI = {
    "batch64": "64 catalogues in one launch sequence: particle counts log-uniform in [1e5, 2e7], seeded "
               "Zel'dovich or Poisson (50/50), grids from {128, 256, 384}^3, L in [300, 1500] Mpc/h, "
               "FP32, 128 shells; persistent deposit and binning kernels + CUDA graph + autotuned tiles",
    "serve": "Poisson arrivals of estimation requests, each its own seeded Poisson catalogue drawn on the "
             "device at arrival, particle counts log-uniform in [1e5, 1.3e8], grids from {128, 256, 512, "
             "1024}^3, FP32, 128 shells, admitted by HBM footprint against 180 GB",
}
# FP32 lanes of the part: 152 SMs x 128 lanes, 2 FLOP per FMA, at the 2070 MHz maximum SM clock
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# warp instructions issued per second at one per SM sub-partition per clock (152 x 4)
ISSUE_PEAK_WARP_INSTR = 152 * 4 * 2.07e9


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


def oracle_step(cat, spec, ng, nbins, dep_frac, slab_frac):
    """One estimate of the oracle as it stands on a bounded sample of the workload: the
    deposit of the first 1/dep_frac of the particles (single-threaded C), the FFT of the
    full grids (scipy, all host cores) and the binning of every slab_frac-th slab (numpy).
    Returns the stage times in seconds and the full-step time they extrapolate to
    (deposit x dep_frac + FFT + binning x slab_frac)."""
    from oracle import estimator as est
    n = len(cat["pos"])
    m = max(1, n // dep_frac)
    t0 = time.perf_counter()
    mom = est.moments(cat["vel"][:m])
    grids = est.assign(cat["pos"][:m], cat["vel"][:m], None, L=spec["L"], ng=ng)
    t1 = time.perf_counter()
    F = est.fft_grids(grids)
    del grids
    t2 = time.perf_counter()
    est.spectra_from_fourier(F, mom, L=spec["L"], ng=ng, nbins=nbins, slabs=range(0, ng, slab_frac))
    t3 = time.perf_counter()
    dep, fft, bins = t1 - t0, t2 - t1, t3 - t2
    return {"deposit_s": dep, "fft_s": fft, "bin_s": bins, "sample_s": t3 - t0,
            "full_step_s": dep * (n / m) + fft + bins * slab_frac}


def sample_fractions(n, ng):
    """(particle fraction, slab fraction) of the oracle's bounded sample: a few seconds
    per sampled step at the largest workloads, the whole estimate for small ones."""
    dep = 1 if n <= 4_000_000 else 64
    slab = 1 if ng <= 128 else 16
    return dep, slab


def cpu_baseline(cat, wl, steps=1, warmup=0):
    """The oracle as it stands, timed on the host cores on a bounded sample of the same
    workload, extrapolated to one full estimate and reported per particle."""
    from oracle import estimator as est
    desc, spec, ng, nbins, _ = WORKLOADS[wl]
    n = len(cat["pos"])
    dep, slab = sample_fractions(n, ng)
    est.estimate(cat["pos"][:1000], cat["vel"][:1000], L=spec["L"], ng=16, nbins=4)  # builds the C part
    for _ in range(warmup):
        oracle_step(cat, spec, ng, nbins, dep, slab)
    runs = [oracle_step(cat, spec, ng, nbins, dep, slab) for _ in range(steps)]
    full = sum(r["full_step_s"] for r in runs) / len(runs)
    sample = (f"deposit of the first 1/{dep} of the catalogue's {n} particles (single-threaded C), FFT of the "
              f"full four {ng}^3 FP64 grids (scipy, {os.cpu_count()} threads) and binning of every {slab}-th "
              f"slab (numpy, one thread), extrapolated to one full estimate: deposit x {dep} + FFT + "
              f"binning x {slab}")
    return {"value": n / full, "unit": "particles/s", "cores": os.cpu_count(),
            "cores_by_stage": {"deposit": 1, "fft": os.cpu_count(), "binning": 1}, "kind": "oracle",
            "sample": sample, "seconds_per_step": full, "sampled_seconds_per_step": runs[-1]["sample_s"],
            "stages_s": {k: runs[-1][k] for k in ("deposit_s", "fft_s", "bin_s")}}


def run_reference(args):
    """The reference arm: the oracle, timed on the host cores, rank 0 only."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = args.workload if args.workload in WORKLOADS else DEFAULT
    desc, spec, ng, nbins, prec = WORKLOADS[wl]
    cat = make_catalog(spec, np.float32 if prec == "f32" else np.float64)
    cb = cpu_baseline(cat, wl, steps=args.steps, warmup=args.warmup)
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


def time_estimates(ctx, pos, vel, p, out, stream, steps, warmup, torch, dev, barrier=lambda: None):
    """W untimed and K timed estimates on one stream; stage times from the library's
    CUDA events recorded on that stream during the timed region."""
    with torch.cuda.stream(stream):
        for _ in range(max(3, warmup)):
            ctx.estimate(pos, vel, p, out=out, stream=stream)
        ctx.sync(stream)
        ctx.timing(True)
        ctx.timing_read()
        clocks = ClockSampler(_clock_id(torch, dev))
        time.sleep(0.3)
        launches0 = ctx.kernel_launches()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(steps):
            ctx.estimate(pos, vel, p, out=out, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        clk = clocks.stop()
        launches = ctx.kernel_launches() - launches0
        stages = ctx.timing_read()
        ctx.timing(False)
        ctx.sync(stream)
    stage_ms = {s: (ms / c if c else 0.0) for s, (ms, c) in stages.items()}
    return e0.elapsed_time(e1), stage_ms, launches, clk


def deposit_kernels(n, ng, prec, bl_radius):
    home = prec == "f32" and ng % 16 == 0 and n >= ng ** 3 / 2 and not bl_radius  # the library's choice
    return "k_deposit_home + k_home_fixup" if home else ("k_deposit_fx" if prec == "f32" else "k_deposit")


def roofline(workload, stage_ms, n, ng, prec, bl_radius, unit_mass=True):
    """Roofline of the deposit, the dominant own kernel: algorithmic bytes per launch
    (24 B per particle read (positions and velocities; 4 more with masses) + 16 B per
    cell written (four FP32 grids)), algorithmic FP32 work (one FMA per node and field:
    64 nodes x 4 fields per particle, 512 FLOP), the launch's average time from the CUDA
    events of the timed region. Bound: instruction issue and the FP32 pipes (ncu: issue
    active well above DRAM throughput), reported against the FP32 peak, with the HBM
    fraction beside it."""
    peak, peak_kind = load_peaks()
    elem = 4 if prec == "f32" else 8
    ms = stage_ms["deposit"]
    alg_bytes = n * (6 + (0 if unit_mass else 1)) * elem + 4 * elem * ng ** 3
    nodes = (2 * bl_radius) ** 3 if bl_radius else 64
    flops = 2.0 * nodes * 4 * n
    gbs = alg_bytes / (ms * 1e-3) / 1e9 if ms > 0 else None
    tflops = flops / (ms * 1e-3) / 1e12 if ms > 0 else None
    traffic = None if bl_radius else MEASURED_TRAFFIC.get((workload, "deposit"))
    kern = deposit_kernels(n, ng, prec, bl_radius)
    issue = None
    ins = MEASURED_INSTRUCTIONS.get(kern.split(" ")[0])
    if ins and ms > 0:
        per_launch = ins[0] * n / ins[1]
        rate = per_launch / (ms * 1e-3)
        issue = {"warp_instructions_per_launch": per_launch, "achieved": rate, "peak": ISSUE_PEAK_WARP_INSTR,
                 "unit": "warp instructions/s", "frac": rate / ISSUE_PEAK_WARP_INSTR,
                 "peak_source": "derived: 152 SMs x 4 schedulers x 2070 MHz", "source": ins[2],
                 "note": "time of the whole stage (with k_home_fixup), so the kernel's own rate is higher"}
    return {"kernel": kern, "bound": "alu", "achieved": tflops,
            "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": (tflops / FP32_PEAK_TFLOPS) if tflops else None,
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 FLOP x 2070 MHz",
            "algorithmic_flops_per_launch": flops,
            "traffic": traffic[0] if traffic else None, "traffic_source": traffic[1] if traffic else None,
            "hbm": {"achieved": gbs, "peak": peak, "unit": "GB/s", "frac": (gbs / peak) if gbs else None,
                    "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                    else "fallback", "algorithmic_bytes_per_launch": alg_bytes},
            "issue": issue, "avg_launch_ms": ms}


def _isqrt(x):
    r = np.floor(np.sqrt(x.astype(np.float64))).astype(np.int64)
    r -= (r * r > x)
    r += ((r + 1) * (r + 1) <= x)
    return r


def in_shell_modes(ng, umin=1.0, umax=None):
    """Modes (n0, n1, l) of the ng^3 half spectrum with umin <= |n| <= umax (umax: ng/2),
    the ones the binning reads: the shells of the bench's workloads span that range."""
    umax = ng / 2 if umax is None else umax
    lo2, hi2 = int(np.ceil(umin * umin)), int(np.floor(umax * umax))
    n = np.arange(-(ng // 2), ng // 2, dtype=np.int64)
    r2 = n[:, None] ** 2 + n[None, :] ** 2
    top = hi2 - r2
    lmax = np.minimum(_isqrt(np.maximum(top, 0)), ng // 2)
    need = lo2 - r2
    lmin = np.where(need <= 0, 0, _isqrt(np.maximum(need - 1, 0)) + 1)
    cnt = np.where(top >= 0, np.maximum(lmax - lmin + 1, 0), 0)
    return int(cnt.sum())


def bin_roofline(stage_ms, ng, prec):
    """The binning stage against HBM. `achieved` counts the bytes the binning must read:
    the four complex values (32 B in FP32) of every half-spectrum mode inside the shell
    range (about pi/6 of the half spectrum when the shells end at the Nyquist frequency);
    `frac_16B_per_cell` counts the whole ng x ng x (ng/2 + 1) half spectra (16 B per grid
    cell), which the kernel does not read in full."""
    peak, _ = load_peaks()
    elem = 4 if prec == "f32" else 8
    full = 4 * 2 * elem * ng * ng * (ng // 2 + 1)
    b = 4 * 2 * elem * in_shell_modes(ng)
    ms = stage_ms["bin"]
    gbs = b / (ms * 1e-3) / 1e9 if ms > 0 else None
    return {"kernel": "k_bin_shells + k_reduce_items", "bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak if gbs else None, "algorithmic_bytes_per_launch": b, "avg_launch_ms": ms,
            "bytes_16B_per_cell": full, "frac_16B_per_cell": full / (ms * 1e-3) / 1e9 / peak if ms > 0 else None}


def e2e_host(ctx, cat, p, stream, torch, k_pipe=30, k_single=7):
    """End to end through the library's host entry points with pinned host buffers: every
    step copies its catalogue in and its spectra out. pkmom_estimate_host_async copies
    catalogue i+1 on the library's copy stream while catalogue i is estimated; its timed
    stream includes the first copy, which nothing overlaps. pkmom_estimate_host (copies
    not overlapped) is reported beside it."""
    from paper_2005_06170_gb300 import pkmom
    from paper_2005_06170_gb300.pipeline import HostPipeline
    n = len(cat["pos"])
    hp = torch.from_numpy(cat["pos"]).pin_memory()
    hv = torch.from_numpy(cat["vel"]).pin_memory()
    pipe = HostPipeline(n_max=n, nbins_max=p.nbins, precision=p.precision)
    # warm-up: plans, tables, buffers and both staging slots (the second is allocated by
    # the second call)
    for _ in range(2):
        pipe.submit(hp, hv, p).result()
    torch.cuda.synchronize()
    # the Python collector paused while the host loops are timed (as timeit does): a full
    # collection of this process's objects takes about as long as several estimates
    gc.collect()
    gc_was = gc.isenabled()
    gc.disable()
    t0 = time.perf_counter()
    prev = None
    done = []  # host time at which each step's result was in hand
    for _ in range(k_pipe):
        cur = pipe.submit(hp, hv, p)
        if prev is not None:
            prev.result()
            done.append(time.perf_counter())
        prev = cur
    prev.result()
    done.append(time.perf_counter())
    dt = (time.perf_counter() - t0) / k_pipe
    gaps = np.diff(np.asarray([t0] + done))
    pipe.close()
    hout = np.empty((pkmom.NROWS, p.nbins))
    hpn, hvn = hp.numpy(), hv.numpy()
    ctx.estimate_host(hpn, hvn, p, out=hout, stream=stream)
    calls = []
    for _ in range(k_single):
        t1 = time.perf_counter()
        ctx.estimate_host(hpn, hvn, p, out=hout, stream=stream)
        calls.append(time.perf_counter() - t1)
    if gc_was:
        gc.enable()
    dt1 = float(np.median(calls))  # a call now and then takes far longer on a shared host
    return {"value": n / dt, "unit": "particles/s", "h2d_bytes_per_step": int(hp.nbytes + hv.nbytes),
            "d2h_bytes_per_step": int(pkmom.NROWS * p.nbins * 8), "ms_per_step": dt * 1e3, "steps": k_pipe,
            "api": "pkmom_estimate_host_async + pkmom_wait (copy of step i+1 overlaps the estimate of step i)",
            "step_intervals_ms": {"median": float(np.median(gaps[1:]) * 1e3), "max": float(gaps.max() * 1e3),
                                  "argmax": int(gaps.argmax()),
                                  "first": float(gaps[0] * 1e3),
                                  "note": "value is the mean over all steps; the first interval holds the "
                                          "first copy, which nothing overlaps"},
            "single_call": {"value": n / dt1, "ms_per_step": dt1 * 1e3, "steps": k_single,
                            "ms_per_call": [round(c * 1e3, 3) for c in calls], "statistic": "median",
                            "api": "pkmom_estimate_host"}}


def batch64(args, torch):
    """Config 4: 64 uneven catalogues, batched (lanes + one CUDA graph + autotuner) vs the
    plain path (one catalogue after another through pkmom_estimate on one stream)."""
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
    origin = torch.cuda.current_stream(dev)
    steps = max(3, args.batch_steps)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    timed = {}
    clk = None
    launches = 0
    for mode in ("fused", "lanes"):
        runner = BatchRunner(cats, params, lanes=8, use_graph=True, tuner=Autotuner(repeats=2),
                             fused=mode == "fused")
        l0 = runner.kernel_launches()
        runner.run()  # tuning, eager pass, capture
        if mode == "fused":
            launches = runner.kernel_launches() - l0
        for _ in range(3):
            runner.run()
        torch.cuda.synchronize()
        clocks = ClockSampler(_clock_id(torch, dev)) if mode == "fused" else None
        e0.record(origin)
        for _ in range(steps):
            runner.run()
        e1.record(origin)
        torch.cuda.synchronize()
        timed[mode] = e0.elapsed_time(e1) / steps
        if clocks is not None:
            clk = clocks.stop()
        runner.close()
    ms = timed["fused"]
    ctx = pkmom.Context(0)
    outs = [torch.empty((pkmom.NROWS, p.nbins), dtype=torch.float64, device=dev) for p in params]
    for c, p, o in zip(cats, params, outs):
        ctx.estimate(c["pos"], c["vel"], p, out=o)
    torch.cuda.synchronize()
    e0.record(origin)
    for _ in range(steps):
        for c, p, o in zip(cats, params, outs):
            ctx.estimate(c["pos"], c["vel"], p, out=o)
    e1.record(origin)
    torch.cuda.synchronize()
    ms_plain = e0.elapsed_time(e1) / steps
    ctx.close()
    return {"workload": MULTI["batch64"], "n_particles": n_total, "cells": cells, "steps": steps,
            "batched_ms": ms, "plain_ms": ms_plain, "batched_over_plain": ms_plain / ms,
            "batched": "pkmom_estimate_batch (persistent deposit and binning kernels) in one CUDA graph",
            "lanes_ms": timed["lanes"], "lanes": "8 lanes (contexts and streams) in one CUDA graph",
            "kernel_launches_per_batch": int(launches),
            "batched_particles_per_s": n_total / (ms * 1e-3), "plain_particles_per_s": n_total / (ms_plain * 1e-3),
            "batched_Mcells_per_s": cells / (ms * 1e-3) / 1e6, "clocks": clk,
            "note": "graph replays launch no kernels from the host; the count is of the eager pass"}


def serve_trace(nreq, rate, seed=1006):
    rng = np.random.Generator(np.random.PCG64(seed))
    t_arr = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    counts = np.round(np.exp(rng.uniform(np.log(1e5), np.log(1.3e8), size=nreq))).astype(np.int64)
    grids = rng.choice([128, 256, 512, 1024], size=nreq)
    return t_arr, counts, grids


def serve(args, torch, rate, nreq, warm=20):
    """Config 5: a Poisson arrival stream served with continuous batching (4 lanes, one
    of them for large requests; admission by footprint against 180 GB) and, on the same
    trace, one request at a time (1 lane). Each request's catalogue is its own seeded
    Poisson catalogue, drawn on the device by the feeder at its arrival time (on the
    feeder's stream; the server orders the estimate after it). Latency runs from arrival
    to the spectra on the host. The first `warm` requests are not counted."""
    from paper_2005_06170_gb300 import catalogs, pkmom
    from paper_2005_06170_gb300.serve import Request, Server, percentiles
    dev = torch.device("cuda", 0)
    total = nreq + warm
    t_arr, counts, grids = serve_trace(total, rate)
    L = 1000.0
    params = [pkmom.params(L, int(g), 128) for g in grids]
    result = {}
    arms = [a for a in (("served", args.serve_lanes), ("plain", 1)) if not args.serve_only or a[0] == args.serve_only]
    for name, lanes in arms:
        srv = Server(lanes=lanes, budget_bytes=180e9, large_priority=args.serve_priority)
        srv.warm((128, 256, 512, 1024), nbins=128, box_L=L)
        # a burst of the extreme sizes before the clock starts: the first launch of every
        # kernel and the allocator's first blocks of each size are not part of the trace
        burst = []
        for g in (128, 256, 512, 1024):
            for k, n in enumerate((100_000, int(counts.max()))):
                c = catalogs.poisson_torch(n, L, seed=90_000 + 10 * g + k, device=dev)
                burst.append(srv.submit(Request(c["pos"], c["vel"], pkmom.params(L, g, 128))))
                del c
        for f in burst:
            f.result(timeout=600)
        srv.completed.clear()
        clocks = ClockSampler(_clock_id(torch, dev)) if name == "served" else None
        futs = []
        reqs = []
        t0 = time.perf_counter()

        def feeder():
            torch.cuda.set_device(dev)
            s = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(s):
                for i in range(total):
                    wait = t0 + t_arr[i] - time.perf_counter()
                    if wait > 0:
                        time.sleep(wait)
                    arrival = time.perf_counter()
                    c = catalogs.poisson_torch(int(counts[i]), L, seed=5000 + i, device=dev)
                    r = Request(c["pos"], c["vel"], params[i], arrival=arrival)
                    reqs.append(r)
                    futs.append(srv.submit(r))
                    del c

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        for f in futs:
            f.result(timeout=600)
        t1 = max(r.done for r in srv.completed)
        counted = reqs[warm:]
        lat = [r.done - r.arrival for r in counted]
        pc = percentiles(lat)
        span = t1 - t0
        result[name] = {"throughput_particles_per_s": float(counts.sum() / span),
                        "p50_ms": pc["p50"] * 1e3, "p99_ms": pc["p99"] * 1e3,
                        "mean_ms": float(np.mean(lat) * 1e3), "max_ms": float(np.max(lat) * 1e3),
                        "wall_s": span, "lanes": lanes, "requests": nreq, "warmup_requests": warm}
        if clocks is not None:
            result["clocks"] = clocks.stop()
        srv.close()
        torch.cuda.empty_cache()
    result["rate_per_s"] = rate
    result["workload"] = MULTI["serve"]
    return result


def run_batch64(args):
    import torch
    b = batch64(args, torch)
    line = {"metric": METRIC, "value": b["batched_particles_per_s"], "unit": "particles/s", "n_gpus": 1,
            "steps": b["steps"], "warmup": 3, "ms_per_step": b["batched_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": MULTI["batch64"], "n_particles": b["n_particles"], "cells": b["cells"],
                       "l2": "inputs larger than L2, no flush"},
            "Mcells_per_s": b["batched_Mcells_per_s"], "plain_value": b["plain_particles_per_s"],
            "plain_ms_per_step": b["plain_ms"], "batched_over_plain": b["batched_over_plain"],
            "lanes_ms_per_step": b["lanes_ms"], "batched": b["batched"], "lanes": b["lanes"],
            "gpu_launches": b["kernel_launches_per_batch"], "clocks": b["clocks"]}
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    import torch
    reps = []
    for k in range(max(1, args.repeats)):
        reps.append(serve(args, torch, args.rate, args.requests))
    sv, pl = reps[0].get("served", {}), reps[0].get("plain", {})
    head = sv or pl
    line = {"metric": METRIC, "value": head["throughput_particles_per_s"], "unit": "particles/s", "n_gpus": 1,
            "steps": args.requests, "warmup": 20, "ms_per_step": head["mean_ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": MULTI["serve"], "requests": args.requests, "rate_per_s": args.rate,
                       "lanes": args.serve_lanes, "large_priority": args.serve_priority},
            "latency_ms": {"p50": head["p50_ms"], "p99": head["p99_ms"]},
            "plain": pl, "served": sv, "repeats": [{a: {k: r[a][k] for k in ("p50_ms", "p99_ms")}
                                                    for a in ("served", "plain") if a in r} for r in reps],
            "clocks": reps[0].get("clocks")}
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--workload", default=DEFAULT, choices=sorted(WORKLOADS) + sorted(MULTI))
    ap.add_argument("--requests", type=int, default=2000, help="serve: requests after 20 warm-up ones")
    ap.add_argument("--rate", type=float, default=20.0, help="serve: mean arrivals per second")
    ap.add_argument("--repeats", type=int, default=1, help="serve: repeats of the whole trace")
    ap.add_argument("--batch-steps", type=int, default=5, help="batch64: timed replays")
    ap.add_argument("--serve-lanes", type=int, default=4, help="serve: lanes of the served run")
    ap.add_argument("--serve-priority", default="low", choices=["low", "same", "high"],
                    help="serve: stream priority of the lane for large requests")
    ap.add_argument("--serve-only", default="", choices=["", "served", "plain"],
                    help="serve: run only one of the two arms")
    ap.add_argument("--tile", type=int, default=-1, help="deposit tile id (pkmom_set_tuning); -1 = automatic")
    ap.add_argument("--bl-radius", type=int, default=0,
                    help="0: exact BL kernel; 2..4: the BL function truncated to that many cells, deposited directly")
    ap.add_argument("--impl", default="pkmom", choices=["pkmom", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="default workload: leave out the 1024^3 grid, batched and served extra keys")
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

    el, stage_ms, launches, clk = time_estimates(ctx, pos, vel, p, out, stream, args.steps, args.warmup, torch, dev,
                                                 barrier)
    elapsed_ms, value = replica_throughput(el, n, args.steps, dist, dev)
    ms_step = elapsed_ms / args.steps
    cells_s = world * ng ** 3 * args.steps / (elapsed_ms * 1e-3)
    elem = 4 if prec == "f32" else 8
    line = {"metric": METRIC, "value": value, "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": prec, "data": "synthetic",
            "config": {"workload": desc + (f"; BL function truncated to {args.bl_radius} cells, direct deposit"
                                           if args.bl_radius else ""),
                       "n_particles": n, "ng": ng, "nbins": nbins, "box_L": L,
                       "bulk": "with and without", "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": f"inputs larger than L2: catalogue {n * 6 * elem / 1e6:.0f} MB, grids "
                             f"{4 * ng * ng * (ng + 2) * elem / 1e6:.0f} MB, no flush"},
            "Mcells_per_s": cells_s / 1e6, "stages_ms_per_step": stage_ms,
            "roofline": roofline(args.workload, stage_ms, n, ng, prec, args.bl_radius),
            "bin_roofline": bin_roofline(stage_ms, ng, prec),
            "gpu_launches": int(launches), "clocks": clk}

    extras = rank == 0 and world == 1 and args.workload == DEFAULT and not args.no_extras and not args.bl_radius
    if extras:
        # the same catalogue on a 1024^3 grid (config 3's second grid)
        p2 = pkmom.params(L, 2 * ng, nbins)
        out2 = torch.empty((pkmom.NROWS, nbins), dtype=torch.float64, device=dev)
        k2 = max(3, args.steps // 4)
        el2, st2, l2, clk2 = time_estimates(ctx, pos, vel, p2, out2, stream, k2, 3, torch, dev)
        line["ng1024"] = {"workload": WORKLOADS["zeldovich512_ng1024"][0], "steps": k2, "ms_per_step": el2 / k2,
                          "particles_per_s": n * k2 / (el2 * 1e-3), "Mcells_per_s": (2 * ng) ** 3 * k2 / el2 / 1e3,
                          "stages_ms_per_step": st2,
                          "roofline": roofline("zeldovich512_ng1024", st2, n, 2 * ng, prec, 0),
                          "bin_roofline": bin_roofline(st2, 2 * ng, prec), "gpu_launches": int(l2), "clocks": clk2}
        from paper_2005_06170_gb300.aliasing import resolution_pair
        line["resolution_pair"] = resolution_pair(ctx, pos, vel, L, ng, nbins, stream=stream)

    if rank == 0 and not args.no_e2e:
        line["e2e"] = e2e_host(ctx, cat, p, stream, torch)
    ctx.close()
    del pos, vel
    torch.cuda.empty_cache()
    if extras:
        line["batch64"] = batch64(args, torch)
        torch.cuda.empty_cache()
        line["serve"] = serve(args, torch, args.rate, args.requests)
        sv, pl = line["serve"]["served"], line["serve"]["plain"]
        line["latency_ms"] = {"served": {"p50": sv["p50_ms"], "p99": sv["p99_ms"]},
                              "plain": {"p50": pl["p50_ms"], "p99": pl["p99_ms"]},
                              "batched_ms": line["batch64"]["batched_ms"], "plain_ms": line["batch64"]["plain_ms"]}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(cat, args.workload)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
