"""Batched estimation of many catalogues of uneven sizes and grids (one GPU).

Two ways to run a batch:

* fused (default): one libpkmom context and one stream; the whole batch is one call of
  pkmom_estimate_batch, which sorts each catalogue, deposits every catalogue that takes
  the gather deposit in ONE persistent kernel (CTAs draw (catalogue, tile) items from a
  work counter) and bins every FP32 catalogue in ONE persistent kernel;
* lanes: the catalogues are dealt to a few lanes (largest first, each to the least
  loaded lane); a lane owns a context (its own cuFFT plans and tables: a cuFFT plan must
  not run on two streams at once) and a CUDA stream, and runs its catalogues one after
  another, so the lanes' catalogues overlap on the device.

Every catalogue has its own grids, scratch, moments and output, allocated once. The
first run is eager (it builds plans and tables and runs the autotuner); it is then
captured into one CUDA graph, which later runs replay with a single launch.
"""
from __future__ import annotations

import torch

from . import pkmom
from .autotune import HOME_TILE, Autotuner


def deal(costs: list[float], lanes: int) -> list[int]:
    """Lane of each item: largest first, each to the least loaded lane (ties: lowest lane)."""
    load = [0.0] * lanes
    out = [0] * len(costs)
    for i in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        lane = min(range(lanes), key=lambda k: (load[k], k))
        out[i] = lane
        load[lane] += costs[i]
    return out


class _Item:
    __slots__ = ("cat", "p", "pos", "vel", "mass", "grids", "mom", "scratch", "out", "tile", "cap", "lane", "cost")


class BatchRunner:
    def __init__(self, catalogs: list[dict], params: list, lanes: int = 4, use_graph: bool = True,
                 tuner: Autotuner | None = None, device: int = 0, fused: bool = True):
        """catalogs: dicts with CUDA tensors pos (n,3), vel (n,3), optional mass (n,);
        params: one pkmom.Params per catalogue. fused: one pkmom_estimate_batch call per
        run (persistent deposit and binning kernels); otherwise `lanes` lanes."""
        if len(catalogs) != len(params):
            raise ValueError("one Params per catalogue")
        self.device = device
        self.use_graph = use_graph
        self.tuner = tuner
        self.fused = fused
        self.gpu = torch.cuda.get_device_name(device)
        nl = 1 if fused else max(1, min(lanes, len(catalogs)))
        self.ctxs = [pkmom.Context(device) for _ in range(nl)]
        self.streams = [torch.cuda.Stream(device=device) for _ in range(nl)]
        self.items: list[_Item] = []
        for c, p in zip(catalogs, params):
            it = _Item()
            it.pos, it.vel, it.mass = c["pos"], c["vel"], c.get("mass")
            it.cat = pkmom.catalog_from_tensors(it.pos, it.vel, it.mass)
            it.p = p
            it.cost = it.cat.n + 2.0 * p.ng ** 3  # rough work estimate: particles + cells
            self.items.append(it)
        for it, lane in zip(self.items, deal([it.cost for it in self.items], nl)):
            it.lane = lane
        self._graph = None
        self._prepared = False

    # -- set-up: tuning and buffers (nothing is allocated after this)
    def _prepare(self):
        for it in self.items:
            ctx = self.ctxs[it.lane]
            if self.tuner is not None:
                # fused: the tiles the persistent deposit takes (16^3 gather) or the home tiles
                it.tile, it.cap = self.tuner.choose(ctx, it.cat, it.p, self.gpu,
                                                    tiles=(0, HOME_TILE) if self.fused else None)
            else:
                it.tile, it.cap = -1, -1
            ctx.set_tuning(it.tile, it.cap)
            n_scratch = ctx.scratch_bytes_tuned(it.p, it.cat.n)
            ctx.set_tuning(-1, -1)
            dt = torch.float32 if it.p.precision == pkmom.F32 else torch.float64
            item = 4 if it.p.precision == pkmom.F32 else 8
            dev = torch.device("cuda", self.device)
            it.grids = torch.empty(pkmom.Context.grid_bytes(it.p.ng, it.p.precision) // item, dtype=dt, device=dev)
            it.mom = torch.zeros(16, dtype=torch.float64, device=dev)
            it.scratch = torch.empty(n_scratch, dtype=torch.uint8, device=dev)
            it.out = torch.empty((pkmom.NROWS, it.p.nbins), dtype=torch.float64, device=dev)
        if self.fused:
            self._chunks = []
            for k in range(0, len(self.items), pkmom.BATCH_MAX):
                part = self.items[k:k + pkmom.BATCH_MAX]
                arr = pkmom.batch_items([(it.cat, it.p, it.grids, it.mom, it.scratch, it.out, it.tile, it.cap)
                                         for it in part])
                work = torch.empty(pkmom.batch_work_bytes(arr), dtype=torch.uint8,
                                   device=torch.device("cuda", self.device))
                self._chunks.append((arr, work))
        self._prepared = True

    def _issue(self, lane: int):
        ctx, s = self.ctxs[lane], self.streams[lane]
        if self.fused:
            for arr, work in self._chunks:
                ctx.estimate_batch(arr, work, stream=s)
            return
        for it in self.items:
            if it.lane != lane:
                continue
            ctx.set_tuning(it.tile, it.cap)
            ctx.assign(it.cat, it.p, it.grids, it.mom, it.scratch, stream=s)
            ctx.fft(it.p, it.grids, stream=s)
            ctx.spectra(it.p, it.grids, it.mom, it.out, stream=s)
        ctx.set_tuning(-1, -1)

    def _issue_all(self, origin: torch.cuda.Stream):
        fork = torch.cuda.Event()
        fork.record(origin)
        joins = []
        for lane, s in enumerate(self.streams):
            s.wait_event(fork)
            self._issue(lane)
            e = torch.cuda.Event()
            e.record(s)
            joins.append(e)
        for e in joins:
            origin.wait_event(e)

    def run(self, stream: torch.cuda.Stream | None = None) -> list[torch.Tensor]:
        """Estimate every catalogue; returns the (NROWS, nbins) outputs (device tensors),
        ready when `stream` (default: current) reaches this point."""
        origin = stream or torch.cuda.current_stream(self.device)
        if not self._prepared:
            self._prepare()
            self._issue_all(origin)  # eager: builds plans and tables
            origin.synchronize()
            for c in self.ctxs:
                c.sync(origin)
            if self.use_graph:
                cap_stream = torch.cuda.Stream(device=self.device)
                cap_stream.wait_stream(origin)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=cap_stream):
                    self._issue_all(cap_stream)
                self._graph = g
                origin.wait_stream(cap_stream)
            return [it.out for it in self.items]
        if self._graph is not None:
            with torch.cuda.stream(origin):
                self._graph.replay()
        else:
            self._issue_all(origin)
        return [it.out for it in self.items]

    def kernel_launches(self) -> int:
        return sum(c.kernel_launches() for c in self.ctxs)

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []
