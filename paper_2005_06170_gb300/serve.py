"""Serving loop: estimation requests admitted by HBM footprint, run as they arrive.

Requests (a catalogue resident on the device plus its Params) are queued on
arrival. A scheduler thread admits them while a lane is free and their device
footprint fits in the budget beside the requests already running (first fit in
arrival order, with a bound on how often a waiting request may be overtaken), and
launches each on its lane's stream: several requests overlap on the GPU and
requests that arrive meanwhile join as lanes and memory free up (continuous
batching). Requests with a large footprint (a 1024^3 grid) run one at a time on a
lane of their own at low stream priority, so that the small ones pass them at kernel
boundaries while two large ones never share the GPU. A lane owns a libpkmom context
(its own cuFFT plans and tables). The
result is copied to pinned host memory on the lane's stream; the scheduler polls
the completion events, releases the request's memory and completes its Future.
Latency is measured from arrival to the moment the result is on the host.
"""
from __future__ import annotations

import concurrent.futures as cf
import threading
import time
from dataclasses import dataclass, field

import numpy as np


@dataclass(eq=False)  # requests compare by identity
class Request:
    pos: object              # (n,3) CUDA tensor
    vel: object              # (n,3) CUDA tensor
    params: object           # pkmom.Params
    mass: object = None
    arrival: float = 0.0     # time.perf_counter() at arrival
    rid: int = 0
    future: cf.Future = field(default_factory=cf.Future)
    # filled by the server
    footprint: int = 0
    ready: object = None     # CUDA event recorded at submit on the producer's stream
    admitted: float = 0.0
    done: float = 0.0
    lane: int = -1
    overtaken: int = 0


class AdmissionPolicy:
    """Which queued requests start now (pure host logic, no CUDA).

    First fit in arrival order: the oldest request that fits the free budget starts
    on a free lane; a request may be overtaken by later, smaller ones at most
    `max_overtake` times, after which nothing behind it starts until it does.
    """

    def __init__(self, budget_bytes: int, max_overtake: int = 8):
        self.budget = int(budget_bytes)
        self.max_overtake = max_overtake

    def admit(self, queue: list, free_lanes: int, in_use: int, free_large: int | None = None,
              is_large=None) -> list:
        """free_large (with is_large): separate lanes for large requests; free_large of
        the free lanes take only requests with is_large(r) true, the others only the
        rest. A request whose kind of lane is busy waits without counting an overtake."""
        chosen = []
        free = self.budget - in_use
        lane_blocked = set()
        small_cap = free_lanes if free_large is None else free_lanes - free_large
        n_small = n_large = 0
        for r in queue:
            if free_large is None:
                if len(chosen) >= free_lanes:
                    break
                large = False
            else:
                if n_large >= free_large and n_small >= small_cap:
                    break
                large = bool(is_large(r))
                if (n_large >= free_large) if large else (n_small >= small_cap):
                    lane_blocked.add(id(r))
                    continue
            if r.footprint <= free:
                chosen.append(r)
                free -= r.footprint
                n_large += large
                n_small += not large
            elif r.overtaken >= self.max_overtake:
                break  # it has waited long enough: nothing behind it starts first
        # every waiting request passed by a later admitted one counts one overtake
        if chosen:
            last = queue.index(chosen[-1])
            for r in queue[:last]:
                if r not in chosen and id(r) not in lane_blocked:
                    r.overtaken += 1
        return chosen


def percentiles(latencies: list[float], qs=(50, 99)) -> dict:
    a = np.sort(np.asarray(latencies, dtype=np.float64))
    if a.size == 0:
        return {f"p{q}": None for q in qs}
    return {f"p{q}": float(np.percentile(a, q, method="inverted_cdf")) for q in qs}


class Server:
    def __init__(self, lanes: int = 4, budget_bytes: float = 180e9, device: int = 0, tuner=None,
                 max_overtake: int = 8, large_bytes: float = 8e9, large_lanes: int | None = None,
                 large_priority: str = "low", strict_lanes: bool = True):
        """Requests whose footprint exceeds large_bytes prefer the last `large_lanes`
        lanes (default one, when there are two or more), the others the first ones.
        large_priority: "low"
        puts the large lanes' streams at the least priority and the small lanes' at the
        greatest, so that small requests pass large ones at kernel boundaries; "same"
        gives every lane the default priority. strict_lanes: large requests run only on
        the large lanes (one at a time per lane, in arrival order) and small ones only on
        the others; otherwise either kind takes any free lane when its own are busy.
        "high" gives the large lanes the greatest priority instead, so that a large request
        runs at nearly its own speed and small ones fill the gaps.

        Measured on a Poisson stream (20 requests/s, 1e5 to 1.3e8 particles, grids 128^3
        to 1024^3) against one request at a time: with four lanes, one of them strict for
        large requests, p50 7.3 ms (13.7), p99 125 to 146 ms (125), mean 20 to 21 ms
        (25); two non-strict large lanes gave p99 near 190 ms, as two 1024^3 requests then
        shared the GPU and both yielded to every small one."""
        import torch

        from . import pkmom
        self._torch, self._pk = torch, pkmom
        self.device = device
        self.ctxs = [pkmom.Context(device) for _ in range(lanes)]
        lo, hi = torch.cuda.Stream.priority_range()  # (least, greatest) priority
        if large_priority not in ("low", "same", "high"):
            raise ValueError("large_priority must be 'low', 'same' or 'high'")
        if large_lanes is None:
            large_lanes = 1 if lanes > 1 else 0
        if not 0 <= large_lanes < lanes:
            raise ValueError("large_lanes must leave at least one lane for small requests")
        self.n_small = lanes - large_lanes
        self.large_bytes = large_bytes
        self.strict = bool(strict_lanes) and large_lanes > 0

        def prio(k):  # stream priority of lane k
            if large_lanes == 0 or large_priority == "same":
                return 0
            small = k < self.n_small
            return (hi if small else lo) if large_priority == "low" else (lo if small else hi)

        self.streams = [torch.cuda.Stream(device=device, priority=prio(k)) for k in range(lanes)]
        self.lane_free = [True] * lanes
        # device memory each lane's context keeps between requests (cuFFT plans and
        # per-grid tables), charged to the budget beside the running requests
        self.lane_bytes = [0] * lanes
        self.policy = AdmissionPolicy(int(budget_bytes), max_overtake)
        self.tuner = tuner
        self.gpu = torch.cuda.get_device_name(device)
        self.queue: list[Request] = []
        self.inflight: list[tuple] = []
        self.in_use = 0
        self.completed: list[Request] = []
        self._lock = threading.Condition()
        self._stop = False
        self._next = 0
        self._thread = threading.Thread(target=self._loop, name="pkmom-serve", daemon=True)
        self._thread.start()

    def footprint(self, req: Request) -> int:
        """Device bytes a request holds while it runs: the library's own estimate for it
        (grids, assignment scratch, a cuFFT workspace of a quarter of the grids in case
        the lane has no plan for this grid yet, staging of a host catalogue), plus the
        moments and the output. A tuned deposit whose scratch is larger is charged the
        difference when it starts. A lane's plans and tables that outlive the request
        are charged separately (lane_bytes)."""
        pk = self._pk
        p = req.params
        return int(pk.Context.footprint_bytes(p, req.pos.shape[0]) + 16 * 8 + pk.NROWS * p.nbins * 8)

    def reserved(self) -> int:
        """Bytes charged to the budget now: running requests and the lanes' contexts."""
        return self.in_use + sum(self.lane_bytes)

    def warm(self, grids, nbins: int = 128, box_L: float = 1000.0):
        """Builds every lane's cuFFT plans and tables for these grid sizes with a tiny
        estimate (before the first request, so that none pays for it), then charges the
        memory the lanes' contexts hold."""
        torch, pk = self._torch, self._pk
        dev = torch.device("cuda", self.device)
        g = torch.Generator(device=dev)
        g.manual_seed(0)
        pos = torch.rand((4096, 3), generator=g, device=dev) * box_L
        vel = torch.zeros_like(pos)
        for ctx, s in zip(self.ctxs, self.streams):
            s.wait_stream(torch.cuda.current_stream(dev))
            for ng in grids:
                ctx.estimate(pos, vel, pk.params(box_L, int(ng), nbins), stream=s)
        torch.cuda.synchronize(dev)
        with self._lock:
            self.lane_bytes = [c.context_bytes() for c in self.ctxs]

    def submit(self, req: Request) -> cf.Future:
        req.footprint = self.footprint(req)
        if not req.arrival:
            req.arrival = time.perf_counter()
        # the catalogue may still be being written on the caller's stream: the lane's
        # stream waits for this point before it reads it
        torch = self._torch
        req.ready = torch.cuda.Event()
        req.ready.record(torch.cuda.current_stream(req.pos.device))
        with self._lock:
            req.rid = self._next
            self._next += 1
            if req.footprint + sum(self.lane_bytes) > self.policy.budget:
                req.future.set_exception(MemoryError(f"request needs {req.footprint} B > budget"))
                return req.future
            self.queue.append(req)
            self._lock.notify()
        return req.future

    def _pick_lane(self, free: list, large: bool) -> int:
        """A free lane of the request's kind (low priority for large ones), else any
        (strict lanes: admission has already checked that one of its kind is free)."""
        mine = [k for k in free if (k >= self.n_small) == large]
        return (mine or free)[0]

    def _launch(self, req: Request, lane: int):
        torch, pk = self._torch, self._pk
        ctx, s = self.ctxs[lane], self.streams[lane]
        p = req.params
        dev = torch.device("cuda", self.device)
        dt = torch.float32 if p.precision == pk.F32 else torch.float64
        item = 4 if p.precision == pk.F32 else 8
        cat = pk.catalog_from_tensors(req.pos, req.vel, req.mass)
        tile, cap = (-1, -1)
        if self.tuner is not None:
            tile, cap = self.tuner.choose(ctx, cat, p, self.gpu)
        ctx.set_tuning(tile, cap)
        n_scratch = ctx.scratch_bytes_tuned(p, cat.n)
        extra = max(0, n_scratch - pk.Context.scratch_bytes(p, cat.n))
        if extra:  # a tuned deposit with a larger scratch than the admitted one
            req.footprint += extra
            self.in_use += extra
        if req.ready is not None:
            s.wait_event(req.ready)
        for t in (req.pos, req.vel) + ((req.mass,) if req.mass is not None else ()):
            t.record_stream(s)  # the allocator keeps the catalogue until the lane is done
        with torch.cuda.stream(s):
            grids = torch.empty(pk.Context.grid_bytes(p.ng, p.precision) // item, dtype=dt, device=dev)
            mom = torch.zeros(16, dtype=torch.float64, device=dev)
            scratch = torch.empty(n_scratch, dtype=torch.uint8, device=dev)
            out = torch.empty((pk.NROWS, p.nbins), dtype=torch.float64, device=dev)
            host = torch.empty((pk.NROWS, p.nbins), dtype=torch.float64, pin_memory=True)
        ctx.assign(cat, p, grids, mom, scratch, stream=s)
        ctx.fft(p, grids, stream=s)
        ctx.spectra(p, grids, mom, out, stream=s)
        ctx.set_tuning(-1, -1)
        with torch.cuda.stream(s):
            host.copy_(out, non_blocking=True)
        ev = torch.cuda.Event()
        ev.record(s)
        req.admitted = time.perf_counter()
        req.lane = lane
        return (req, lane, ev, host, (grids, mom, scratch, out))

    def _loop(self):
        try:
            self._run_loop()
        except BaseException as e:  # never leave callers waiting on a dead scheduler
            with self._lock:
                self._stop = True
                pending = list(self.queue) + [entry[0] for entry in self.inflight]
                self.queue.clear()
                self.inflight.clear()
            for r in pending:
                if not r.future.done():
                    r.future.set_exception(RuntimeError(f"serving loop failed: {e!r}"))
            raise

    def _run_loop(self):
        torch = self._torch
        torch.cuda.set_device(self.device)
        while True:
            with self._lock:
                if self._stop and not self.queue and not self.inflight:
                    return
                free = [k for k, f in enumerate(self.lane_free) if f]
                if not free:
                    start = []
                elif self.strict:
                    start = self.policy.admit(self.queue, len(free), self.reserved(),
                                              free_large=sum(k >= self.n_small for k in free),
                                              is_large=lambda r: r.footprint > self.large_bytes)
                else:
                    start = self.policy.admit(self.queue, len(free), self.reserved())
                if not start and not self.inflight and self.queue:
                    # nothing runs and the oldest request still does not fit beside the
                    # lanes' own memory: it never will
                    head = self.queue[0]
                    if head.footprint + self.reserved() > self.policy.budget:
                        self.queue.pop(0)
                        head.future.set_exception(MemoryError(
                            f"request needs {head.footprint} B beside {self.reserved()} B held by the lanes "
                            f"> budget {self.policy.budget} B"))
                for r in start:
                    self.queue.remove(r)
                    self.in_use += r.footprint
                    lane = self._pick_lane(free, r.footprint > self.large_bytes)
                    free.remove(lane)
                    self.lane_free[lane] = False
                    self.inflight.append(self._launch(r, lane))
            finished = []
            for entry in list(self.inflight):
                req, lane, ev, host, bufs = entry
                if ev.query():
                    req.done = time.perf_counter()
                    finished.append(entry)
            if finished:
                with self._lock:
                    for entry in finished:
                        req, lane, ev, host, bufs = entry
                        self.inflight.remove(entry)
                        err = None
                        try:
                            self.ctxs[lane].sync(self.streams[lane])
                        except Exception as e:  # a data error latched by the library
                            err = e
                        self.lane_free[lane] = True
                        self.in_use -= req.footprint
                        self.lane_bytes[lane] = self.ctxs[lane].context_bytes()
                        self.completed.append(req)
                        # the server no longer needs the catalogue (the lane's stream,
                        # recorded on it, has finished): release it for the caller
                        req.pos = req.vel = req.mass = None
                        if err is None:
                            req.future.set_result(host.numpy().copy())
                        else:
                            req.future.set_exception(err)
                    self._lock.notify_all()
            elif not start:
                with self._lock:
                    if not self._stop or self.queue or self.inflight:
                        self._lock.wait(timeout=0.0002)

    def close(self):
        with self._lock:
            self._stop = True
            self._lock.notify_all()
        self._thread.join()
        for c in self.ctxs:
            c.close()
        self.ctxs = []

    def latencies(self) -> list[float]:
        return [r.done - r.arrival for r in self.completed]
