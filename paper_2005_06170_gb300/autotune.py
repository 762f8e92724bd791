"""Autotuner for the assignment step: deposit tile shape and per-tile particle list.

For each (GPU, grid size, precision, particle-density class) it times the candidate
settings of ``pkmom_set_tuning`` on the first catalogue of that class with CUDA
events and keeps the fastest. Results are cached in memory and, if a path is given,
in a JSON file (keyed by GPU name, ng, precision and density class), so later runs
skip the measurement. The estimate itself does not depend on the choice.
"""
from __future__ import annotations

import json
import math
import os
import threading

# deposit tile shapes of the library (x, y, z nodes), by tile id
TILES = {0: (16, 16, 16), 1: (16, 16, 32), 2: (8, 8, 32), 3: (8, 8, 8),
         4: (8, 8, 16), 5: (16, 16, 16), 6: (8, 8, 8), 7: (16, 16, 16)}
F32_TILES = (0, 1, 2, 3, 7)
HOME_TILE = 7  # each particle deposited once by the tile owning its cell (no list)
F64_TILES = (4, 5, 6)


def density_class(n: int, ng: int) -> int:
    """log2 of particles per cell, rounded and clipped to [-10, 10]."""
    ppc = max(n, 1) / float(ng) ** 3
    return int(max(-10, min(10, round(math.log2(ppc)))))


def candidates(ng: int, precision: int) -> list[tuple[int, int]]:
    """(tile, list_cap) pairs valid for this grid; list_cap -1 = the library's choice, 0 = none."""
    tiles = F32_TILES if precision == 0 else F64_TILES
    out = []
    for t in tiles:
        d = TILES[t]
        if all(ng % x == 0 for x in d):
            out.append((t, -1))
            if precision == 0 and t != HOME_TILE:
                out.append((t, 0))
    return out


class Autotuner:
    def __init__(self, path: str | None = None, repeats: int = 3, timer=None):
        """timer(ctx, cat, p, tile, list_cap) -> milliseconds; default times pkmom_assign."""
        self.path = path
        self.repeats = repeats
        self.timer = timer or self._time_assign
        self.table: dict[str, dict] = {}
        self._lock = threading.Lock()
        if path and os.path.exists(path):
            with open(path) as fh:
                self.table = json.load(fh)

    @staticmethod
    def key(gpu: str, ng: int, precision: int, n: int) -> str:
        return f"{gpu}|ng={ng}|prec={precision}|dc={density_class(n, ng)}"

    def choose(self, ctx, cat, p, gpu: str = "gpu", tiles=None) -> tuple[int, int]:
        """Tuning for this request: cached, or measured now (cat: the pkmom Catalog).
        tiles: the deposit tiles to choose from (default all that divide the grid)."""
        k = self.key(gpu, p.ng, p.precision, cat.n)
        cands = candidates(p.ng, p.precision)
        if tiles is not None:
            k += "|tiles=" + ",".join(str(t) for t in sorted(tiles))
            cands = [c for c in cands if c[0] in tiles] or cands
        with self._lock:
            if k in self.table:
                e = self.table[k]
                return e["tile"], e["list_cap"]
        best = None
        trials = {}
        for tile, cap in cands:
            ms = self.timer(ctx, cat, p, tile, cap)
            trials[f"{tile},{cap}"] = ms
            if best is None or ms < best[0]:
                best = (ms, tile, cap)
        with self._lock:
            self.table[k] = {"tile": best[1], "list_cap": best[2], "ms": best[0], "trials": trials}
            self._save()
        return best[1], best[2]

    def _save(self):
        if not self.path:
            return
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        tmp = self.path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(self.table, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def _time_assign(self, ctx, cat, p, tile, cap) -> float:
        import torch
        from . import pkmom
        ctx.set_tuning(tile, cap)
        try:
            dt = torch.float32 if p.precision == pkmom.F32 else torch.float64
            item = 4 if p.precision == pkmom.F32 else 8
            grids = torch.empty(pkmom.Context.grid_bytes(p.ng, p.precision) // item, dtype=dt, device="cuda")
            mom = torch.zeros(16, dtype=torch.float64, device="cuda")
            scratch = torch.empty(ctx.scratch_bytes_tuned(p, cat.n), dtype=torch.uint8, device="cuda")
            s = torch.cuda.current_stream()
            ctx.assign(cat, p, grids, mom, scratch, stream=s)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            for _ in range(self.repeats):
                ctx.assign(cat, p, grids, mom, scratch, stream=s)
            e1.record(s)
            e1.synchronize()
            return e0.elapsed_time(e1) / self.repeats
        finally:
            ctx.set_tuning(-1, -1)
