"""Estimates of a stream of host catalogues with the transfers hidden behind the compute.

The host-device link of this part moves about 210 GB/s (measured, pinned copies and
kernel reads of mapped host memory alike), so copying a catalogue of 256^3 particles
(403 MB) takes about as long as estimating it. HostPipeline keeps two device staging
slots: the copy of catalogue i+1 (copy stream) runs while catalogue i is estimated
(compute stream, the libpkmom context's own grids and scratch), and each result is
copied back to pinned host memory on the compute stream. A slot is refilled only after
the estimate that read it has finished (an event per slot).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import pkmom


@dataclass
class Pending:
    done: torch.cuda.Event
    out_host: torch.Tensor  # (NROWS, nbins) view of a pinned buffer

    def result(self) -> np.ndarray:
        """The (NROWS, nbins) spectra, once the estimate and its copy have finished."""
        self.done.synchronize()
        return self.out_host.numpy().copy()


class HostPipeline:
    def __init__(self, n_max: int, nbins_max: int, precision: int = pkmom.F32, device: int = 0):
        """n_max: the largest catalogue (particles); nbins_max: the most shells requested."""
        self.device = device
        dev = torch.device("cuda", device)
        dt = torch.float32 if precision == pkmom.F32 else torch.float64
        self.precision = precision
        self.ctx = pkmom.Context(device)
        self.copy_stream = torch.cuda.Stream(device=device)
        self.compute_stream = torch.cuda.Stream(device=device)
        self.slots = [{"pos": torch.empty((n_max, 3), dtype=dt, device=dev),
                       "vel": torch.empty((n_max, 3), dtype=dt, device=dev),
                       "mass": None,
                       "free": torch.cuda.Event()} for _ in range(2)]
        # flat buffers: the first NROWS * nbins doubles viewed as (NROWS, nbins)
        self.out_dev = [torch.empty(pkmom.NROWS * nbins_max, dtype=torch.float64, device=dev) for _ in range(2)]
        self.out_host = [torch.empty(pkmom.NROWS * nbins_max, dtype=torch.float64).pin_memory() for _ in range(2)]
        self.n_max, self.nbins_max = n_max, nbins_max
        self.count = 0

    def submit(self, pos: torch.Tensor, vel: torch.Tensor, p, mass: torch.Tensor | None = None) -> Pending:
        """Queue the estimate of a host catalogue: pos, vel (n, 3) pinned CPU tensors of the
        pipeline's precision, optional mass (n,). The result of the submit before the
        previous one must have been read (two output buffers)."""
        n = pos.shape[0]
        if n > self.n_max or p.nbins > self.nbins_max:
            raise ValueError("catalogue or shell count beyond the pipeline's sizes")
        k = self.count % 2
        self.count += 1
        slot = self.slots[k]
        cs, ks = self.copy_stream, self.compute_stream
        cs.wait_event(slot["free"])  # the estimate that last read this slot has finished
        with torch.cuda.stream(cs):
            dpos = slot["pos"][:n]
            dvel = slot["vel"][:n]
            dpos.copy_(pos, non_blocking=True)
            dvel.copy_(vel, non_blocking=True)
            dmass = None
            if mass is not None:
                if slot["mass"] is None or slot["mass"].shape[0] < n:
                    slot["mass"] = torch.empty(self.n_max, dtype=dpos.dtype, device=dpos.device)
                dmass = slot["mass"][:n]
                dmass.copy_(mass, non_blocking=True)
        ready = torch.cuda.Event()
        ready.record(cs)
        ks.wait_event(ready)
        size = pkmom.NROWS * p.nbins
        out = self.out_dev[k][:size].view(pkmom.NROWS, p.nbins)
        host = self.out_host[k][:size].view(pkmom.NROWS, p.nbins)
        with torch.cuda.stream(ks):
            self.ctx.estimate(dpos, dvel, p, mass=dmass, out=out, stream=ks)
            slot["free"].record(ks)
            host.copy_(out, non_blocking=True)
        done = torch.cuda.Event()
        done.record(ks)
        return Pending(done, host)

    def close(self):
        torch.cuda.synchronize(self.device)
        self.ctx.close()
