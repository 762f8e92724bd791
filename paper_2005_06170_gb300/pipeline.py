"""Estimates of a stream of host catalogues with the transfers hidden behind the compute.

The host-device link of this part moves about 210 GB/s (measured, pinned copies and
kernel reads of mapped host memory alike), so copying a catalogue of 256^3 particles
(403 MB) takes about as long as estimating it. HostPipeline queues each catalogue with
the library's pkmom_estimate_host_async: the library copies catalogue i+1 on its own
copy stream, into the one of its two device staging slots that the estimate of
catalogue i-1 has finished reading, while catalogue i is estimated on the compute
stream, and copies each result to a pinned host buffer. Python only marshals the
arguments and keeps the buffers alive until the result has been read.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import pkmom


@dataclass
class Pending:
    ctx: pkmom.Context
    ticket: int
    out_host: np.ndarray  # (NROWS, nbins) view of a pinned buffer
    keep: tuple           # host arrays the library reads until the ticket completes

    def result(self) -> np.ndarray:
        """The (NROWS, nbins) spectra, once the estimate and its copy have finished."""
        self.ctx.wait(self.ticket)
        return self.out_host.copy()


class HostPipeline:
    def __init__(self, n_max: int, nbins_max: int, precision: int = pkmom.F32, device: int = 0, depth: int = 2):
        """n_max: the largest catalogue (particles); nbins_max: the most shells requested;
        depth: results that may be pending at once (one pinned output buffer each)."""
        self.device = device
        self.precision = precision
        self.ctx = pkmom.Context(device)
        self.compute_stream = torch.cuda.Stream(device=device)
        self.out_host = [torch.empty(pkmom.NROWS * nbins_max, dtype=torch.float64).pin_memory()
                         for _ in range(depth)]
        self.n_max, self.nbins_max = n_max, nbins_max
        self.count = 0

    def submit(self, pos: torch.Tensor, vel: torch.Tensor, p, mass: torch.Tensor | None = None) -> Pending:
        """Queue the estimate of a host catalogue: pos, vel (n, 3) pinned CPU tensors of the
        pipeline's precision, optional mass (n,). The result of the submit `depth` calls
        back must have been read (its output buffer is reused)."""
        n = pos.shape[0]
        if n > self.n_max or p.nbins > self.nbins_max:
            raise ValueError("catalogue or shell count beyond the pipeline's sizes")
        buf = self.out_host[self.count % len(self.out_host)]
        self.count += 1
        size = pkmom.NROWS * p.nbins
        host = buf[:size].view(pkmom.NROWS, p.nbins).numpy()
        arrays = (pos, vel) + ((mass,) if mass is not None else ())
        t = self.ctx.estimate_host_async(pos.numpy(), vel.numpy(), p, host,
                                         mass=None if mass is None else mass.numpy(), stream=self.compute_stream)
        return Pending(self.ctx, t, host, arrays)

    def close(self):
        torch.cuda.synchronize(self.device)
        self.ctx.close()
