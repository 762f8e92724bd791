"""HostPipeline: host catalogues copied while the previous one is estimated give the same
spectra as the plain device estimate of each (the deposit's integer sums and fixed-order
reductions make repeated estimates identical up to the FP64 rounding of the shell
tables)."""
import numpy as np
import pytest

from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu


def test_pipelined_host_estimates_equal_device_estimates(gpu_lib):
    import torch

    from paper_2005_06170_gb300.pipeline import HostPipeline
    pk = gpu_lib
    specs = [(32, 300.0, 32, 12), (24, 200.0, 48, 10), (40, 500.0, 64, 16), (16, 100.0, 32, 8), (32, 250.0, 40, 12)]
    cats = [catalogs.zeldovich(ns, L, seed=400 + i, dtype=np.float32) for i, (ns, L, _, _) in enumerate(specs)]
    params = [pk.params(L, ng, nb) for (_, L, ng, nb) in specs]
    pipe = HostPipeline(n_max=max(len(c["pos"]) for c in cats), nbins_max=16)
    pending, results = [], []
    for c, p in zip(cats, params):
        pending.append(pipe.submit(torch.from_numpy(c["pos"]).pin_memory(), torch.from_numpy(c["vel"]).pin_memory(), p))
        if len(pending) == 2:
            results.append(pending.pop(0).result())
    results += [q.result() for q in pending]
    pipe.close()
    ctx = pk.Context(0)
    for c, p, got in zip(cats, params, results):
        ref = ctx.estimate(torch.from_numpy(c["pos"]).cuda(), torch.from_numpy(c["vel"]).cuda(), p)
        ctx.sync()
        ref = ref.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(ref)), equal_nan=True)
    ctx.close()
