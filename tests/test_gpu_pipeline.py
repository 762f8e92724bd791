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


def test_estimate_host_async_through_the_c_abi(gpu_lib):
    """pkmom_estimate_host_async + pkmom_wait against pkmom_estimate_host on catalogues of
    growing size (the staging slots grow), FP64 with masses, and an unknown ticket."""
    import torch
    pk = gpu_lib
    ctx = pk.Context(0)
    ref_ctx = pk.Context(0)
    stream = torch.cuda.Stream()
    outs, tickets, refs, keep = [], [], [], []
    for i, (n, ng, prec) in enumerate([(5000, 32, pk.F32), (40000, 48, pk.F32), (20000, 32, pk.F64),
                                       (60000, 64, pk.F32)]):
        dt = np.float32 if prec == pk.F32 else np.float64
        c = catalogs.poisson(n, 300.0, seed=700 + i, dtype=dt, unit_mass=(prec == pk.F32))
        pos = torch.from_numpy(c["pos"]).pin_memory().numpy()
        vel = torch.from_numpy(c["vel"]).pin_memory().numpy()
        mass = None if "mass" not in c else torch.from_numpy(c["mass"]).pin_memory().numpy()
        p = pk.params(300.0, ng, 10, precision=prec)
        out = np.full((pk.NROWS, 10), -1.0)
        tickets.append(ctx.estimate_host_async(pos, vel, p, out, mass=mass, stream=stream))
        outs.append(out)
        keep.append((pos, vel, mass))
        refs.append(ref_ctx.estimate_host(pos, vel, p, mass=mass))
    assert tickets == [0, 1, 2, 3]
    ctx.wait(tickets[-1])  # waits for every earlier ticket too
    for got, ref in zip(outs, refs):
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(ref)), equal_nan=True)
    for t in tickets:
        ctx.wait(t)
    with pytest.raises(pk.PkmomError) as e:
        ctx.wait(99)
    assert e.value.status == -1
    assert ctx.context_bytes() > 0
    ctx.close()
    ref_ctx.close()
