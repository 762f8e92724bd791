"""Batched and served estimation on the GPU give the same spectra as single runs.

The deposit accumulates in integers with order-independent scales and the other
reductions of the data have a fixed order, so with the same tuning a catalogue's
spectra do not depend on what runs beside it: batched, graph-replayed and served
results equal the single-catalogue results up to the FP64 rounding of each
context's shell tables (1e-12). Catalogues are also checked against the oracle.
"""
import numpy as np
import pytest

from oracle import estimator as est
from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu


def _mixed(seed=0):
    specs = [("p", 3000, 80.0, 32), ("z", 24, 200.0, 48), ("p", 20000, 150.0, 64), ("z", 32, 300.0, 32),
             ("p", 500, 60.0, 16), ("z", 16, 100.0, 64), ("p", 8000, 120.0, 40)]
    out = []
    for i, (kind, n, L, ng) in enumerate(specs):
        if kind == "p":
            c = catalogs.poisson(n, L, seed=500 + i + seed, dtype=np.float32)
        else:
            c = catalogs.zeldovich(n, L, seed=600 + i + seed, dtype=np.float32)
        out.append((c, L, ng))
    return out


def _dev(c, torch):
    return {"pos": torch.from_numpy(c["pos"]).cuda(), "vel": torch.from_numpy(c["vel"]).cuda()}


def _single(pk, ctx, d, p):
    out = ctx.estimate(d["pos"], d["vel"], p)
    ctx.sync()
    return out.cpu().numpy()


@pytest.mark.parametrize("fused", [True, False])
def test_batch_graph_equals_single_runs(gpu_lib, fused):
    import torch

    from paper_2005_06170_gb300.batch import BatchRunner
    pk = gpu_lib
    items = _mixed()
    devs = [_dev(c, torch) for c, _, _ in items]
    params = [pk.params(L, ng, 12, theta_scale=0.02) for _, L, ng in items]
    ctx = pk.Context(0)
    ref = [_single(pk, ctx, d, p) for d, p in zip(devs, params)]
    runner = BatchRunner(devs, params, lanes=3, use_graph=True, fused=fused)
    first = [o.cpu().numpy() for o in runner.run()]  # eager run, then capture
    torch.cuda.synchronize()
    for o in runner.run():  # graph replay
        o.zero_()
    torch.cuda.synchronize()
    replay = [o.cpu().numpy() for o in runner.run()]
    torch.cuda.synchronize()
    for r, a, b in zip(ref, first, replay):
        # integer deposit sums and fixed-order reductions: equal up to the FP64 rounding
        # of the shell tables each context builds
        np.testing.assert_allclose(a, r, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(r)), equal_nan=True)
        np.testing.assert_allclose(b, r, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(r)), equal_nan=True)
    runner.close()
    ctx.close()


def test_batch_with_autotuner_matches_oracle(gpu_lib):
    import torch

    from paper_2005_06170_gb300.autotune import Autotuner
    from paper_2005_06170_gb300.batch import BatchRunner
    pk = gpu_lib
    items = _mixed(seed=7)[:3]
    devs = [_dev(c, torch) for c, _, _ in items]
    params = [pk.params(L, ng, 10) for _, L, ng in items]
    runner = BatchRunner(devs, params, lanes=2, use_graph=True, tuner=Autotuner(repeats=1))
    outs = [pk.as_dict(o) for o in runner.run()]
    torch.cuda.synchronize()
    for (c, L, ng), g in zip(items, outs):
        o = est.estimate(c["pos"], c["vel"], L=L, ng=ng, nbins=10)
        for key in ("P_dd", "P_pp", "P_tt", "P_pp_b", "P_tt_b"):
            sn = o["SN" + key[1:]]
            scale = np.maximum(np.abs(o[key]), sn / np.sqrt(o["n_modes"]))
            assert np.all(np.abs(g[key] - o[key]) <= 1e-4 * scale), key
    runner.close()


def test_served_results_same_alone_and_in_the_mix(gpu_lib):
    import torch

    from paper_2005_06170_gb300.serve import Request, Server
    pk = gpu_lib
    items = _mixed(seed=3)
    devs = [_dev(c, torch) for c, _, _ in items]
    params = [pk.params(L, ng, 12) for _, L, ng in items]
    alone = []
    srv = Server(lanes=1)
    for d, p in zip(devs, params):
        alone.append(srv.submit(Request(d["pos"], d["vel"], p)).result(timeout=120))
    srv.close()
    srv = Server(lanes=4)
    futs = [srv.submit(Request(d["pos"], d["vel"], p)) for d, p in zip(devs, params)]
    mixed = [f.result(timeout=120) for f in futs]
    lanes_used = {r.lane for r in srv.completed}
    srv.close()
    assert len(lanes_used) > 1  # the requests did overlap on several lanes
    for a, b in zip(alone, mixed):
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(a)), equal_nan=True)


def test_large_requests_keep_their_own_lane(gpu_lib):
    """Strict lanes: requests above large_bytes run only on the last lane, one at a time
    and in arrival order; the others never take that lane; every result equals the one
    computed alone."""
    import torch

    from paper_2005_06170_gb300.serve import Request, Server
    pk = gpu_lib
    items = _mixed(seed=7)[:6]
    devs = [_dev(c, torch) for c, _, _ in items]
    params = [pk.params(L, 64 if k % 2 else 32, 8) for k, (_, L, _) in enumerate(items)]
    srv = Server(lanes=1)
    alone = [srv.submit(Request(d["pos"], d["vel"], p)).result(timeout=120) for d, p in zip(devs, params)]
    fps = [srv.footprint(Request(d["pos"], d["vel"], p)) for d, p in zip(devs, params)]
    srv.close()
    cut = (max(f for f, p in zip(fps, params) if p.ng == 32) + min(f for f, p in zip(fps, params) if p.ng == 64)) / 2
    assert max(f for f, p in zip(fps, params) if p.ng == 32) < cut < min(f for f, p in zip(fps, params) if p.ng == 64)
    srv = Server(lanes=3, large_bytes=cut)
    futs = [srv.submit(Request(d["pos"], d["vel"], p)) for d, p in zip(devs, params)]
    mixed = [f.result(timeout=120) for f in futs]
    done = list(srv.completed)
    srv.close()
    large = sorted((r for r in done if r.footprint > cut), key=lambda r: r.admitted)
    assert large and all(r.lane == 2 for r in large)
    assert all(r.lane in (0, 1) for r in done if r.footprint <= cut)
    assert [r.rid for r in large] == sorted(r.rid for r in large)  # arrival order
    for a, b in zip(large, large[1:]):
        assert b.admitted >= a.done - 1e-3  # never two large ones at once
    for a, b in zip(alone, mixed):
        np.testing.assert_allclose(b, a, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(a)), equal_nan=True)


def test_serving_admits_by_footprint(gpu_lib):
    import torch

    from paper_2005_06170_gb300.serve import Request, Server
    pk = gpu_lib
    items = _mixed(seed=5)[:4]
    devs = [_dev(c, torch) for c, _, _ in items]
    params = [pk.params(L, 64, 8) for _, L, _ in items]
    probe = Server(lanes=1)
    fp = max(probe.footprint(Request(d["pos"], d["vel"], p)) for d, p in zip(devs, params))
    probe.close()
    srv = Server(lanes=4, budget_bytes=1e12)
    srv.warm((64,), nbins=8)  # every lane's plan and tables, charged to the budget
    assert all(b > 0 for b in srv.lane_bytes) and srv.reserved() == sum(srv.lane_bytes)
    srv.policy.budget = srv.reserved() + int(1.5 * fp)  # room for one request at a time
    futs = [srv.submit(Request(d["pos"], d["vel"], p)) for d, p in zip(devs, params)]
    for f in futs:
        f.result(timeout=120)
    done = sorted(srv.completed, key=lambda r: r.admitted)
    for a, b in zip(done, done[1:]):
        assert b.admitted >= a.done - 1e-3  # never two at once
    big = Request(devs[0]["pos"], devs[0]["vel"], pk.params(100.0, 1024, 8))
    with pytest.raises(MemoryError):
        srv.submit(big).result(timeout=10)
    srv.close()


def test_served_catalogue_written_on_the_callers_stream(gpu_lib):
    """A request whose catalogue is still being written on the caller's stream when it is
    submitted: the lane waits for that point of the caller's stream before reading it."""
    import torch

    from paper_2005_06170_gb300.serve import Request, Server
    pk = gpu_lib
    c, L, ng = _mixed(seed=9)[2]
    d = _dev(c, torch)
    p = pk.params(L, ng, 10)
    ctx = pk.Context(0)
    ref = _single(pk, ctx, d, p)
    ctx.close()
    srv = Server(lanes=2)
    side = torch.cuda.Stream()
    pos = torch.zeros_like(d["pos"])
    vel = torch.zeros_like(d["vel"])
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        torch.cuda._sleep(20_000_000)  # the copy below lands well after the submit
        pos.copy_(d["pos"])
        vel.copy_(d["vel"])
        fut = srv.submit(Request(pos, vel, p))
    got = fut.result(timeout=120)
    srv.close()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(ref)), equal_nan=True)


def test_estimate_batch_through_the_c_abi(gpu_lib):
    """pkmom_estimate_batch on catalogues that take every deposit path (16^3 gather tiles
    in the persistent kernel, home tiles, another order, FP64, the direct BL stencil, an
    8^3 tile by tuning) equals pkmom_estimate on each, in the same context (bit for bit:
    the same kernels per tile and per binning item, reductions in the same order)."""
    import torch
    pk = gpu_lib
    specs = [  # (kind, size, L, ng, precision, order, bl_radius, tile)
        ("p", 3000, 80.0, 32, pk.F32, 4, 0, -1), ("z", 32, 200.0, 32, pk.F32, 4, 0, -1),
        ("p", 40000, 150.0, 64, pk.F32, 4, 0, 0), ("p", 5000, 100.0, 48, pk.F32, 2, 0, -1),
        ("p", 4000, 90.0, 32, pk.F64, 4, 0, -1), ("z", 16, 100.0, 32, pk.F32, 4, 3, -1),
        ("p", 20000, 120.0, 64, pk.F32, 4, 0, 3), ("z", 24, 300.0, 48, pk.F32, 4, 0, -1)]
    ctx = pk.Context(0)
    entries, refs = [], []
    keep = []
    for i, (kind, size, L, ng, prec, order, blr, tile) in enumerate(specs):
        dt = np.float32 if prec == pk.F32 else np.float64
        c = (catalogs.poisson(size, L, seed=800 + i, dtype=dt) if kind == "p"
             else catalogs.zeldovich(size, L, seed=900 + i, dtype=dt))
        pos, vel = torch.from_numpy(c["pos"]).cuda(), torch.from_numpy(c["vel"]).cuda()
        p = pk.params(L, ng, 10, precision=prec, order=order, bl_radius=blr, theta_scale=0.01)
        ctx.set_tuning(tile, -1)
        ref = ctx.estimate(pos, vel, p)
        ctx.sync()
        ctx.set_tuning(-1, -1)
        refs.append(ref.cpu().numpy())
        tdt = torch.float32 if prec == pk.F32 else torch.float64
        grids = torch.empty(pk.Context.grid_bytes(ng, prec) // (4 if prec == pk.F32 else 8), dtype=tdt,
                            device="cuda")
        mom = torch.zeros(16, dtype=torch.float64, device="cuda")
        cat = pk.catalog_from_tensors(pos, vel)
        ctx.set_tuning(tile, -1)
        scratch = torch.empty(ctx.scratch_bytes_tuned(p, cat.n), dtype=torch.uint8, device="cuda")
        ctx.set_tuning(-1, -1)
        out = torch.full((pk.NROWS, 10), -1.0, dtype=torch.float64, device="cuda")
        entries.append((cat, p, grids, mom, scratch, out, tile, -1))
        keep.append((pos, vel))
    arr = pk.batch_items(entries)
    work = torch.empty(pk.batch_work_bytes(arr), dtype=torch.uint8, device="cuda")
    l0 = ctx.kernel_launches()
    ctx.estimate_batch(arr, work)
    ctx.sync()
    assert ctx.kernel_launches() > l0
    for e, ref in zip(entries, refs):
        got = e[5].cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(ref)), equal_nan=True)
    ctx.close()
