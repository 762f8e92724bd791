"""The checked build (libpkmom_checked.so): index tests before every grid, halo,
shared-buffer, sort-key, record and bin access. On valid inputs no test fails, and the
results equal the unchecked build's (to the last bit of its FP64 shell tables) and the
oracle's within the usual tolerance, through every deposit path (home tiles, gather
tiles, the dense cell-block path, FP64, another order, the direct BL stencil) and the
batched entry point; the reporting path raises PKMOM_EDATA for the self-test's failed
test."""
import numpy as np
import pytest

from oracle import estimator as est
from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu


CASES = [  # (kind, size, L, ng, precision, order, bl_radius)
    ("z", 32, 200.0, 32, 0, 4, 0),      # one particle per cell: home tiles
    ("p", 3000, 100.0, 32, 0, 4, 0),    # sparse: gather tiles
    ("c", 20000, 100.0, 32, 0, 4, 0),   # all in one cell: the dense path
    ("p", 4000, 90.0, 32, 1, 4, 0),     # FP64
    ("p", 5000, 100.0, 48, 0, 2, 0),    # cloud in cell
    ("z", 16, 100.0, 32, 0, 4, 3),      # direct truncated BL
]


def _cat(kind, size, L, prec, seed):
    dt = np.float32 if prec == 0 else np.float64
    if kind == "z":
        return catalogs.zeldovich(size, L, seed=seed, dtype=dt)
    if kind == "p":
        return catalogs.poisson(size, L, seed=seed, dtype=dt)
    rng = np.random.default_rng(seed)
    pos = (10.0 + rng.uniform(0, L / 32, size=(size, 3))).astype(dt)
    return {"pos": pos, "vel": rng.normal(0, 100, size=(size, 3)).astype(dt), "L": L}


@pytest.mark.parametrize("case", CASES)
def test_checked_build_equals_unchecked_and_oracle(gpu_lib, case):
    import torch
    pk = gpu_lib
    kind, size, L, ng, prec, order, blr = case
    c = _cat(kind, size, L, prec, seed=1200 + ng + size % 97)
    pos, vel = torch.from_numpy(c["pos"]).cuda(), torch.from_numpy(c["vel"]).cuda()
    p = pk.params(L, ng, 8, precision=prec, order=order, bl_radius=blr)
    outs = []
    for checked in (False, True):
        ctx = pk.Context(0, checked=checked)
        outs.append(ctx.estimate(pos, vel, p).cpu().numpy())
        ctx.sync()  # raises PKMOM_EDATA if an index test failed
        ctx.close()
    # the same grids and per-mode sums; the shell tables, built in FP64 by each library's
    # own code, may differ in the last bit
    np.testing.assert_allclose(outs[1], outs[0], rtol=1e-12, atol=1e-12 * np.nanmax(np.abs(outs[0])),
                               equal_nan=True)
    o = est.estimate(c["pos"], c["vel"], L=L, ng=ng, nbins=8, order=order, bl_radius=blr)
    g = pk.as_dict(outs[1])
    rtol = 1e-9 if prec == 1 else 1e-4
    for key in ("P_dd", "P_pp", "P_tt"):
        floor = o["SN" + key[1:]] / np.sqrt(np.maximum(o["n_modes"], 1))
        scale = np.maximum(np.abs(o[key]), floor)
        ok = o["n_modes"] > 0
        assert np.all(np.abs(g[key][ok] - o[key][ok]) <= rtol * scale[ok]), key


def test_checked_batch_and_selftest(gpu_lib):
    import torch
    pk = gpu_lib
    ctx = pk.Context(0, checked=True)
    entries, keep = [], []
    for i, (kind, size, L, ng) in enumerate([("p", 3000, 80.0, 32), ("z", 24, 200.0, 48), ("p", 500, 60.0, 16)]):
        c = _cat(kind, size, L, 0, 1300 + i)
        pos, vel = torch.from_numpy(c["pos"]).cuda(), torch.from_numpy(c["vel"]).cuda()
        p = pk.params(L, ng, 8)
        cat = pk.catalog_from_tensors(pos, vel)
        grids = torch.empty(pk.Context.grid_bytes(ng) // 4, dtype=torch.float32, device="cuda")
        mom = torch.zeros(16, dtype=torch.float64, device="cuda")
        scratch = torch.empty(ctx.scratch_bytes_tuned(p, cat.n), dtype=torch.uint8, device="cuda")
        out = torch.empty((pk.NROWS, 8), dtype=torch.float64, device="cuda")
        entries.append((cat, p, grids, mom, scratch, out, -1, -1))
        keep.append((pos, vel))
    arr = pk.batch_items(entries)
    work = torch.empty(pk.batch_work_bytes(arr), dtype=torch.uint8, device="cuda")
    ctx.estimate_batch(arr, work)
    ctx.sync()
    ctx.checked_selftest()
    with pytest.raises(pk.PkmomError) as e:
        ctx.sync()
    assert e.value.status == -8 and "checked" in str(e.value)
    ctx.sync()  # the word was cleared: the context stays usable
    ctx.close()


def test_unchecked_build_has_no_selftest(gpu_lib):
    pk = gpu_lib
    ctx = pk.Context(0)
    with pytest.raises(pk.PkmomError) as e:
        ctx.checked_selftest()
    assert e.value.status == -6
    ctx.close()
