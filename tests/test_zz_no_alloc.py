"""The binning entry point that allocates nothing (pkmom_spectra_static).

Callers that cannot allocate device memory while they run (a host application that
owns a fixed device pool and forbids allocator calls, a plug-in that must not grow
the footprint of the program it runs in) use this entry point; its scratch is a
fixed device array inside the library. Through the C-ABI, its output
must equal that of pkmom_spectra on the same transformed grids and moments, on two
calls in a row (the second call reuses the array the first one left behind). The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu


def _prepared(pk, ctx, cat, p):
    import torch
    pos = torch.from_numpy(cat["pos"]).cuda()
    vel = torch.from_numpy(cat["vel"]).cuda()
    dt = torch.float32 if p.precision == pk.F32 else torch.float64
    grids = torch.empty((4, p.ng, p.ng, p.ng + 2), dtype=dt, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pk.Context.scratch_bytes(p, len(cat["pos"])), dtype=torch.uint8, device="cuda")
    ctx.assign(pk.catalog_from_tensors(pos, vel), p, grids, mom, scratch)
    ctx.fft(p, grids)
    return grids, mom


@pytest.mark.parametrize("prec,order,bl_radius", [("f32", 4, 0), ("f64", 4, 0), ("f32", 1, 0), ("f32", 5, 0),
                                                  ("f64", 5, 0), ("f32", 4, 3)])
def test_static_scratch_spectra_match_regular_spectra_twice(gpu_lib, prec, order, bl_radius):
    """Every window table the entry point builds on the device: the B-spline orders 1 and
    5 and the truncated BL function's Sigma / Bhat^2 window (bl_radius 3)."""
    import torch
    pk = gpu_lib
    ctx = pk.Context(0)
    L = 400.0
    dtype = np.float32 if prec == "f32" else np.float64
    cat = catalogs.zeldovich(48, L, seed=77, dtype=dtype)
    cat["vel"] = cat["vel"] + dtype(25.0)
    p = pk.params(L, 48, 20, precision=pk.F32 if prec == "f32" else pk.F64, theta_scale=0.02, order=order,
                  bl_radius=bl_radius)
    grids, mom = _prepared(pk, ctx, cat, p)
    ref = torch.empty((pk.NROWS, p.nbins), dtype=torch.float64, device="cuda")
    ctx.spectra(p, grids, mom, ref)
    ctx.sync()
    ref = ref.cpu().numpy()
    # a different request in between leaves other contents in the shared array
    p_other = pk.params(L, 48, 7, precision=p.precision, kmin_kf=3.0, kmax_kf=20.0,
                        order=3 if order != 3 else 2)
    junk = torch.empty((pk.NROWS, 7), dtype=torch.float64, device="cuda")
    pk.spectra_static(p_other, grids, mom, junk)
    for _ in range(2):
        out = torch.full((pk.NROWS, p.nbins), -1.0, dtype=torch.float64, device="cuda")
        pk.spectra_static(p, grids, mom, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # the same per-mode values, summed in another order (and, with FP32 grids, by
        # another reduction kernel): the suite's parity tolerance for each precision
        rtol = 1e-4 if prec == "f32" else 1e-9
        np.testing.assert_allclose(got, ref, rtol=rtol, atol=rtol * np.nanmax(np.abs(ref)), equal_nan=True)
    ctx.close()


def test_static_scratch_rejects_sizes_beyond_its_limit(gpu_lib):
    import torch
    pk = gpu_lib
    p = pk.params(100.0, 32, 300)  # more shells than the static array holds
    g = torch.zeros((4, 32, 32, 34), dtype=torch.float32, device="cuda")
    m = torch.zeros(16, dtype=torch.float64, device="cuda")
    o = torch.zeros((pk.NROWS, 300), dtype=torch.float64, device="cuda")
    with pytest.raises(pk.PkmomError) as e:
        pk.spectra_static(p, g, m, o)
    assert e.value.status == -6


def test_static_scratch_rejects_non_finite_parameters(gpu_lib):
    import torch
    pk = gpu_lib
    g = torch.zeros((4, 32, 32, 34), dtype=torch.float32, device="cuda")
    m = torch.zeros(16, dtype=torch.float64, device="cuda")
    o = torch.zeros((pk.NROWS, 8), dtype=torch.float64, device="cuda")
    for field, value in (("box_L", float("inf")), ("theta_scale", float("nan"))):
        p = pk.params(100.0, 32, 8)
        setattr(p, field, value)
        with pytest.raises(pk.PkmomError) as e:
            pk.spectra_static(p, g, m, o)
        assert e.value.status == -1
