"""Direct real-space assignment with the BL function truncated to R cells (the literal
stencil of Sec. 2.4.1, (2R)^3 nodes per particle) against the oracle, and its bias
relative to the exact (factored) BL kernel."""
import numpy as np
import pytest

from oracle import estimator as est
from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def _dev(cat, torch):
    return torch.from_numpy(cat["pos"]).cuda(), torch.from_numpy(cat["vel"]).cuda()


@pytest.mark.parametrize("radius", [2, 3, 4])
@pytest.mark.parametrize("dtype,ng", [(np.float32, 32), (np.float32, 24), (np.float64, 32), (np.float64, 24)])
def test_direct_bl_grids_match_oracle(ctx, gpu_lib, radius, dtype, ng):
    """Grids of the 16^3 (ng = 32) and 8^3 (ng = 24) tiles against the oracle: FP64 within
    1e-12 of the grid maximum; FP32 within 1e-5 (R/2)^3. The FP32 grids are 32-bit fixed
    point: each of a node's contributions is rounded once, at a step set by the tile's
    worst-case node sum, and both the contributions per node and that bound grow with the
    stencil volume (2R)^3, eight times the cubic B-spline's at R = 4."""
    import torch
    pk = gpu_lib
    L = 150.0
    cat = catalogs.poisson(6000, L, seed=70 + radius + ng, dtype=dtype)
    prec = pk.F32 if dtype == np.float32 else pk.F64
    p = pk.params(L, ng, 8, precision=prec, bl_radius=radius)
    pos, vel = _dev(cat, torch)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    grids = torch.empty((4, ng, ng, ng + 2), dtype=tdt, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pk.Context.scratch_bytes(p, len(cat["pos"])), dtype=torch.uint8, device="cuda")
    ctx.assign(pk.catalog_from_tensors(pos, vel, None), p, grids, mom, scratch)
    ctx.sync()
    g = grids[..., :ng].double().cpu().numpy()
    ref = est.assign_bl_direct(cat["pos"], cat["vel"], None, L=L, ng=ng, radius=radius)
    tol = 1e-5 * (radius / 2) ** 3 if dtype == np.float32 else 1e-12
    for f in range(4):
        scale = np.abs(ref[f]).max()
        assert np.max(np.abs(g[f] - ref[f])) <= tol * scale, (f, np.max(np.abs(g[f] - ref[f])) / scale)


@pytest.mark.parametrize("radius", [2, 4])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_direct_bl_spectra_match_oracle(ctx, gpu_lib, radius, dtype):
    from test_gpu_parity import compare
    import torch
    pk = gpu_lib
    L, ng, nb = 200.0, 32, 10
    cat = catalogs.zeldovich(24, L, seed=80 + radius, dtype=dtype)
    prec = pk.F32 if dtype == np.float32 else pk.F64
    pos, vel = _dev(cat, torch)
    g = pk.as_dict(ctx.estimate(pos, vel, pk.params(L, ng, nb, precision=prec, bl_radius=radius)))
    ctx.sync()
    o = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, nbins=nb, bl_radius=radius)
    compare(g, o, 1e-4 if dtype == np.float32 else 1e-9)


def test_truncation_bias_shrinks_with_radius(ctx, gpu_lib):
    """Raw spectra of a 64^3 Zel'dovich catalogue with the truncated kernel against the
    exact kernel: the deviation (the truncation bias of a real-space BL stencil) falls
    as R grows; printed for the record."""
    import torch
    pk = gpu_lib
    L, ng, nb = 250.0, 64, 16
    cat = catalogs.zeldovich(64, L, seed=90, dtype=np.float32)
    pos, vel = _dev(cat, torch)
    exact = pk.as_dict(ctx.estimate(pos, vel, pk.params(L, ng, nb, subtract_shot_noise=False)))
    worst = {}
    for R in (2, 3, 4):
        d = pk.as_dict(ctx.estimate(pos, vel, pk.params(L, ng, nb, subtract_shot_noise=False, bl_radius=R)))
        ctx.sync()
        dev = {k: np.abs(d[k] / exact[k] - 1) for k in ("P_dd", "P_pp", "P_tt")}
        worst[R] = max(float(v.max()) for v in dev.values())
        half = nb // 2
        print(f"R={R}: max |P_R/P - 1| below k_N/2 "
              f"{max(float(v[:half].max()) for v in dev.values()):.2e}, up to k_N {worst[R]:.2e}")
    assert worst[2] > worst[3] > worst[4]
