"""GPU library vs the FP64 CPU oracle, through the C-ABI, on the same seeded inputs.

Tolerances: FP64 mode 1e-9 and FP32 grids 1e-4, relative
per k-shell, with a floor at the shell's shot-noise fluctuation scale SN_b/sqrt(n_b)
for shells whose noise-subtracted value is near zero.
"""
import ctypes

import numpy as np
import pytest

from oracle import estimator as est
from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu

SN_OF = {"P_dd": "SN_dd", "P_pp": "SN_pp", "P_tt": "SN_tt", "P_pp_b": "SN_pp_b", "P_tt_b": "SN_tt_b"}
KEYS = ("P_dd", "P_pp", "P_tt", "P_dt")
KEYS_B = ("P_pp_b", "P_tt_b", "P_dt_b")


def compare(gpu: dict, ora: dict, rtol: float, bulk: bool = True):
    """Per-shell relative error with the shot-noise floor; returns the worst value."""
    n = ora["n_modes"]
    np.testing.assert_array_equal(gpu["n_modes"], n)
    ok = n > 0
    np.testing.assert_allclose(gpu["k"][ok], ora["k_mean"][ok], rtol=1e-13)
    assert np.all(np.isnan(gpu["k"][~ok]))
    worst = 0.0
    for key in KEYS + (KEYS_B if bulk else ()):
        o, g = ora[key][ok], gpu[key][ok]
        if key in SN_OF:
            floor = ora[SN_OF[key]][ok] / np.sqrt(n[ok])
        else:
            sfx = "_b" if key.endswith("_b") else ""
            floor = np.sqrt(ora["SN_dd"][ok] * ora["SN_tt" + sfx][ok]) / np.sqrt(n[ok])
        if key.endswith("_b"):
            # F_p' = F_p - v_b F_d cancels when v_b dominates (one particle: exactly):
            # its rounding is set by the unsubtracted fields, a few ulps of them
            eps = 2.2e-16 if rtol <= 1e-9 else 1.2e-7
            base = key[:-2]
            unsub = np.abs(ora[base][ok]) + (ora[SN_OF[base]][ok] if base in SN_OF else
                                             np.sqrt(ora["SN_dd"][ok] * ora["SN_tt"][ok]))
            floor = np.maximum(floor, 100.0 * eps / rtol * unsub)
        scale = np.maximum(np.abs(o), floor)
        err = np.abs(g - o) / scale
        worst = max(worst, float(err.max()))
        assert np.all(err <= rtol), (key, float(err.max()), int(err.argmax()))
    # shot-noise rows depend only on the moments: FP64 sums of FP64 values, or of FP32
    # values summed 16 at a time in FP32 before each FP64 add
    sn_rtol = 1e-12 if rtol <= 1e-9 else 1e-6
    for key, skey in SN_OF.items():
        if bulk or not key.endswith("_b"):
            np.testing.assert_allclose(gpu[skey][ok], ora[skey][ok], rtol=sn_rtol)
    return worst


def to_dev(cat, torch):
    pos = torch.from_numpy(cat["pos"]).cuda()
    vel = torch.from_numpy(cat["vel"]).cuda()
    mass = torch.from_numpy(cat["mass"]).cuda() if "mass" in cat else None
    return pos, vel, mass


def run_gpu(ctx, pkmom, cat, p):
    import torch
    pos, vel, mass = to_dev(cat, torch)
    out = ctx.estimate(pos, vel, p, mass=mass)
    ctx.sync()
    return pkmom.as_dict(out)


def run_oracle(cat, L, ng, nbins, **kw):
    return est.estimate(cat["pos"], cat["vel"], cat.get("mass"), L=L, ng=ng, nbins=nbins, **kw)


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


# ------------------------------------------------------------------ stages

@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_moments_match_oracle(ctx, gpu_lib, dtype):
    import torch
    pk = gpu_lib
    cat = catalogs.poisson(100003, 300.0, seed=41, dtype=dtype, bulk=(120.0, -40.0, 7.0), unit_mass=False)
    prec = pk.F32 if dtype == np.float32 else pk.F64
    p = pk.params(300.0, 32, 8, precision=prec)
    pos, vel, mass = to_dev(cat, torch)
    grids = torch.empty(pk.Context.grid_bytes(32, prec) // 4, dtype=torch.int32, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pk.Context.scratch_bytes(p, len(cat["pos"])), dtype=torch.uint8, device="cuda")
    ctx.assign(pk.catalog_from_tensors(pos, vel, mass), p, grids, mom, scratch)
    ctx.sync()
    m = mom.cpu().numpy()
    ref = est.moments(cat["vel"], cat["mass"])
    rt = 2e-6 if dtype == np.float32 else 1e-12
    np.testing.assert_allclose(m[0], ref["M"], rtol=rt)
    np.testing.assert_allclose(m[1], ref["S2"], rtol=rt)
    np.testing.assert_allclose(m[2:5] / m[0], ref["vb"], rtol=rt * 10, atol=rt * 300)
    Q = ref["Q"]
    np.testing.assert_allclose(m[8:14], [Q[0, 0], Q[1, 1], Q[2, 2], Q[0, 1], Q[0, 2], Q[1, 2]], rtol=rt * 10,
                               atol=rt * np.trace(Q))
    assert m[14] == len(cat["pos"])


@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("dtype,ng", [(np.float32, 32), (np.float64, 24), (np.float32, 40)])
def test_assigned_grids_match_oracle(ctx, gpu_lib, order, dtype, ng):
    import torch
    pk = gpu_lib
    L = 123.0
    cat = catalogs.poisson(7777, L, seed=43 + order, dtype=dtype, unit_mass=(order != 2))
    prec = pk.F32 if dtype == np.float32 else pk.F64
    p = pk.params(L, ng, 8, precision=prec, order=order)
    pos, vel, mass = to_dev(cat, torch)
    tdt = torch.float32 if dtype == np.float32 else torch.float64
    grids = torch.empty((4, ng, ng, ng + 2), dtype=tdt, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pk.Context.scratch_bytes(p, len(cat["pos"])), dtype=torch.uint8, device="cuda")
    ctx.assign(pk.catalog_from_tensors(pos, vel, mass), p, grids, mom, scratch)
    ctx.sync()
    g = grids[..., :ng].double().cpu().numpy()
    ref = est.assign(cat["pos"], cat["vel"], cat.get("mass"), L=L, ng=ng, order=order)
    # FP32 grids are accumulated in 32-bit fixed point per tile: each contribution is
    # rounded to 2^-s with 2^s * (largest possible node value of the tile) < 2^30, about
    # 2^-20 of the tile's sum of |q|; FP64 grids use FP64 atomics
    for f in range(4):
        scale = np.abs(ref[f]).max()
        tol = (1e-5 if dtype == np.float32 else 1e-12) * scale
        assert np.max(np.abs(g[f] - ref[f])) <= tol, (f, np.max(np.abs(g[f] - ref[f])) / scale)


@pytest.mark.parametrize("order", [3, 4, 5])
@pytest.mark.parametrize("kind", ["uniform", "clustered"])
def test_bank_grouped_list_equals_per_node_path(ctx, gpu_lib, order, kind):
    """Sparse tiles of the gather deposit (16^3 cells) regroup their particle list by the
    shared-memory bank of each stencil's first node and add every node at an immediate
    offset from it. Each contribution is the same rounded integer as on the per-node path
    of unlisted tiles (list capacity 0), so the grids agree bit for bit. Against the oracle:
    1e-5 of the largest node for the uniform catalogue; the clustered one (listed, unlisted
    and dense tiles in one launch) gets 5e-5, because a blob tile rounds each of its
    thousands of contributions per node at 2^-30 of its own bound (sum of |q| over its
    reach times the largest weight), which is many times the largest node value. Orders 3
    and 5 move the first node with the offset in the cell."""
    import torch
    pk = gpu_lib
    ng, n, L = 64, 30000, 300.0
    cat = catalogs.poisson(n, L, seed=70 + order, dtype=np.float32) if kind == "uniform" else _clustered(n, L, 71)
    p = pk.params(L, ng, 8, order=order)
    pos, vel, mass = to_dev(cat, torch)
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    out = []
    for list_cap in (-1, 0):
        grids = torch.empty((4, ng, ng, ng + 2), dtype=torch.float32, device="cuda")
        ctx.set_tuning(0, list_cap)
        try:
            scratch = torch.empty(ctx.scratch_bytes_tuned(p, n), dtype=torch.uint8, device="cuda")
            ctx.assign(pk.catalog_from_tensors(pos, vel, mass), p, grids, mom, scratch)
            ctx.sync()
        finally:
            ctx.set_tuning(-1, -1)
        out.append(grids[..., :ng].clone())
    assert torch.equal(out[0], out[1])
    g = out[0].double().cpu().numpy()
    ref = est.assign(cat["pos"], cat["vel"], None, L=L, ng=ng, order=order)
    rtol = 1e-5 if kind == "uniform" else 5e-5
    for f in range(4):
        scale = np.abs(ref[f]).max()
        assert np.max(np.abs(g[f] - ref[f])) <= rtol * scale, (f, np.max(np.abs(g[f] - ref[f])) / scale)


def _clustered(n, L, seed):
    """Half the particles in a Gaussian blob (sigma = L/16) at the centre, 40 % uniform in
    the slab x < L/3, 10 % uniform in the box: 16^3-cell tiles of every density class."""
    rng = np.random.Generator(np.random.PCG64(seed))
    nb, ns = n // 2, (2 * n) // 5
    nu = n - nb - ns
    blob = rng.normal(L / 2, L / 16, (nb, 3))
    slab = rng.uniform(0, L, (ns, 3))
    slab[:, 0] /= 3
    pos = np.mod(np.concatenate([blob, slab, rng.uniform(0, L, (nu, 3))]), L).astype(np.float32)
    pos[pos >= np.float32(L)] = 0
    vel = rng.normal(0, 300, (n, 3)).astype(np.float32)
    return {"pos": pos, "vel": vel}


@pytest.mark.parametrize("kind,ng,n,tile", [("uniform", 32, 40000, -1), ("clustered", 48, 66355, -1),
                                            ("uniform", 64, 20000, 7), ("clustered", 32, 20000, 7)])
def test_home_tile_grids_match_oracle(ctx, gpu_lib, kind, ng, n, tile):
    """Home-tile deposit (each particle once by the tile owning its cell, halos added by a
    fix-up pass): uniform catalogues (one particle per lane of a 2 x 16 cell block, extra
    particles queued), clustered ones (dense, medium and sparse tiles in one launch), and
    the tile forced below half a particle per cell."""
    import torch
    pk = gpu_lib
    L = 200.0
    cat = catalogs.poisson(n, L, seed=90 + ng, dtype=np.float32) if kind == "uniform" else _clustered(n, L, 91 + ng)
    p = pk.params(L, ng, 8)
    pos, vel, mass = to_dev(cat, torch)
    grids = torch.empty((4, ng, ng, ng + 2), dtype=torch.float32, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    ctx.set_tuning(tile, -1)
    try:
        scratch = torch.empty(ctx.scratch_bytes_tuned(p, n), dtype=torch.uint8, device="cuda")
        ctx.assign(pk.catalog_from_tensors(pos, vel, mass), p, grids, mom, scratch)
        ctx.sync()
    finally:
        ctx.set_tuning(-1, -1)
    g = grids[..., :ng].double().cpu().numpy()
    ref = est.assign(cat["pos"], cat["vel"], None, L=L, ng=ng, order=4)
    for f in range(4):
        scale = np.abs(ref[f]).max()
        assert np.max(np.abs(g[f] - ref[f])) <= 1e-5 * scale, (f, np.max(np.abs(g[f] - ref[f])) / scale)


# ------------------------------------------------------------------ whole estimator

def test_config1_fp64_poisson(ctx, gpu_lib):
    """32768 Poisson particles in L = 256, sigma_v = 300, unit mass, 64^3 grid, BL3,
    32 bins from k_f to k_N, FP64: parity 1e-9."""
    pk = gpu_lib
    cat = catalogs.poisson(32768, 256.0, sigma_v=300.0, seed=1000, dtype=np.float64)
    p = pk.params(256.0, 64, 32, precision=pk.F64)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, 256.0, 64, 32)
    compare(g, o, 1e-9)


@pytest.mark.parametrize("seed", [1, 2])
def test_zeldovich_fp32_small(ctx, gpu_lib, seed):
    pk = gpu_lib
    L = 500.0
    cat = catalogs.zeldovich(64, L, seed=seed, dtype=np.float32)
    p = pk.params(L, 64, 32, theta_scale=1.0 / 50.0)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, L, 64, 32, theta_scale=1.0 / 50.0)
    compare(g, o, 1e-4)


def test_ragged_fp32_masses_odd_order(ctx, gpu_lib):
    """ng = 40 (no 16-wide tile divides it), n not a multiple of any block, 7 shells
    over an inner k range, TSC order, random masses, isotropic theta noise."""
    pk = gpu_lib
    L = 77.0
    cat = catalogs.poisson(12345, L, seed=45, dtype=np.float32, bulk=(30.0, 0.0, -60.0), unit_mass=False)
    kw = dict(kmin_kf=2.3, kmax_kf=15.5, theta_scale=0.37, theta_sn="isotropic", order=3)
    p = pk.params(L, 40, 7, **kw)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, L, 40, 7, kmin_kf=2.3, kmax_kf=15.5, theta_scale=0.37, theta_sn="isotropic", order=3)
    compare(g, o, 1e-4)


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_more_shells_than_radii(ctx, gpu_lib, prec):
    """128 shells from k_f to k_N on a 32^3 grid (width 0.12 k_f): the inner shells that
    no integer |n|^2 reaches are empty (no mode, k NaN), and every (slab, shell) item of
    the work list is either binned or skipped by the same geometry."""
    pk = gpu_lib
    L = 100.0
    dt = np.float32 if prec == "f32" else np.float64
    cat = catalogs.poisson(20000, L, seed=61, dtype=dt, bulk=(40.0, -25.0, 10.0))
    p = pk.params(L, 32, 128, precision=pk.F32 if prec == "f32" else pk.F64)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, L, 32, 128)
    assert (o["n_modes"] == 0).sum() > 10
    compare(g, o, 1e-4 if prec == "f32" else 1e-9)


@pytest.mark.parametrize("order", [1, 2, 4, 5])
def test_orders_fp64(ctx, gpu_lib, order):
    pk = gpu_lib
    L = 64.0
    cat = catalogs.poisson(5000, L, seed=47, dtype=np.float64, bulk=(0.0, 341.0, 0.0))
    p = pk.params(L, 32, 10, precision=pk.F64, order=order)
    compare(run_gpu(ctx, pk, cat, p), run_oracle(cat, L, 32, 10, order=order), 1e-9)


def test_no_shot_noise_no_bulk(ctx, gpu_lib):
    pk = gpu_lib
    L = 200.0
    cat = catalogs.zeldovich(32, L, seed=5, dtype=np.float64)
    p = pk.params(L, 32, 12, precision=pk.F64, subtract_shot_noise=False, bulk=False)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, L, 32, 12, subtract_shot_noise=False, bulk=False)
    compare(g, o, 1e-9, bulk=False)
    for key in KEYS_B:
        assert np.all(np.isnan(g[key]))


# ------------------------------------------------------------------ edge cases

def test_single_particle_and_wrapped_positions(ctx, gpu_lib):
    pk = gpu_lib
    L = 50.0
    pos = np.array([[-3.25, 49.999, 123.5]], dtype=np.float64)  # outside [0, L): wrapped
    cat = {"pos": pos, "vel": np.array([[10.0, -20.0, 5.0]]), "L": L}
    p = pk.params(L, 16, 4, precision=pk.F64)
    compare(run_gpu(ctx, pk, cat, p), run_oracle(cat, L, 16, 4), 1e-9)


def test_all_particles_in_one_cell(ctx, gpu_lib):
    """Dense catalogue: every particle in two neighbouring cells (shared-memory
    contention, 2e4 contributions per node whose momentum sums cancel), held to the
    normal shot-noise floor. An FP64 emulation of FP32 grids and an FP32 FFT of the same
    catalogue stays within 2e-6 of that floor, so FP32 arithmetic needs no wider one."""
    pk = gpu_lib
    rng = np.random.default_rng(51)
    L, ng, n = 100.0, 32, 20000
    pos = (10.0 + rng.uniform(0, L / ng, size=(n, 3))).astype(np.float32)
    vel = rng.normal(0, 100, size=(n, 3)).astype(np.float32)
    cat = {"pos": pos, "vel": vel, "L": L}
    p = pk.params(L, ng, 8)
    worst = compare(run_gpu(ctx, pk, cat, p), run_oracle(cat, L, ng, 8), 1e-4)
    print(f"all particles in one cell: worst normalised shell error {worst:.3e}")


def test_positions_on_the_box_edge_fp32(ctx, gpu_lib):
    pk = gpu_lib
    L, ng = 256.0, 16
    pos = np.array([[0.0, 0.0, 0.0], [np.float32(L), 255.99998, 16.0], [1e-30, 128.0, 240.0]], dtype=np.float32)
    vel = np.array([[1.0, 2.0, 3.0], [4.0, 5.0, 6.0], [7.0, 8.0, 9.0]], dtype=np.float32)
    cat = {"pos": pos, "vel": vel, "L": L}
    for order in (1, 4):
        p = pk.params(L, ng, 4, order=order)
        compare(run_gpu(ctx, pk, cat, p), run_oracle(cat, L, ng, 4, order=order), 1e-4)


def test_non_finite_position_is_reported(ctx, gpu_lib):
    import torch
    pk = gpu_lib
    pos = torch.tensor([[1.0, 2.0, 3.0], [float("nan"), 1.0, 1.0]], dtype=torch.float32, device="cuda")
    vel = torch.zeros_like(pos)
    with pytest.raises(pk.PkmomError) as e:
        ctx.estimate(pos, vel, pk.params(10.0, 16, 4))
        ctx.sync()
    assert e.value.status == -8
    # the context stays usable
    out = ctx.estimate(pos[:1].contiguous(), vel[:1].contiguous(), pk.params(10.0, 16, 4))
    ctx.sync()
    assert np.isfinite(out[pk.ROW["P_pp"]].cpu().numpy()).all()


def test_invalid_arguments(ctx, gpu_lib):
    import torch
    pk = gpu_lib
    pos = torch.zeros((4, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(pk.PkmomError) as e:
        ctx.estimate(pos, pos, pk.params(10.0, 16, 4, precision=pk.F64))  # dtype mismatch
    assert e.value.status == -1
    p = pk.params(10.0, 16, 4)
    grids = torch.empty(pk.Context.grid_bytes(16, 0) // 4, dtype=torch.float32, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    small = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(pk.PkmomError) as e:
        ctx.assign(pk.catalog_from_tensors(pos, pos), p, grids, mom, small)
    assert e.value.status == -7


def test_host_entry_point_equals_device_entry_point(ctx, gpu_lib):
    pk = gpu_lib
    L = 300.0
    cat = catalogs.zeldovich(32, L, seed=9, dtype=np.float32)
    p = pk.params(L, 32, 10)
    d = run_gpu(ctx, pk, cat, p)
    h = pk.as_dict(ctx.estimate_host(cat["pos"], cat["vel"], p))
    for k in pk.ROW:
        np.testing.assert_allclose(h[k], d[k], rtol=1e-6, equal_nan=True)


def test_kernels_come_from_the_in_tree_library(ctx, gpu_lib):
    import os
    pk = gpu_lib
    before = ctx.kernel_launches()
    cat = catalogs.poisson(1000, 10.0, seed=3)
    run_gpu(ctx, pk, cat, pk.params(10.0, 16, 4))
    assert ctx.kernel_launches() - before >= 9
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    assert pk.library_path().startswith(root)
    with open("/proc/self/maps") as fh:
        assert pk.library_path() in fh.read()


# ------------------------------------------------------------------ full-size workload

def test_config2_full_size_both_bulk_variants(ctx, gpu_lib):
    """Zel'dovich 256^3 particles in L = 1000, 256^3 FP32 grid, 128 shells, with and
    without the bulk flow: the launch configuration the benchmark times."""
    pk = gpu_lib
    L = 1000.0
    cat = catalogs.zeldovich(256, L, seed=1001, dtype=np.float32)
    p = pk.params(L, 256, 128)
    g = run_gpu(ctx, pk, cat, p)
    o = run_oracle(cat, L, 256, 128)
    worst = compare(g, o, 1e-4)
    print(f"config 2 worst normalised shell error {worst:.3e}")


def test_misaligned_grids_are_rejected(ctx, gpu_lib):
    """The deposit writes grid rows in 8-byte pairs: grids and scratch must be 16-byte
    aligned, and a pointer that is not gives PKMOM_EINVAL (nothing is launched)."""
    import torch
    pk = gpu_lib
    p = pk.params(100.0, 16, 4)
    pos = torch.rand((100, 3), device="cuda") * 100.0
    vel = torch.zeros_like(pos)
    cat = pk.catalog_from_tensors(pos, vel)
    grids = torch.empty(pk.Context.grid_bytes(16) // 4 + 4, dtype=torch.float32, device="cuda")
    mom = torch.zeros(16, dtype=torch.float64, device="cuda")
    scratch = torch.empty(pk.Context.scratch_bytes(p, 100), dtype=torch.uint8, device="cuda")
    with pytest.raises(pk.PkmomError) as e:
        ctx.assign(cat, p, grids[1:], mom, scratch)
    assert e.value.status == -1
    ctx.assign(cat, p, grids[4:], mom, scratch)  # 16 bytes in: fine
    ctx.sync()
