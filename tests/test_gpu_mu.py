"""Spectra in (|k|, mu) bins on the GPU (pkmom_spectra_mu) against the FP64 oracle
(oracle/mu.py), and at full size against the shell-averaged estimate and the bulk-flow
relation of Eq. bfpp."""
import numpy as np
import pytest

from oracle import mu as omu
from paper_2005_06170_gb300 import catalogs

pytestmark = pytest.mark.gpu

DIR = (0.3, -0.5, 0.81)


@pytest.fixture(scope="module")
def ctx(gpu_lib):
    c = gpu_lib.Context(0)
    yield c
    c.close()


def _cat(n_side, L, dtype, masses=False, seed=21):
    c = catalogs.zeldovich(n_side, L, seed=seed, dtype=dtype)
    c["vel"] = (c["vel"].astype(np.float64) + 51.5 * np.array([2.0, -1.0, 2.0]) / 3.0).astype(dtype)
    if masses:
        c["mass"] = np.random.default_rng(5).uniform(0.5, 1.5, len(c["vel"])).astype(dtype)
    return c


def _run(ctx, pk, c, p, nmu, direction):
    import torch
    pos = torch.from_numpy(c["pos"]).cuda()
    vel = torch.from_numpy(c["vel"]).cuda()
    mass = torch.from_numpy(c["mass"]).cuda() if "mass" in c else None
    out = ctx.estimate_mu(pos, vel, p, nmu, direction=direction, mass=mass)
    ctx.sync()
    return pk.as_mu_dict(out, p.nbins, nmu)


@pytest.mark.parametrize("dtype,masses,direction", [(np.float32, False, DIR), (np.float32, True, DIR),
                                                    (np.float64, False, DIR), (np.float64, True, DIR),
                                                    (np.float64, False, None)])
def test_mu_spectra_match_oracle(ctx, gpu_lib, dtype, masses, direction):
    """Every (shell, mu) cell: counts exact, spectra within 1e-4 (FP32 grids) / 1e-9 (FP64)
    of max(|P|, its shot-noise fluctuation scale SN/sqrt(n)). With no direction the bins
    follow the bulk flow each side computes from its own moments (FP64 catalogue only: an
    FP32 catalogue's moments agree to FP32 rounding, which can move a mode at a bin edge)."""
    pk = gpu_lib
    L, ng, nb, nmu = 100.0, 32, 6, 5
    c = _cat(24, L, dtype, masses)
    prec = pk.F32 if dtype == np.float32 else pk.F64
    p = pk.params(L, ng, nb, precision=prec, theta_scale=0.02)
    g = _run(ctx, pk, c, p, nmu, direction)
    o = omu.spectra_mu(c["pos"], c["vel"], c.get("mass"), L=L, ng=ng, nbins=nb, nmu=nmu, direction=direction,
                       theta_scale=0.02)
    rtol = 1e-4 if dtype == np.float32 else 1e-9
    n = o["n_modes"]
    np.testing.assert_array_equal(g["n_modes"], n)
    ok = n > 0
    np.testing.assert_allclose(g["k"][ok], o["k_mean"][ok], rtol=1e-6 if dtype == np.float32 else 1e-13)
    np.testing.assert_allclose(g["mu"][ok], o["mu_mean"][ok], rtol=0, atol=1e-6 if dtype == np.float32 else 1e-12)
    mom = o["moments"]
    sn_dd = o["SN_dd"]
    sn_pp = sn_dd * np.trace(mom["Q"]) / mom["S2"]
    sn_tt = o["SN_tt"]
    floors = {"P_dd": sn_dd, "P_pp": sn_pp, "P_pp_b": sn_pp, "P_tt": sn_tt, "P_tt_b": sn_tt,
              "Re_dt": np.sqrt(sn_dd * sn_tt), "Im_dt": np.sqrt(sn_dd * sn_tt), "Re_dt_b": np.sqrt(sn_dd * sn_tt),
              "Im_dt_b": np.sqrt(sn_dd * sn_tt), "Re_dpb_b": np.sqrt(sn_dd * sn_pp)}
    for key, fl in floors.items():
        scale = np.maximum(np.abs(o[key][ok]), fl[ok] / np.sqrt(n[ok]))
        err = np.abs(g[key][ok] - o[key][ok]) / scale
        assert np.all(err <= rtol), (key, float(err.max()))
    # shot-noise rows: sums of per-mode window factors in the grid precision; the odd
    # Im_SN_dt cancels between mirrored modes, down to the sum's rounding
    f32 = dtype == np.float32
    for key in ("SN_dd", "SN_tt", "Im_SN_dt"):
        np.testing.assert_allclose(g[key][ok], o[key][ok], rtol=1e-6 if f32 else 1e-12,
                                   atol=(1e-6 if f32 else 1e-12) * np.abs(o[key][ok]).max(), err_msg=key)


def test_mu_spectra_full_size_properties(ctx, gpu_lib):
    """Zel'dovich 256^3 in L = 1000 with a 51.5 km/s bulk flow, 256^3 grid, 32 shells x 8
    mu bins: the mu bins of each shell collapse to the shell average of pkmom_estimate
    (below the Nyquist shell), and Eq. bfpp holds in every cell. Prints the time."""
    import torch
    pk = gpu_lib
    L, ng, nb, nmu = 1000.0, 256, 32, 8
    c = _cat(256, L, np.float32, seed=1001)
    pos = torch.from_numpy(c["pos"]).cuda()
    vel = torch.from_numpy(c["vel"]).cuda()
    p = pk.params(L, ng, nb, kmax_kf=ng / 2 - 0.5, theta_scale=0.02)
    iso = pk.as_dict(ctx.estimate(pos, vel, p))
    ctx.estimate_mu(pos, vel, p, nmu)  # warm-up (tables, work arrays)
    ctx.sync()
    ctx.timing(True)
    ctx.timing_read()
    g = pk.as_mu_dict(ctx.estimate_mu(pos, vel, p, nmu), nb, nmu)
    ctx.sync()
    t = ctx.timing_read()
    ctx.timing(False)
    print(f"(|k|, mu) binning, 256^3 grid, {nb} x {nmu} cells: {t['bin'][0]:.3f} ms")
    n = g["n_modes"]
    np.testing.assert_array_equal(n.sum(axis=1), iso["n_modes"])
    for key in ("P_dd", "P_pp", "P_tt", "P_pp_b", "P_tt_b"):
        s = np.nansum(g[key] * n, axis=1) / n.sum(axis=1)
        np.testing.assert_allclose(s, iso[key], rtol=1e-5, atol=1e-6 * np.abs(iso[key]).max(), err_msg=key)
    for key, ikey in (("Re_dt", "P_dt"), ("Re_dt_b", "P_dt_b")):
        s = np.nansum(g[key] * n, axis=1) / n.sum(axis=1)
        tol = 1e-5 * np.sqrt(iso["SN_dd"] * iso["SN_tt"]) + 1e-5 * np.abs(iso[ikey])
        assert np.all(np.abs(s - iso[ikey]) <= tol), key
    vbn = np.linalg.norm(np.asarray(c["vel"], np.float64).mean(axis=0))
    ok = n > 0
    lhs = (g["P_pp"] - g["P_pp_b"])[ok]
    rhs = (2 * vbn * g["Re_dpb_b"] + vbn ** 2 * g["P_dd"])[ok]
    assert np.all(np.abs(lhs - rhs) <= 1e-4 * np.abs(g["P_pp"][ok]) + 1e-4 * np.abs(lhs).max())
