"""Pins for the oracle's estimator (oracle/estimator.py) against things that do not
come from the oracle itself: brute force, closed forms, exact identities of the
paper, and statistics of catalogues whose true spectrum is known.
"""
import numpy as np
import pytest

from oracle import _clib, direct
from oracle import bspline as bs
from oracle import estimator as est
from paper_2005_06170_gb300 import catalogs


# ---------------------------------------------------------------- assignment

@pytest.mark.parametrize("order", [1, 2, 3, 4, 5])
def test_deposit_conserves_each_field(order):
    rng = np.random.default_rng(3)
    u = rng.uniform(-20, 40, size=(300, 3))
    q = rng.normal(size=(300, 4))
    g = _clib.deposit_bspline(u, q, order, 16)
    np.testing.assert_allclose(g.reshape(4, -1).sum(axis=1), q.sum(axis=0), rtol=1e-12)


def test_deposit_single_particle_weights_are_bspline_samples():
    # a particle at u = 5.25 on each axis: weights B_4(5.25 - n) per axis
    u = np.array([[5.25, 5.25, 5.25]])
    g = _clib.deposit_bspline(u, np.ones(1), 4, 16)[0]
    t = 0.25
    ref1 = np.zeros(16)
    ref1[4:8] = [(1 - t) ** 3 / 6, (3 * t ** 3 - 6 * t ** 2 + 4) / 6, (-3 * t ** 3 + 3 * t ** 2 + 3 * t + 1) / 6, t ** 3 / 6]
    np.testing.assert_allclose(g, np.einsum("i,j,k->ijk", ref1, ref1, ref1), atol=1e-15)


def test_deposit_ngp_half_open_cells():
    u = np.array([[2.5, 2.4999, 0.0], [15.5, 7.0, 3.0]])
    g = _clib.deposit_bspline(u, np.ones(2), 1, 16)[0]
    assert g[3, 2, 0] == 1.0  # 2.5 rounds up, 2.4999 down
    assert g[0, 7, 3] == 1.0  # 15.5 -> node 16 -> wraps to 0
    assert g.sum() == 2.0


def test_fp32_grid_coordinates_are_formed_in_fp32():
    pos = np.array([[999.99994, 0.1, 500.0]], dtype=np.float32)
    u = est.grid_coordinates(pos, 1000.0, 256)
    ref = (pos * np.float32(256 / 1000.0)).astype(np.float64)
    assert np.array_equal(u, ref)
    assert u.dtype == np.float64


@pytest.mark.parametrize("radius", [2, 3, 4])
def test_truncated_bl_deposit_keeps_the_nearest_image_within_the_radius(radius):
    """Direct truncated BL deposit of one particle: the weight of node n on each axis is
    phi(d) for the nearest image distance d when |d| < R, else 0, whereas the untruncated
    deposit folds every image (Sec. 2.4.1, the literal real-space stencil)."""
    rng = np.random.default_rng(11 + radius)
    ng = 16
    for _ in range(4):
        u = rng.uniform(0, ng, size=(1, 3))
        g = direct.deposit_bl_direct(u, np.ones((1, 1)), ng, 4, radius=radius)[0]
        nodes = np.arange(ng)
        w = []
        for a in range(3):
            d = u[0, a] - nodes
            d = d - ng * np.round(d / ng)  # nearest image
            w.append(np.where(np.abs(d) < radius, bs.phi(d, 4), 0.0))
        ref = w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
        np.testing.assert_allclose(g, ref, rtol=0, atol=1e-13)
        assert np.count_nonzero(np.abs(g) > 0) <= (2 * radius) ** 3


def test_truncated_bl_estimate_converges_to_the_exact_kernel():
    """As the radius grows the direct truncated-BL spectra approach those of the exact
    (factored, Fourier-space) BL kernel, an independent route: the truncation bias
    shrinks with the tail of phi (about 0.5^R)."""
    cat = catalogs.poisson(3000, 100.0, seed=3, dtype=np.float64)
    kw = dict(L=100.0, ng=16, nbins=6, subtract_shot_noise=False)
    exact = est.estimate(cat["pos"], cat["vel"], **kw)
    dev = {}
    for R in (4, 8, 16):
        d = est.estimate(cat["pos"], cat["vel"], bl_radius=R, **kw)
        dev[R] = max(float(np.max(np.abs(d[k] / exact[k] - 1))) for k in ("P_dd", "P_pp", "P_tt", "P_dt"))
    assert dev[4] > dev[8] > dev[16]
    assert dev[16] < 1e-4, dev


@pytest.mark.parametrize("order", [3, 4, 5])
def test_factored_bl_equals_direct_real_space_bl(order):
    """The oracle's BL field (B-spline deposit x periodic Fourier factor) equals the
    deposit with phi itself, summed over periodic images (direct, no Fourier factor)."""
    rng = np.random.default_rng(7)
    ng = 8
    u = rng.uniform(0, ng, size=(12, 3))
    q = rng.normal(size=(12, 2))
    gd = direct.deposit_bl_direct(u, q, ng, order, reach=40, nmax=40)
    gb = _clib.deposit_bspline(u, q, order, ng)
    Fd = np.fft.rfftn(gd, axes=(1, 2, 3))
    Fb = np.fft.rfftn(gb, axes=(1, 2, 3))
    nf = est.signed_freq(ng)
    nh = np.arange(ng // 2 + 1)
    cf = bs.alias_sum(2 * np.pi * nf / ng, order) ** -0.5
    ch = bs.alias_sum(2 * np.pi * nh / ng, order) ** -0.5
    C = cf[:, None, None] * cf[None, :, None] * ch[None, None, :]
    assert np.max(np.abs(Fd - Fb * C)) < 1e-9 * np.max(np.abs(Fd))


# ---------------------------------------------------------------- FFT

def test_fft_matches_brute_force_dft():
    rng = np.random.default_rng(11)
    g = rng.normal(size=(2, 8, 8, 8))
    F = est.fft_grids(g, workers=1)
    for f in range(2):
        full = direct.dft3(g[f])
        np.testing.assert_allclose(F[f], full[:, :, :5], atol=1e-11)


# ---------------------------------------------------------------- binning

def test_bin_index_edges():
    n2 = np.array([0, 1, 2, 3, 4, 63, 64, 65])
    b = est.bin_index(n2, 4, 1.0, 8.0)
    # u = 0 excluded, 1 -> bin 0, 8 (=umax) -> last bin, >8 excluded
    assert b[0] == -1 and b[1] == 0 and b[6] == 3 and b[7] == -1


def test_half_spectrum_binning_matches_full_sphere():
    """Mode counts, <|k|> and a deconvolved auto spectrum from the half spectrum with
    weights 1/2/1 equal a plain average over every mode of the full complex FFT."""
    rng = np.random.default_rng(5)
    ng, L, nb = 16, 100.0, 6
    cat = catalogs.poisson(400, L, seed=9, dtype=np.float64)
    grids = est.assign(cat["pos"], cat["vel"], None, L=L, ng=ng, order=4)
    F = est.fft_grids(grids, workers=1)
    mom = est.moments(cat["vel"])
    out = est.spectra_from_fourier(F, mom, L=L, ng=ng, nbins=nb, subtract_shot_noise=False, bulk=False)
    Ffull = np.fft.fftn(grids[1])
    f = est.signed_freq(ng)
    w = 2 * np.pi * f / ng
    bh2 = bs.bspline_hat(w, 4) ** 2
    B2 = bh2[:, None, None] * bh2[None, :, None] * bh2[None, None, :]
    # the x-momentum part of P_pp only: compare against one component via linearity
    vals = L ** 3 * np.abs(Ffull) ** 2 / mom["M"] ** 2 / B2
    cnt, mean = direct.full_sphere_bins(vals, ng, nb, 1.0, ng / 2, est.bin_index)
    np.testing.assert_array_equal(out["n_modes"], cnt)
    out_x = est.spectra_from_fourier(np.stack([F[0], F[1], 0 * F[2], 0 * F[3]]), mom, L=L, ng=ng, nbins=nb,
                                     subtract_shot_noise=False, bulk=False)
    np.testing.assert_allclose(out_x["P_pp"], mean, rtol=1e-11)
    kf = 2 * np.pi / L
    kk = np.sqrt(f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2) * kf
    _, kmean = direct.full_sphere_bins(kk, ng, nb, 1.0, ng / 2, est.bin_index)
    np.testing.assert_allclose(out["k_mean"], kmean, rtol=1e-13)
    rng.normal()


# ---------------------------------------------------------------- closed forms

def _lattice_expected(ng, L, kint, amp, order=4):
    """Deconvolved P_pp at +-k0 for one particle per node with v = amp e cos(k0.q).

    The lattice-sampled B_m has DFT H(w) = sum_d B_m(d) cos(w d) (B_4: (2 + cos w)/3);
    the deconvolved mode is F_B / prod Bhat_m, with |F_B| = amp ng^3 / 2 prod H.
    """
    V = L ** 3
    val = V * amp ** 2 / 4.0
    samples = {4: lambda w: (2 + np.cos(w)) / 3.0, 2: lambda w: np.ones_like(w), 1: lambda w: np.ones_like(w),
               3: lambda w: (3 + np.cos(w)) / 4.0, 5: lambda w: (115 + 76 * np.cos(w) + np.cos(2 * w)) / 192.0}
    for a in range(3):
        w = 2 * np.pi * kint[a] / ng
        val *= (samples[order](np.array(w)) / bs.bspline_hat(w, order)) ** 2
    return float(val)


@pytest.mark.parametrize("order", [5, 4, 3, 2])
@pytest.mark.parametrize("kint,e,kind", [((1, 2, 0), (2, -1, 0), "curl"), ((1, 2, 0), (1, 2, 0), "grad"),
                                         ((0, 0, 3), (0, 0, 1), "grad"), ((2, 1, 1), (0, 1, -1), "curl")])
def test_lattice_plane_wave_closed_form(order, kint, e, kind):
    ng, L, amp = 16, 16.0, 50.0
    e = np.asarray(e, dtype=np.float64)
    e = e / np.linalg.norm(e)
    cat = catalogs.lattice_wave(ng, L, kint, e, amp)
    out = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, order=order, nbins=8, subtract_shot_noise=False,
                       theta_scale=0.01, workers=1)
    P0 = _lattice_expected(ng, L, kint, amp, order)
    nsq = sum(k * k for k in kint)
    b = est.bin_index(np.array([nsq]), 8, 1.0, ng / 2)[0]
    expect = np.zeros(8)
    expect[b] = 2 * P0 / out["n_modes"][b]
    np.testing.assert_allclose(out["P_pp"], expect, rtol=1e-10, atol=1e-10 * expect.max())
    # D(n) is constant (partition of unity): no density or cross power at k != 0
    assert np.max(np.abs(out["P_dd"])) < 1e-20 * P0 + 1e-12
    assert np.max(np.abs(out["P_dt"])) < 1e-12 * expect.max()
    k0 = 2 * np.pi / L * np.sqrt(nsq)
    if kind == "grad":
        np.testing.assert_allclose(out["P_tt"], expect * (0.01 * k0) ** 2, rtol=1e-10, atol=1e-10 * expect.max())
    else:
        assert np.max(np.abs(out["P_tt"])) < 1e-13 * expect.max() * (0.01 * k0) ** 2


def test_b3_integer_samples():
    # the (3 + cos w)/4 used above: B_3 at the integers is (1/8, 3/4, 1/8)
    v = bs.bspline(np.array([-1.0, 0.0, 1.0]) + 0.0, 3)
    np.testing.assert_allclose(v, [1 / 8, 3 / 4, 1 / 8], atol=1e-15)


def test_b5_integer_samples():
    # the (115 + 76 cos w + cos 2w)/192 used above: the centred quartic B-spline at the
    # integers is (1/384, 19/96, 115/192, 19/96, 1/384) (textbook values)
    v = bs.bspline(np.arange(-2.0, 3.0), 5)
    np.testing.assert_allclose(v, [1 / 384, 19 / 96, 115 / 192, 19 / 96, 1 / 384], atol=1e-15)


# ---------------------------------------------------------------- Poisson shot noise

def _z_scores(out, key, sn_key, n_modes):
    # each mode's deconvolved estimate fluctuates by ~ its shot noise; the bin mean
    # over n_b/2 independent (k, -k) pairs by SN_b / sqrt(n_b / 2)
    sigma = out[sn_key] / np.sqrt(n_modes / 2.0)
    return out[key] / sigma


@pytest.mark.parametrize("order", [5, 4, 1])
def test_poisson_catalog_deconvolved_spectra_vanish(order):
    """Eq. psn / rawPp: for a Poisson catalogue the raw spectrum is pure shot noise,
    so the deconvolved, noise-subtracted spectra scatter around zero. (NGP, order 1,
    is exact for uniform random samples, Sec. 2.4.2.)"""
    L, ng = 200.0, 32
    cat = catalogs.poisson(20000, L, sigma_v=300.0, seed=21, dtype=np.float64)
    out = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, order=order, nbins=12, workers=1)
    for key, sn in (("P_dd", "SN_dd"), ("P_pp", "SN_pp"), ("P_tt", "SN_tt"), ("P_pp_b", "SN_pp_b")):
        z = _z_scores(out, key, sn, out["n_modes"])
        assert np.all(np.abs(z) < 5.0), (key, z)
        chi2 = float((z ** 2).mean())
        assert 0.2 < chi2 < 3.0, (key, chi2)
    # raw power, not subtracted, is biased high by exactly the shot noise
    raw = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, order=order, nbins=12, workers=1,
                       subtract_shot_noise=False)
    ratio = raw["P_pp"] / raw["SN_pp"]
    assert np.all(np.abs(ratio - 1.0) < 5.0 / np.sqrt(raw["n_modes"] / 2.0))


def test_poisson_with_added_bulk_flow():
    """Sec. 2.2 and Fig. vbnoise: a bulk flow of 341 km/s makes the theta shot noise
    direction dependent (Eq. thetanoise); with the exact per-mode noise the
    subtracted spectra still vanish, and Re P_dtheta is unchanged (Eq. rawPx)."""
    L, ng = 200.0, 32
    base = catalogs.poisson(20000, L, sigma_v=300.0, seed=23, dtype=np.float64)
    vb = 341.0 * np.array([1.0, 1.0, 0.0]) / np.sqrt(2.0)
    moved = dict(base, vel=base["vel"] + vb[None, :])
    o0 = est.estimate(base["pos"], base["vel"], L=L, ng=ng, nbins=10, workers=1)
    o1 = est.estimate(moved["pos"], moved["vel"], L=L, ng=ng, nbins=10, workers=1)
    np.testing.assert_allclose(o1["P_dt"], o0["P_dt"], rtol=1e-9, atol=1e-9 * np.abs(o0["P_dt"]).max())
    for key, sn in (("P_tt", "SN_tt"), ("P_pp", "SN_pp"), ("P_tt_b", "SN_tt_b")):
        z = _z_scores(o1, key, sn, o1["n_modes"])
        assert np.all(np.abs(z) < 5.0), (key, z)
    # the noise grows by v_b^2 (Sec. 3.1: sigma_v^2 = sigma_v'^2 + v_b^2)
    m = o1["moments"]
    np.testing.assert_allclose(np.trace(m["Q"]) / m["n"], np.trace(m["Qp"]) / m["n"] + m["vb"] @ m["vb"], rtol=1e-12)


def test_shell_average_of_tensor_noise_equals_isotropic_noise():
    """Sec. 2.2: in the isotropic (shell-averaged) spectrum the direction dependence of
    the theta shot noise averages out to sigma_v^2/3 -- the shells are cubic-symmetric."""
    L, ng = 100.0, 16
    cat = catalogs.poisson(3000, L, seed=29, dtype=np.float64, bulk=(400.0, -100.0, 50.0))
    ot = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, nbins=6, workers=1)
    oi = est.estimate(cat["pos"], cat["vel"], L=L, ng=ng, nbins=6, workers=1, theta_sn="isotropic")
    np.testing.assert_allclose(ot["SN_tt"], oi["SN_tt"], rtol=1e-12)
    np.testing.assert_allclose(ot["P_tt"], oi["P_tt"], rtol=1e-9, atol=1e-12 * np.abs(ot["SN_tt"]).max())


# ---------------------------------------------------------------- bulk-flow identities

def test_bulk_flow_relations_per_mode():
    """Eqs. bfpp and bfpdpx hold per mode for the estimator (linearity), to rounding:
    P_p = P_p' + v_b [P_dp'b + c.c.] + v_b^2 P,
    P_theta = P_theta' + i k mu_b v_b/(Haf) [P_dtheta' - c.c.] + k^2 mu_b^2 (v_b/Haf)^2 P,
    P_dtheta = P_dtheta' - i k mu_b v_b/(Haf) P."""
    L, ng, ts = 150.0, 16, 0.02
    cat = catalogs.zeldovich(16, L, seed=31, dtype=np.float64)
    cat["vel"] = cat["vel"] + np.array([51.5, -20.0, 10.0])[None, :]
    mom = est.moments(cat["vel"])
    F = est.fft_grids(est.assign(cat["pos"], cat["vel"], None, L=L, ng=ng), workers=1)
    out = est.spectra_from_fourier(F, mom, L=L, ng=ng, nbins=8, theta_scale=ts, per_mode=True)
    md = out["modes"]
    vb = mom["vb"]
    vbn = np.linalg.norm(vb)
    kdotvb = sum(md["kvec"][:, a] * vb[a] for a in range(3))
    Pdd = md["P_dd"]
    scale_p = np.abs(md["P_pp"]).max()
    lhs = md["P_pp"]
    rhs = md["P_pp_b"] + vbn * 2.0 * np.real(md["D_pb_b"]) + vbn ** 2 * Pdd
    mask = md["bin"] >= 0
    assert np.max(np.abs(lhs - rhs)[mask]) < 1e-9 * scale_p
    lhs = md["P_tt"]
    rhs = md["P_tt_b"] + 1j * kdotvb * ts * (md["X_b"] - np.conj(md["X_b"])) + (kdotvb * ts) ** 2 * Pdd
    assert np.max(np.abs(lhs - rhs)[mask]) < 1e-9 * np.abs(md["P_tt"]).max()
    # Re P_dtheta is immune to the bulk flow (Eq. bfpdpx, second line)
    np.testing.assert_allclose(np.real(md["X"])[mask], np.real(md["X_b"])[mask], atol=1e-10 * np.abs(md["X"]).max())
    np.testing.assert_allclose(md["P_dt"][mask], md["P_dt_b"][mask], atol=1e-10 * np.abs(md["X"]).max())
    d_im = np.imag(md["X"] - md["X_b"])
    # Im part: X - X_b = -i ts (k.v_b) |F_delta|^2 V/M^2/W^2 = -i ts (k.v_b) (P_dd + SN_dd/W^2)
    unsub = est.spectra_from_fourier(F, mom, L=L, ng=ng, nbins=8, theta_scale=ts, per_mode=True,
                                     subtract_shot_noise=False)["modes"]["P_dd"]
    np.testing.assert_allclose(d_im[mask], (-ts * kdotvb * unsub)[mask], atol=1e-10 * np.abs(d_im).max())


# ---------------------------------------------------------------- linear theory sanity

@pytest.mark.slow
def test_zeldovich_linear_theory_ratios():
    """Loose physics check (Sec. 4, linear theory): with theta_scale = 1/(H a f) the
    momentum divergence follows the density at low k, so P_dtheta/P_delta and
    P_thetatheta/P_delta are close to 1 in the first bins, and P_dtheta > 0.
    A displaced lattice is not a Poisson sample, so no shot noise is subtracted."""
    L, n = 1000.0, 64
    cat = catalogs.zeldovich(n, L, seed=1002, dtype=np.float32)
    out = est.estimate(cat["pos"], cat["vel"], L=L, ng=64, nbins=16, theta_scale=1.0 / 50.0,
                       subtract_shot_noise=False)
    r1 = out["P_dt"][:4] / out["P_dd"][:4]
    r2 = out["P_tt"][:4] / out["P_dd"][:4]
    assert np.all(out["P_dt"][:8] > 0)
    assert np.all(np.abs(r1 - 1) < 0.02), r1
    assert np.all(np.abs(r2 - 1) < 0.03), r2


def test_fp32_grids_meet_the_shot_noise_floor_on_a_one_cell_catalogue():
    """The parity tolerance for FP32 grids (1e-4 of max(|P_b|, SN_b / sqrt(n_b))) is met
    by FP32 arithmetic itself on the most degenerate catalogue the GPU tests use: 2e4
    particles in two neighbouring cells, whose momentum node sums cancel. The oracle's
    grids rounded to FP32 and transformed by an FP32 FFT stay within 1e-5 of that
    floor (measured 1.6e-6), so the GPU test holds that case to the normal floor."""
    import scipy.fft
    rng = np.random.default_rng(51)
    L, ng, n = 100.0, 32, 20000
    pos = (10.0 + rng.uniform(0, L / ng, size=(n, 3))).astype(np.float32)
    vel = rng.normal(0, 100, size=(n, 3)).astype(np.float32)
    ref = est.estimate(pos, vel, L=L, ng=ng, nbins=8)
    mom = est.moments(vel)
    grids = est.assign(pos, vel, None, L=L, ng=ng)
    F32 = np.stack([scipy.fft.rfftn(g.astype(np.float32)) for g in grids])
    assert F32.dtype == np.complex64
    emu = est.spectra_from_fourier(F32.astype(np.complex128), mom, L=L, ng=ng, nbins=8)
    nm = ref["n_modes"]
    for key in ("P_dd", "P_pp", "P_tt", "P_dt", "P_pp_b", "P_tt_b", "P_dt_b"):
        sfx = "_b" if key.endswith("_b") else ""
        if key.startswith("P_dt"):
            floor = np.sqrt(ref["SN_dd"] * ref["SN_tt" + sfx]) / np.sqrt(nm)
        else:
            floor = ref["SN_" + key[2:]] / np.sqrt(nm)
        err = np.abs(emu[key] - ref[key]) / np.maximum(np.abs(ref[key]), floor)
        assert np.max(err) < 1e-5, (key, np.max(err))
