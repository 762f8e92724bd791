"""Pins of the (|k|, mu)-binned oracle (oracle/mu.py) against independent routes and the
paper's bulk-flow relations (Sec. 2.2 Eq. thetanoise, Sec. 3.1 Eq. bfpp, Sec. 3.2 Eq.
bfpdpx)."""
import numpy as np
import pytest

from oracle import estimator as est
from oracle import mu as omu
from paper_2005_06170_gb300 import catalogs


def _cat(masses=False):
    """Zel'dovich 16^3 in L = 100 with an added bulk flow of 51.5 km/s (the paper's
    artificial bulk flow, Sec. 3.3) along (2, -1, 2)/3; optional random masses."""
    c = catalogs.zeldovich(16, 100.0, seed=21, dtype=np.float64)
    c["vel"] = c["vel"] + 51.5 * np.array([2.0, -1.0, 2.0]) / 3.0
    if masses:
        c["mass"] = np.random.default_rng(5).uniform(0.5, 1.5, len(c["vel"]))
    return c


# shells up to just below the Nyquist frequency: the mu-binned spectra leave out the
# Nyquist axis modes, whose direction has no sign
KW = dict(L=100.0, ng=16, nbins=6, theta_scale=0.02, kmax_kf=7.5)


@pytest.mark.parametrize("masses", [False, True])
def test_mu_bins_collapse_to_the_isotropic_spectra(masses):
    """Summing the mu bins of a shell (mode-weighted) gives the isotropic oracle, which
    works on the half spectrum with weights instead of the full FFT."""
    c = _cat(masses)
    iso = est.estimate(c["pos"], c["vel"], c.get("mass"), **KW)
    mu = omu.spectra_mu(c["pos"], c["vel"], c.get("mass"), nmu=5, **KW)
    n = mu["n_modes"]
    np.testing.assert_array_equal(n.sum(axis=1), iso["n_modes"])
    for key, ikey in (("P_dd", "P_dd"), ("P_pp", "P_pp"), ("P_tt", "P_tt"), ("Re_dt", "P_dt"),
                      ("P_pp_b", "P_pp_b"), ("P_tt_b", "P_tt_b"), ("Re_dt_b", "P_dt_b")):
        s = np.nansum(mu[key] * n, axis=1) / n.sum(axis=1)
        np.testing.assert_allclose(s, iso[ikey], rtol=1e-10, atol=1e-12 * np.abs(iso[ikey]).max(), err_msg=key)
    # the imaginary cross spectrum is odd in mu: its shell average vanishes
    s = np.nansum(mu["Im_dt"] * n, axis=1) / n.sum(axis=1)
    assert np.all(np.abs(s) <= 1e-10 * np.nanmax(np.abs(mu["Im_dt"])))


@pytest.mark.parametrize("masses", [False, True])
def test_bulk_flow_relations_per_bin_and_per_mode(masses):
    """Eq. bfpp per (k, mu) bin: P_p - P_p' = 2 v_b Re P_dp'b + v_b^2 P; Eq. bfpdpx per
    mode: Im(P_dtheta - P_dtheta') = -(k.v_b) ts P and P_theta - P_theta' =
    -2 (k.v_b) ts Im P_dtheta' + (k.v_b)^2 ts^2 P, all with shot noise removed."""
    c = _cat(masses)
    mu = omu.spectra_mu(c["pos"], c["vel"], c.get("mass"), nmu=5, per_mode=True, **KW)
    vb = mu["moments"]["vb"]
    vbn = np.sqrt(vb @ vb)
    lhs = mu["P_pp"] - mu["P_pp_b"]
    rhs = 2 * vbn * mu["Re_dpb_b"] + vbn ** 2 * mu["P_dd"]
    ok = mu["n_modes"] > 0
    np.testing.assert_allclose(lhs[ok], rhs[ok], rtol=1e-9, atol=1e-9 * np.abs(lhs[ok]).max())
    md = mu["modes"]
    kv = np.einsum("a,a...->...", vb, md["kvec"])
    ts = KW["theta_scale"]
    im_lhs = md["Im_dt"] - md["Im_dt_b"]
    np.testing.assert_allclose(im_lhs, -kv * ts * md["P_dd"], rtol=1e-9, atol=1e-9 * np.abs(im_lhs).max())
    tt_lhs = md["P_tt"] - md["P_tt_b"]
    tt_rhs = -2 * kv * ts * md["Im_dt_b"] + kv ** 2 * ts ** 2 * md["P_dd"]
    np.testing.assert_allclose(tt_lhs, tt_rhs, rtol=1e-9, atol=1e-9 * np.abs(tt_lhs).max())


def test_imaginary_cross_spectrum_follows_mu():
    """Eq. bfpdpx in bins: Im(P_dtheta - P_dtheta') is close to -k mu_b v_b ts P (the
    bin means of k mu and of P stand in for the mean of their product) and changes sign
    with mu_b; the shot noise of theta grows with mu_b^2 (Eq. thetanoise)."""
    c = _cat()
    mu = omu.spectra_mu(c["pos"], c["vel"], nmu=6, **KW)
    vb = mu["moments"]["vb"]
    vbn = np.sqrt(vb @ vb)
    ok = mu["n_modes"] > 0
    d = (mu["Im_dt"] - mu["Im_dt_b"])[ok]
    approx = (-mu["k_mean"] * mu["mu_mean"] * vbn * KW["theta_scale"] * mu["P_dd"])[ok]
    assert np.all(np.sign(d[np.abs(approx) > 0.1 * np.abs(approx).max()]) ==
                  np.sign(approx[np.abs(approx) > 0.1 * np.abs(approx).max()]))
    sn = mu["SN_tt"]
    assert np.all(sn[:, 0] > sn[:, 2]) and np.all(sn[:, 5] > sn[:, 3])  # |mu| ~ 1 above mu ~ 0


def test_mu_bin_decision_matches_the_exact_cosine():
    """The FP32 decision equals floor((mu + 1) nmu / 2) of the FP64 cosine except within
    FP32 rounding of a bin edge."""
    rng = np.random.default_rng(3)
    n = rng.integers(-64, 65, size=(3, 20000))
    n = n[:, (n ** 2).sum(axis=0) > 0]
    e = omu.unit_direction([0.3, -0.5, 0.81])
    for nmu in (2, 5, 8):
        m32 = omu.mu_bin32(n[0], n[1], n[2], e, nmu)
        mu = (e @ n) / np.sqrt((n ** 2).sum(axis=0))
        t = (mu + 1) * nmu / 2
        m64 = np.clip(np.floor(t), 0, nmu - 1)
        bad = m32 != m64
        assert np.all(np.abs(t[bad] - np.round(t[bad])) < 1e-5)
