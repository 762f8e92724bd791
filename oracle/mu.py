"""FP64 oracle of the spectra binned in |k| and mu = k.e / (k |e|).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

With a bulk flow v_b the momentum-divergence shot noise depends on mu_b, the cosine
between k and v_b (Sec. 2.2, Eq. thetanoise), and the cross spectrum of density and
momentum divergence gains an imaginary part -i k mu_b (v_b/Haf) P (Sec. 3.2, Eq.
bfpdpx; Fig. bfPpdiff). Shell averages cancel both (the terms are odd in mu_b), so
they are measured in bins of (|k|, mu).

The steps are those of estimator.py (moments, B-spline deposit and BL factor, FFT,
window deconvolution, shot-noise subtraction), evaluated on the FULL complex FFT of
each grid, so that every mode n appears once with weight 1 and its own mu; no
half-spectrum bookkeeping. Per mode, in the paper's e^{+ikr} convention:

* P_dd  = V|F_d|^2/M^2/W^2 - V S2/M^2 A/W^2
* P_pp  = V|F_p|^2/M^2/W^2 - V tr Q/M^2 A/W^2, and with F_p' = F_p - v_b F_d, Q'
* P_tt  = V ts^2 |k.F_p|^2/M^2/W^2 - V ts^2 k.Q.k/M^2 A/W^2 (Eq. rawPtheta), and '
* X     = -i V ts conj(F_d)(k.F_p)/M^2/W^2 - (-i V ts (k.R)/M^2 A/W^2), the complex
          <delta theta*> with its (imaginary) shot noise removed (Eq. rawPx:
          <v mu> = v_b mu_b at unit mass; R = sum m^2 v), and X' with R' = R - S2 v_b
* D_pb' = V conj(F_d)(e_b.F_p')/M^2/W^2 - V (e_b.R')/M^2 A/W^2, the cross spectrum of
          density and the bulk-direction momentum p'_b of Eq. bfpp (e_b = v_b/|v_b|)

Modes with a component at the Nyquist index (-ng/2, which is also +ng/2) are their own
mirror image, so the sign of their direction cosine, and of their imaginary cross
spectrum, is not defined: they are left out (inside |n| <= ng/2 they are the three axis
points of the last shell).

mu bins: linear in [-1, 1]; the bin of a mode is decided in FP32, in the order
d = (n0 e0 + n1 e1) + n2 e2, mu = d / sqrt(|n|^2), m = floor((mu + 1) * (nmu/2)),
clipped to [0, nmu - 1], with e normalised in FP64 and rounded to FP32 (the precision
and order the GPU kernel uses, so that both sides put every mode in the same bin).
"""
from __future__ import annotations

import numpy as np

from . import bspline as _bs
from . import estimator as _est


def unit_direction(e) -> np.ndarray:
    e = np.asarray(e, dtype=np.float64)
    nrm = np.sqrt(float(e @ e))
    return e / nrm if nrm > 0 else np.zeros(3)


def mu_bin32(n0, n1, n2, e, nmu: int) -> np.ndarray:
    """FP32 mu bin of integer wave vectors (arrays) for the unit direction e (FP64)."""
    f = np.float32
    e32 = np.asarray(e, dtype=np.float64).astype(f)
    a = (np.asarray(n0).astype(f) * e32[0]).astype(f)
    b = (np.asarray(n1).astype(f) * e32[1]).astype(f)
    c = (np.asarray(n2).astype(f) * e32[2]).astype(f)
    d = ((a + b).astype(f) + c).astype(f)
    nn = (np.asarray(n0) ** 2 + np.asarray(n1) ** 2 + np.asarray(n2) ** 2).astype(f)
    r = np.sqrt(nn).astype(f)
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = (d / r).astype(f)
    t = ((mu + f(1)).astype(f) * f(nmu / 2)).astype(f)
    # the k = 0 mode has no direction (0/0); callers leave it out, so give it bin 0
    # rather than cast a NaN to an integer
    t = np.where(nn > 0, t, f(0))
    m = np.floor(t).astype(np.int64)
    return np.clip(m, 0, nmu - 1)


def spectra_mu(pos, vel, mass=None, *, L: float, ng: int, nbins: int, nmu: int, direction=None,
               order: int = 4, kmin_kf: float = 1.0, kmax_kf: float | None = None, theta_scale: float = 1.0,
               per_mode: bool = False, workers: int = -1) -> dict:
    """(nbins, nmu) arrays of the spectra listed in the module docstring, bins in |k|
    (the shells of estimator.bin_index) and mu (relative to `direction`, default the
    bulk flow). Small grids only (four full complex FFTs in memory)."""
    import scipy.fft
    mom = _est.moments(vel, mass)
    grids = _est.assign(pos, vel, mass, L=L, ng=ng, order=order)
    F = np.stack([scipy.fft.fftn(g, workers=workers) for g in grids])
    del grids
    V = float(L) ** 3
    kf = 2.0 * np.pi / L
    M2 = mom["M"] ** 2
    S2 = mom["S2"]
    ts = theta_scale
    umin = float(kmin_kf)
    umax = float(ng // 2 if kmax_kf is None else kmax_kf)
    vb = mom["vb"]
    vbn = float(np.sqrt(vb @ vb))
    eb = vb / vbn if vbn > 0 else np.zeros(3)
    e = unit_direction(vb if direction is None else direction)
    R = mom["R"]
    Rp = R - S2 * vb
    Q, Qp = mom["Q"], mom["Qp"]

    nf = _est.signed_freq(ng)
    n0 = nf[:, None, None] * np.ones((1, ng, ng), dtype=np.int64)
    n1 = nf[None, :, None] * np.ones((ng, 1, ng), dtype=np.int64)
    n2 = nf[None, None, :] * np.ones((ng, ng, 1), dtype=np.int64)
    nsq = n0 * n0 + n1 * n1 + n2 * n2
    b = _est.bin_index(nsq, nbins, umin, umax)
    m = mu_bin32(n0, n1, n2, e, nmu)
    w = 2.0 * np.pi * nf / ng
    C1 = _bs.alias_sum(w, order) ** -0.5
    W1 = _bs.phi_hat(w, order) ** 2
    A1 = _bs.phi_alias_sum(w, order)
    Cfac = C1[:, None, None] * C1[None, :, None] * C1[None, None, :]
    W2 = W1[:, None, None] * W1[None, :, None] * W1[None, None, :]
    A = A1[:, None, None] * A1[None, :, None] * A1[None, None, :]
    h = A / W2

    Fd = F[0] * Cfac
    Fp = [F[1 + a] * Cfac for a in range(3)]
    Fq = [Fp[a] - vb[a] * Fd for a in range(3)]
    nvec = (n0, n1, n2)
    kP = sum(kf * nvec[a] * Fp[a] for a in range(3))
    kQ = sum(kf * nvec[a] * Fq[a] for a in range(3))
    c = V / M2

    def kTk(T):
        return sum(kf * kf * nvec[a] * nvec[c2] * T[a, c2] for a in range(3) for c2 in range(3))

    def kdot(v):
        return sum(kf * nvec[a] * v[a] for a in range(3))

    vals = {
        "P_dd": c * np.abs(Fd) ** 2 / W2 - c * S2 * h,
        "P_pp": c * sum(np.abs(Fp[a]) ** 2 for a in range(3)) / W2 - c * np.trace(Q) * h,
        "P_pp_b": c * sum(np.abs(Fq[a]) ** 2 for a in range(3)) / W2 - c * np.trace(Qp) * h,
        "P_tt": c * ts * ts * np.abs(kP) ** 2 / W2 - c * ts * ts * kTk(Q) * h,
        "P_tt_b": c * ts * ts * np.abs(kQ) ** 2 / W2 - c * ts * ts * kTk(Qp) * h,
    }
    X = -1j * c * ts * np.conj(Fd) * kP / W2 - (-1j * c * ts * kdot(R) * h)
    Xb = -1j * c * ts * np.conj(Fd) * kQ / W2 - (-1j * c * ts * kdot(Rp) * h)
    Dpb = c * np.conj(Fd) * sum(eb[a] * Fq[a] for a in range(3)) / W2 - c * float(eb @ Rp) * h
    vals.update({"Re_dt": X.real, "Im_dt": X.imag, "Re_dt_b": Xb.real, "Im_dt_b": Xb.imag,
                 "Re_dpb_b": Dpb.real,
                 "SN_dd": c * S2 * h, "SN_tt": c * ts * ts * kTk(Q) * h, "Im_SN_dt": -c * ts * kdot(R) * h})
    with np.errstate(invalid="ignore", divide="ignore"):
        mu_exact = np.where(nsq > 0, (n0 * e[0] + n1 * e[1] + n2 * e[2]) / np.sqrt(nsq), 0.0)
    h2 = -(ng // 2)
    ok = (b >= 0) & (n0 != h2) & (n1 != h2) & (n2 != h2)
    cell = (b * nmu + m)[ok]
    ncell = nbins * nmu
    cnt = np.bincount(cell, minlength=ncell).astype(np.float64)
    out = {"n_modes": cnt.reshape(nbins, nmu)}
    with np.errstate(invalid="ignore", divide="ignore"):
        out["k_mean"] = (np.bincount(cell, weights=kf * np.sqrt(nsq[ok]), minlength=ncell) / cnt).reshape(nbins, nmu)
        out["mu_mean"] = (np.bincount(cell, weights=mu_exact[ok], minlength=ncell) / cnt).reshape(nbins, nmu)
        for key, v in vals.items():
            out[key] = (np.bincount(cell, weights=v[ok], minlength=ncell) / cnt).reshape(nbins, nmu)
    out["moments"] = mom
    out["direction"] = e
    if per_mode:
        out["modes"] = dict(vals, shell=b, mu_bin=m, kvec=np.stack([kf * n0, kf * n1, kf * n2]))
    return out
