"""FP64 CPU oracle of the momentum power-spectrum estimator.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The steps follow the paper in its own order:

1. moments of the catalogue: total weight, bulk flow v_b (Sec. 2.2, Eq. thetanoise),
   sigma_v^2 (Eq. rawppnoise), the velocity tensor behind <v^2 mu^2> (Eq. rawPtheta);
2. assignment of the density and the three momentum components to the FFT grid
   with the BL scaling function W (Sec. 2.1, Eq. rawFFTed; Sec. 2.4.1);
3. FFT of each grid (Sec. 2.4.1);
4. raw per-mode spectra |p|^2, |k.p|^2 theta_scale^2, Re<delta theta*> and |delta|^2
   (Eqs. 3, rawPp, rawPtheta, rawPx);
5. shot noise times sum_J W^2(k + 2 k_N J) subtracted (Eqs. psn, rawPp, rawPtheta,
   rawPx), then division by W^2(k) (the window deconvolution of Sec. 2.1);
6. shell average in |k|;
7. the same with the bulk flow removed, v' = v - v_b, p' = p - (1+delta) v_b
   (Sec. 3.1), which on the grid is F_p' = F_p - v_b F_delta.

Conventions (readings of the paper where it is silent or ambiguous):
* Positions: grid coordinate u = x * (ng / L). For an FP32 catalogue u is formed in
  FP32 (u = fl32(x * fl32(ng/L))), the precision in which the GPU takes the
  cell decision; for an FP64 catalogue in FP64. Everything after that is FP64.
* BL kernel of B-spline order m (default 4): the grid field deposited with phi is
  the field deposited with B_m times, in Fourier space, prod_a Sigma_m(w_a)^{-1/2}
  (exact on a periodic grid: phi = sum_n c_n B_m(. - n) and the c_n are the Fourier
  coefficients of Sigma_m^{-1/2}).
* Normalisation: p_hat(k) = (1/M) sum_j m_j v_j e^{i k.r_j} with M = sum_j m_j
  (the paper's 1/N at unit mass); spectra are returned times the box volume V, so
  P_pp is in (Mpc/h)^3 (km/s)^2. Shot noise V sum_j m_j^2 v_j^2 / M^2 (= V sigma_v^2/N).
* Transform sign: numpy's FFT uses e^{-ikr}, the paper e^{+ikr}; for real fields
  the paper's transform is the complex conjugate, so the cross spectrum's real part
  Re<delta theta*> = theta_scale * Im(conj(F_delta) (k.F_p)) with theta = i k.p * theta_scale
  (theta_scale = 1/(H a f) in the paper).
* Bins: linear in u = |k|/k_f between umin and umax (defaults 1 and ng/2), index
  floor(((u - umin) * nbins) / (umax - umin)) in FP64, the last bin closed; the
  k = 0 mode is always excluded. Half-spectrum modes carry weight 2 except the
  planes n_2 = 0 and n_2 = ng/2 (weight 1), which reproduces the full-sphere count.
"""
from __future__ import annotations

import numpy as np

from . import bspline as _bs
from . import _clib

FIELDS = ("delta", "px", "py", "pz")


def grid_coordinates(pos: np.ndarray, L: float, ng: int) -> np.ndarray:
    """Particle positions (n,3) -> grid units, in the catalogue's own precision."""
    if pos.dtype == np.float32:
        s = np.float32(ng / L)
        u = pos * s  # FP32 multiply, rounded once
        return u.astype(np.float64)
    return np.asarray(pos, dtype=np.float64) * (ng / L)


def moments(vel: np.ndarray, mass: np.ndarray | None = None) -> dict:
    """Catalogue moments in FP64 (Secs. 2.1-2.2 and 3.1).

    M = sum m, S2 = sum m^2, v_b = sum m v / M (Eq. thetanoise's bulk flow at unit
    mass), Q = sum m^2 v v^T, R = sum m^2 v, and the same for v' = v - v_b.
    sigma_v^2 = tr(Q) / S2 at unit mass (Eq. rawppnoise).
    """
    v = np.asarray(vel, dtype=np.float64)
    m = np.ones(len(v)) if mass is None else np.asarray(mass, dtype=np.float64)
    M = m.sum()
    S2 = (m * m).sum()
    vb = (m[:, None] * v).sum(axis=0) / M
    m2 = m * m
    Q = np.einsum("j,ja,jb->ab", m2, v, v)
    R = (m2[:, None] * v).sum(axis=0)
    vp = v - vb
    Qp = np.einsum("j,ja,jb->ab", m2, vp, vp)
    return {"M": M, "S2": S2, "vb": vb, "Q": Q, "R": R, "Qp": Qp, "n": len(v)}


def assign(pos, vel, mass, *, L: float, ng: int, order: int = 4) -> np.ndarray:
    """B-spline deposit of (m, m vx, m vy, m vz) onto four ng^3 FP64 grids."""
    u = grid_coordinates(np.asarray(pos), L, ng)
    v = np.asarray(vel, dtype=np.float64)
    m = np.ones(len(v)) if mass is None else np.asarray(mass, dtype=np.float64)
    q = np.concatenate([m[:, None], m[:, None] * v], axis=1)
    return _clib.deposit_bspline(u, q, order, ng)


def fft_grids(grids: np.ndarray, workers: int = -1) -> np.ndarray:
    """R2C FFT (e^{-ikr}, unnormalised) of each grid over its three axes, one grid at a
    time into one output array (so that a 1024^3 run holds one transform beside it)."""
    import scipy.fft
    out = None
    for f, g in enumerate(grids):
        t = scipy.fft.rfftn(g, workers=workers)
        if out is None:
            out = np.empty((len(grids),) + t.shape, dtype=t.dtype)
        out[f] = t
        del t
    return out


def signed_freq(ng: int) -> np.ndarray:
    """Integer frequency of each full-axis FFT index: i for i < ng/2, i - ng otherwise."""
    i = np.arange(ng)
    return np.where(i < ng // 2, i, i - ng)


def bin_index(n2: np.ndarray, nbins: int, umin: float, umax: float) -> np.ndarray:
    """Shell index of modes with |n|^2 = n2 (in units of k_f); -1 if outside."""
    u = np.sqrt(n2.astype(np.float64))
    t = np.floor(((u - umin) * nbins) / (umax - umin))
    b = np.minimum(t, nbins - 1).astype(np.int64)
    ok = (n2 > 0) & (u >= umin) & (u <= umax)
    return np.where(ok, b, -1)


class _Accum:
    def __init__(self, nbins):
        self.nbins = nbins
        self.s = {}

    def add(self, key, b, w, vals):
        acc = self.s.setdefault(key, np.zeros(self.nbins))
        acc += np.bincount(b, weights=w * vals, minlength=self.nbins + 1)[1:]


def spectra_from_fourier(F: np.ndarray, mom: dict, *, L: float, ng: int, order: int = 4,
                         nbins: int, kmin_kf: float = 1.0, kmax_kf: float | None = None,
                         theta_scale: float = 1.0, subtract_shot_noise: bool = True,
                         theta_sn: str = "tensor", bulk: bool = True,
                         per_mode: bool = False, bl_assigned: bool = False, slabs=None) -> dict:
    """Steps 4-7 on the Fourier transforms F[4] of the B-spline-deposited grids.

    bl_assigned: F holds grids already assigned with the BL function itself (the direct
    real-space deposit), so the Fourier-space factor prod Sigma^{-1/2} is not applied.
    Returns shell averages. With per_mode=True also returns the per-mode arrays
    (only sensible for small grids). slabs: the first-axis indices to visit (default
    all); a subset gives partial sums, used only to time a bounded sample.
    """
    umin = float(kmin_kf)
    umax = float(ng // 2 if kmax_kf is None else kmax_kf)
    V = float(L) ** 3
    kf = 2.0 * np.pi / L
    M2 = mom["M"] ** 2
    nfull = signed_freq(ng).astype(np.float64)
    nhalf = np.arange(ng // 2 + 1, dtype=np.float64)
    w_full = 2.0 * np.pi * nfull / ng
    w_half = 2.0 * np.pi * nhalf / ng
    # per-axis factors of the BL window
    C_full = _bs.alias_sum(w_full, order) ** -0.5
    C_half = _bs.alias_sum(w_half, order) ** -0.5
    W2_full = _bs.phi_hat(w_full, order) ** 2
    W2_half = _bs.phi_hat(w_half, order) ** 2
    A_full = _bs.phi_alias_sum(w_full, order)
    A_half = _bs.phi_alias_sum(w_half, order)
    wt_half = np.where((np.arange(ng // 2 + 1) == 0) | (np.arange(ng // 2 + 1) == ng // 2), 1.0, 2.0)

    acc = _Accum(nbins)
    modes = {} if per_mode else None
    vb = mom["vb"]
    variants = [("", mom["Q"])] + ([("_b", mom["Qp"])] if bulk else [])
    for i0 in (range(ng) if slabs is None else slabs):
        n1 = nfull[:, None]
        n2 = nhalf[None, :]
        n0 = nfull[i0]
        nsq = (n0 * n0 + n1 * n1 + n2 * n2).astype(np.int64)
        b = bin_index(nsq, nbins, umin, umax) + 1  # 0 = excluded
        wmode = np.broadcast_to(wt_half[None, :], nsq.shape)
        Cfac = 1.0 if bl_assigned else C_full[i0] * C_full[:, None] * C_half[None, :]
        W2 = W2_full[i0] * W2_full[:, None] * W2_half[None, :]
        A = A_full[i0] * A_full[:, None] * A_half[None, :]
        kvec = [kf * n0 * np.ones_like(n1 * n2), kf * n1 * np.ones_like(n2), kf * n2 * np.ones_like(n1)]
        # the BL-assigned fields (Eq. rawFFTed): B-spline field times the periodic factor
        Fd = F[0, i0] * Cfac
        Fp0 = [F[1 + a, i0] * Cfac for a in range(3)]
        bb = b.ravel()
        ww = wmode.ravel()
        raw_dd = V * np.abs(Fd) ** 2 / M2
        sn_dd = V * mom["S2"] / M2 * A
        P_dd = (raw_dd - (sn_dd if subtract_shot_noise else 0.0)) / W2
        acc.add("n_modes", bb, ww, np.ones_like(ww))
        acc.add("k_sum", bb, ww, np.sqrt(nsq.astype(np.float64)).ravel() * kf)
        acc.add("P_dd", bb, ww, P_dd.ravel())
        acc.add("SN_dd", bb, ww, (sn_dd / W2).ravel())
        if per_mode:
            modes.setdefault("P_dd", []).append(P_dd)
        for suffix, Q in variants:
            Fp = Fp0 if suffix == "" else [Fp0[a] - vb[a] * Fd for a in range(3)]
            raw_pp = V * sum(np.abs(Fp[a]) ** 2 for a in range(3)) / M2
            kp = sum(kvec[a] * Fp[a] for a in range(3))
            raw_tt = V * theta_scale ** 2 * np.abs(kp) ** 2 / M2
            raw_dt = V * theta_scale * np.imag(np.conj(Fd) * kp) / M2
            sn_pp = V * np.trace(Q) / M2 * A
            if theta_sn == "tensor":
                kQk = sum(kvec[a] * kvec[c] * Q[a, c] for a in range(3) for c in range(3))
            elif theta_sn == "isotropic":
                kQk = (kvec[0] ** 2 + kvec[1] ** 2 + kvec[2] ** 2) * np.trace(Q) / 3.0
            else:
                raise ValueError(theta_sn)
            sn_tt = V * theta_scale ** 2 * kQk / M2 * A
            sub = 1.0 if subtract_shot_noise else 0.0
            P_pp = (raw_pp - sub * sn_pp) / W2
            P_tt = (raw_tt - sub * sn_tt) / W2
            P_dt = raw_dt / W2  # the cross shot noise is purely imaginary (Eq. rawPx)
            for name, arr in (("P_pp", P_pp), ("P_tt", P_tt), ("P_dt", P_dt),
                              ("SN_pp", sn_pp / W2), ("SN_tt", sn_tt / W2)):
                acc.add(name + suffix, bb, ww, arr.ravel())
                if per_mode:
                    modes.setdefault(name + suffix, []).append(arr)
            if per_mode:
                # complex <delta theta*> (paper's e^{+ikr} convention), deconvolved,
                # and <delta p_b*> with p_b = p . v_b / |v_b| (Sec. 3.1)
                X = -1j * V * theta_scale * np.conj(Fd) * kp / M2 / W2
                vbn = np.linalg.norm(vb)
                e_b = vb / vbn if vbn > 0 else np.zeros(3)
                D_pb = V * np.conj(Fd) * sum(e_b[a] * Fp[a] for a in range(3)) / M2 / W2
                modes.setdefault("X" + suffix, []).append(X)
                modes.setdefault("D_pb" + suffix, []).append(D_pb)
                if suffix == "":
                    modes.setdefault("kvec", []).append(np.stack(kvec))
                    modes.setdefault("bin", []).append(b - 1)
                    modes.setdefault("weight", []).append(np.array(wmode))
    out = {}
    n = acc.s["n_modes"]
    with np.errstate(invalid="ignore", divide="ignore"):
        for key, val in acc.s.items():
            if key == "n_modes":
                out[key] = val
            elif key == "k_sum":
                out["k_mean"] = val / n
            else:
                out[key] = val / n
    out["SN_dt"] = np.zeros(nbins)
    if bulk:
        out["SN_dt_b"] = np.zeros(nbins)
    if per_mode:
        out["modes"] = {k: np.stack(v) for k, v in modes.items()}
    return out


def assign_bl_direct(pos, vel, mass, *, L: float, ng: int, radius: float) -> np.ndarray:
    """Direct real-space assignment with the BL function truncated to |x| < radius cells
    (cubic order), onto four ng^3 FP64 grids."""
    from . import direct
    u = grid_coordinates(np.asarray(pos), L, ng)
    v = np.asarray(vel, dtype=np.float64)
    m = np.ones(len(v)) if mass is None else np.asarray(mass, dtype=np.float64)
    q = np.concatenate([m[:, None], m[:, None] * v], axis=1)
    return direct.deposit_bl_direct(u, q, ng, 4, radius=radius)


def estimate(pos, vel, mass=None, *, L: float, ng: int, order: int = 4, nbins: int,
             kmin_kf: float = 1.0, kmax_kf: float | None = None, theta_scale: float = 1.0,
             subtract_shot_noise: bool = True, theta_sn: str = "tensor", bulk: bool = True,
             workers: int = -1, bl_radius: float = 0) -> dict:
    """The whole estimator on one catalogue: steps 1-7 of the module docstring.

    bl_radius > 0: step 2 with the BL function truncated to |x| < bl_radius cells and
    deposited directly in real space (cubic order; small catalogues only)."""
    mom = moments(vel, mass)
    if bl_radius:
        if order != 4:
            raise ValueError("the direct BL deposit is of cubic order")
        grids = assign_bl_direct(pos, vel, mass, L=L, ng=ng, radius=bl_radius)
    else:
        grids = assign(pos, vel, mass, L=L, ng=ng, order=order)
    F = fft_grids(grids, workers=workers)
    del grids
    out = spectra_from_fourier(F, mom, L=L, ng=ng, order=order, nbins=nbins, kmin_kf=kmin_kf,
                               kmax_kf=kmax_kf, theta_scale=theta_scale,
                               subtract_shot_noise=subtract_shot_noise, theta_sn=theta_sn, bulk=bulk,
                               bl_assigned=bool(bl_radius))
    out["moments"] = mom
    return out
