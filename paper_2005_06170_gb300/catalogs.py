"""Seeded synthetic particle catalogues (inputs only; none of the estimator's arithmetic).

These stand in for the paper's Gadget-2 snapshots (Sec. 2.4.1: 1024^3 particles in
a 1000 Mpc/h periodic box), which are not available here. Both the GPU library's
tests/benchmark and the CPU oracle's tests draw their inputs from this module.

All generators return a dict with ``pos`` (n,3), ``vel`` (n,3), optional ``mass``
(n,), and ``L``; arrays are C-contiguous numpy arrays in the requested dtype.
Positions are wrapped into [0, L).

* poisson   - uniform positions, iid Gaussian velocities (plus an optional bulk
              flow), the analogue of the paper's position-randomised samples
              (Sec. 2.4.2);
* zeldovich - a lattice displaced by a Gaussian random field with a given P(k),
              velocities v = f H psi (linear theory), the stand-in for the
              simulation snapshots;
* lattice_wave - particles on grid nodes with a single plane-wave velocity field
              (gradient or curl), for closed-form spectra.
"""
from __future__ import annotations

import numpy as np


def _wrap(pos: np.ndarray, L: float) -> np.ndarray:
    pos = np.mod(pos, L)
    pos[pos >= L] -= L  # np.mod can return L for tiny negative inputs
    return pos


def poisson(n: int, L: float, sigma_v: float = 300.0, seed: int = 1000, dtype=np.float32,
            bulk=(0.0, 0.0, 0.0), unit_mass: bool = True) -> dict:
    rng = np.random.Generator(np.random.PCG64(seed))
    pos = rng.uniform(0.0, L, size=(n, 3))
    vel = rng.normal(0.0, sigma_v, size=(n, 3)) + np.asarray(bulk, dtype=np.float64)[None, :]
    out = {"L": float(L)}
    pos = pos.astype(dtype)
    pos[pos >= dtype(L)] = 0  # rounding to the narrower type may land on L
    out["pos"] = np.ascontiguousarray(pos)
    out["vel"] = np.ascontiguousarray(vel.astype(dtype))
    if not unit_mass:
        out["mass"] = np.ascontiguousarray(rng.uniform(0.5, 1.5, size=n).astype(dtype))
    return out


def linear_power(k: np.ndarray, amp: float = 2.0e4, k0: float = 0.02) -> np.ndarray:
    """P(k) = amp (k/k0) / (1 + (k/k0)^3.5) in (Mpc/h)^3."""
    x = k / k0
    return amp * x / (1.0 + x ** 3.5)


def zeldovich(n_side: int, L: float, seed: int = 1001, f: float = 0.5, H: float = 100.0,
              dtype=np.float32, amp: float = 2.0e4, k0: float = 0.02, workers: int = -1) -> dict:
    """Zel'dovich catalogue: n_side^3 particles on the lattice q = i L / n_side.

    A white-noise field (seeded PCG64) is coloured to delta(k) with power P(k)
    (delta(0) = 0, Nyquist planes zeroed), displaced by psi(k) = i k delta(k) / k^2
    (numpy's e^{-ikx} forward convention, so delta = -div psi), x = q + psi
    wrapped into the box, and v = f H psi.
    """
    import scipy.fft

    rng = np.random.Generator(np.random.PCG64(seed))
    N = n_side
    V = L ** 3
    white = rng.standard_normal((N, N, N))
    wk = scipy.fft.rfftn(white, workers=workers)
    del white
    kf = 2.0 * np.pi / L
    kx = kf * np.fft.fftfreq(N, d=1.0 / N)
    kz = kf * np.arange(N // 2 + 1)
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    amp_k = np.sqrt(linear_power(np.sqrt(k2), amp, k0) * N ** 3 / V)
    amp_k[0, 0, 0] = 0.0
    amp_k[N // 2, :, :] = 0.0
    amp_k[:, N // 2, :] = 0.0
    amp_k[:, :, N // 2] = 0.0
    dk = wk * amp_k
    del wk, amp_k
    q1 = np.arange(N, dtype=np.float64) * (L / N)
    pos = np.empty((N, N, N, 3), dtype=np.float64)
    vel = np.empty((N, N, N, 3), dtype=dtype)
    kvecs = (kx[:, None, None], kx[None, :, None], kz[None, None, :])
    for a in range(3):
        psi = scipy.fft.irfftn(1j * kvecs[a] / k2 * dk, s=(N, N, N), workers=workers)
        qa = q1.reshape([N if i == a else 1 for i in range(3)])
        pos[..., a] = qa + psi
        vel[..., a] = (f * H * psi).astype(dtype)
        del psi
    pos = _wrap(pos.reshape(-1, 3), L).astype(dtype)
    pos[pos >= dtype(L)] = 0
    return {"L": float(L), "pos": np.ascontiguousarray(pos), "vel": np.ascontiguousarray(vel.reshape(-1, 3))}


def lattice_wave(ng: int, L: float, kvec_int=(1, 0, 0), e=(1.0, 0.0, 0.0), amp: float = 100.0,
                 dtype=np.float64) -> dict:
    """One particle on every grid node, v_j = amp * e * cos(k0 . q_j), k0 = k_f * kvec_int."""
    i = np.arange(ng, dtype=np.float64)
    g0, g1, g2 = np.meshgrid(i, i, i, indexing="ij")
    q = np.stack([g0, g1, g2], axis=-1).reshape(-1, 3) * (L / ng)
    k0 = (2.0 * np.pi / L) * np.asarray(kvec_int, dtype=np.float64)
    c = np.cos(q @ k0)
    vel = amp * c[:, None] * np.asarray(e, dtype=np.float64)[None, :]
    return {"L": float(L), "pos": np.ascontiguousarray(q.astype(dtype)),
            "vel": np.ascontiguousarray(vel.astype(dtype))}


def log_uniform_counts(n_catalogs: int, lo: float, hi: float, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.round(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_catalogs))).astype(np.int64)


# ---------------------------------------------------------------------------
# Device-side generators (PyTorch): the same recipes drawn with torch's generator
# on the GPU, for the batched and serving workloads whose many large catalogues
# would take minutes to draw on the host. They are not bit-identical to the numpy
# generators above (different random streams); tests that compare with the CPU
# oracle use the numpy ones, or copy these to the host.

def poisson_torch(n: int, L: float, sigma_v: float = 300.0, seed: int = 1000, device="cuda",
                  dtype=None) -> dict:
    import torch
    dtype = dtype or torch.float32
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    pos = torch.rand((n, 3), generator=g, device=device, dtype=torch.float64) * L
    vel = torch.randn((n, 3), generator=g, device=device, dtype=torch.float64) * sigma_v
    pos = pos.to(dtype)
    pos[pos >= L] = 0
    return {"L": float(L), "pos": pos.contiguous(), "vel": vel.to(dtype).contiguous()}


def zeldovich_torch(n_side: int, L: float, seed: int = 1001, f: float = 0.5, H: float = 100.0, device="cuda",
                    dtype=None, amp: float = 2.0e4, k0: float = 0.02) -> dict:
    """The recipe of zeldovich() (same P(k), delta(0) = 0, Nyquist planes zeroed,
    psi(k) = i k delta(k) / k^2, v = f H psi), drawn on the device."""
    import torch
    dtype = dtype or torch.float32
    N = n_side
    V = L ** 3
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    white = torch.randn((N, N, N), generator=g, device=device, dtype=torch.float32)
    wk = torch.fft.rfftn(white)
    del white
    kf = 2.0 * torch.pi / L
    kx = kf * torch.fft.fftfreq(N, d=1.0 / N, device=device)
    kz = kf * torch.arange(N // 2 + 1, device=device, dtype=torch.float32)
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    k2[0, 0, 0] = 1.0
    x = torch.sqrt(k2) / k0
    amp_k = torch.sqrt(amp * x / (1.0 + x ** 3.5) * (N ** 3) / V)
    amp_k[0, 0, 0] = 0.0
    amp_k[N // 2, :, :] = 0.0
    amp_k[:, N // 2, :] = 0.0
    amp_k[:, :, N // 2] = 0.0
    dk = wk * amp_k
    del wk, amp_k, x
    q1 = torch.arange(N, device=device, dtype=torch.float64) * (L / N)
    pos = torch.empty((N, N, N, 3), device=device, dtype=dtype)
    vel = torch.empty((N, N, N, 3), device=device, dtype=dtype)
    kvecs = (kx[:, None, None], kx[None, :, None], kz[None, None, :])
    for a in range(3):
        psi = torch.fft.irfftn(1j * kvecs[a] / k2 * dk, s=(N, N, N)).to(torch.float64)
        qa = q1.reshape([N if i == a else 1 for i in range(3)])
        pos[..., a] = torch.remainder(qa + psi, L).to(dtype)
        vel[..., a] = (f * H * psi).to(dtype)
        del psi
    pos = pos.reshape(-1, 3)
    pos[pos >= L] = 0
    return {"L": float(L), "pos": pos.contiguous(), "vel": vel.reshape(-1, 3).contiguous()}
