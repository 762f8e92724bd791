"""Brute-force references that pin the oracle (small sizes only).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

* deposit_bl_direct - real-space assignment with the orthonormalised scaling
  function phi itself (from its B-spline expansion), summed over periodic images, no
  Fourier-space factor. Untruncated it pins the factored form used by estimator.py;
  with a radius R it is the oracle of the direct truncated BL assignment (phi set to
  zero beyond R cells, the literal real-space stencil of Sec. 2.4.1), which
  estimator.estimate(bl_radius=R) uses.
* dft3           - O(M^2) discrete Fourier transform by its definition.
* full_sphere_bins - binning over every mode of a full complex FFT (no half-spectrum
  weights), using the same bin definition.
"""
from __future__ import annotations

import numpy as np

from . import bspline as _bs


def _folded_weights(x: np.ndarray, ng: int, order: int, reach: int, nmax: int, radius: float | None) -> np.ndarray:
    """Weights phi(x_j - n) for all integer n within `reach` of each x_j, zero where
    |x_j - n| >= radius (if given), folded onto ng periodic nodes: (len(x), ng)."""
    x = np.asarray(x, dtype=np.float64)
    base = np.floor(x).astype(np.int64)
    nodes = base[:, None] + np.arange(-reach, reach + 1)[None, :]
    d = x[:, None] - nodes
    w = _bs.phi(d, order, nmax=nmax)
    if radius is not None:
        w = np.where(np.abs(d) < radius, w, 0.0)
    out = np.zeros((len(x), ng))
    rows = np.repeat(np.arange(len(x)), nodes.shape[1])
    np.add.at(out, (rows, np.mod(nodes, ng).ravel()), w.ravel())
    return out


def deposit_bl_direct(u: np.ndarray, q: np.ndarray, ng: int, order: int = 4,
                      reach: int = 40, nmax: int = 40, radius: float | None = None) -> np.ndarray:
    """Grid G_f(n) = sum_j q_jf sum_images phi_R(u_j - n) (separable product), FP64,
    with phi_R = phi truncated to |x| < radius (no truncation if radius is None)."""
    u = np.asarray(u, dtype=np.float64)
    q = np.asarray(q, dtype=np.float64)
    if q.ndim == 1:
        q = q[:, None]
    if radius is not None:
        reach = int(np.ceil(radius)) + 1
    grids = np.zeros((q.shape[1], ng, ng, ng))
    for j0 in range(0, len(u), 512):
        sl = slice(j0, j0 + 512)
        wx = _folded_weights(u[sl, 0], ng, order, reach, nmax, radius)
        wy = _folded_weights(u[sl, 1], ng, order, reach, nmax, radius)
        wz = _folded_weights(u[sl, 2], ng, order, reach, nmax, radius)
        grids += np.einsum("jf,ja,jb,jc->fabc", q[sl], wx, wy, wz, optimize=True)
    return grids


def dft3(g: np.ndarray) -> np.ndarray:
    """F(k) = sum_n g(n) exp(-2 pi i k.n / N) by the definition (full spectrum)."""
    n0, n1, n2 = g.shape
    out = np.zeros(g.shape, dtype=np.complex128)
    i0 = np.arange(n0)[:, None, None]
    i1 = np.arange(n1)[None, :, None]
    i2 = np.arange(n2)[None, None, :]
    for k0 in range(n0):
        for k1 in range(n1):
            for k2 in range(n2):
                ph = np.exp(-2j * np.pi * (k0 * i0 / n0 + k1 * i1 / n1 + k2 * i2 / n2))
                out[k0, k1, k2] = (g * ph).sum()
    return out


def full_sphere_bins(values: np.ndarray, ng: int, nbins: int, umin: float, umax: float,
                     bin_index) -> tuple[np.ndarray, np.ndarray]:
    """Mode counts and mean of `values` (full ng^3 array) per shell, every mode weight 1."""
    f = np.fft.fftfreq(ng, d=1.0 / ng).astype(np.int64)
    f = np.where(f == -(ng // 2), -(ng // 2), f)
    n2 = f[:, None, None] ** 2 + f[None, :, None] ** 2 + f[None, None, :] ** 2
    b = bin_index(n2, nbins, umin, umax).ravel() + 1
    cnt = np.bincount(b, minlength=nbins + 1)[1:].astype(np.float64)
    s = np.bincount(b, weights=values.ravel(), minlength=nbins + 1)[1:]
    with np.errstate(invalid="ignore", divide="ignore"):
        return cnt, s / cnt
