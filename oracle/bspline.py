"""Assignment kernels of the estimator, written out from their definitions (FP64).

TEST INFRASTRUCTURE ONLY. This module belongs to the CPU oracle: only tests, the
smoke check and the CPU-baseline leg of the benchmark may import it. The GPU
library never calls it and shares no code with it.

Paper: objects are assigned to the FFT grid with the third-order orthogonalised
Battle-Lemarie (BL3) scaling function (Sec. 2.4.1, also the abstract and Sec. 5).
The paper does not write the function down. Reading used here: the orthonormalised
centred B-spline scaling function on the unit-spaced grid,

    phi_hat(w) = Bhat_m(w) / sqrt(Sigma_m(w)),
    Bhat_m(w)  = [sin(w/2) / (w/2)]^m,
    Sigma_m(w) = sum_J Bhat_m(w + 2 pi J)^2 = sum_n B_{2m}(n) cos(n w),

with B-spline order m = 4 (cubic, polynomial degree 3) by default and m as a
parameter. Sigma_m is the alias sum that appears as sum_J W^2(k + 2 k_N J) in the
shot-noise terms of Eqs. rawPp, rawPtheta and rawPx (per axis, for a
separable window). With it, sum_J phi_hat(w + 2 pi J)^2 = 1 identically.

Parity pins (tests/test_oracle_kernel.py): brute-force alias sums, the textbook
CIC alias sum, exact rational integer samples, partition of unity and
orthonormality of the real-space phi by quadrature.
"""
from __future__ import annotations

import math
from fractions import Fraction

import functools

import numpy as np


def bspline_int_samples(order: int) -> dict[int, Fraction]:
    """Exact values B_order(n) of the centred B-spline at the integers n.

    Uses the truncated-power form B_m(x) = 1/(m-1)! sum_k (-1)^k C(m,k)
    (x + m/2 - k)_+^(m-1), evaluated in rational arithmetic. Only valid for even
    order (integer nodes fall on the knots' midpoints otherwise); 2m is always even.
    """
    if order % 2:
        raise ValueError("integer samples are computed for even orders only")
    half = order // 2
    out = {}
    for n in range(-half, half + 1):
        s = Fraction(0)
        for k in range(order + 1):
            t = n + half - k
            if t > 0:
                s += (-1) ** k * math.comb(order, k) * Fraction(t) ** (order - 1)
        out[n] = s / math.factorial(order - 1)
    return out


def bspline(x, m: int):
    """Centred B-spline B_m(x) of order m (support [-m/2, m/2]), FP64, vectorised.

    Truncated-power formula. B_1 is the box on [-1/2, 1/2) (half-open, so that
    every point belongs to exactly one NGP node).
    """
    x = np.asarray(x, dtype=np.float64)
    if m == 1:
        return ((x >= -0.5) & (x < 0.5)).astype(np.float64)
    s = np.zeros_like(x)
    for k in range(m + 1):
        t = x + m / 2.0 - k
        s += (-1) ** k * math.comb(m, k) * np.where(t > 0, t, 0.0) ** (m - 1)
    out = s / math.factorial(m - 1)
    out = np.where(np.abs(x) < m / 2.0, out, 0.0)
    return out


def bspline_hat(w, m: int):
    """Fourier transform of the centred B_m: [sin(w/2)/(w/2)]^m (value 1 at w = 0)."""
    w = np.asarray(w, dtype=np.float64)
    return np.sinc(w / (2.0 * np.pi)) ** m


def alias_sum(w, m: int):
    """Sigma_m(w) = sum_n B_{2m}(n) cos(n w), the closed form of sum_J Bhat_m(w+2piJ)^2."""
    w = np.asarray(w, dtype=np.float64)
    samples = bspline_int_samples(2 * m)
    out = np.full_like(w, float(samples[0]))
    for n in range(1, m + 1):
        out += 2.0 * float(samples[n]) * np.cos(n * w)
    return out


def alias_sum_brute(w, m: int, jmax: int = 2000):
    """sum_{|J|<=jmax} Bhat_m(w + 2 pi J)^2 by direct summation (pin for alias_sum)."""
    w = np.asarray(w, dtype=np.float64)
    J = np.arange(-jmax, jmax + 1, dtype=np.float64)
    return (bspline_hat(w[..., None] + 2.0 * np.pi * J, m) ** 2).sum(axis=-1)


def phi_hat(w, m: int = 4):
    """Fourier transform of the orthonormalised (Battle-Lemarie) scaling function."""
    return bspline_hat(w, m) / np.sqrt(alias_sum(w, m))


def phi_alias_sum(w, m: int = 4):
    """sum_J phi_hat(w + 2 pi J)^2: the per-axis factor of sum_J W^2(k + 2 k_N J) in
    the shot-noise terms (Eq. rawPp). Since Sigma_m is 2 pi-periodic, this is
    [sum_J Bhat_m(w + 2 pi J)^2] / Sigma_m(w), with the numerator in its closed form
    (pinned to brute force and to Jing 2005 in the tests). It equals 1 for the
    orthonormal scaling function, up to rounding."""
    w = np.asarray(w, dtype=np.float64)
    return alias_sum(w, m) / alias_sum(w, m)


def phi_alias_sum_brute(w, m: int = 4, jmax: int = 200):
    """sum_{|J|<=jmax} phi_hat(w + 2 pi J)^2 by direct summation (pin for phi_alias_sum)."""
    w = np.asarray(w, dtype=np.float64)
    J = np.arange(-jmax, jmax + 1, dtype=np.float64)
    return (phi_hat(w[..., None] + 2.0 * np.pi * J, m) ** 2).sum(axis=-1)


@functools.lru_cache(maxsize=None)
def bl_coefficients(m: int = 4, nmax: int = 40, nquad: int = 4096):
    """Coefficients c_n of phi(x) = sum_n c_n B_m(x - n), n = -nmax..nmax.

    c_n = (1/2pi) int_{-pi}^{pi} Sigma_m(w)^{-1/2} e^{i n w} dw, by the periodic
    trapezoid rule (spectrally accurate for this smooth periodic integrand).
    """
    w = 2.0 * np.pi * np.arange(nquad) / nquad
    f = 1.0 / np.sqrt(alias_sum(w, m))
    n = np.arange(-nmax, nmax + 1)
    c = (f[None, :] * np.cos(n[:, None] * w[None, :])).mean(axis=1)
    return n, c


def phi(x, m: int = 4, nmax: int = 40):
    """Real-space orthonormalised scaling function, truncated to |n| <= nmax terms."""
    x = np.asarray(x, dtype=np.float64)
    n, c = bl_coefficients(m, nmax)
    out = np.zeros_like(x)
    for nn, cc in zip(n, c):
        out += cc * bspline(x - nn, m)
    return out
