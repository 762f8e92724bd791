"""Pins for the oracle's assignment kernel (oracle/bspline.py).

The BL scaling function is not written down in the paper (Sec. 2.4.1 cites it);
these tests pin the oracle's reading of it to mathematics that does not depend on
the oracle's own code: exact textbook samples, brute-force alias sums, the
textbook NGP/CIC/TSC alias sums (Jing 2005), partition of unity and
orthonormality of phi by quadrature.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import bspline as bs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_integer_samples_match_textbook():
    for order, n, num, den in _read("bspline_integer_samples.txt"):
        got = bs.bspline_int_samples(int(order))[int(n)]
        assert got == Fraction(int(num), int(den)), (order, n, got)


@pytest.mark.parametrize("m", [2, 3, 4, 5, 6])
def test_integer_samples_sum_to_one(m):
    # partition of unity of B_m at integer shifts, exact
    if m % 2 == 0:
        assert sum(bs.bspline_int_samples(m).values()) == 1


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_bspline_partition_of_unity_and_integral(m):
    x = np.linspace(-0.5, 0.5, 101)
    s = sum(bs.bspline(x - n, m) for n in range(-6, 7))
    np.testing.assert_allclose(s, 1.0, atol=1e-13)
    t = np.linspace(-m / 2, m / 2, 200001)
    integral = np.trapezoid(bs.bspline(t, m), t)
    assert abs(integral - 1.0) < 1e-5  # trapezoid error at the box edges ~ h/2


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_bspline_convolution_recursion(m):
    # B_m = B_{m-1} * B_1 by numerical convolution on a fine grid
    h = 1e-3
    t = np.arange(-4, 4 + h / 2, h)
    lhs = bs.bspline(t, m)
    box = bs.bspline(t, 1)
    prev = bs.bspline(t, m - 1)
    conv = np.convolve(prev, box, mode="same") * h
    assert np.max(np.abs(conv - lhs)) < 5e-3


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_bspline_hat_is_fourier_transform(m):
    # direct quadrature of int B_m(x) cos(w x) dx
    x = np.linspace(-m / 2, m / 2, 40001)
    for w in (0.3, 1.7, 3.1):
        ft = np.trapezoid(bs.bspline(x, m) * np.cos(w * x), x)
        assert abs(ft - bs.bspline_hat(w, m)) < 1e-7


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_alias_sum_closed_form_vs_brute_force(m):
    w = np.linspace(-np.pi, np.pi, 41)
    np.testing.assert_allclose(bs.alias_sum(w, m), bs.alias_sum_brute(w, m, jmax=4000), rtol=0, atol=1e-12)


def test_alias_sum_ngp_brute_force_tail_bound():
    # NGP: sum_J sinc^2 = 1; the brute sum's tail is bounded by ~ 2/(pi^2 J)
    w = np.linspace(-3.0, 3.0, 13)
    jmax = 20000
    err = np.abs(bs.alias_sum_brute(w, 1, jmax=jmax) - bs.alias_sum(w, 1))
    assert np.all(err < 4.0 / (np.pi ** 2 * jmax))


def test_alias_sums_match_jing2005():
    w = np.linspace(-np.pi, np.pi, 33)
    s2 = np.sin(w / 2) ** 2
    for order, c0, c1, c2 in _read("alias_sums_jing2005.txt"):
        ref = float(c0) + float(c1) * s2 + float(c2) * s2 ** 2
        np.testing.assert_allclose(bs.alias_sum(w, int(order)), ref, atol=1e-15)


@pytest.mark.parametrize("m", [1, 2, 3, 4, 5])
def test_phi_hat_orthonormal_and_partition(m):
    w = np.linspace(-np.pi, np.pi, 29)
    np.testing.assert_allclose(bs.phi_alias_sum_brute(w, m, jmax=400 if m > 1 else 20000), 1.0,
                               atol=1e-4 if m == 1 else 1e-12)
    np.testing.assert_allclose(bs.phi_alias_sum(w, m), 1.0, atol=1e-15)
    assert abs(bs.phi_hat(0.0, m) - 1.0) < 1e-15
    for J in (1, 2, 3, -1):
        assert abs(bs.phi_hat(2 * np.pi * J, m)) < 1e-15


def test_phi_real_space_orthonormality_and_partition_of_unity():
    m = 4
    x = np.linspace(-0.5, 0.5, 21)
    pou = np.array([bs.phi(xx - np.arange(-45, 46), m).sum() for xx in x])
    np.testing.assert_allclose(pou, 1.0, atol=1e-10)
    # <phi(x) phi(x - n)> = delta_n by quadrature over the (numerical) support
    h = 1.0 / 64
    t = np.arange(-30, 30 + h / 2, h)
    f = bs.phi(t, m)
    for n in range(0, 4):
        g = bs.phi(t - n, m)
        inner = np.trapezoid(f * g, t)
        assert abs(inner - (1.0 if n == 0 else 0.0)) < 1e-8, (n, inner)


def test_phi_decay_of_bl3_coefficients():
    # c_n decays geometrically; the first values are those of Sigma_4^{-1/2}
    n, c = bs.bl_coefficients(4, nmax=40)
    c = dict(zip(n, c))
    assert abs(c[0] - 1.9697616) < 1e-6
    assert abs(c[1] - c[-1]) < 1e-15
    assert abs(c[30]) < 1e-7 and abs(c[40]) < 1e-9


@pytest.mark.parametrize("m", [2, 3, 4, 5])
def test_phi_alias_sum_brute_force_converges_to_closed_form(m):
    w = np.linspace(-np.pi, np.pi, 17)
    err = np.abs(bs.phi_alias_sum_brute(w, m, jmax=3000) - bs.phi_alias_sum(w, m))
    assert np.all(err < 1e-11)
