"""The byte counts behind bench.py's binning roofline: the half-spectrum modes inside the
shell range (1 <= |n| <= ng/2), counted row by row with exact integer square roots,
against brute force over every mode of small grids, and the count's approach to pi/6 of
the half spectrum."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def brute(ng, umin, umax):
    n = np.arange(-(ng // 2), ng // 2)
    l = np.arange(ng // 2 + 1)
    nsq = n[:, None, None] ** 2 + n[None, :, None] ** 2 + l[None, None, :] ** 2
    return int(((nsq >= math.ceil(umin * umin)) & (nsq <= math.floor(umax * umax))).sum())


@pytest.mark.parametrize("ng", [2, 4, 8, 14, 16, 22, 32])
def test_in_shell_modes_equals_brute_force(ng):
    assert bench.in_shell_modes(ng) == brute(ng, 1.0, ng / 2)


@pytest.mark.parametrize("ng,umin,umax", [(16, 2.5, 6.0), (20, 1.0, 9.99), (24, 0.0, 12.0)])
def test_in_shell_modes_other_ranges(ng, umin, umax):
    assert bench.in_shell_modes(ng, umin, umax) == brute(ng, umin, umax)


def test_in_shell_fraction_tends_to_pi_over_6():
    ng = 512
    frac = bench.in_shell_modes(ng) / (ng * ng * (ng // 2 + 1))
    assert abs(frac - math.pi / 6) < 2e-3
