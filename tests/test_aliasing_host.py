"""Host logic of the resolution-pair report (Sec. 2.4.3, Fig. simalias): the crossing
scale and the maxima below 0.5 and 0.7 k_N, on arrays with known answers."""
import numpy as np

from paper_2005_06170_gb300.aliasing import compare_pair


def test_compare_pair_finds_the_first_shell_above_the_threshold():
    kN = 2.0
    k = np.linspace(0.05, 2.0, 40)            # k / k_N from 0.025 to 1
    n = np.full(40, 10.0)
    x = k / kN
    base = {"k": k, "n_modes": n, "P_pp": np.ones(40), "P_dd": 5.0 * np.ones(40)}
    dev = 0.02 * x ** 4                       # 1 % first exceeded where x^4 > 0.5
    fine = {"k": k, "n_modes": n, "P_pp": 1.0 + dev, "P_dd": 5.0 * (1.0 - 0.001 * x)}
    rep = compare_pair(base, fine, kN)
    first = x[np.nonzero(dev > 0.01)[0][0]]
    assert rep["P_pp"]["first_k_over_kN_above"] == first
    assert abs(rep["P_pp"]["max_dev_k_le_0.5kN"] - np.max(dev[x <= 0.5])) < 1e-15
    assert abs(rep["P_pp"]["max_dev_k_le_0.7kN"] - np.max(dev[x <= 0.7])) < 1e-15
    assert rep["P_dd"]["first_k_over_kN_above"] is None
    assert abs(rep["P_dd"]["max_dev_k_le_0.7kN"] - 0.001 * np.max(x[x <= 0.7])) < 1e-12
    assert "P_tt" not in rep


def test_compare_pair_skips_empty_shells():
    k = np.array([np.nan, 0.5, 1.0, 1.5])
    n = np.array([0.0, 4.0, 4.0, 4.0])
    a = {"k": k, "n_modes": n, "P_pp": np.array([np.nan, 1.0, 1.0, 1.0])}
    b = {"k": k, "n_modes": n, "P_pp": np.array([np.nan, 1.0, 1.0, 1.5])}
    rep = compare_pair(a, b, 2.0)
    assert rep["P_pp"]["first_k_over_kN_above"] == 0.75
    assert rep["P_pp"]["max_dev_k_le_0.5kN"] == 0.0
