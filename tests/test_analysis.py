"""The verification statistics (Sec. 3): the Gaussian difference test
against every Q value the paper prints, and binning / tau_int against the
exact results of a first-order autoregressive process."""
import os

import numpy as np
import pytest

from paper_0904_0642_gb300 import analysis

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_q_values.txt")


def paper_q_rows():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        rows.append((t[0], *map(float, t[1:6])))
    return rows


@pytest.mark.parametrize("row", paper_q_rows(), ids=lambda r: r[0])
def test_gaussian_difference_reproduces_printed_q(row):
    """Printed Q has two digits and the printed error bars are rounded up in
    their second digit: the recomputed Q agrees within 0.006."""
    _, x1, e1, x2, e2, q = row
    assert analysis.gaussian_difference_q(x1, e1, x2, e2) == pytest.approx(q, abs=0.006)


def test_gaussian_difference_properties():
    q = analysis.gaussian_difference_q
    assert q(1.0, 0.1, 1.0, 0.2) == 1.0
    assert q(1.0, 0.1, 1.3, 0.0) == q(1.3, 0.0, 1.0, 0.1)  # symmetric
    # |x1 - x2| = 1.96 standard deviations of the difference: Q = 0.05
    assert q(0.0, 0.3, 1.96 * 0.5, 0.4) == pytest.approx(0.05, abs=1e-4)
    # Q is uniform for correct error bars: mean 1/2 over many pairs
    rng = np.random.default_rng(1)
    e = rng.uniform(0.5, 2.0, (20000, 2))
    x = rng.normal(0.0, e)
    qs = np.array([q(a, ea, b, eb) for (a, b), (ea, eb) in zip(x, e)])
    assert abs(qs.mean() - 0.5) < 0.01 and abs((qs < 0.1).mean() - 0.1) < 0.01


def ar1(n, rho, seed):
    """x_t = rho x_{t-1} + sqrt(1 - rho^2) eps_t, stationary, unit variance;
    its autocorrelation is rho^t and tau_int = (1 + rho) / (1 - rho)."""
    rng = np.random.default_rng(seed)
    eps = rng.standard_normal(n)
    x = np.empty(n)
    x[0] = eps[0]
    a = np.sqrt(1 - rho * rho)
    for t in range(1, n):
        x[t] = rho * x[t - 1] + a * eps[t]
    return x


def test_autocorrelation_of_ar1():
    x = ar1(1 << 18, 0.9, 3)
    r = analysis.autocorrelation(x, 20)
    assert r[0] == 1.0
    assert np.allclose(r, 0.9 ** np.arange(21), atol=0.03)


@pytest.mark.parametrize("rho", [0.0, 0.5, 0.9])
def test_tau_int_of_ar1(rho):
    x = ar1(1 << 19, rho, 7)
    exact = (1 + rho) / (1 - rho)
    tw, w = analysis.tau_int_window(x)
    assert tw == pytest.approx(exact, rel=0.06), (tw, w)
    # binning: 1024 bins of 512 samples (bins >> tau); the estimate of a
    # variance from 1024 bins has a relative error of sqrt(2/1023) ~ 4 %
    assert analysis.tau_int_binning(x, 1024) == pytest.approx(exact, rel=0.15)


def test_binned_error_of_ar1_mean():
    """Error of the mean of N AR(1) samples: sqrt(tau_int / N) (unit
    variance).  32 bins estimate it within the scatter of a 31-degree-of-
    freedom variance (~13 % on the error), here checked over 40 series."""
    rho, n = 0.8, 1 << 15
    exact = np.sqrt((1 + rho) / (1 - rho) / n)
    ratios = []
    for s in range(40):
        m, e = analysis.binned_mean_error(ar1(n, rho, 100 + s), 32)
        ratios.append(e / exact)
    assert np.mean(ratios) == pytest.approx(1.0, abs=0.06)


def test_bin_means_brute_force():
    x = np.arange(100, dtype=float)
    b = analysis.bin_means(x, 4)  # 4 bins of 25
    assert np.array_equal(b, [12.0, 37.0, 62.0, 87.0])
    m, e = analysis.binned_mean_error(x, 4)
    assert m == 49.5 and e == pytest.approx(np.std(b, ddof=1) / 2)
    with pytest.raises(ValueError):
        analysis.bin_means([1.0], 2)


def test_format_value_rounds_error_up():
    assert analysis.format_value(0.538547, 0.0000692) == "0.538547 (70)"
    assert analysis.format_value(0.53811, 0.000181) == "0.53811 (19)"
