"""Statistical analysis of Monte Carlo time series, as the paper's
verification section uses it (Sec. 3): error bars from binning, the
integrated autocorrelation time tau_int, and the Gaussian difference test
whose Q values Tables 1-3 print.

All functions are plain numpy on host data (measurement series read back
from the device); none of them touches the GPU.
"""
from __future__ import annotations

from math import erfc, sqrt

import numpy as np


def gaussian_difference_q(x1: float, e1: float, x2: float, e2: float) -> float:
    """Q of the Gaussian difference test between two estimates x1 +- e1 and
    x2 +- e2 (Sec. 3): the probability that two Gaussian estimates of the
    same mean differ by at least |x1 - x2|,
    Q = erfc(|x1 - x2| / sqrt(2 (e1^2 + e2^2))).
    Q is uniformly distributed on (0, 1] when both estimates are correct."""
    s = sqrt(2.0 * (e1 * e1 + e2 * e2))
    if s == 0.0:
        return 1.0 if x1 == x2 else 0.0
    return erfc(abs(x1 - x2) / s)


def bin_means(series, nbins: int) -> np.ndarray:
    """Means of nbins contiguous bins of equal length; samples beyond
    nbins * (len // nbins) at the end are dropped."""
    x = np.asarray(series, dtype=np.float64)
    if nbins < 2 or len(x) < nbins:
        raise ValueError(f"need at least {nbins} >= 2 samples")
    n = len(x) // nbins
    return x[: n * nbins].reshape(nbins, n).mean(axis=1)


def binned_mean_error(series, nbins: int = 32) -> tuple[float, float]:
    """Mean and its error bar from nbins bins (the paper uses 32): the
    standard deviation of the bin means over sqrt(nbins).  Valid when a bin
    is much longer than tau_int, so that bin means are independent."""
    b = bin_means(series, nbins)
    return float(b.mean()), float(b.std(ddof=1) / np.sqrt(nbins))


def naive_error(series) -> float:
    """Error bar of the mean as if the samples were independent."""
    x = np.asarray(series, dtype=np.float64)
    return float(x.std(ddof=1) / np.sqrt(len(x)))


def tau_int_binning(series, nbins: int = 32) -> float:
    """tau_int from binning: (binned error / naive error)^2, which tends to
    tau_int = 1 + 2 sum_{t>=1} rho(t) for bins much longer than the
    autocorrelation time (the variance of a mean of N correlated samples is
    sigma^2 tau_int / N)."""
    return (binned_mean_error(series, nbins)[1] / naive_error(series)) ** 2


def autocorrelation(series, tmax: int) -> np.ndarray:
    """Normalised autocorrelation function rho(t), t = 0..tmax, by FFT."""
    x = np.asarray(series, dtype=np.float64)
    x = x - x.mean()
    n = len(x)
    m = 1 << int(np.ceil(np.log2(2 * n)))
    f = np.fft.rfft(x, m)
    c = np.fft.irfft(f * np.conj(f), m)[: tmax + 1]
    c /= np.arange(n, n - tmax - 1, -1)  # unbiased: n - t pairs at lag t
    return c / c[0]


def tau_int_window(series, c: float = 6.0, tmax: int | None = None) -> tuple[float, int]:
    """tau_int = 1 + 2 sum_{t=1}^{W} rho(t), with the window W the smallest
    lag for which W >= c * tau_int(W) (the self-consistent window of Madras
    and Sokal).  Returns (tau_int, W)."""
    x = np.asarray(series, dtype=np.float64)
    tmax = min(len(x) // 4, 100000) if tmax is None else tmax
    rho = autocorrelation(x, tmax)
    tau = 1.0 + 2.0 * np.cumsum(rho[1:])
    for w in range(1, tmax + 1):
        if w >= c * tau[w - 1]:
            return float(tau[w - 1]), w
    return float(tau[-1]), tmax


def format_value(x: float, e: float) -> str:
    """x (e) with the error in units of the last two digits, rounded up in
    the second digit as the paper does (Sec. 3.1.1)."""
    if not np.isfinite(e) or e <= 0:
        return f"{x:.6f}"
    digits = max(0, 1 - int(np.floor(np.log10(e))))
    scale = 10.0 ** digits
    return f"{x:.{digits}f} ({int(np.ceil(e * scale - 1e-9))})"
