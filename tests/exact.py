"""Closed forms and generic numerics that the statistical tests compare to.

Nothing here restates the heatbath: these are mathematical facts about the
distributions the method must sample.

* SU(2) heatbath: with Haar measure on SU(2), the weight exp(alpha x0) gives
  x0 the density  alpha / (pi I_1(alpha)) * sqrt(1 - x0^2) * exp(alpha x0)
  on [-1, 1], with mean I_2(alpha)/I_1(alpha).  One Kennedy-Pendleton hit is
  accepted with probability sqrt(2 pi alpha) exp(-alpha) I_1(alpha).
* SU(3) one-link integrals: z(g) = int dU exp((g/3) Re Tr U) over Haar SU(3),
  evaluated by the Weyl integration formula over the eigenphases
  (theta1, theta2, -theta1-theta2) with density prod_{j<k} |e^{i theta_j} -
  e^{i theta_k}|^2; the periodic trapezoid rule converges exponentially.
  <(1/3) Re Tr U>_g = z'(g)/z(g).
"""
from __future__ import annotations

import numpy as np
from scipy import special

# ---------------------------------------------------------------- SU(2)


def su2_a0_density(x: np.ndarray, alpha: float) -> np.ndarray:
    return alpha / (np.pi * special.iv(1, alpha)) * np.sqrt(np.clip(1 - x * x, 0, None)) * np.exp(alpha * x)


def su2_a0_cdf_bins(edges: np.ndarray, alpha: float, n_sub: int = 2000) -> np.ndarray:
    """Probability of each histogram bin (Gauss-Legendre per bin)."""
    xg, wg = np.polynomial.legendre.leggauss(64)
    probs = []
    for a, b in zip(edges[:-1], edges[1:]):
        # substitute x = cos(t) near the endpoints is unnecessary with 64 nodes for these bin widths
        xm = 0.5 * (b - a) * xg + 0.5 * (a + b)
        probs.append(0.5 * (b - a) * np.sum(wg * su2_a0_density(xm, alpha)))
    return np.array(probs)


def su2_a0_mean(alpha: float) -> float:
    return float(special.iv(2, alpha) / special.iv(1, alpha))


def kp_acceptance(alpha: float) -> float:
    return float(np.sqrt(2 * np.pi * alpha) * special.ive(1, alpha))


# ---------------------------------------------------------------- SU(3) Weyl integrals

_N = 240
_th = 2 * np.pi * np.arange(_N) / _N
_T1, _T2 = np.meshgrid(_th, _th, indexing="ij")
_E1, _E2, _E3 = np.exp(1j * _T1), np.exp(1j * _T2), np.exp(-1j * (_T1 + _T2))
_HAAR = (np.abs(_E1 - _E2) ** 2 * np.abs(_E1 - _E3) ** 2 * np.abs(_E2 - _E3) ** 2)
_RETR = np.cos(_T1) + np.cos(_T2) + np.cos(_T1 + _T2)
_TR = _E1 + _E2 + _E3


def su3_haar_average(f_of_trace) -> complex:
    """<f(Tr U)> over Haar SU(3)."""
    return complex(np.sum(_HAAR * f_of_trace(_TR)) / np.sum(_HAAR))


def su3_plaquette_mean(g: float) -> float:
    """<(1/3) Re Tr U> for the weight exp((g/3) Re Tr U) on SU(3)."""
    w = _HAAR * np.exp(g / 3.0 * (_RETR - 3.0))
    return float(np.sum(w * _RETR / 3.0) / np.sum(w))


def su3_plaquette_var(g: float) -> float:
    w = _HAAR * np.exp(g / 3.0 * (_RETR - 3.0))
    m = np.sum(w * _RETR / 3.0) / np.sum(w)
    return float(np.sum(w * (_RETR / 3.0 - m) ** 2) / np.sum(w))


# ---------------------------------------------------------------- statistics


def binned_mean(series: np.ndarray, nbins: int = 32):
    """Mean and its error from nbins equal bins (bins long against the
    autocorrelation time make the bin means independent)."""
    series = np.asarray(series, dtype=np.float64)
    n = (len(series) // nbins) * nbins
    bins = series[:n].reshape(nbins, -1).mean(axis=1)
    return float(bins.mean()), float(bins.std(ddof=1) / np.sqrt(nbins))


def chi2_pvalue(counts: np.ndarray, probs: np.ndarray) -> float:
    n = counts.sum()
    expected = probs / probs.sum() * n
    keep = expected > 5
    chi2 = float(np.sum((counts[keep] - expected[keep]) ** 2 / expected[keep]))
    dof = int(keep.sum()) - 1
    return float(special.gammaincc(dof / 2.0, chi2 / 2.0))
