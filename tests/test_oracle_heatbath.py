"""Pins of the oracle's SU(2) and Cabibbo-Marinari heatbath (Sec. 2.1).

The paper only cites the FHKP algorithm; what fixes the result is the
distribution it must sample.  These tests compare the draws with closed forms
(Bessel functions for SU(2), Weyl integrals for SU(3)) rather than with a
second copy of the algorithm.
"""
import numpy as np
import pytest

import oracle
from tests import exact


@pytest.mark.parametrize("alpha", [0.5, 2.0, 8.0, 40.0])
def test_su2_a0_histogram(alpha):
    x, acc = oracle.su2_samples(alpha, hits=200, seed=11, n=200_000)
    a0 = x[acc, 0]
    assert acc.mean() > 0.999
    edges = np.linspace(-1, 1, 81) if alpha < 10 else np.linspace(0.8, 1, 81)
    counts, _ = np.histogram(a0, bins=edges)
    probs = exact.su2_a0_cdf_bins(edges, alpha)
    assert exact.chi2_pvalue(counts, probs) > 1e-4
    m = a0.mean()
    err = a0.std() / np.sqrt(len(a0))
    assert abs(m - exact.su2_a0_mean(alpha)) < 5 * err


@pytest.mark.parametrize("alpha", [1.0, 4.0, 24.0])
def test_su2_one_hit_acceptance(alpha):
    _, acc = oracle.su2_samples(alpha, hits=1, seed=5, n=200_000)
    p = exact.kp_acceptance(alpha)
    err = np.sqrt(p * (1 - p) / len(acc))
    assert abs(acc.mean() - p) < 5 * err


@pytest.mark.parametrize("subgroup", [0, 1, 2])
def test_su2_draw_is_unit_and_isotropic(subgroup):
    x, acc = oracle.su2_samples(3.0, hits=50, seed=2, n=100_000, subgroup=subgroup)
    x = x[acc]
    np.testing.assert_allclose(np.sum(x * x, axis=1), 1.0, atol=1e-14)
    # the vector part points uniformly on the sphere: mean 0, equal second moments
    v = x[:, 1:]
    assert np.all(np.abs(v.mean(axis=0)) < 5 * v.std(axis=0) / np.sqrt(len(v)))
    m2 = (v ** 2).mean(axis=0)
    target = (1 - x[:, 0] ** 2).mean() / 3
    assert np.all(np.abs(m2 - target) < 0.01 * target + 5 * (v ** 2).std(axis=0) / np.sqrt(len(v)))


def test_su2_directions_of_the_three_subgroups_are_independent():
    """The three subgroups of one link update draw their directions from two
    random-number blocks (two words each; subgroups 0 and 1 share a block).
    At the same counter the three unit directions must be uncorrelated: a
    subgroup reading another one's words would repeat its direction."""
    n = 50_000
    dirs = []
    for sg in range(3):
        x, acc = oracle.su2_samples(3.0, hits=50, seed=4, n=n, subgroup=sg)
        assert acc.all()
        v = x[:, 1:]
        dirs.append(v / np.linalg.norm(v, axis=1, keepdims=True))
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        dot = np.sum(dirs[a] * dirs[b], axis=1)  # 1/3 variance for independent isotropic directions
        assert abs(dot.mean()) < 5 * np.sqrt(1 / 3 / n)
        cos_theta = dirs[a][:, 2] * dirs[b][:, 2]
        assert abs(cos_theta.mean()) < 5 * np.sqrt(1 / 9 / n)


def _random_su3(rng):
    z = (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1 / 3)


@pytest.mark.parametrize("gamma,hits", [(1.0, 20), (6.0, 20), (24.0, 1), (24.0, 20)])
def test_frozen_staple_matches_weyl_integral(gamma, hits):
    """A link in a fixed staple A = c V (V in SU(3)) must be distributed as
    exp((beta/3) Re Tr(U A)), so <Re Tr(U A)>/(3c) = z'(g)/z(g) with
    g = beta c.  A non-unit V checks that the subgroups are taken from
    W = U A, and hits=1 checks the Fredenhagen-Marcu variant."""
    rng = np.random.default_rng(7)
    V = _random_su3(rng)
    c = 6.0
    beta = gamma / c
    series = oracle.link_chain(c * V, beta, hits, seed=3, n=120_000)
    m, err = exact.binned_mean(series[2000:] / (3 * c), nbins=40)
    assert abs(m - exact.su3_plaquette_mean(gamma)) < 4.5 * err + 1e-12


def test_link_update_stays_in_su3():
    rng = np.random.default_rng(1)
    u = _random_su3(rng)
    A = sum(_random_su3(rng) for _ in range(6))
    for t in range(50):
        u, _ = oracle.link_heatbath(u, A, 6.0, 2, seed=9, site_key=3, sweep=t, colour=1, mu=2)
        np.testing.assert_allclose(u @ u.conj().T, np.eye(3), atol=1e-13)
        assert abs(np.linalg.det(u) - 1) < 1e-13


def test_link_update_is_deterministic_in_counter():
    rng = np.random.default_rng(4)
    u = _random_su3(rng)
    A = sum(_random_su3(rng) for _ in range(6))
    a, _ = oracle.link_heatbath(u, A, 6.0, 2, seed=9, site_key=3, sweep=5, colour=0, mu=1)
    b, _ = oracle.link_heatbath(u, A, 6.0, 2, seed=9, site_key=3, sweep=5, colour=0, mu=1)
    c, _ = oracle.link_heatbath(u, A, 6.0, 2, seed=9, site_key=3, sweep=6, colour=0, mu=1)
    assert np.array_equal(a, b)
    assert not np.allclose(a, c)
