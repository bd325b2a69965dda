"""Pins of the oracle's double-layered torus with two couplings (Sec. 2.2):
a plaquette gets beta1 when any of its links lies in the second layer, else
beta0."""
import numpy as np
import pytest

import oracle


def _random_su3(rng):
    z = (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1 / 3)


def test_beta1_plaquette_count_time_glued():
    """Cold links (every plaquette = 1): the weighted action is
    beta0 N0 + beta1 N1.  Glued in time only, N1 = 6V (all of layer 1) +
    3V/n_t (layer-0 time-like plaquettes on the last time slice, whose
    forward time link starts in layer 1)."""
    dims = [4, 2, 4, 6]
    lat = oracle.Lattice(dims, nlayers=2, glue_mask=0b1000).cold_start()
    V = lat.V
    n1 = 6 * V + 3 * V // dims[3]
    n0 = 12 * V - n1
    assert lat.action_weighted(5.0, 2.0) == pytest.approx(5.0 * n0 + 2.0 * n1, rel=1e-14)


def test_beta1_plaquette_count_all_glued():
    """Glued in all directions: a layer-0 plaquette in plane (mu, nu) touches
    layer 1 when x^mu or x^nu sits on the upper boundary."""
    dims = [4, 6, 2, 4]
    lat = oracle.Lattice(dims, nlayers=2, glue_mask=0b1111).cold_start()
    V = lat.V
    n1 = 6 * V
    for mu in range(4):
        for nu in range(mu + 1, 4):
            n1 += round(V * (1 - (1 - 1 / dims[mu]) * (1 - 1 / dims[nu])))
    n0 = 12 * V - n1
    assert lat.action_weighted(6.0, 1.5) == pytest.approx(6.0 * n0 + 1.5 * n1, rel=1e-14)


@pytest.mark.parametrize("glue", [0b1111, 0b1000, 0b0101])
def test_weighted_staple_gives_local_weighted_action(glue):
    rng = np.random.default_rng(17)
    lat = oracle.Lattice([2, 4, 2, 4], nlayers=2, glue_mask=glue).hot_start(3)
    b0, b1 = 5.7, 3.1
    for _ in range(12):
        layer, site, mu = int(rng.integers(2)), int(rng.integers(lat.V)), int(rng.integers(4))
        A = lat.staple_weighted(layer, site, mu, b0, b1)
        s0 = lat.action_weighted(b0, b1)
        M = lat.links()
        old = M[layer, site, mu].copy()
        new = _random_su3(rng)
        M[layer, site, mu] = new
        lat.set_links(M)
        s1 = lat.action_weighted(b0, b1)
        assert abs(3 * (s1 - s0) - np.real(np.trace((new - old) @ A))) < 1e-10


def test_equal_couplings_reduce_to_one_beta():
    lat = oracle.Lattice([2, 4, 2, 4], nlayers=2, glue_mask=0b1011).hot_start(8)
    for site in range(0, lat.V, 7):
        np.testing.assert_allclose(lat.staple_weighted(1, site, 2, 5.5, 5.5), 5.5 * lat.staple(1, site, 2),
                                   atol=1e-12)
    a = oracle.Lattice([2, 4, 2, 4], nlayers=2, glue_mask=0b1011).hot_start(8)
    b = oracle.Lattice([2, 4, 2, 4], nlayers=2, glue_mask=0b1011).hot_start(8)
    a.sweep(5.5, 2, 4, n=2)
    b.sweep(5.5, 2, 4, n=2, beta1=5.5)
    assert np.array_equal(a.U, b.U)


def test_two_couplings_change_only_the_weighted_sweep():
    a = oracle.Lattice([2, 4, 2, 4], nlayers=2).hot_start(8)
    b = oracle.Lattice([2, 4, 2, 4], nlayers=2).hot_start(8)
    a.sweep(5.5, 2, 4, n=1)
    b.sweep(5.5, 2, 4, n=1, beta1=4.0)
    assert not np.array_equal(a.U, b.U)
    M = b.links().reshape(-1, 3, 3)
    np.testing.assert_allclose(M @ M.conj().transpose(0, 2, 1), np.broadcast_to(np.eye(3), M.shape), atol=1e-13)
