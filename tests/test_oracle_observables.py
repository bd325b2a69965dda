"""Pins of the oracle's staple, plaquette, Polyakov loop, start
configurations and re-unitarisation, against exact identities."""
import numpy as np
import pytest

import oracle
from tests import exact

GEOMS = [
    dict(dims=[4, 4]),
    dict(dims=[4, 2, 4]),
    dict(dims=[2, 4, 2, 4]),
    dict(dims=[2, 4, 2, 4], nlayers=2, glue_mask=0b1111),
    dict(dims=[2, 4, 2, 4], nlayers=2, glue_mask=0b1000),
    dict(dims=[4, 2, 4], nlayers=2, glue_mask=0b011),
]


def _random_su3(rng, n=None):
    shape = (3, 3) if n is None else (n, 3, 3)
    z = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    d = np.diagonal(r, axis1=-2, axis2=-1)
    q = q * (d / np.abs(d))[..., None, :]
    det = np.linalg.det(q)
    return q / (det ** (1 / 3))[..., None, None]


def _action_sum(lat):
    """sum over plaquettes of Re Tr U_p, from the averaged plaquette."""
    tot = lat.plaquette(-1)[0]
    nplaq = lat.nlayers * lat.V * lat.D * (lat.D - 1) // 2
    return 3.0 * tot * nplaq


@pytest.mark.parametrize("g", GEOMS)
def test_cold_start_observables_are_one(g):
    lat = oracle.Lattice(**g).cold_start()
    for layer in range(-1, lat.nlayers):
        t, s, ti = lat.plaquette(layer)
        assert t == 1.0 and ti == 1.0 and (s == 1.0 or lat.D == 2)
        assert lat.polyakov(layer) == 1.0


@pytest.mark.parametrize("g", GEOMS)
def test_staple_gives_local_action(g):
    """sum_p Re Tr U_p changes by Re Tr((U' - U) A) when one link U_mu(x)
    is replaced by U': A is the staple sum of that link."""
    rng = np.random.default_rng(3)
    lat = oracle.Lattice(**g).hot_start(5)
    for trial in range(12):
        layer = int(rng.integers(lat.nlayers))
        site = int(rng.integers(lat.V))
        mu = int(rng.integers(lat.D))
        A = lat.staple(layer, site, mu)
        s0 = _action_sum(lat)
        M = lat.links()
        old = M[layer, site, mu].copy()
        new = _random_su3(rng)
        M[layer, site, mu] = new
        lat.set_links(M)
        s1 = _action_sum(lat)
        assert abs((s1 - s0) - np.real(np.trace((new - old) @ A))) < 1e-10


@pytest.mark.parametrize("g", GEOMS)
def test_gauge_invariance(g):
    """U_mu(x) -> g(x) U_mu(x) g(x+mu)^+ leaves plaquettes and the trace of
    closed Polyakov lines unchanged."""
    rng = np.random.default_rng(8)
    lat = oracle.Lattice(**g).hot_start(21)
    lat.sweep(5.0, 2, 4, n=1)
    p0 = [lat.plaquette(layer) for layer in range(-1, lat.nlayers)]
    q0 = [lat.polyakov(layer) for layer in range(-1, lat.nlayers)]
    tab = lat.neighbour_table().reshape(lat.nlayers * lat.V, lat.D, 2)
    G = _random_su3(rng, lat.nlayers * lat.V)
    M = lat.links().reshape(lat.nlayers * lat.V, lat.D, 3, 3)
    for mu in range(lat.D):
        M[:, mu] = G @ M[:, mu] @ G[tab[:, mu, 1]].conj().transpose(0, 2, 1)
    lat.set_links(M.reshape(lat.nlayers, lat.V, lat.D, 3, 3))
    p1 = [lat.plaquette(layer) for layer in range(-1, lat.nlayers)]
    q1 = [lat.polyakov(layer) for layer in range(-1, lat.nlayers)]
    np.testing.assert_allclose(np.array(p1), np.array(p0), atol=1e-13)
    np.testing.assert_allclose(np.array(q1), np.array(q0), atol=1e-13)


def test_plaquette_of_constant_field_strength():
    """U_1 = 1, U_2(x) = diag(e^{i phi x1}, e^{-i phi x1}, 1), phi = 2 pi/n1:
    the (1,2) plaquettes are diag(e^{i phi}, e^{-i phi}, 1) -> (1 + 2 cos phi)/3,
    every other plaquette is 1."""
    dims = [6, 4, 2, 4]
    lat = oracle.Lattice(dims).cold_start()
    M = lat.links()
    phi = 2 * np.pi / dims[0]
    for s in range(lat.V):
        x1 = lat.site_coords(s)[0]
        M[0, s, 1] = np.diag([np.exp(1j * phi * x1), np.exp(-1j * phi * x1), 1.0])
    lat.set_links(M)
    p12 = (1 + 2 * np.cos(phi)) / 3
    total, space, time = lat.plaquette()
    assert abs(total - (p12 + 5) / 6) < 1e-14
    assert abs(space - (p12 + 2) / 3) < 1e-14
    assert time == 1.0


@pytest.mark.parametrize("nlayers,glue,length", [(1, 0, 4), (2, 0b0111, 4), (2, 0b1000, 8), (2, 0b1111, 8)])
def test_polyakov_of_constant_time_links(nlayers, glue, length):
    """U_D = diag(e^{i t}, e^{i t}, e^{-2 i t}) everywhere: the closed line of
    length L gives (2 e^{i L t} + e^{-2 i L t})/3, with L = n^D, or 2 n^D on a
    DLT glued in the time direction."""
    dims = [2, 4, 2, 4]
    lat = oracle.Lattice(dims, nlayers=nlayers, glue_mask=glue).cold_start()
    M = lat.links()
    t = 0.37
    M[:, :, 3] = np.diag([np.exp(1j * t), np.exp(1j * t), np.exp(-2j * t)])
    lat.set_links(M)
    want = (2 * np.exp(1j * length * t) + np.exp(-2j * length * t)) / 3
    for layer in range(-1, nlayers):
        assert abs(lat.polyakov(layer) - want) < 1e-14


def test_hot_start_is_haar_su3():
    """Haar SU(3): <Tr U> = 0, <|Tr U|^2> = 1, <|Tr U|^4> = 2 and, special to
    SU(3) (zero for U(3)), <(Tr U)^3> = 1."""
    lat = oracle.Lattice([8, 8, 8, 8]).hot_start(12345)
    M = lat.links().reshape(-1, 3, 3)
    n = len(M)
    np.testing.assert_allclose(M @ M.conj().transpose(0, 2, 1), np.broadcast_to(np.eye(3), M.shape), atol=1e-14)
    np.testing.assert_allclose(np.linalg.det(M), 1.0, atol=1e-14)
    tr = np.trace(M, axis1=1, axis2=2)
    for f, want in [(lambda t: t, 0), (lambda t: np.abs(t) ** 2, 1), (lambda t: np.abs(t) ** 4, 2),
                    (lambda t: t ** 3, 1)]:
        v = f(tr)
        assert abs(v.mean() - want) < 5 * np.std(v) / np.sqrt(n) + 1e-12
        assert abs(exact.su3_haar_average(f) - want) < 1e-10


def test_reunitarize_matches_qr():
    """Gram-Schmidt of rows 1,2 equals the first two rows of the QR factor of
    the transpose (phases fixed so R has a positive diagonal); row 3 then
    makes the determinant one."""
    rng = np.random.default_rng(2)
    for _ in range(50):
        m = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
        r = oracle.reunitarize_matrix(m)
        q, rr = np.linalg.qr(m.T)
        ph = np.diag(rr) / np.abs(np.diag(rr))
        q = q * ph
        np.testing.assert_allclose(r[:2], q.T[:2], atol=1e-13)
        np.testing.assert_allclose(r @ r.conj().T, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(r) - 1) < 1e-14


def test_reunitarize_fixes_drift_and_keeps_su3():
    rng = np.random.default_rng(5)
    u = _random_su3(rng)
    np.testing.assert_allclose(oracle.reunitarize_matrix(u), u, atol=1e-14)
    noisy = u + 1e-6 * (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3)))
    r = oracle.reunitarize_matrix(noisy)
    np.testing.assert_allclose(r @ r.conj().T, np.eye(3), atol=1e-14)
    assert np.max(np.abs(r - u)) < 1e-5
