"""The oracle's pins must catch plausible mistakes.

Each case plants one mistake (a dropped term, a wrong sign, index or
operand order) in a temporary copy of oracle/su3_oracle.c, builds it, and
requires that at least one of the quick pin checks below fails.  This runs on
the CPU only and never touches the GPU path.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from tests import exact

SRC = os.path.join(os.path.dirname(oracle.__file__), "su3_oracle.c")

MUTATIONS = {
    "alpha_factor": ("double alpha = 2.0 * beta * k / 3.0;", "double alpha = beta * k / 3.0;"),
    "a2_sign": ("a[2] = 0.5 * (creal(W.m[i][j]) - creal(W.m[j][i]));",
                "a[2] = 0.5 * (creal(W.m[i][j]) + creal(W.m[j][i]));"),
    "a1_sign": ("a[1] = 0.5 * (cimag(W.m[i][j]) + cimag(W.m[j][i]));",
                "a[1] = 0.5 * (cimag(W.m[i][j]) - cimag(W.m[j][i]));"),
    "w_operand_order": ("mat3 W = m_mul(U, A);", "mat3 W = m_mul(A, U);"),
    "r_not_daggered": ("r[p][q] = xm[p][0] * conj(vm[q][0]) + xm[p][1] * conj(vm[q][1]);",
                       "r[p][q] = xm[p][0] * vm[0][q] + xm[p][1] * vm[1][q];"),
    "staple_missing_dagger": ("mat3 b = link_at(g, U, ln, sn, mu); b = m_dag(&b);",
                              "mat3 b = link_at(g, U, ln, sn, mu);"),
    "staple_wrong_site": ("orc_neighbour(g, lp, sp, nu, -1, &lpm, &spm);",
                          "orc_neighbour(g, layer, s, nu, -1, &lpm, &spm);"),
    "staple_dropped_lower": ("    A = m_add(&A, &dn);\n", "\n"),
    "kp_dropped_cos2": ("X = -(log(u[0]) + c * c * log(u[2])) / alpha;", "X = -(log(u[0]) + log(u[2])) / alpha;"),
    "kp_accept_not_squared": ("double lhs = u[3] * u[3], rhs", "double lhs = u[3], rhs"),
    "direction_radius": ("double rho = sqrt(X * (2.0 - X));", "double rho = sqrt(X * (1.0 - X));"),
    "direction_not_isotropic": ("double costh = 2.0 * u5 - 1.0;", "double costh = u5;"),
    "direction_words_repeated": ("double u5 = subgroup == 1 ? u[2] : u[0], u6 = subgroup == 1 ? u[3] : u[1];",
                                 "double u5 = u[0], u6 = u[1];"),
    "plaquette_missing_dagger": ("mat3 c = link_at(g, U, ln, sn, mu); c = m_dag(&c);\n  mat3 d",
                                 "mat3 c = link_at(g, U, ln, sn, mu);\n  mat3 d"),
    "plaquette_time_split": ("if (nu == D - 1) { sum_t", "if (mu == 0) { sum_t"),
    "dlt_no_layer_flip": ("l = 1 - layer;", "l = layer;"),
    "philox_constant": ("uint64_t p0 = (uint64_t)0xD2511F53u * c0;", "uint64_t p0 = (uint64_t)0xD2511F55u * c0;"),
    "philox_key_bump": ("k0 += 0x9E3779B9u;", "k0 += 0x9E3779B8u;"),
    "reunit_inner_product": ("p += conj(a->m[0][k]) * a->m[1][k];", "p += a->m[0][k] * conj(a->m[1][k]);"),
    "third_row_not_conjugated": ("a->m[2][2] = conj(a->m[0][0] * a->m[1][1] - a->m[0][1] * a->m[1][0]);",
                                 "a->m[2][2] = a->m[0][0] * a->m[1][1] - a->m[0][1] * a->m[1][0];"),
    "hot_start_rows_equal": ("a.m[1][k] = gauss[6 + 2 * k] + I * gauss[6 + 2 * k + 1];",
                             "a.m[1][k] = gauss[2 * k] + I * gauss[2 * k + 1] + 1e-9;"),
    "sweep_ignores_colour": ("if (orc_colour(g, x) != colour) continue;", ""),
    "polyakov_open_line": ("} while (!(cl == l && cs == s));", "} while (0);"),
    "two_beta_tag_base_only": ("double b_up = (layer + lp + ln + layer) ? beta1 : beta0;",
                               "double b_up = (layer) ? beta1 : beta0;"),
    "two_beta_lower_tags": ("double b_dn = (lm + lpm + layer + lm) ? beta1 : beta0;",
                            "double b_dn = (lm + layer) ? beta1 : beta0;"),
}


def _random_su3(rng):
    z = (rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))) / np.sqrt(2)
    q, r = np.linalg.qr(z)
    q = q * (np.diag(r) / np.abs(np.diag(r)))
    return q / np.linalg.det(q) ** (1 / 3)


# ----------------------------------------------------------- quick pin checks


def check_philox():
    assert oracle.philox4x32_10([0, 0, 0, 0], [0, 0]) == [0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]


def check_dlt_neighbours():
    lat = oracle.Lattice([4, 2], nlayers=2, glue_mask=0b11)
    tab = lat.neighbour_table()
    assert tab[0, 3, 0, 1] == lat.V + 0  # x1 = 3 -> 0 crosses into layer 1


def check_su2():
    x, acc = oracle.su2_samples(2.0, 100, 1, 60_000)
    a = x[acc]
    np.testing.assert_allclose(np.sum(a * a, axis=1), 1.0, atol=1e-13)
    assert abs(a[:, 0].mean() - exact.su2_a0_mean(2.0)) < 5 * a[:, 0].std() / np.sqrt(len(a))
    assert np.all(np.abs(a[:, 1:].mean(axis=0)) < 5 * a[:, 1:].std(axis=0) / np.sqrt(len(a)))
    _, acc1 = oracle.su2_samples(4.0, 1, 2, 60_000)
    p = exact.kp_acceptance(4.0)
    assert abs(acc1.mean() - p) < 5 * np.sqrt(p * (1 - p) / len(acc1))
    # the subgroups' directions at one counter are independent
    v = [oracle.su2_samples(3.0, 50, 4, 20_000, subgroup=sg)[0][:, 1:] for sg in range(3)]
    v = [w / np.linalg.norm(w, axis=1, keepdims=True) for w in v]
    for a, b in [(0, 1), (0, 2), (1, 2)]:
        assert abs(np.sum(v[a] * v[b], axis=1).mean()) < 5 * np.sqrt(1 / 3 / 20_000)


def check_frozen_staple():
    rng = np.random.default_rng(7)
    V = _random_su3(rng)
    series = oracle.link_chain(6.0 * V, 1.0, 20, 3, 40_000)
    m, err = exact.binned_mean(series[1000:] / 18.0, nbins=20)
    assert abs(m - exact.su3_plaquette_mean(6.0)) < 5 * err


def check_local_action_and_gauge():
    rng = np.random.default_rng(3)
    for kw in (dict(dims=[2, 4, 2, 4]), dict(dims=[2, 4, 2, 4], nlayers=2, glue_mask=0b1010)):
        lat = oracle.Lattice(**kw).hot_start(5)
        nplaq = lat.nlayers * lat.V * 6
        for _ in range(4):
            layer, site, mu = int(rng.integers(lat.nlayers)), int(rng.integers(lat.V)), int(rng.integers(4))
            A = lat.staple(layer, site, mu)
            s0 = 3 * nplaq * lat.plaquette()[0]
            M = lat.links()
            old = M[layer, site, mu].copy()
            new = _random_su3(rng)
            M[layer, site, mu] = new
            lat.set_links(M)
            s1 = 3 * nplaq * lat.plaquette()[0]
            assert abs((s1 - s0) - np.real(np.trace((new - old) @ A))) < 1e-9
        p0 = lat.plaquette()
        tab = lat.neighbour_table().reshape(lat.nlayers * lat.V, 4, 2)
        G = np.array([_random_su3(rng) for _ in range(lat.nlayers * lat.V)])
        M = lat.links().reshape(lat.nlayers * lat.V, 4, 3, 3)
        for mu in range(4):
            M[:, mu] = G @ M[:, mu] @ G[tab[:, mu, 1]].conj().transpose(0, 2, 1)
        lat.set_links(M.reshape(lat.nlayers, lat.V, 4, 3, 3))
        np.testing.assert_allclose(lat.plaquette(), p0, atol=1e-12)


def check_closed_form_configs():
    lat = oracle.Lattice([6, 4, 2, 4]).cold_start()
    M = lat.links()
    phi = 2 * np.pi / 6
    for s in range(lat.V):
        x1 = lat.site_coords(s)[0]
        M[0, s, 1] = np.diag([np.exp(1j * phi * x1), np.exp(-1j * phi * x1), 1.0])
    lat.set_links(M)
    p12 = (1 + 2 * np.cos(phi)) / 3
    t, s_, ti = lat.plaquette()
    assert abs(s_ - (p12 + 2) / 3) < 1e-13 and ti == 1.0
    lat = oracle.Lattice([2, 2, 2, 4]).cold_start()
    M = lat.links()
    M[:, :, 3] = np.diag([np.exp(0.3j), np.exp(0.3j), np.exp(-0.6j)])
    lat.set_links(M)
    assert abs(lat.polyakov() - (2 * np.exp(1.2j) + np.exp(-2.4j)) / 3) < 1e-13


def check_reunit_and_hot_start():
    rng = np.random.default_rng(2)
    m = rng.standard_normal((3, 3)) + 1j * rng.standard_normal((3, 3))
    r = oracle.reunitarize_matrix(m)
    np.testing.assert_allclose(r @ r.conj().T, np.eye(3), atol=1e-13)
    assert abs(np.linalg.det(r) - 1) < 1e-13
    lat = oracle.Lattice([2, 2, 2, 2]).hot_start(4)
    M = lat.links().reshape(-1, 3, 3)
    np.testing.assert_allclose(M @ M.conj().transpose(0, 2, 1), np.broadcast_to(np.eye(3), M.shape), atol=1e-13)


def check_sweep():
    lat = oracle.Lattice([4, 4, 2, 2]).hot_start(3)
    prop, acc = lat.sweep(6.0, 1, 5, n=2)
    assert prop == 2 * 3 * lat.nlinks  # one hit per subgroup: every link updated once per sweep
    M = lat.links().reshape(-1, 3, 3)
    np.testing.assert_allclose(M @ M.conj().transpose(0, 2, 1), np.broadcast_to(np.eye(3), M.shape), atol=1e-12)
    lat = oracle.Lattice([4, 4, 4, 4]).hot_start(1)
    lat.sweep(1.0, 12, 2, n=10)
    series = []
    for _ in range(150):
        lat.sweep(1.0, 12, 2, n=1)
        series.append(lat.plaquette()[0])
    m, err = exact.binned_mean(np.array(series), nbins=15)
    assert abs(m - exact.su3_plaquette_mean(1.0)) < 5 * err


def check_two_beta():
    rng = np.random.default_rng(5)
    lat = oracle.Lattice([2, 4, 2, 4], nlayers=2, glue_mask=0b1111).hot_start(3)
    for _ in range(6):
        layer, site, mu = int(rng.integers(2)), int(rng.integers(lat.V)), int(rng.integers(4))
        A = lat.staple_weighted(layer, site, mu, 5.0, 2.0)
        s0 = lat.action_weighted(5.0, 2.0)
        M = lat.links()
        old = M[layer, site, mu].copy()
        new = _random_su3(rng)
        M[layer, site, mu] = new
        lat.set_links(M)
        s1 = lat.action_weighted(5.0, 2.0)
        assert abs(3 * (s1 - s0) - np.real(np.trace((new - old) @ A))) < 1e-9


CHECKS = [check_philox, check_dlt_neighbours, check_closed_form_configs, check_reunit_and_hot_start,
          check_local_action_and_gauge, check_su2, check_sweep, check_frozen_staple, check_two_beta]


def test_unmutated_oracle_passes_quick_checks():
    for check in CHECKS:
        check()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = tmp_path / "mut.c"
    mutated.write_text(src.replace(old, new, 1))
    so = tmp_path / f"libmut_{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so),
                           str(mutated), "-lm"])
    caught = []
    with oracle.use_library(str(so)):
        for check in CHECKS:
            try:
                with np.errstate(all="ignore"):
                    check()
            except (AssertionError, ValueError, FloatingPointError, np.linalg.LinAlgError):
                caught.append(check.__name__)
                break
    assert caught, f"mutation {name} passed every pin"
