"""Pins of the oracle's full checkerboard sweep.

* Symmetry tests that the paper itself uses (Sec. 3): identical random
  numbers on sublattices reproduce the small-lattice run (Sec. 3.1.1), and a
  DLT with identical numbers on both layers reproduces the PBC run (lat2test,
  Sec. 3.2).  A DLT glued only in time is the torus with twice the time
  extent, link by link.
* Closed forms: in D=2 the plaquettes of a large torus decouple, so
  <(1/3) Re Tr U_p> = z'(beta)/z(beta) (Weyl integral); in D=4 at strong
  coupling the same one-plaquette value holds up to O(u^5) (the first closed
  surface, a cube, has six plaquettes), beta/18 at leading order.
* The paper's own numbers: 4^4, beta = 5.6, ordered start (Sec. 3.1.1).
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
from tests import exact


def _paper_values():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")
    vals = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        vals[t[0]] = (float(t[1]), float(t[2]))
    return vals


def test_sweep_keeps_links_in_su3():
    lat = oracle.Lattice([4, 4, 4, 4]).hot_start(3)
    lat.sweep(6.0, 2, 1, n=3)
    M = lat.links().reshape(-1, 3, 3)
    np.testing.assert_allclose(M @ M.conj().transpose(0, 2, 1), np.broadcast_to(np.eye(3), M.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(M), 1.0, atol=1e-13)


def test_identical_random_numbers_on_sublattices():
    """Sec. 3.1.1: with identical random numbers on every 4^4 sublattice the
    8x8x4x4 lattice reproduces the 4^4 PBC run, tile by tile, bitwise."""
    small = oracle.Lattice([4, 4, 4, 4]).hot_start(77)
    big = oracle.Lattice([8, 8, 4, 4], rng_period=[4, 4, 4, 4]).hot_start(77)
    for sweep in range(3):
        small.sweep(5.7, 2, 99, n=1)
        big.sweep(5.7, 2, 99, n=1)
    s = small.links()[0]
    b = big.links()[0]
    for site in range(big.V):
        x = big.site_coords(site)
        y = [xi % 4 for xi in x]
        assert np.array_equal(b[site], s[small.site_index(y)])
    assert big.plaquette() == pytest.approx(small.plaquette(), abs=1e-15)


@pytest.mark.parametrize("glue", [0b1111, 0b0111, 0b1000])
def test_lat2test_reproduces_pbc(glue):
    """Sec. 3.2 (lat2test): identical starts and random numbers on both DLT
    layers reproduce the PBC run on each layer, bitwise."""
    dims = [4, 2, 4, 4]
    pbc = oracle.Lattice(dims).hot_start(8)
    dlt = oracle.Lattice(dims, nlayers=2, glue_mask=glue, layer_blind=True).hot_start(8)
    assert np.array_equal(dlt.U[0], pbc.U[0]) and np.array_equal(dlt.U[1], pbc.U[0])
    pbc.sweep(5.65, 2, 31, n=3)
    dlt.sweep(5.65, 2, 31, n=3)
    assert np.array_equal(dlt.U[0], pbc.U[0])
    assert np.array_equal(dlt.U[1], pbc.U[0])


def test_time_glued_dlt_is_double_time_torus():
    """Two 4x2x2x4 layers glued only in time form the 4x2x2x8 torus: the
    random-number site key is layer*V + i_s - 1, which is the site number on
    the doubled torus, so the runs agree link by link."""
    dlt = oracle.Lattice([4, 2, 2, 4], nlayers=2, glue_mask=0b1000).hot_start(5)
    tor = oracle.Lattice([4, 2, 2, 8]).hot_start(5)
    assert np.array_equal(dlt.U.reshape(-1), tor.U.reshape(-1))
    dlt.sweep(5.7, 2, 13, n=2)
    tor.sweep(5.7, 2, 13, n=2)
    assert np.array_equal(dlt.U.reshape(-1), tor.U.reshape(-1))
    assert dlt.polyakov(0) == pytest.approx(tor.polyakov(), abs=1e-15)


@pytest.mark.slow
def test_two_dimensional_plaquette_closed_form():
    beta = 3.0
    lat = oracle.Lattice([32, 32]).cold_start()
    lat.sweep(beta, 4, 17, n=50)
    series = []
    for _ in range(1200):
        lat.sweep(beta, 4, 17, n=1)
        series.append(lat.plaquette()[0])
    m, err = exact.binned_mean(np.array(series), nbins=30)
    assert abs(m - exact.su3_plaquette_mean(beta)) < 4.5 * err


@pytest.mark.slow
@pytest.mark.parametrize("beta", [0.3, 1.0])
def test_strong_coupling_four_dimensions(beta):
    lat = oracle.Lattice([4, 4, 4, 4]).hot_start(1)
    lat.sweep(beta, 12, 23, n=20)
    series = []
    for _ in range(500):
        lat.sweep(beta, 12, 23, n=1)
        series.append(lat.plaquette()[0])
    m, err = exact.binned_mean(np.array(series), nbins=25)
    assert abs(m - exact.su3_plaquette_mean(beta)) < 4.5 * err
    assert abs(m - beta / 18) < 4.5 * err + beta ** 2 / 216 * 1.2


@pytest.mark.slow
def test_paper_4x4x4x4_beta_5p6():
    """Sec. 3.1.1: act = 0.53770(18) (single process) and 0.53811(19) (MPI)
    at beta = 5.6 from an ordered start.  With a few thousand sweeps the
    oracle reaches a few 1e-3, which still rules out a wrong action."""
    vals = _paper_values()
    ref, ref_err = vals["act_4x4x4x4_b5p6_cold_single"]
    lat = oracle.Lattice([4, 4, 4, 4]).cold_start()
    lat.sweep(5.6, 1, 2024, n=300)
    series = []
    for _ in range(1500):
        lat.sweep(5.6, 1, 2024, n=2)
        series.append(lat.plaquette()[0])
    m, err = exact.binned_mean(np.array(series), nbins=15)
    assert abs(m - ref) < 4.5 * np.hypot(err, ref_err)


def test_acceptance_in_scaling_region():
    """Sec. 2.1: the 1-hit acceptance is about 97 per cent in the scaling
    region of SU(3)."""
    lat = oracle.Lattice([4, 4, 4, 4]).cold_start()
    lat.sweep(6.0, 1, 3, n=30)
    prop, acc = lat.sweep(6.0, 1, 3, n=20)
    assert 0.95 < acc / prop < 0.995


def test_threads_give_identical_sweeps():
    """OpenMP over the sites of a phase (the all-cores oracle timing): the
    links of one phase are independent and every random number is a
    function of its counter, so threads change nothing, bit for bit.  Run in
    a fresh interpreter, so that this process never starts OpenMP threads
    (later tests fork)."""
    code = (
        "import numpy as np, oracle\n"
        "dims = [4, 4, 2, 4]\n"
        "a = oracle.Lattice(dims).hot_start(3); b = oracle.Lattice(dims).hot_start(3)\n"
        "ma = np.full(a.nlinks, np.inf); mb = np.full(b.nlinks, np.inf)\n"
        "oracle.set_threads(1); sa = a.sweep(5.7, 3, 11, n=2, margins=ma)\n"
        "oracle.set_threads(4); sb = b.sweep(5.7, 3, 11, n=2, margins=mb)\n"
        "assert sa == sb, (sa, sb)\n"
        "assert np.array_equal(a.U, b.U) and np.array_equal(ma, mb)\n"
        "print('identical')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "identical" in r.stdout, r.stderr
