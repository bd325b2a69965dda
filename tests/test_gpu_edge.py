"""Degenerate and extreme cases of the method against the oracle: beta = 0
(no proposal is ever accepted, links never move), zero sweeps, strong
coupling with many hits, weak coupling where the FP32 path takes its
double-precision draw (alpha >= 32), and the largest hit count."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3
from tests.test_gpu_parity import FP32_TOL, STRONG_CEILING, _flip_check, _sensitivity

pytestmark = pytest.mark.gpu

DIMS = [4, 4, 2, 4]


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18])
def test_beta_zero_never_moves_links(storage):
    lat = su3.Lattice(DIMS, beta=0.0, seed=4, storage=storage, start=su3.SU3_START_HOT, hits=3)
    start = lat.get_links()
    lat.sweep(3)
    prop, acc, sweeps = lat.stats()
    assert np.array_equal(lat.get_links(), start)
    assert acc == 0 and prop == 3 * 3 * 3 * lat.nlinks and sweeps == 3
    booked, direct = lat.action()
    assert booked == direct == 0.0  # S = beta * (...) = 0
    o = oracle.Lattice(DIMS).hot_start(4)
    o.U[...] = start
    p, a = o.sweep(0.0, 3, 4, n=1)
    assert a == 0 and np.array_equal(o.U, start)


def test_zero_sweeps_is_a_no_op():
    lat = su3.Lattice(DIMS, beta=6.0, seed=4, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, measure_every=1)
    start = lat.get_links()
    lat.sweep(0)
    assert np.array_equal(lat.get_links(), start) and lat.stats() == (0, 0, 0)
    assert lat.measurements().shape[0] == 0


@pytest.mark.parametrize("beta,hits,start", [(0.05, 20, "hot"), (0.3, 254, "hot"), (50.0, 2, "cold"),
                                             (400.0, 1, "cold")])
def test_extreme_couplings_one_sweep(beta, hits, start):
    """FP64 link by link within 1e-11.  FP32 within 1e-5, with accept flips
    and ill-conditioned updates counted as in the parity tests; at beta = 50
    and 400 from an ordered start alpha = 2 beta k / 3 is far above 32, so
    the FP32 path runs its double-precision draw; at beta = 0.05 and 0.3
    alpha < 2 and it takes the accurate logarithm (X = -(ln u1 + c^2 ln u3)
    / alpha divides the absolute error of each logarithm by alpha)."""
    o = oracle.Lattice(DIMS)
    o = o.hot_start(21) if start == "hot" else o.cold_start()
    U0 = o.U.copy()
    margins = np.full(o.nlinks, np.inf)
    o.sweep(beta, hits, 5, n=1, margins=margins)
    for storage in (su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18):
        lat = su3.Lattice(DIMS, beta=beta, seed=5, hits=hits, storage=storage)
        lat.set_links(U0)
        lat.sweep(1)
        got = lat.get_links()
        if storage == su3.SU3_FP64_18:
            assert np.max(np.abs(got - o.U)) <= 1e-11
        else:
            probe = su3.Lattice(DIMS, storage=storage)
            probe.set_links(U0)
            start32 = probe.get_links()  # the float-rounded start (12-real: row 3 rebuilt) both sides use
            lat = su3.Lattice(DIMS, beta=beta, seed=5, hits=hits, storage=storage)
            lat.set_links(start32)
            lat.sweep(1)
            got = lat.get_links()
            sens = _sensitivity(lambda: oracle.Lattice(DIMS), start32, beta=beta, hits=hits, seed=5, n=1)
            o32 = oracle.Lattice(DIMS)
            o32.U[...] = start32
            m32 = np.full(o32.nlinks, np.inf)
            o32.sweep(beta, hits, 5, n=1, margins=m32)
            counted = _flip_check(got, o32.U, m32, sens, FP32_TOL, ceiling=STRONG_CEILING)
            # Strong coupling with many hits is ill-conditioned: at beta = 0.3
            # and 254 hits the median link moves by ~1e-6 under a one-ulp
            # perturbation of the start (six times more than at beta = 6).
            # The FP32 arithmetic of an update acts like a perturbation of
            # 10-30 ulp, so the links beyond the tolerance are at most those
            # whose sensitivity times 10 already exceeds it (measured: 83 and
            # 91 of 512 links at beta = 0.3), and every one is explained link
            # by link above.
            expected = int(np.count_nonzero(10.0 * sens > FP32_TOL))
            assert counted <= max(2, o32.nlinks // 100, expected), (counted, expected)
