"""Action bookkeeping (Sec. 2.1): the action booked update by update agrees
with a direct recalculation."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu


def test_booked_action_matches_direct_fp64():
    lat = su3.Lattice([8, 8, 8, 8], beta=5.8, seed=12, storage=su3.SU3_FP64_18, start=su3.SU3_START_HOT, hits=2)
    b0, d0 = lat.action()
    assert b0 == pytest.approx(d0, rel=1e-14)
    lat.sweep(20)
    b1, d1 = lat.action()
    assert abs(b1 - d1) <= 1e-11 * abs(d1)
    assert abs(d1 - d0) > 1e4  # the action did move (hot start relaxes)


def test_booked_action_matches_direct_fp32():
    """FP32-12 links: each update books (beta/3) * dReTr(U A) from the values
    in registers, while the direct sum sees the stored link, rounded to FP32
    and with its third row rebuilt from the first two.  Per update the two
    differ by at most (beta/3) |dU|_F |A|_F with |dU|_F <= sqrt(18) * 2^-23 * 2
    (rounding of two stored rows, rebuilt row) and |A|_F <= 2(D-1) sqrt(3)
    (2(D-1) SU(3) staples).  On links that drift from SU(3) the rebuilt row
    no longer matches the rotated one, so the comparison starts from a
    reunitarized lattice with a fresh reference and runs a few sweeps.

    The kernel sums the changes of a warp's 32 updates in FP32 (a 5-level
    tree) before one double add per warp: each level rounds by at most
    2^-24 times the sum of magnitudes.  One update's change of Re Tr(U A) is
    at most 3 subgroups x 2(k + |a0|) <= 12 k with k <= |A|_F / sqrt(2)."""
    beta, D, sweeps = 5.8, 4, 4
    lat = su3.Lattice([8, 8, 8, 8], beta=beta, seed=12, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, hits=2)
    lat.sweep(10)
    lat.reunitarize()
    lat.action_reset()
    _, d0 = lat.action()
    lat.sweep(sweeps)
    b1, d1 = lat.action()
    a_frob = 2 * (D - 1) * np.sqrt(3)
    per_update = beta / 3 * (np.sqrt(18) * 2.0 ** -23 * 2) * a_frob
    per_warp = beta / 3 * 5 * 2.0 ** -24 * 32 * 12 * a_frob / np.sqrt(2)
    updates = lat.nlinks * sweeps
    bound = per_update * updates + per_warp * updates / 32
    assert abs(b1 - d1) <= bound, (b1 - d1, bound)
    assert abs(d1 - d0) > 10 * bound  # the action did move


def test_cold_start_action_is_zero_then_grows():
    lat = su3.Lattice([6, 6, 6, 6], beta=6.0, seed=3, storage=su3.SU3_FP64_18)
    assert lat.action() == (0.0, 0.0)
    lat.sweep(3)
    b, d = lat.action()
    assert d > 0 and b == pytest.approx(d, rel=1e-11)


def test_reset_and_set_links():
    lat = su3.Lattice([6, 6, 6, 6], beta=6.0, seed=3, storage=su3.SU3_FP64_18, start=su3.SU3_START_HOT)
    lat.sweep(2)
    lat.reunitarize()  # not booked
    lat.action_reset()
    b, d = lat.action()
    assert b == d
    o = oracle.Lattice([6, 6, 6, 6]).hot_start(77)
    lat.set_links(o.U)  # resets the reference
    b, d = lat.action()
    assert b == d
    np_ = 6 ** 4 * 6
    assert d == pytest.approx(6.0 * np_ * (1 - o.plaquette()[0]), rel=1e-12)


def test_two_couplings_booked_change_matches_oracle_weighted_action():
    dims = [4, 4, 4, 4]
    lat = su3.Lattice(dims, boundary=su3.SU3_DLT, beta=6.0, beta1=4.5, seed=8, storage=su3.SU3_FP64_18,
                      start=su3.SU3_START_HOT, hits=2)
    o = oracle.Lattice(dims, nlayers=2)
    o.U[...] = lat.get_links()
    # S_w = sum_p beta_p (1 - P_p) = sum_p beta_p - sum_p beta_p P_p; sum_p beta_p from a cold lattice
    cold = oracle.Lattice(dims, nlayers=2).cold_start()
    sum_beta = cold.action_weighted(6.0, 4.5)
    s_before = sum_beta - o.action_weighted(6.0, 4.5)
    lat.sweep(5)
    booked, direct = lat.action()
    assert np.isnan(direct)
    o.U[...] = lat.get_links()
    s_after = sum_beta - o.action_weighted(6.0, 4.5)
    assert booked == pytest.approx(s_after - s_before, rel=1e-10)


@pytest.mark.parametrize("storage,rel,ndiv", [(su3.SU3_FP64_18, 1e-11, None), (su3.SU3_FP32_12, 2e-6, None),
                                              (su3.SU3_FP64_18, 1e-11, [2, 1, 1, 2])])
def test_apply_links_restarts_bookkeeping_at_next_measurement(storage, rel, ndiv):
    """A lattice that records measurements restarts the bookkeeping after
    su3_apply_links at its next measurement (which measures the action
    anyway): the booked action then follows the direct one from there.
    Asked before any measurement, su3_action restarts it on the spot.  Also
    for a lattice divided into sublattice boxes (measured in the boxes)."""
    dims = [4, 6, 6, 4] if ndiv else [6, 6, 6, 6]
    lat = su3.Lattice(dims, beta=6.0, seed=3, storage=storage, start=su3.SU3_START_HOT, measure_every=5,
                      reunit_every=5, ndiv=ndiv)
    start = oracle.Lattice(dims).hot_start(77).U
    lat.sweep(7)
    lat.stage_links(start)
    lat.apply_links()
    lat.sweep(8)  # the restart is the measurement after sweep 5 of these
    meas = lat.measurements()[-2]  # that measurement (the last one is after sweep 10)
    b, d = lat.action()
    assert b == pytest.approx(d, rel=rel)
    np_ = int(np.prod(dims)) * 6
    assert meas.shape == (2, 5)
    lat.stage_links(start)
    lat.apply_links()
    b, d = lat.action()  # no measurement since: restarted now
    assert b == d
    assert d == pytest.approx(6.0 * np_ * (1 - oracle.Lattice(dims).hot_start(77).plaquette()[0]), rel=1e-6)
    lat.sweep(3)
    b, d = lat.action()
    assert b == pytest.approx(d, rel=rel)


def test_autotune_leaves_the_bookkeeping_alone():
    """The autotuner's timing sweeps run on saved links and restore them
    afterwards, together with the booked changes: the booked action still
    follows the direct one."""
    lat = su3.Lattice([8, 8, 8, 8], beta=5.8, seed=21, storage=su3.SU3_FP64_18, start=su3.SU3_START_HOT, hits=2)
    lat.sweep(3)
    b0, d0 = lat.action()
    lat.autotune()
    b1, d1 = lat.action()
    assert d1 == d0 and b1 == pytest.approx(b0, rel=1e-15)
    lat.sweep(2)
    b2, d2 = lat.action()
    assert b2 == pytest.approx(d2, rel=1e-11)
