"""The GPU path (FP32 links) against the paper's published plaquette values.

Each check runs an ensemble of independent chains: equilibration sweeps,
then measurements every 2 sweeps.  The error of the mean comes from the
spread of the chain means (chains are independent), and the comparison is
the paper's Gaussian difference test (Sec. 3.1): the two values must agree
within 4 combined standard deviations.  The paper's runs use nhit = 1
(mc.par, Sec. 2.3).
"""
import os

import numpy as np
import pytest

import paper_0904_0642_gb300 as su3

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


def paper_values():
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_values.txt")
    vals = {}
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        t = line.split()
        vals[t[0]] = (float(t[1]), float(t[2]))
    return vals


def run_ensemble(dims, beta, nchains, equil, nmeas_sweeps, start, boundary=su3.SU3_PBC, glue_mask=0, seed0=1,
                 hits=1):
    every = 2
    cfgs = [su3.make_config(dims, boundary=boundary, glue_mask=glue_mask, beta=beta, seed=seed0 + c,
                            storage=su3.SU3_FP32_12, start=start, hits=hits, reunit_every=10, measure_every=every,
                            measure_capacity=(equil + nmeas_sweeps) // every + 8) for c in range(nchains)]
    ens = su3.Ensemble(cfgs)
    ens.sweep(equil + nmeas_sweeps)
    skip = equil // every
    means = []
    for c in range(nchains):
        m = ens.measurements(c)[skip:, -1, :3]  # whole lattice: total, space, time
        means.append(m.mean(axis=0))
    means = np.array(means)
    return means.mean(axis=0), means.std(axis=0, ddof=1) / np.sqrt(nchains)


def gaussian_difference_ok(a, ea, b, eb, nsigma=4.0):
    return abs(a - b) < nsigma * np.hypot(ea, eb)


def test_sec311_four_to_the_four_beta_5p6():
    """Sec. 3.1.1, eqs. (act1MPI), (act1noMPI): 4^4, beta = 5.6, ordered start."""
    v = paper_values()
    mean, err = run_ensemble([4, 4, 4, 4], 5.6, 128, 500, 4000, su3.SU3_START_COLD)
    for key in ("act_4x4x4x4_b5p6_cold_single", "act_4x4x4x4_b5p6_cold_mpi"):
        ref, ref_err = v[key]
        assert gaussian_difference_ok(mean[0], err[0], ref, ref_err), (key, mean[0], err[0])


def test_table1_8x8x8x4_beta_5p65():
    """Table 1, first row: periodic 8^3 x 4 at beta = 5.65, 0.538547(70)."""
    v = paper_values()
    ref, ref_err = v["act_8x8x8x4_b5p65_nonmpi"]
    mean, err = run_ensemble([8, 8, 8, 4], 5.65, 64, 500, 4000, su3.SU3_START_COLD, seed0=100)
    assert gaussian_difference_ok(mean[0], err[0], ref, ref_err), (mean[0], err[0])


def test_table2_16x16x16x4_space_and_time():
    """Table 2: 16^3 x 4 at beta = 5.65, space- and time-like plaquettes
    against the literature values (row B) and the paper's non-MPI run."""
    v = paper_values()
    mean, err = run_ensemble([16, 16, 16, 4], 5.65, 64, 400, 3000, su3.SU3_START_COLD, seed0=300)
    for key, k in (("plaq_16x16x16x4_b5p65_space_Bo96", 1), ("plaq_16x16x16x4_b5p65_time_Bo96", 2),
                   ("plaq_16x16x16x4_b5p65_space_nonmpi", 1), ("plaq_16x16x16x4_b5p65_time_nonmpi", 2)):
        ref, ref_err = v[key]
        assert gaussian_difference_ok(mean[k], err[k], ref, ref_err), (key, mean[k], err[k])


def test_table3_double_layered_torus_beta_5p55():
    """Table 3, first row: two 8^3 x 4 layers glued in all directions (the
    paper's first DLT option), beta = 5.55, disordered start: 0.510608(33)."""
    v = paper_values()
    ref, ref_err = v["act_dlt_8x8x8x4_b5p55_hot_np2"]
    mean, err = run_ensemble([8, 8, 8, 4], 5.55, 64, 600, 4000, su3.SU3_START_HOT, boundary=su3.SU3_DLT,
                             glue_mask=0b1111, seed0=700)
    assert gaussian_difference_ok(mean[0], err[0], ref, ref_err), (mean[0], err[0])
