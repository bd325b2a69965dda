"""Over many sweeps the FP32 GPU chains must sample what the FP64 oracle
chains sample: plaquette and |Polyakov loop| averages agree within two
combined standard deviations (the chains' trajectories themselves separate
after a few sweeps, as FP32 and FP64 rounding differ).

4^4 PBC at beta = 5.7, 2 hits, disordered starts; 8 oracle chains on the
host CPU and 128 GPU chains (one fused ensemble), 100 equilibration sweeps
and 500 measured sweeps each.  The error of each mean is the spread of the
chain means (independent chains) over sqrt(number of chains)."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3
from paper_0904_0642_gb300 import analysis

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DIMS, BETA, HITS = [4, 4, 4, 4], 5.7, 2
EQUIL, MEAS = 100, 500


def oracle_chain_means(nchains=8):
    means = []
    for c in range(nchains):
        seed = 900 + c
        o = oracle.Lattice(DIMS).hot_start(seed)
        o.sweep(BETA, HITS, seed, n=EQUIL)
        plaq, poly = [], []
        for _ in range(MEAS):
            o.sweep(BETA, HITS, seed, n=1)
            plaq.append(o.plaquette()[0])
            poly.append(abs(o.polyakov()))
        means.append((np.mean(plaq), np.mean(poly)))
    return np.array(means)


def gpu_chain_means(nchains=128):
    cfgs = [su3.make_config(DIMS, beta=BETA, seed=5000 + c, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                            hits=HITS, reunit_every=10, measure_every=1, measure_capacity=EQUIL + MEAS + 8)
            for c in range(nchains)]
    ens = su3.Ensemble(cfgs)
    ens.sweep(EQUIL + MEAS)
    means = []
    for c in range(nchains):
        m = ens.measurements(c)[EQUIL:, -1, :]  # whole lattice: total, space, time, poly re, poly im
        means.append((m[:, 0].mean(), np.hypot(m[:, 3], m[:, 4]).mean()))
    ens.close()
    return np.array(means)


def test_fp32_chains_sample_like_fp64_oracle_chains():
    g = gpu_chain_means()
    o = oracle_chain_means()
    for k, name in enumerate(("plaquette", "|Polyakov|")):
        mg, eg = g[:, k].mean(), g[:, k].std(ddof=1) / np.sqrt(len(g))
        mo, eo = o[:, k].mean(), o[:, k].std(ddof=1) / np.sqrt(len(o))
        q = analysis.gaussian_difference_q(mg, eg, mo, eo)
        assert abs(mg - mo) < 2.0 * np.hypot(eg, eo), (name, mg, eg, mo, eo, q)
        assert eo < 0.01 and eg < 0.01  # the comparison has teeth
