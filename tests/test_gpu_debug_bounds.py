"""The debug-bounds build (SU3_DEBUG_BOUNDS, libsu3gb300_dbg.so): device
index checks record the first violation and skip the access, with no trap.
The smallest parity geometries (one sweep against the oracle in every
storage form), re-unitarisation, measurements, a divided lattice, an
ensemble, the server and the allocation-free measurement run under the
checks without a violation; a deliberate violation (the self-test, which
checks an out-of-range index but accesses nothing) is reported by
su3_synchronize.  Runs in a child process, which loads the debug library."""
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_runs_record_no_violation_and_a_violation_is_reported():
    env = dict(os.environ, SU3_DEBUG_BOUNDS="1")
    out = subprocess.run([sys.executable, "-c", "import tests.test_gpu_debug_bounds as t; t.checked_cases()"],
                         cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-3000:]
    assert "checked ok" in out.stdout


def checked_cases():
    import oracle
    import paper_0904_0642_gb300 as su3
    from tests.test_gpu_parity import GEOMS, gpu_lattice, oracle_lattice

    assert "debug bounds" in su3.su3_version(), su3.su3_version()
    assert su3.su3_bounds_status()[0] == 0
    small = [GEOMS[i] for i in (1, 2, 3, 4, 5, 6, 7)]  # ragged tile, 2^4, D = 2, D = 3, the three DLT masks
    for g in small:
        o = oracle_lattice(g).hot_start(11)
        start = o.U.copy()
        o.sweep(6.0, 2, 99, n=1)
        for storage in (su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18):
            with gpu_lattice(g, storage, beta=6.0, seed=99, hits=2, reunit_every=1, measure_every=1) as lat:
                lat.set_links(start)
                lat.sweep(1)
                got = lat.get_links()
                lat.plaquette()
                lat.polyakov()
                lat.reunitarize()
                lat.synchronize()
            tol = 1e-11 if storage == su3.SU3_FP64_18 else 1e-3  # the FP32 forms run; their parity is tested elsewhere
            assert np.max(np.abs(got - o.U)) <= tol, (g, storage)
    # a divided lattice (sublattice boxes and halo copies), all three forms
    for storage in (su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18):
        with su3.Lattice([8, 4, 4, 4], storage=storage, start=su3.SU3_START_HOT, ndiv=[2, 2, 1, 1], seed=3,
                         reunit_every=1, measure_every=1) as lat:
            lat.sweep(2)
            lat.plaquette()
            lat.get_links()
            lat.synchronize()
    # an ensemble of mixed chains
    cfgs = [su3.make_config(d, boundary=b, seed=40 + i, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                            reunit_every=1, measure_every=1)
            for i, (d, b) in enumerate([([4, 4, 4, 4], su3.SU3_PBC), ([6, 4, 2], su3.SU3_PBC),
                                        ([4, 2, 4, 4], su3.SU3_DLT)])]
    ens = su3.Ensemble(cfgs)
    ens.sweep(2)
    ens.measure()
    ens.close()
    # the server
    srv = su3.Server(max_slots=2)
    ids = [srv.submit(c, 3) for c in cfgs]
    assert all(srv.wait(j, timeout_s=120).status == su3.SU3_OK for j in ids)
    srv.close()
    # the allocation-free measurement
    import torch
    cfg = su3.make_config([4, 4, 4, 4], storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT)
    buf = torch.empty(su3.su3_link_bytes(cfg), dtype=torch.uint8, device="cuda")
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    with su3.Lattice([4, 4, 4, 4], storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, buffer=buf) as lat:
        su3.su3_measure_noalloc(lat.cfg, buf.data_ptr(), out.data_ptr())
        lat.synchronize()
    assert su3.su3_bounds_status()[0] == 0  # raises on a recorded violation
    # the reporting path: a deliberate, recorded but never accessed violation
    su3.su3_bounds_selftest()
    with su3.Lattice([4, 4, 4, 4]) as lat:
        try:
            lat.synchronize()
        except su3.Su3Error as e:
            assert e.status == su3.SU3_ECUDA and "self-test" in str(e), str(e)
        else:
            raise AssertionError("the recorded violation was not reported")
    print("checked ok")
