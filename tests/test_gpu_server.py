"""The continuous-batching job server: results equal the same job run alone,
admission respects the HBM budget, and errors are reported, not thrown."""
import time

import numpy as np
import pytest

import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu

JOBS = [
    ([8, 8, 8, 8], su3.SU3_PBC, 5.7, 40),
    ([12, 12, 12], su3.SU3_PBC, 6.2, 25),
    ([6, 6, 6, 4], su3.SU3_DLT, 5.9, 33),
    ([4, 4, 4, 4], su3.SU3_PBC, 6.0, 70),
    ([8, 8, 8, 4], su3.SU3_DLT, 5.6, 17),
    ([16, 8, 8, 8], su3.SU3_PBC, 6.4, 21),
]


def job_config(i, dims, boundary, beta):
    return su3.make_config(dims, boundary=boundary, beta=beta, seed=4242 + i, storage=su3.SU3_FP32_12,
                           start=su3.SU3_START_HOT, hits=1 + i % 2, reunit_every=10)


def alone(i, dims, boundary, beta, sweeps):
    lat = su3.Lattice(dims, boundary=boundary, beta=beta, seed=4242 + i, storage=su3.SU3_FP32_12,
                      start=su3.SU3_START_HOT, hits=1 + i % 2, reunit_every=10)
    lat.sweep(sweeps)
    return lat.plaquette(), lat.polyakov(), lat.stats()


def test_jobs_in_the_mix_equal_jobs_alone():
    srv = su3.Server(max_slots=4)
    ids = []
    for i, (dims, b, beta, sweeps) in enumerate(JOBS):
        ids.append(srv.submit(job_config(i, dims, b, beta), sweeps))
        time.sleep(0.002)  # arrivals while earlier jobs run
    results = [srv.wait(j, timeout_s=120) for j in ids]
    srv.close()
    for i, ((dims, b, beta, sweeps), r) in enumerate(zip(JOBS, results)):
        assert r.status == su3.SU3_OK
        plaq, poly, (prop, acc, _) = alone(i, dims, b, beta, sweeps)
        assert abs(r.plaquette[0] - plaq[0]) < 1e-14 and abs(r.plaquette[1] - plaq[1]) < 1e-14
        assert abs(complex(r.polyakov[0], r.polyakov[1]) - poly) < 1e-14
        assert (r.proposals, r.accepts) == (prop, acc)
        assert r.submit_s <= r.start_s <= r.finish_s


def test_admission_waits_for_memory():
    cfg = job_config(0, [16, 16, 16, 16], su3.SU3_PBC, 6.0)
    one_job = su3.su3_link_bytes(cfg)
    srv = su3.Server(hbm_budget_bytes=int(2.5 * one_job), max_slots=8)
    ids = [srv.submit(job_config(k, [16, 16, 16, 16], su3.SU3_PBC, 6.0), 30) for k in range(6)]
    most = 0
    deadline = time.time() + 120
    done = set()
    while len(done) < len(ids) and time.time() < deadline:
        q, r, f = srv.load()
        most = max(most, r)
        for j in ids:
            if j not in done and srv.poll(j) is not None:
                done.add(j)
        time.sleep(0.001)
    srv.close()
    assert len(done) == len(ids)
    assert 1 <= most <= 2  # at most two 16^4 jobs fit the budget at once


def test_errors():
    srv = su3.Server(hbm_budget_bytes=1 << 20, max_slots=2)
    with pytest.raises(su3.Su3Error) as ei:
        srv.submit(job_config(0, [16, 16, 16, 16], su3.SU3_PBC, 6.0), 10)  # larger than the budget
    assert ei.value.status == su3.SU3_ENOMEM
    with pytest.raises(su3.Su3Error) as ei:
        srv.submit(job_config(0, [4, 4, 5, 4], su3.SU3_PBC, 6.0), 10)
    assert ei.value.status == su3.SU3_EINVAL
    with pytest.raises(su3.Su3Error) as ei:
        srv.poll(987654321)
    assert ei.value.status == su3.SU3_ENOTFOUND
    j = srv.submit(job_config(0, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 100000)
    with pytest.raises(su3.Su3Error) as ei:
        srv.wait(j, timeout_s=0.05)
    assert ei.value.status == su3.SU3_ETIMEOUT
    srv.close()  # a running job ends with EBUSY when the server stops
