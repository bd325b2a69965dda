"""The continuous-batching job server: results equal the same job run alone
and match the double-precision oracle, admission respects the HBM budget,
and errors are reported, not thrown, nor left to time out."""
import time

import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3
from tests.test_gpu_parity import FLIP_MARGIN, FP32_TOL, SENS_FACTOR, _flip_check, _sensitivity

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
    rounds, device_ms = srv.stats()
    srv.close()
    # every job's ticks ran inside the worker's rounds, timed on the device
    assert rounds >= max(sweeps for *_, sweeps in JOBS) * 2 * 4 // 16
    assert 0.0 < device_ms < 1e3 * max(r.finish_s for r in results)
    for i, ((dims, b, beta, sweeps), r) in enumerate(zip(JOBS, results)):
        assert r.status == su3.SU3_OK
        plaq, poly, (prop, acc, _) = alone(i, dims, b, beta, sweeps)
        assert abs(r.plaquette[0] - plaq[0]) < 1e-14 and abs(r.plaquette[1] - plaq[1]) < 1e-14
        assert abs(complex(r.polyakov[0], r.polyakov[1]) - poly) < 1e-14
        assert (r.proposals, r.accepts) == (prop, acc)
        assert r.submit_s <= r.start_s <= r.finish_s


def test_job_alone_on_a_grid_captured_for_more_tiles():
    """The worker keeps its captured graph of ticks across admissions and
    retirements, so a job that outlives a larger one runs alone on a grid
    sized for more tiles: some CTAs run no tile.  The job must finish and
    equal the same job run alone."""
    big = (0, [8, 8, 8, 8], su3.SU3_PBC, 5.8, 12)  # 16 tiles of 128 sites
    small = (3, [4, 4, 4, 4], su3.SU3_PBC, 6.0, 60)  # 1 tile, outlives the big job
    srv = su3.Server(max_slots=4)
    ib = srv.submit(job_config(*big[:4]), big[4])
    t0 = time.time()
    while srv.stats()[0] < 1 and time.time() - t0 < 30:  # the graph is captured in the big job's first round
        time.sleep(0.001)
    js = srv.submit(job_config(*small[:4]), small[4])
    rb, rs = srv.wait(ib, timeout_s=60), srv.wait(js, timeout_s=60)
    srv.close()
    assert rb.status == su3.SU3_OK and rs.status == su3.SU3_OK
    for job, r in ((big, rb), (small, rs)):
        plaq, poly, (prop, acc, _) = alone(*job)
        assert abs(r.plaquette[0] - plaq[0]) < 1e-14
        assert (r.proposals, r.accepts) == (prop, acc)


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


# ---------------------------------------------------------------- against the oracle

SERVED = [  # dims, boundary, glue_mask, beta, seed
    ([4, 4, 4, 4], su3.SU3_PBC, 0, 5.8, 811),
    ([4, 4, 4, 4], su3.SU3_DLT, 0b1000, 5.7, 812),  # two 4^3 x 4 layers glued in time
    ([6, 6, 6], su3.SU3_PBC, 0, 6.1, 813),           # D = 3
]


def float_start(U):
    """The oracle's start as two-row float storage holds it: rows 1, 2
    rounded to float, row 3 = conj(row1 x row2) (in double here; the GPU
    rebuilds it in float, a difference of rounding size that the
    sensitivity rule of the parity tests covers)."""
    W = U.copy()
    r = W[..., :2, :, :].astype(np.float32).astype(np.float64)
    W[..., :2, :, :] = r
    c = r[..., 0] + 1j * r[..., 1]
    r3 = np.conj(np.cross(c[..., 0, :], c[..., 1, :]))
    W[..., 2, :, 0] = r3.real
    W[..., 2, :, 1] = r3.imag
    return np.ascontiguousarray(W)


def test_served_jobs_match_the_oracle():
    """Jobs submitted while others run (continuous batching; the Sec. 2.1
    update): after one sweep every link against the oracle as in the FP32
    parity tests, the proposal and acceptance counts equal unless a decision
    sits at its threshold; after three sweeps the plaquette (total, per
    layer) and the Polyakov loop within the FP32 tolerance, or within the
    sensitivity bound where that is larger."""
    srv = su3.Server(max_slots=8)
    background = [srv.submit(job_config(20 + k, [8, 8, 8, 8], su3.SU3_PBC, 6.0), 300) for k in range(3)]
    time.sleep(0.01)
    runs = []
    for dims, b, glue, beta, seed in SERVED:
        nl = 2 if b == su3.SU3_DLT else 1

        def make(dims=dims, nl=nl, glue=glue):
            return oracle.Lattice(dims, nlayers=nl, glue_mask=glue or None)

        start = float_start(make().hot_start(seed).U)
        cfg = su3.make_config(dims, boundary=b, glue_mask=glue, beta=beta, seed=seed, storage=su3.SU3_FP32_12,
                              hits=2)
        out1 = np.zeros_like(start)
        j1 = srv.submit(cfg, 1, links_in=start, links_out=out1)
        j3 = srv.submit(cfg, 3, links_in=start)
        runs.append((make, beta, seed, start, out1, j1, j3, nl))
    results = [(srv.wait(r[5], timeout_s=300), srv.wait(r[6], timeout_s=300)) for r in runs]
    bg = [srv.wait(j, timeout_s=300) for j in background]
    srv.close()
    assert all(r.status == su3.SU3_OK for r in bg)
    for (make, beta, seed, start, out1, _, _, nl), (r1, r3) in zip(runs, results):
        assert r1.status == su3.SU3_OK and r3.status == su3.SU3_OK
        # the job ran in the mix: some background job was resident meanwhile
        assert any(g.start_s <= r3.finish_s and r3.start_s <= g.finish_s for g in bg)
        # one sweep, link by link
        o1 = make()
        o1.U[...] = start
        m1 = np.full(o1.nlinks, np.inf)
        p1, a1 = o1.sweep(beta, 2, seed, n=1, margins=m1)
        sens = _sensitivity(make, start, beta=beta, hits=2, seed=seed, n=1)
        counted = _flip_check(out1, o1.U, m1, sens, FP32_TOL)
        assert counted <= max(2, o1.nlinks // 100)
        near1 = int(np.count_nonzero(m1 < FLIP_MARGIN))
        assert abs(int(r1.proposals) - p1) <= near1 and abs(int(r1.accepts) - a1) <= near1
        # three sweeps, observables
        o3 = make()
        o3.U[...] = start
        m3 = np.full(o3.nlinks, np.inf)
        p3, a3 = o3.sweep(beta, 2, seed, n=3, margins=m3)
        near3 = int(np.count_nonzero(m3 < FLIP_MARGIN))
        assert abs(int(r3.proposals) - p3) <= near3 and abs(int(r3.accepts) - a3) <= near3
        # sensitivity of the observables: the oracle from perturbed starts
        rng = np.random.default_rng(7)
        ds = 0.0
        for _ in range(4):
            q = make()
            q.U[...] = start * (1 + 2.0 ** -24 * rng.uniform(-1, 1, start.shape))
            q.sweep(beta, 2, seed, n=3)
            ds = max(ds, abs(q.plaquette()[0] - o3.plaquette()[0]), abs(q.polyakov() - o3.polyakov()))
        tol = max(FP32_TOL, SENS_FACTOR * ds)
        if near3 == 0:
            assert abs(r3.plaquette[0] - o3.plaquette()[0]) <= tol
            assert abs(r3.plaquette[1] - o3.plaquette()[1]) <= tol
            assert abs(r3.plaquette[2] - o3.plaquette()[2]) <= tol
            assert abs(complex(r3.polyakov[0], r3.polyakov[1]) - o3.polyakov()) <= tol
            for layer in range(nl):
                assert abs(r3.layer_plaquette[layer] - o3.plaquette(layer)[0]) <= tol


# ---------------------------------------------------------------- failures, injected on the host

@pytest.fixture
def disarm():
    yield
    su3.su3_inject_fault("server_admit", 0)
    su3.su3_inject_fault("server_round", 0)


def test_worker_failure_is_reported_not_a_timeout(disarm):
    srv = su3.Server(max_slots=4)
    j0 = srv.submit(job_config(0, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 5)
    assert srv.wait(j0, timeout_s=60).status == su3.SU3_OK  # the worker runs
    su3.su3_inject_fault("server_round", 1)
    j1 = srv.submit(job_config(1, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 5)
    t0 = time.time()
    with pytest.raises(su3.Su3Error) as ei:
        srv.wait(j1, timeout_s=30)
    assert ei.value.status == su3.SU3_ECUDA and "injected" in str(ei.value)
    assert time.time() - t0 < 10  # reported when it happens, not at the timeout
    with pytest.raises(su3.Su3Error) as ei:
        srv.poll(j1)
    assert ei.value.status == su3.SU3_ECUDA
    with pytest.raises(su3.Su3Error) as ei:  # the stopped worker takes no new jobs
        srv.submit(job_config(2, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 5)
    assert ei.value.status == su3.SU3_ECUDA and "worker" in str(ei.value)
    srv.close()


def test_failed_admission_fails_only_that_job(disarm):
    srv = su3.Server(max_slots=4)
    su3.su3_inject_fault("server_admit", 1)
    j1 = srv.submit(job_config(0, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 5)
    r1 = srv.wait(j1, timeout_s=60)
    assert r1.status == su3.SU3_ENOMEM
    j2 = srv.submit(job_config(1, [4, 4, 4, 4], su3.SU3_PBC, 6.0), 5)
    assert srv.wait(j2, timeout_s=60).status == su3.SU3_OK
    srv.close()

