"""The multi-rank (replica) path on CPU: two gloo ranks, each advancing its
own chain (the oracle stands in for the GPU step), with the barrier and
max-over-ranks timing that bench.py uses on GPUs."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import time

    import oracle
    from paper_0904_0642_gb300.replicas import Replicas

    reps = Replicas("gloo")
    lat = oracle.Lattice([4, 4, 4, 4]).hot_start(reps.seed(100))
    reps.barrier()
    t0 = time.perf_counter()
    for _ in range(2 + rank):  # rank 1 is deliberately slower
        lat.sweep(6.0, 2, reps.seed(100), n=1)
    dt = time.perf_counter() - t0
    tmax = reps.max(dt)
    value = reps.rate(2 * lat.nlinks, dt)
    out[rank] = (dt, tmax, value, lat.plaquette()[0])
    reps.close()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_time_by_the_slowest_rank():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
    (dt0, max0, v0, p0), (dt1, max1, v1, p1) = out[0], out[1]
    assert max0 == max1 == max(dt0, dt1)              # every rank agrees on the slowest time
    assert v0 == v1 == pytest.approx(world * 2 * 1024 / max(dt0, dt1))
    assert p0 != p1                                    # independent chains (seed per rank)


def test_single_process_is_a_world_of_one():
    from paper_0904_0642_gb300.replicas import Replicas
    r = Replicas()
    assert (r.world, r.rank) == (1, 0)
    assert r.max(2.5) == 2.5
    assert r.rate(100, 2.0) == 50.0
    assert r.seed(7) == 7
