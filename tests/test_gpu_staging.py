"""Asynchronous link input (su3_stage_links / su3_apply_links): the same
result as su3_set_links, with the copy overlapping queued sweeps."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage,ndiv", [(su3.SU3_FP64_18, None), (su3.SU3_FP32_12, None),
                                          (su3.SU3_FP32_12, [2, 1, 2, 1]), (su3.SU3_FP32_18, None),
                                          (su3.SU3_FP32_18, [2, 1, 2, 1])])
def test_stage_apply_equals_set_links(storage, ndiv):
    dims = [8, 8, 4, 4]
    l1 = oracle.Lattice(dims).hot_start(41).U.copy()
    l2 = oracle.Lattice(dims).hot_start(42).U.copy()
    kw = dict(beta=5.9, seed=3, storage=storage, start=su3.SU3_START_HOT, ndiv=ndiv)
    ref = su3.Lattice(dims, **kw)
    ref.set_links(l1)
    ref.sweep(4)
    ref.set_links(l2)
    ref.sweep(3)
    lat = su3.Lattice(dims, **kw)
    lat.stage_links(l1)
    lat.apply_links()
    lat.sweep(4)
    lat.stage_links(l2)  # copied while the four sweeps run
    lat.apply_links()
    lat.sweep(3)
    assert np.array_equal(lat.get_links(), ref.get_links())
    assert lat.stats() == ref.stats()
    b, d = lat.action()
    br, dr = ref.action()
    assert d == dr and b == pytest.approx(br, rel=1e-13)


def test_pinned_host_buffer_and_measurement_in_stream_order():
    torch = pytest.importorskip("torch")
    dims = [16, 16, 16, 16]
    start = su3.Lattice(dims, seed=5, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT).get_links()
    host = torch.empty(start.size, dtype=torch.float64, pin_memory=True).numpy()
    host[:] = start.reshape(-1)
    stream = torch.cuda.Stream()
    lat = su3.Lattice(dims, beta=6.0, seed=6, storage=su3.SU3_FP32_12, stream=stream)
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    lat.stage_links(host)
    vals = []
    for k in range(3):
        lat.apply_links()
        lat.sweep(2)
        if k < 2:
            lat.stage_links(host)
        lat.measure_into(out.data_ptr())
        with torch.cuda.stream(stream):
            vals.append(out.cpu().numpy().copy())
    ref = su3.Lattice(dims, beta=6.0, seed=6, storage=su3.SU3_FP32_12)
    for k in range(3):
        ref.set_links(start)
        ref.sweep(2)
        t, s_, ti = ref.plaquette()
        p = ref.polyakov()
        assert np.allclose(vals[k][5:], [t, s_, ti, p.real, p.imag], rtol=0, atol=1e-15)


def test_staging_errors():
    lat = su3.Lattice([4, 4, 4, 4], storage=su3.SU3_FP32_12)
    with pytest.raises(su3.Su3Error) as ei:
        lat.apply_links()
    assert ei.value.status == su3.SU3_EINVAL
    links = lat.get_links()
    lat.stage_links(links)
    with pytest.raises(su3.Su3Error) as ei:
        lat.stage_links(links)
    assert ei.value.status == su3.SU3_EBUSY
    lat.apply_links()
    with pytest.raises(su3.Su3Error) as ei:
        lat.stage_links(links[:, :10])
    assert ei.value.status == su3.SU3_EINVAL


@pytest.mark.parametrize("storage", [su3.SU3_FP32_12, su3.SU3_FP64_18, su3.SU3_FP32_18])
def test_two_row_float_input(storage):
    """SU3_LINKS_FP32_12: rows 1, 2 as float, row 3 rebuilt.  For FP32 12-real
    storage this is exactly what set_links stores from the same values."""
    dims = [6, 4, 4, 4]
    canon = oracle.Lattice(dims).hot_start(8).U
    rows = canon[..., :2, :, :].astype(np.float32)  # [layer, site, mu, row 1..2, col, re/im]
    a = su3.Lattice(dims, storage=storage)
    a.stage_links(rows, fmt=su3.SU3_LINKS_FP32_12)
    a.apply_links()
    got = a.get_links()
    if storage == su3.SU3_FP32_12:
        b = su3.Lattice(dims, storage=storage)
        b.set_links(canon.astype(np.float32).astype(np.float64))
        assert np.array_equal(got, b.get_links())
    # row 3 = conj(row1 x row2) of the float rows, within float rounding
    assert np.max(np.abs(got - canon)) < 2e-6


def test_latest_measurement():
    lat = su3.Lattice([6, 6, 6, 6], beta=6.0, seed=2, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                      measure_every=2, measure_capacity=3)
    with pytest.raises(su3.Su3Error) as ei:
        lat.latest_measurement()
    assert ei.value.status == su3.SU3_ENOTFOUND
    lat.sweep(10)  # 5 measurements in a ring of 3
    assert np.array_equal(lat.latest_measurement(), lat.measurements()[-1])


def test_latest_measurement_async_pipeline():
    """su3_measurement_latest_async copies, in stream order, the measurement
    of the sweeps queued before it: a pipelined loop that reads step k's
    result while step k+1 runs gets every step's result, equal to the ring
    read afterwards; sweeps no longer wait for the queued work."""
    import torch
    stream = torch.cuda.Stream()
    lat = su3.Lattice([6, 6, 6, 4], beta=5.9, seed=7, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                      measure_every=5, measure_capacity=64, reunit_every=5, stream=stream)
    out = np.zeros(4, dtype=np.float64)
    with pytest.raises(su3.Su3Error) as ei:
        lat.latest_measurement_async(np.zeros(10))
    assert ei.value.status == su3.SU3_ENOTFOUND
    with pytest.raises(su3.Su3Error):
        lat.sweep(5)
        lat.latest_measurement_async(out)  # too small for 5 * 2 values
    lat.synchronize()
    bufs = [torch.empty(10, dtype=torch.float64, pin_memory=True).numpy() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    got = []
    for k in range(6):
        lat.sweep(5)
        lat.latest_measurement_async(bufs[k % 2])
        evs[k % 2].record(stream)
        if k >= 1:
            evs[(k - 1) % 2].synchronize()
            got.append(bufs[(k - 1) % 2].copy())
    evs[1].synchronize()
    got.append(bufs[1].copy())
    ring = lat.measurements()  # one per 5 sweeps: the first from the sweep above, then six
    assert ring.shape[0] == 7
    for k in range(6):
        assert np.array_equal(got[k].reshape(2, 5), ring[k + 1])
