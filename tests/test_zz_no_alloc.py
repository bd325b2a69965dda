"""The allocation-free measurement entry point, su3_measure_noalloc.

Some callers cannot call cudaMalloc: a host framework whose memory pool must
own all device memory, loops that cannot take the synchronisation an
allocation may cause, plug-ins under a fixed memory budget.  For them the
library measures links the caller holds, with its scratch in a fixed array
inside the library.  These tests compare it with the allocating entry point
su3_measure_async on the same links, on two calls in a row.  The file sorts
last so that a run stopping at the first failure has run every other test.
"""
import numpy as np
import pytest

import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

CASES = [
    dict(dims=[8, 8, 8, 8], boundary=su3.SU3_PBC, storage=su3.SU3_FP32_12),
    dict(dims=[6, 4, 8, 6], boundary=su3.SU3_PBC, storage=su3.SU3_FP64_18),
    dict(dims=[6, 4, 8, 6], boundary=su3.SU3_PBC, storage=su3.SU3_FP32_18),
    dict(dims=[8, 8, 8, 4], boundary=su3.SU3_DLT, storage=su3.SU3_FP32_12),
    dict(dims=[32, 32, 32, 32], boundary=su3.SU3_PBC, storage=su3.SU3_FP32_12),
    # exactly the capacity of the static scratch: 64^4 / 2 / 256 = 32768 tiles
    dict(dims=[64, 64, 64, 64], boundary=su3.SU3_PBC, storage=su3.SU3_FP32_12, sweeps=0),
]


def geometry_only_config(dims, boundary, storage):
    """A zero-filled config with only the fields the call reads: hits = 0,
    start = 0 and every cadence 0, which a lattice would reject."""
    c = su3.su3_config()
    c.D = len(dims)
    for i, n in enumerate(dims):
        c.dims[i] = n
    c.boundary = boundary
    c.storage = storage
    return c


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{'x'.join(map(str, c['dims']))}-b{c['boundary']}-s{c['storage']}")
def test_noalloc_matches_allocating_entry_point(case):
    stream = torch.cuda.Stream()
    cfg = su3.make_config(case["dims"], boundary=case["boundary"], storage=case["storage"], beta=5.8, seed=31,
                          start=su3.SU3_START_HOT)
    nbytes = su3.su3_link_bytes(cfg)
    buf = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    lat = su3.Lattice(case["dims"], boundary=case["boundary"], storage=case["storage"], beta=5.8, seed=31,
                      start=su3.SU3_START_HOT, stream=stream, buffer=buf)
    nvals = 5 * (lat.nlayers + 1)
    bare = geometry_only_config(case["dims"], case["boundary"], case["storage"])
    for call in range(2):  # two calls in a row share the static scratch
        lat.sweep(case.get("sweeps", 2))
        want = torch.zeros(nvals, dtype=torch.float64, device="cuda")
        got = torch.full((nvals,), float("nan"), dtype=torch.float64, device="cuda")
        su3.su3_measure_async(lat.h, want.data_ptr())
        # the lattice's own config on the first call, the bare geometry on the second
        su3.su3_measure_noalloc(lat.cfg if call == 0 else bare, buf.data_ptr(), got.data_ptr(), stream=stream)
        stream.synchronize()
        np.testing.assert_allclose(got.cpu().numpy(), want.cpu().numpy(), rtol=0, atol=1e-13)
        assert abs(got[-5].item() - lat.plaquette()[0]) < 1e-13
    lat.close()


@pytest.mark.parametrize("dims,boundary", [([64, 64, 64, 66], su3.SU3_PBC),   # 33792 tiles
                                           ([64, 64, 64, 34], su3.SU3_DLT)])  # 2 layers x 17408 tiles
def test_noalloc_rejects_lattices_beyond_the_scratch(dims, boundary):
    # rejected before anything is launched: the buffer is never read
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")
    out = torch.empty(15, dtype=torch.float64, device="cuda")
    cfg = su3.make_config(dims, boundary=boundary, storage=su3.SU3_FP32_12)
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_measure_noalloc(cfg, buf.data_ptr(), out.data_ptr())
    assert ei.value.status == su3.SU3_EINVAL
    assert "static scratch" in str(ei.value)


def test_noalloc_validates_only_the_geometry():
    buf = torch.empty(1024, dtype=torch.uint8, device="cuda")
    out = torch.empty(15, dtype=torch.float64, device="cuda")
    bad = geometry_only_config([4, 4, 5, 4], su3.SU3_PBC, su3.SU3_FP32_12)  # odd extent
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_measure_noalloc(bad, buf.data_ptr(), out.data_ptr())
    assert ei.value.status == su3.SU3_EINVAL and "even" in str(ei.value)
    bad = geometry_only_config([4, 4, 4, 4], su3.SU3_PBC, 7)  # unknown storage
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_measure_noalloc(bad, buf.data_ptr(), out.data_ptr())
    assert ei.value.status == su3.SU3_EINVAL and "storage" in str(ei.value)
