"""The C ABI library loads and exports every symbol include/su3.h declares;
host-side validation rejects bad arguments before any GPU work."""
import os
import re

import pytest

import paper_0904_0642_gb300 as su3
from paper_0904_0642_gb300 import build as su3_build

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "su3.h")


@pytest.fixture(scope="module", autouse=True)
def built():
    su3_build.build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(su3_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert len(names) >= 30
    L = su3.lib()
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(su3.EXPORTED)


def test_version_and_defaults():
    assert "sm_103a" in su3.su3_version()
    c = su3.su3_config_init()
    assert c.D == 4 and list(c.dims) == [4, 4, 4, 4] and c.beta == 6.0 and c.hits == 2
    assert su3.su3_link_bytes(c) == 4 ** 4 * 4 * 144
    c.storage = su3.SU3_FP32_12
    assert su3.su3_link_bytes(c) == 4 ** 4 * 4 * 48
    c.storage = su3.SU3_FP32_18
    assert su3.su3_link_bytes(c) == 4 ** 4 * 4 * 72
    c.storage = su3.SU3_FP32_12
    c.boundary = su3.SU3_DLT
    assert su3.su3_link_bytes(c) == 2 * 4 ** 4 * 4 * 48


@pytest.mark.parametrize("change,msg", [
    (dict(dims=[4, 4, 5, 4]), "even"),
    (dict(dims=[4, 4, 0, 4]), "even"),
    (dict(beta=-1.0), "beta"),
    (dict(beta=float("nan")), "beta"),
    (dict(hits=0), "hits"),
    (dict(storage=7), "storage"),
    (dict(storage=3), "storage"),
    (dict(boundary=3), "boundary"),
    (dict(rng_period=[3, 4, 4, 4]), "rng_period"),
    (dict(glue_mask=1 << 4), "glue_mask"),
    (dict(hits=255), "hits"),
    (dict(beta1=float("inf")), "beta1"),
    (dict(reunit_every=-1), "negative"),
    (dict(dims=[256, 256, 256, 64]), "too large"),  # 2^30 sites: link storage beyond 2^31 vectors
])
def test_invalid_configs_are_rejected(change, msg):
    kw = dict(dims=[4, 4, 4, 4])
    kw.update(change)
    dims = kw.pop("dims")
    cfg = su3.make_config(dims, **kw)
    assert su3.su3_link_bytes(cfg) == 0
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_lattice_create_ex(cfg)
    assert ei.value.status == su3.SU3_EINVAL
    assert msg in str(ei.value)


def test_dimension_out_of_range():
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_lattice_create(5, [2, 2, 2, 2, 2], su3.SU3_PBC, 6.0, 1)
    assert ei.value.status == su3.SU3_EINVAL
    with pytest.raises(su3.Su3Error):
        su3.su3_lattice_create(1, [4], su3.SU3_PBC, 6.0, 1)


def test_null_handles_are_errors():
    L = su3.lib()
    assert L.su3_sweep(None, 1, 1) == su3.SU3_EINVAL
    assert L.su3_reunitarize(None) == su3.SU3_EINVAL
    assert L.su3_ensemble_sweep(None, 1) == su3.SU3_EINVAL
    assert L.su3_server_poll(None, 1, None) == su3.SU3_EINVAL
    assert "NULL" in su3.su3_last_error()


@pytest.mark.parametrize("dims,ndiv,ok", [
    ([8, 8, 8, 8], [2, 2, 1, 1], True),
    ([8, 8, 8, 8], [2, 2, 2, 2], True),
    ([12, 12, 4, 4], [3, 3, 1, 1], True),    # the paper's (mpifactor, ndmpi) = (3, 2) on 4^4 sublattices
    ([8, 8, 8, 8], [0, 1, 0, 1], True),      # 0 and 1 both mean undivided
    ([8, 8, 8, 8], [4, 1, 1, 1], True),      # sublattice extent 2
    ([6, 8, 8, 8], [3, 1, 1, 1], True),      # sublattice extent 2
    ([8, 8, 8, 8], [3, 1, 1, 1], False),     # 3 does not divide 8
    ([6, 8, 8, 8], [2, 1, 1, 1], False),     # sublattice extent 3 is odd
    ([8, 8, 8], [1, 1, 1, 2], False),        # a direction beyond D
    ([8, 8, 8, 8], [-1, 1, 1, 1], False),
])
def test_sublattice_validation(dims, ndiv, ok):
    """Sec. 2.4: sublattices of even extent (the checkerboard needs it)
    that divide the lattice exactly."""
    c = su3.make_config(dims, storage=su3.SU3_FP32_12, ndiv=ndiv)
    nbytes = su3.su3_link_bytes(c)
    if not ok:
        assert nbytes == 0
        assert "ndiv" in su3.su3_last_error()
        return
    plain = su3.su3_link_bytes(su3.make_config(dims, storage=su3.SU3_FP32_12))
    if max(ndiv) <= 1:
        assert nbytes == plain
        return
    # boxes: every sublattice padded by one halo layer per side of each cut direction
    V = 1
    nb = 1
    for n, k in zip(dims, ndiv):
        k = max(k, 1)
        nb *= k
        V *= n // k + (2 if k > 1 else 0)
    assert nbytes == plain + len(dims) * nb * V * 48


def test_sublattice_rejections():
    # a caller-owned buffer, and two couplings on a DLT cut along a glued direction
    c = su3.make_config([8, 8, 8, 8], storage=su3.SU3_FP32_12, ndiv=[2, 1, 1, 1], buffer=(1 << 20, 1 << 30))
    assert su3.su3_link_bytes(c) == 0 and "link_buffer" in su3.su3_last_error()
    c = su3.make_config([8, 8, 8, 8], boundary=su3.SU3_DLT, beta1=5.0, storage=su3.SU3_FP32_12, ndiv=[2, 1, 1, 1])
    assert su3.su3_link_bytes(c) == 0 and "two couplings" in su3.su3_last_error()
    c = su3.make_config([8, 8, 8, 8], boundary=su3.SU3_DLT, glue_mask=0b1000, beta1=5.0, storage=su3.SU3_FP32_12,
                        ndiv=[2, 1, 1, 1])
    assert su3.su3_link_bytes(c) > 0  # direction 0 is not glued


def test_fault_sites_are_validated():
    """Host-side fault injection (the server's error-path tests) accepts only
    its known sites and non-negative counts; arming and disarming needs no GPU."""
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_inject_fault("nowhere", 1)
    assert ei.value.status == su3.SU3_EINVAL
    with pytest.raises(su3.Su3Error):
        su3.su3_inject_fault("server_round", -1)
    su3.su3_inject_fault("server_round", 0)
    su3.su3_inject_fault("server_admit", 0)


def test_release_build_has_no_bounds_checks():
    """The release library compiles the device bounds checks out: no
    violation can be recorded, and the self-test is refused."""
    if os.environ.get("SU3_DEBUG_BOUNDS") == "1":
        pytest.skip("the debug-bounds library is loaded")
    assert su3.su3_bounds_status() == (0, 0, 0)
    with pytest.raises(su3.Su3Error) as ei:
        su3.su3_bounds_selftest()
    assert ei.value.status == su3.SU3_EINVAL
    assert "debug bounds" not in su3.su3_version()
