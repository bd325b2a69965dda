"""Sublattice decomposition on one device (the paper's MPI sublattices with
face and corner exchange, Sec. 2.4): a lattice cut into sublattice boxes
with halo layers must reproduce the undivided lattice bit for bit, and with
identical random numbers on every sublattice each sublattice must reproduce
the single-sublattice run (Sec. 3.1.1)."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu

CASES = [
    dict(dims=[8, 8, 8, 8], ndiv=[2, 2, 1, 1]),            # two cut directions: faces and corners
    dict(dims=[8, 8, 8, 8], ndiv=[2, 2, 2, 2]),            # every direction cut, time included
    dict(dims=[12, 8, 4, 4], ndiv=[3, 2, 1, 1]),
    dict(dims=[8, 4, 4, 8], ndiv=[1, 1, 1, 4]),            # sublattice extent 2 in time
    dict(dims=[8, 8, 8], ndiv=[2, 1, 2]),                  # D = 3
    dict(dims=[12, 8], ndiv=[3, 2]),                       # D = 2
    dict(dims=[4, 4, 4, 4], ndiv=[2, 1, 1, 1], boundary=su3.SU3_DLT, glue_mask=0b1111),
    dict(dims=[4, 4, 4, 4], ndiv=[1, 2, 1, 2], boundary=su3.SU3_DLT, glue_mask=0b1000),
    dict(dims=[4, 4, 4, 4], ndiv=[2, 2, 1, 1], boundary=su3.SU3_DLT, glue_mask=0b0111),
]


def pair(case, storage, **kw):
    base = dict(boundary=case.get("boundary", su3.SU3_PBC), glue_mask=case.get("glue_mask", 0), storage=storage,
                start=su3.SU3_START_HOT, **kw)
    return su3.Lattice(case["dims"], **base), su3.Lattice(case["dims"], ndiv=case["ndiv"], **base)


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18])
@pytest.mark.parametrize("case", CASES)
def test_divided_lattice_equals_undivided(case, storage):
    plain, div = pair(case, storage, beta=5.8, seed=17, hits=2, reunit_every=2)
    assert np.array_equal(plain.get_links(), div.get_links())  # same start
    plain.sweep(5)
    div.sweep(5)
    assert np.array_equal(plain.get_links(), div.get_links())
    assert plain.stats() == div.stats()
    for layer in range(-1, plain.nlayers):
        assert div.plaquette(layer) == plain.plaquette(layer)
        assert div.polyakov(layer) == plain.polyakov(layer)


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18])
def test_divided_from_given_links_and_launch_shapes(storage):
    """set_links scatters into the boxes and refills every halo; graphs,
    launch shapes and resuming do not change the result."""
    dims, ndiv = [8, 8, 4, 8], [2, 2, 1, 2]
    start = oracle.Lattice(dims).hot_start(123).U
    ref = su3.Lattice(dims, beta=6.1, seed=5, storage=storage)
    ref.set_links(start)
    ref.sweep(4)
    want = ref.get_links()
    for threads, ctas, graph in ((128, 0, True), (64, 2, False), (256, 1, True)):
        d = su3.Lattice(dims, beta=6.1, seed=5, storage=storage, ndiv=ndiv)
        d.set_links(start)
        d.set_launch(threads, ctas)
        d.use_graph(graph)
        d.sweep(2)
        saved, (_, _, n) = d.get_links(), d.stats()
        d.set_links(saved)
        d.set_sweep_counter(n)
        d.sweep(2)
        assert np.array_equal(d.get_links(), want), (threads, ctas, graph)


@pytest.mark.parametrize("mpifactor,ndmpi", [(1, 1), (2, 1), (2, 2), (2, 3), (2, 4), (3, 1), (3, 2)])
def test_identical_random_numbers_on_sublattices(mpifactor, ndmpi):
    """Sec. 3.1.1: with identical random numbers on every 4^4 sublattice
    (lsd2mpi false) the run over the (mpifactor, ndmpi) MPI lattice agrees on
    every sublattice with the run of a single 4^4 lattice."""
    ndiv = [mpifactor if i < ndmpi else 1 for i in range(4)]
    dims = [4 * k for k in ndiv]
    single = su3.Lattice([4, 4, 4, 4], beta=5.6, seed=9, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                         reunit_every=3)
    div = su3.Lattice(dims, beta=5.6, seed=9, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, reunit_every=3,
                      ndiv=ndiv, rng_period=[4, 4, 4, 4])
    single.sweep(4)
    div.sweep(4)
    s = single.get_links()[0]
    b = div.get_links()[0]
    o = oracle.Lattice(dims)
    os_ = oracle.Lattice([4, 4, 4, 4])
    for site in range(o.V):
        x = o.site_coords(site)
        assert np.array_equal(b[site], s[os_.site_index([xi % 4 for xi in x])])
    assert div.plaquette() == pytest.approx(single.plaquette(), abs=1e-14)


def test_measurements_recorded_inside_the_sweep():
    """measure_every on a divided lattice: plaquettes from the boxes and
    their forward halos; Polyakov lines when time is not cut, NaN when it is."""
    for ndiv, time_cut in (([2, 2, 2, 1], False), ([1, 2, 1, 2], True)):
        kw = dict(beta=5.9, seed=8, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, measure_every=2,
                  measure_capacity=4)
        plain = su3.Lattice([8, 8, 8, 8], **kw)
        div = su3.Lattice([8, 8, 8, 8], ndiv=ndiv, **kw)
        plain.sweep(4)
        div.sweep(4)
        mp, md = plain.measurements(), div.measurements()
        assert md.shape == mp.shape == (2, 2, 5)
        assert np.allclose(md[..., :3], mp[..., :3], rtol=0, atol=1e-14)
        if time_cut:
            assert np.isnan(md[..., 3:]).all()
        else:
            assert np.allclose(md[..., 3:], mp[..., 3:], rtol=0, atol=1e-14)


def test_action_bookkeeping_on_sublattices():
    """Sec. 2.1: each update books its action change in its own sublattice;
    the total agrees with the undivided lattice and with a direct sum."""
    plain, div = pair(dict(dims=[8, 8, 8, 8], ndiv=[2, 2, 2, 1]), su3.SU3_FP64_18, beta=5.8, seed=12, hits=2)
    plain.sweep(6)
    div.sweep(6)
    bp, dp = plain.action()
    bd, dd = div.action()
    assert dd == dp
    assert bd == pytest.approx(dd, rel=1e-11) and bd == pytest.approx(bp, rel=1e-12)


def test_divided_lattices_are_single_chains():
    cfg = su3.make_config([8, 8, 8, 8], storage=su3.SU3_FP32_12, ndiv=[2, 1, 1, 1])
    with pytest.raises(su3.Su3Error) as ei:
        su3.Ensemble([cfg])
    assert ei.value.status == su3.SU3_EINVAL
    srv = su3.Server(max_slots=2)
    with pytest.raises(su3.Su3Error) as ei:
        srv.submit(cfg, 10)
    assert ei.value.status == su3.SU3_EINVAL
    srv.close()
