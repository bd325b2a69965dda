"""GPU engine behaviour: invariances that must hold bit for bit (the paper's
sublattice and lat2test checks, graphs, launch shapes, batching, resume),
and full-size parity on sampled links against the oracle."""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18])
def test_identical_random_numbers_on_sublattices(storage):
    """Sec. 3.1.1: with the random-number site key taken modulo a 4^4
    sublattice, the 8x8x8x4 lattice reproduces the 4^4 run on every tile."""
    small = su3.Lattice([4, 4, 4, 4], beta=5.6, seed=9, storage=storage, start=su3.SU3_START_HOT)
    big = su3.Lattice([8, 8, 8, 4], beta=5.6, seed=9, storage=storage, start=su3.SU3_START_HOT,
                      rng_period=[4, 4, 4, 4])
    small.sweep(3)
    big.sweep(3)
    s = small.get_links()[0]
    b = big.get_links()[0]
    o = oracle.Lattice([8, 8, 8, 4])
    os_ = oracle.Lattice([4, 4, 4, 4])
    for site in range(o.V):
        x = o.site_coords(site)
        assert np.array_equal(b[site], s[os_.site_index([xi % 4 for xi in x])])


@pytest.mark.parametrize("glue", [0b1111, 0b1000, 0b0111])
def test_lat2test_reproduces_pbc(glue):
    """Sec. 3.2: identical numbers on both DLT layers reproduce the PBC run."""
    dims = [4, 4, 2, 4]
    pbc = su3.Lattice(dims, beta=5.65, seed=4, start=su3.SU3_START_HOT, storage=su3.SU3_FP32_12)
    dlt = su3.Lattice(dims, boundary=su3.SU3_DLT, glue_mask=glue, beta=5.65, seed=4, start=su3.SU3_START_HOT,
                      storage=su3.SU3_FP32_12, layer_blind=True)
    pbc.sweep(4)
    dlt.sweep(4)
    p = pbc.get_links()[0]
    d = dlt.get_links()
    assert np.array_equal(d[0], p) and np.array_equal(d[1], p)
    assert dlt.plaquette(0) == pbc.plaquette() and dlt.plaquette(1) == pbc.plaquette()


def test_time_glued_dlt_is_double_time_torus():
    """Two 16^3 x 4 layers glued in time are the 16^3 x 8 torus, link by link
    (the random-number site key layer*V + i_s - 1 is the torus site number)."""
    dlt = su3.Lattice([16, 16, 16, 4], boundary=su3.SU3_DLT, glue_mask=0b1000, beta=5.7, seed=3,
                      start=su3.SU3_START_HOT, storage=su3.SU3_FP32_12)
    tor = su3.Lattice([16, 16, 16, 8], beta=5.7, seed=3, start=su3.SU3_START_HOT, storage=su3.SU3_FP32_12)
    dlt.sweep(3)
    tor.sweep(3)
    assert np.array_equal(dlt.get_links().reshape(-1), tor.get_links().reshape(-1))
    assert dlt.polyakov(0) == pytest.approx(tor.polyakov(), abs=1e-15)


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18, su3.SU3_FP32_12, su3.SU3_FP32_18])
def test_graph_and_launch_shape_do_not_change_links(storage):
    kw = dict(beta=6.0, seed=21, storage=storage, start=su3.SU3_START_HOT, reunit_every=3)
    dims = [8, 6, 4, 6]
    ref = su3.Lattice(dims, **kw)
    ref.use_graph(False)
    ref.sweep(7)
    want = ref.get_links()
    shapes = [(0, 32, 1), (0, 64, 0), (0, 128, 2), (0, 256, 0)]
    if storage == su3.SU3_FP32_12:
        shapes += [(1, 128, 0), (1, 96, 3), (2, 64, 0), (2, 128, 1), (3, 256, 2), (4, 256, 0), (4, 128, 3)]
    for variant, threads, ctas in shapes:
        for pdl in (True, False):
            lat = su3.Lattice(dims, **kw)
            lat.set_launch(threads, ctas, variant=variant)
            lat.use_pdl(pdl)
            lat.sweep(7)
            assert np.array_equal(lat.get_links(), want), (variant, threads, ctas, pdl)
            assert lat.stats() == ref.stats()


def test_resume_is_bitwise():
    """Save links and the sweep counter after 5 sweeps, restore them into a
    fresh lattice, 5 more sweeps: identical to 10 sweeps in one go."""
    kw = dict(beta=5.8, seed=77, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT)
    a = su3.Lattice([8, 8, 8, 8], **kw)
    a.sweep(10)
    b = su3.Lattice([8, 8, 8, 8], **kw)
    b.sweep(5)
    saved, (_, _, n) = b.get_links(), b.stats()
    c = su3.Lattice([8, 8, 8, 8], **kw)
    c.set_links(saved)
    c.set_sweep_counter(n)
    c.sweep(5)
    assert np.array_equal(a.get_links(), c.get_links())


def _mixed_configs(storage=su3.SU3_FP32_12):
    rng = np.random.default_rng(42)
    shapes = [[8, 8, 8, 8], [6, 4, 8, 4], [8, 8, 8], [4, 4, 4, 4], [12, 12, 12]]
    cfgs = []
    for i, dims in enumerate(shapes * 2):
        boundary = su3.SU3_DLT if i in (3, 7) else su3.SU3_PBC
        cfgs.append(su3.make_config(dims, boundary=boundary, beta=float(rng.uniform(5.5, 6.5)), seed=1000 + i,
                                    storage=storage, start=su3.SU3_START_HOT, hits=1 + i % 3,
                                    reunit_every=4))
    return cfgs


@pytest.mark.parametrize("storage", [su3.SU3_FP32_12, su3.SU3_FP32_18, su3.SU3_FP64_18])
def test_chain_alone_equals_chain_in_mixed_ensemble(storage):
    """Chains of different D, shape, boundary, beta, seed and hits advanced
    in one fused launch per tick give the same links as each chain alone."""
    cfgs = _mixed_configs(storage)
    ens = su3.Ensemble(cfgs)
    ens.sweep(6)
    meas = ens.measure()
    for i, cfg in enumerate(cfgs):
        dims = [cfg.dims[k] for k in range(cfg.D)]
        alone = su3.Lattice(dims, boundary=cfg.boundary, beta=cfg.beta, seed=cfg.seed, storage=cfg.storage,
                            start=cfg.start, hits=cfg.hits, reunit_every=cfg.reunit_every)
        alone.sweep(6)
        assert np.array_equal(ens.get_links(i), alone.get_links()), i
        assert abs(meas[i, 0] - alone.plaquette()[0]) < 1e-14


def test_ensemble_matches_sequential_single_chains_256x8x8x8x8():
    """The batched-ensemble workload (256 chains of 8^4, beta in [5.5, 6.5])
    against single-chain runs of a sample of its chains."""
    rng = np.random.default_rng(2009)
    betas = rng.uniform(5.5, 6.5, 256)
    cfgs = [su3.make_config([8, 8, 8, 8], beta=float(b), seed=5000 + i, storage=su3.SU3_FP32_12,
                            start=su3.SU3_START_HOT, hits=2) for i, b in enumerate(betas)]
    ens = su3.Ensemble(cfgs)
    ens.sweep(3)
    for i in [0, 17, 128, 255]:
        alone = su3.Lattice([8, 8, 8, 8], beta=float(betas[i]), seed=5000 + i, storage=su3.SU3_FP32_12,
                            start=su3.SU3_START_HOT, hits=2)
        alone.sweep(3)
        assert np.array_equal(ens.get_links(i), alone.get_links())


def test_staged_chain_switches_in_a_persistent_torus_ensemble():
    """A persistent grid (one CTA per SM) over 64 torus chains of 16 tiles:
    nearly every tile of a CTA belongs to another chain, so the multi-chain
    torus form stages the next chain's descriptor and state in shared memory
    at every tile.  Links equal each chain alone bit for bit, and the
    measurements (every 2 sweeps, finished by the launch's last warp from
    the list of measuring chains) agree."""
    rng = np.random.default_rng(7)
    betas = rng.uniform(5.6, 6.4, 64)
    kw = dict(storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, hits=2, reunit_every=3, measure_every=2)
    cfgs = [su3.make_config([8, 8, 8, 8], beta=float(b), seed=7000 + i, **kw) for i, b in enumerate(betas)]
    ens = su3.Ensemble(cfgs)
    ens.set_launch(128, 1, variant=0)
    ens.sweep(5)
    for i in [0, 1, 31, 63]:
        alone = su3.Lattice([8, 8, 8, 8], beta=float(betas[i]), seed=7000 + i, **kw)
        alone.sweep(5)
        assert np.array_equal(ens.get_links(i), alone.get_links()), i
        m_ens, m_alone = ens.measurements(i), alone.measurements()
        assert m_ens.shape == m_alone.shape == (2, 2, 5)
        np.testing.assert_allclose(m_ens, m_alone, rtol=0, atol=1e-14)
        alone.close()
    ens.close()


def test_measurement_stage_records_every_k_sweeps():
    lat = su3.Lattice([6, 6, 6, 6], beta=6.0, seed=2, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                      reunit_every=2, measure_every=3, measure_capacity=8)
    lat.sweep(12)
    m = lat.measurements()
    assert m.shape == (4, 2, 5)
    assert np.allclose(m[-1, 1], [*lat.plaquette(), lat.polyakov().real, lat.polyakov().imag], atol=1e-14)
    assert np.allclose(m[:, 0], m[:, 1])  # one layer: the layer slot equals the whole lattice


FULL_SIZE = [  # (dims, layers, glue_mask, beta, storage, tol): the benchmark lattice and both config-3 workloads
    ([32, 32, 32, 32], 1, 0, 6.0, su3.SU3_FP64_18, 1e-11),
    ([32, 32, 32, 32], 1, 0, 6.0, su3.SU3_FP32_12, 1e-5),
    ([32, 32, 32, 32], 1, 0, 6.0, su3.SU3_FP32_18, 1e-5),
    ([16, 16, 16, 4], 2, 0b1000, 5.7, su3.SU3_FP32_12, 1e-5),   # two 16^3 x 4 layers glued in time
    ([16, 16, 16, 4], 2, 0b1000, 5.7, su3.SU3_FP64_18, 1e-11),
    ([64, 64, 64], 1, 0, 10.0, su3.SU3_FP32_12, 1e-5),           # D = 3
]


@pytest.mark.parametrize("dims,layers,glue,beta,storage,tol", FULL_SIZE,
                         ids=lambda v: "x".join(map(str, v)) if isinstance(v, list) else str(v))
def test_full_size_sampled_links(dims, layers, glue, beta, storage, tol):
    """Full-size lattices, hot start, one sweep at the default launch shape:
    links of the first phase (colour 0, direction 1) were updated from the
    start configuration, links of the last phase (colour 1, direction D) from
    the final configuration of all other links.  The oracle recomputes a
    sample of both, in every layer, link by link (the random-number site key
    is layer * V + i_s - 1)."""
    boundary = su3.SU3_DLT if layers == 2 else su3.SU3_PBC
    lat = su3.Lattice(dims, boundary=boundary, glue_mask=glue, beta=beta, seed=20090406, storage=storage,
                      start=su3.SU3_START_HOT, hits=2)
    c0 = lat.get_links()
    lat.sweep(1)
    c1 = lat.get_links()
    lat.close()
    o = oracle.Lattice(dims, nlayers=layers, glue_mask=glue or None)
    D = len(dims)
    rng = np.random.default_rng(0)
    checked = bad = 0
    for phase, mu, src in ((0, 0, c0), (1, D - 1, c1)):
        o.U[...] = src
        for layer, s in zip(rng.integers(0, layers, 400), rng.integers(0, o.V, 400)):
            layer, s = int(layer), int(s)
            if sum(o.site_coords(s)) % 2 != phase:
                continue
            A = o.staple(layer, s, mu)
            old = oracle.to_complex(c0[layer, s, mu])
            new, _ = oracle.link_heatbath(old, A, beta, 2, 20090406, layer * o.V + s, 0, phase, mu)
            err = np.max(np.abs(oracle.from_complex(new) - c1[layer, s, mu]))
            checked += 1
            bad += err > tol
    assert checked > 300
    assert bad <= (0 if storage == su3.SU3_FP64_18 else 1)


def test_acceptance_counters():
    lat = su3.Lattice([8, 8, 8, 8], beta=6.0, seed=3, storage=su3.SU3_FP32_12, hits=1)
    lat.sweep(20)
    prop, acc, sweeps = lat.stats()
    assert sweeps == 20
    assert prop == 20 * 3 * lat.nlinks  # one proposal per subgroup per link at hits = 1
    assert 0.95 < acc / prop < 0.995    # about 97 per cent in the scaling region (Sec. 2.1)


def test_two_coupling_chain_in_ensemble_leaves_others_bitwise():
    """A two-coupling DLT chain switches the fused launch to the tick
    kernel's weighted form; the other chains (and the weighted chain itself)
    must still equal their runs alone, bit for bit."""
    cfgs = [su3.make_config([4, 4, 4, 4], boundary=su3.SU3_DLT, beta=6.0, beta1=4.5, seed=31,
                            storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, hits=2),
            su3.make_config([8, 8, 8, 8], beta=5.9, seed=32, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                            hits=2),
            su3.make_config([6, 6, 6, 4], boundary=su3.SU3_DLT, beta=5.7, seed=33, storage=su3.SU3_FP32_12,
                            start=su3.SU3_START_HOT, hits=1)]
    ens = su3.Ensemble(cfgs)
    ens.sweep(4)
    for i, cfg in enumerate(cfgs):
        dims = [cfg.dims[k] for k in range(cfg.D)]
        alone = su3.Lattice(dims, boundary=cfg.boundary, beta=cfg.beta, beta1=(cfg.beta1 if cfg.beta1 >= 0 else None),
                            seed=cfg.seed, storage=cfg.storage, start=cfg.start, hits=cfg.hits)
        alone.sweep(4)
        assert np.array_equal(ens.get_links(i), alone.get_links()), i


def test_autotune_cache(tmp_path):
    """A cached launch shape is applied without timing, and gives the same
    links as any other shape."""
    import time
    path = str(tmp_path / "tune.json")
    kw = dict(beta=6.0, seed=4, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT, reunit_every=5)
    a = su3.Lattice([16, 16, 16, 16], **kw)
    first = a.autotune(cache=path)
    b = su3.Lattice([16, 16, 16, 16], **kw)
    t0 = time.perf_counter()
    second = b.autotune(cache=path)
    assert second == first and time.perf_counter() - t0 < 0.5
    a.sweep(3)
    b.sweep(3)
    assert np.array_equal(a.get_links(), b.get_links())


def test_wait_with_deadline():
    """Host watchdog: a deadline that passes before the queued work ends
    gives SU3_ETIMEOUT and leaves the work running; a later wait succeeds."""
    lat = su3.Lattice([32, 32, 32, 32], beta=6.0, seed=1, storage=su3.SU3_FP32_12, start=su3.SU3_START_HOT,
                      reunit_every=10)
    lat.sweep(1)
    lat.synchronize()
    lat.sweep(40)  # ~30 ms queued
    with pytest.raises(su3.Su3Error) as ei:
        lat.wait(0.0)
    assert ei.value.status == su3.SU3_ETIMEOUT
    lat.wait(120.0)
    assert lat.stats()[2] == 41
    with pytest.raises(su3.Su3Error) as ei:
        lat.wait(-1.0)
    assert ei.value.status == su3.SU3_EINVAL
