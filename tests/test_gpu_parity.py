"""GPU parity: the CUDA path against the double-precision CPU oracle, link by
link, through the C ABI.

Tolerances: FP64 storage <= 1e-11 per link element after one sweep; FP32
12-real storage <= 1e-5, where a link outside it is counted (and must be
explained by the oracle): an accept/reject decision within the float
rounding of its threshold, or an ill-conditioned update - one whose oracle
result moves by much under a rounding-level perturbation of the start (a
subgroup with a small norm k, whose direction a/k amplifies the float
rounding of W = U A).
"""
import numpy as np
import pytest

import oracle
import paper_0904_0642_gb300 as su3

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-11
FP32_TOL = 1e-5
FLIP_MARGIN = 1e-4  # an FP32 decision this close to the threshold may flip
# An ill-conditioned link is excused when its error is at most SENS_FACTOR
# times its sensitivity (its response in the oracle to a one-ulp relative
# perturbation of the start) and at most an absolute ceiling.  Measured on
# GB300 over 52 one-sweep cases (every geometry below, both float forms,
# three seeds each, the two-coupling DLT and the edge couplings; about
# 40,000 links): the ratio error / sensitivity of every link not near an
# accept threshold was at most 27.6, the per-case maxima 8-21; the FP32
# arithmetic of one update acts like a perturbation of 10-30 ulp of the
# start.  The largest excused error was 1.4e-5 at beta = 6 (ceiling 5e-5)
# and 9.7e-5 at beta = 0.3 with 254 hits, where the sensitivity itself
# reaches 4.6e-5 (ceiling 2e-4, STRONG_CEILING).
SENS_FACTOR = 30.0
CEILING = 5e-5
STRONG_CEILING = 2e-4

GEOMS = [
    dict(dims=[4, 4, 4, 4]),
    dict(dims=[6, 4, 2, 8]),          # 192 sites per colour: one full 128-tile + a ragged tail
    dict(dims=[2, 2, 2, 2]),          # smallest 4-D lattice: x+mu and x-mu coincide
    dict(dims=[8, 6]),                # D = 2
    dict(dims=[6, 4, 8]),             # D = 3
    dict(dims=[4, 2, 4, 4], nlayers=2, glue_mask=0b1111),
    dict(dims=[4, 2, 4, 4], nlayers=2, glue_mask=0b1000),
    dict(dims=[4, 4, 2, 4], nlayers=2, glue_mask=0b0111),
]


def gpu_lattice(g, storage, **kw):
    boundary = su3.SU3_DLT if g.get("nlayers", 1) == 2 else su3.SU3_PBC
    return su3.Lattice(g["dims"], boundary=boundary, glue_mask=g.get("glue_mask", 0), storage=storage, **kw)


def oracle_lattice(g, **kw):
    return oracle.Lattice(g["dims"], nlayers=g.get("nlayers", 1), glue_mask=g.get("glue_mask"), **kw)


FLOAT_FORMS = [su3.SU3_FP32_12, su3.SU3_FP32_18]


@pytest.mark.parametrize("storage", [su3.SU3_FP64_18] + FLOAT_FORMS)
@pytest.mark.parametrize("g", GEOMS[:1] + GEOMS[5:6])
def test_cold_start_observables(g, storage):
    with gpu_lattice(g, storage) as lat:
        for layer in range(-1, lat.nlayers):
            t, s, ti = lat.plaquette(layer)
            assert t == 1.0 and s == 1.0 and ti == 1.0
            assert lat.polyakov(layer) == 1.0
        U = lat.get_links()
        assert np.array_equal(U, oracle_lattice(g).cold_start().U)


@pytest.mark.parametrize("g", GEOMS)
def test_hot_start_matches_oracle(g):
    o = oracle_lattice(g).hot_start(2024)
    with gpu_lattice(g, su3.SU3_FP64_18, seed=2024, start=su3.SU3_START_HOT) as lat:
        assert np.max(np.abs(lat.get_links() - o.U)) < 1e-13
    for storage in FLOAT_FORMS:
        with gpu_lattice(g, storage, seed=2024, start=su3.SU3_START_HOT) as lat:
            assert np.max(np.abs(lat.get_links() - o.U)) < 1e-6


@pytest.mark.parametrize("storage,tol", [(su3.SU3_FP64_18, 0.0), (su3.SU3_FP32_12, 2e-7), (su3.SU3_FP32_18, 0.0)])
def test_set_get_round_trip(storage, tol):
    """FP64 keeps every bit; FP32_18 rounds each real to float (compared with
    numpy's float32 rounding, bit for bit); FP32_12 also rebuilds row 3."""
    g = GEOMS[1]
    o = oracle_lattice(g).hot_start(5)
    want = o.U.astype(np.float32).astype(np.float64) if storage == su3.SU3_FP32_18 else o.U
    with gpu_lattice(g, storage) as lat:
        lat.set_links(o.U)
        assert np.max(np.abs(lat.get_links() - want)) <= tol


def _sensitivity(make, start, samples=4, **sweep_kw):
    """Each link's response, in the oracle, to perturbations of the start at
    float rounding level (every element times 1 + 2^-24 r, r uniform in
    [-1, 1]): the empirical condition of the one-sweep update, the largest
    response over `samples` independent perturbations (one perturbation can
    miss the sensitive direction: at beta = 0.3 with 254 hits single samples
    differ from the largest of eight by up to a factor 16)."""
    rng = np.random.default_rng(99)
    a = make()
    a.U[...] = start
    a.sweep(**sweep_kw)
    out = np.zeros(a.U.size // 18)
    for _ in range(samples):
        b = make()
        b.U[...] = start * (1 + 2.0 ** -24 * rng.uniform(-1, 1, start.shape))
        b.sweep(**sweep_kw)
        out = np.maximum(out, np.max(np.abs(a.U - b.U).reshape(-1, 18), axis=1))
    return out


def _flip_check(got, want, margins, sens, tol, ceiling=CEILING):
    """Links beyond tol are counted, not failed, when the oracle explains
    them: an accept/reject decision within FLIP_MARGIN of its threshold (a
    flip: the subgroup's rotation differs entirely, so no bound applies), or
    a link whose own response to rounding-level perturbations of the start is
    large (an ill-conditioned update, e.g. a subgroup with small k, whose
    direction a/k amplifies the rounding of W); such a link must stay within
    SENS_FACTOR times that response and within the absolute ceiling.
    Returns the number counted."""
    err = np.max(np.abs(got - want).reshape(-1, 18), axis=1)
    margins = margins.reshape(-1)
    over = err > tol
    flip = margins < FLIP_MARGIN
    conditioned = (err <= SENS_FACTOR * sens) & (err <= ceiling)
    unexplained = over & ~flip & ~conditioned
    assert not unexplained.any(), (
        f"{int(unexplained.sum())} links differ beyond the FP32 bound: err={err[unexplained][:5]}, "
        f"margin={margins[unexplained][:5]}, sensitivity={sens[unexplained][:5]}")
    return int(over.sum())


@pytest.mark.parametrize("g", GEOMS)
@pytest.mark.parametrize("beta,hits", [(6.0, 2), (0.8, 3)])
def test_one_sweep_fp64(g, beta, hits):
    o = oracle_lattice(g).hot_start(11)
    start = o.U.copy()
    o.sweep(beta, hits, 99, n=1)
    with gpu_lattice(g, su3.SU3_FP64_18, beta=beta, seed=99, hits=hits) as lat:
        lat.set_links(start)
        lat.sweep(1)
        got = lat.get_links()
        prop, acc, sweeps = lat.stats()
    assert np.max(np.abs(got - o.U)) <= FP64_TOL
    assert sweeps == 1


@pytest.mark.parametrize("storage", FLOAT_FORMS)
@pytest.mark.parametrize("g", GEOMS)
def test_one_sweep_fp32(g, storage):
    o = oracle_lattice(g).hot_start(12)
    with gpu_lattice(g, storage, beta=6.0, seed=7, hits=2) as lat:
        lat.set_links(o.U)
        start = lat.get_links()  # the float-rounded start both sides use
    o.U[...] = start
    margins = np.full(o.nlinks, np.inf)
    o.sweep(6.0, 2, 7, n=1, margins=margins)
    sens = _sensitivity(lambda: oracle_lattice(g), start, beta=6.0, hits=2, seed=7, n=1)
    with gpu_lattice(g, storage, beta=6.0, seed=7, hits=2) as lat:
        lat.set_links(start)
        lat.sweep(1)
        got = lat.get_links()
    counted = _flip_check(got, o.U, margins, sens, FP32_TOL)
    assert counted <= max(2, o.nlinks // 100)


def test_config1_cold_start_hundred_sweeps_fp64():
    """4^4 PBC, beta = 6.0, cold start, hits = 2, seed 1: all link elements
    after sweep 1, and the plaquette after each of 100 sweeps."""
    o = oracle.Lattice([4, 4, 4, 4]).cold_start()
    with su3.Lattice([4, 4, 4, 4], beta=6.0, seed=1, hits=2) as lat:
        lat.sweep(1)
        o.sweep(6.0, 2, 1, n=1)
        assert np.max(np.abs(lat.get_links() - o.U)) <= FP64_TOL
        diffs = []
        for _ in range(99):
            lat.sweep(1)
            o.sweep(6.0, 2, 1, n=1)
            diffs.append(abs(lat.plaquette()[0] - o.plaquette()[0]))
    assert max(diffs) < 1e-9, max(diffs)


@pytest.mark.parametrize("storage,tol", [(su3.SU3_FP64_18, 1e-13), (su3.SU3_FP32_12, 2e-6), (su3.SU3_FP32_18, 2e-6)])
@pytest.mark.parametrize("g", GEOMS)
def test_observables_match_oracle(g, storage, tol):
    o = oracle_lattice(g).hot_start(3)
    o.sweep(5.7, 2, 3, n=2)
    with gpu_lattice(g, storage) as lat:
        lat.set_links(o.U)
        o.U[...] = lat.get_links()  # storage-rounded links on both sides
        for layer in range(-1, o.nlayers):
            np.testing.assert_allclose(lat.plaquette(layer), o.plaquette(layer), atol=tol)
            assert abs(lat.polyakov(layer) - o.polyakov(layer)) < tol


@pytest.mark.parametrize("storage,tol", [(su3.SU3_FP64_18, 1e-14), (su3.SU3_FP32_12, 1e-6), (su3.SU3_FP32_18, 1e-6)])
def test_reunitarize_matches_oracle(storage, tol):
    """Float storage: the double-precision Gram-Schmidt result rounded to
    nearest float, so the stored floats equal numpy's float32 rounding of
    the oracle's result except where the two double computations (summation
    order, one Newton step) straddle a rounding boundary: rare, and then one
    ulp.  Rows 1, 2 for the 12-real form (row 3 is rebuilt on load), all
    three for the 18-real form."""
    g = GEOMS[1]
    o = oracle_lattice(g).hot_start(4)
    rng = np.random.default_rng(0)
    o.U += 1e-4 * rng.standard_normal(o.U.shape)
    with gpu_lattice(g, storage) as lat:
        lat.set_links(o.U)
        o.U[...] = lat.get_links()
        lat.reunitarize()
        o.reunitarize()
        got = lat.get_links()
        assert np.max(np.abs(got - o.U)) < tol
    if storage != su3.SU3_FP64_18:
        rows = 2 if storage == su3.SU3_FP32_12 else 3
        g32 = got[..., :rows, :, :].astype(np.float32)
        w32 = o.U[..., :rows, :, :].astype(np.float32)
        exact = np.mean(g32 == w32)
        ulps = np.abs(g32.view(np.int32).astype(np.int64) - w32.view(np.int32).astype(np.int64))
        assert exact >= 0.999 and ulps.max() <= 1, (exact, ulps.max())


@pytest.mark.parametrize("glue", [0b1111, 0b1000])
def test_two_couplings_one_sweep(glue):
    """DLT with beta0 != beta1 (Sec. 2.2): FP64 link by link against the
    oracle; FP32 within the FP32 tolerance, every link beyond it explained by
    the oracle as in test_one_sweep_fp32 (the beta-weighted staple sums terms
    of size beta_p, so a few ill-conditioned links land just above 1e-5)."""
    g = dict(dims=[4, 2, 4, 4], nlayers=2, glue_mask=glue)
    o = oracle_lattice(g).hot_start(19)
    start = o.U.copy()
    o.sweep(6.0, 2, 5, n=1, beta1=4.2)
    with gpu_lattice(g, su3.SU3_FP64_18, beta=6.0, beta1=4.2, seed=5, hits=2) as lat:
        lat.set_links(start)
        lat.sweep(1)
        assert np.max(np.abs(lat.get_links() - o.U)) <= FP64_TOL
    o2 = oracle_lattice(g)
    with gpu_lattice(g, su3.SU3_FP32_12, beta=6.0, beta1=4.2, seed=5, hits=2) as lat:
        lat.set_links(start)
        start32 = lat.get_links()
        o2.U[...] = start32
        margins = np.full(o2.nlinks, np.inf)
        o2.sweep(6.0, 2, 5, n=1, beta1=4.2, margins=margins)
        sens = _sensitivity(lambda: oracle_lattice(g), start32, beta=6.0, hits=2, seed=5, n=1, beta1=4.2)
        lat.sweep(1)
        counted = _flip_check(lat.get_links(), o2.U, margins, sens, FP32_TOL)
    assert counted <= max(2, o2.nlinks // 100)
