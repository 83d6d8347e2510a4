"""GPU parity: the CUDA path through the C ABI against the FP64 oracle, element by element.

Counts must be bit-identical; weighted sums and ravg within 1e-6 relative.  Inputs are seeded
synthetic catalogues sized so the oracle finishes in seconds while cells still hold several
128-point tiles plus a ragged tail.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import TOL, assert_match, gpu_count, to_dev
from tests.test_oracle_pins import LATTICE, PERIODIC, RPPI, Cat

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    yield c
    cf.cf_destroy(c)


def both(ctx, kind, edges, d1, d2=None, **kw):
    got = gpu_count(ctx, kind, edges, d1, d2, **kw)
    okw = {k: v for k, v in kw.items() if k not in ("refine", "device")}
    exp = oracle.count(kind, edges, d1, d2, **okw)
    return got, exp


# ---- exact ties (every separation is exact: all of them sit on edges or wrap boundaries) ----

def _f32(cat):
    for a in ("x", "y", "z"):
        setattr(cat, a, getattr(cat, a).astype(np.float32))
    if cat.w is not None:
        cat.w = cat.w.astype(np.float32)
    return cat


@pytest.mark.parametrize("f32", [False, True])
def test_hand_lattices(ctx, f32):
    conv = _f32 if f32 else (lambda c: c)
    d = conv(Cat(LATTICE, w=[1.0, 2.0, 0.5, 4.0]))
    got, exp = both(ctx, "r", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, weighted=True, ravg=True)
    assert got["npairs"].tolist() == [2, 4, 4, 2]
    assert_match(got, exp, True, True)
    d = conv(Cat(PERIODIC))
    got, exp = both(ctx, "r", [0, 1, 2, 4, 5], d, autocorr=True, periodic=True, box=8.0)
    assert got["npairs"].tolist() == [7, 4, 2, 10]
    got, exp = both(ctx, "r", [0, 1, 2, 4, 5], d, d, autocorr=False, periodic=True, box=8.0)
    assert got["npairs"].tolist() == [7, 4, 2, 10]
    d = conv(Cat(RPPI))
    got, exp = both(ctx, "rppi", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, pimax=3.0, npibins=3)
    assert_match(got, exp)
    got, exp = both(ctx, "wp", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, pimax=3.0, npibins=3)
    assert got["npairs"].tolist() == [2, 4, 4, 0]
    d = conv(Cat([(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)]))
    got, exp = both(ctx, "theta", [60, 90, 180], d, autocorr=True, periodic=False, ravg=True)
    assert got["npairs"].tolist() == [0, 10]
    assert_match(got, exp, ravg=True)


# ---- randomised parity over every kind and option ----

def _catalogue(kind, n_centres, seed, dtype=np.float32, box=40.0):
    if kind == "theta":
        return gen.sphere_patch(n_centres * 60, 0.0, 25.0, -5.0, 20.0, seed)
    d = gen.clustered_box(n_centres, 60, 1.2, box, seed, dtype=dtype)
    u = gen.uniform_box(n_centres * 20, box, seed + 1, dtype=dtype)
    return gen.Catalogue(*(np.concatenate([getattr(d, a), getattr(u, a)]) for a in "xyz"))


CASES = []
for kind in ("r", "rppi", "wp", "theta"):
    for autocorr in (True, False):
        for periodic in ((False,) if kind == "theta" else (True, False)):
            for weighted, ravg in ((False, False), (True, False), (False, True), (True, True)):
                CASES.append((kind, autocorr, periodic, weighted, ravg))


@pytest.mark.parametrize("kind,autocorr,periodic,weighted,ravg", CASES)
def test_random_parity(ctx, kind, autocorr, periodic, weighted, ravg):
    seed = 1000 + len(kind) * 10 + int(autocorr) * 3 + int(periodic)
    d1 = _catalogue(kind, 40, seed)
    d2 = _catalogue(kind, 30, seed + 7)
    d1.w = gen.uniform_weights(d1.n, 0.5, 1.5, seed + 2)
    d2.w = gen.uniform_weights(d2.n, 0.5, 1.5, seed + 3)
    edges = gen.log_edges(0.01, 2.5, 14) if kind == "theta" else gen.log_edges(0.05, 7.0, 12)
    kw = dict(autocorr=autocorr, periodic=periodic, box=40.0, pimax=9.0, npibins=9, weighted=weighted, ravg=ravg)
    got, exp = both(ctx, kind, edges, d1, None if autocorr else d2, **kw)
    assert_match(got, exp, weighted, ravg)
    assert int(np.asarray(got["npairs"]).sum()) > 1000


@pytest.mark.parametrize("kind", ["r", "rppi", "theta"])
def test_float64_inputs(ctx, kind):
    d = _catalogue(kind, 30, 77, dtype=np.float64)
    if kind == "theta":
        d = gen.Catalogue(*(getattr(d, a).astype(np.float64) for a in "xyz"))
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 78).astype(np.float64)
    edges = gen.log_edges(0.01, 2.5, 10) if kind == "theta" else gen.log_edges(0.05, 7.0, 10)
    kw = dict(autocorr=True, periodic=kind != "theta", box=40.0, pimax=9.0, npibins=9)
    for weighted, ravg in ((False, False), (True, True)):
        got, exp = both(ctx, kind, edges, d, weighted=weighted, ravg=ravg, **kw)
        assert_match(got, exp, weighted, ravg)


def test_uniform_20k_float64_full(ctx):
    """The correctness workload in full: N=20000 uniform float64, periodic L=250, 20 log bins."""
    wl = gen.workload("uniform_r_20k")
    got, exp = both(ctx, "r", wl.edges, wl.d1, autocorr=True, periodic=True, box=wl.box)
    assert_match(got, exp)


@pytest.mark.parametrize("refine", [(1, 1, 1), (2, 2, 2), (3, 1, 2), (4, 4, 4)])
def test_refinement_does_not_change_results(ctx, refine):
    d = _catalogue("r", 40, 5)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 6)
    edges = gen.log_edges(0.05, 7.0, 12)
    got, exp = both(ctx, "r", edges, d, autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True,
                    refine=refine)
    assert_match(got, exp, True, True)
    got, exp = both(ctx, "rppi", edges, d, autocorr=True, periodic=True, box=40.0, pimax=9.0, npibins=9,
                    refine=refine)
    assert_match(got, exp)


def test_rmax_spans_box(ctx):
    """Cells fewer than 2k+1 per axis: explicit minimum image; totals are N(N-1) / N1*N2."""
    d = gen.uniform_box(700, 10.0, 3)
    e = gen.uniform_box(500, 10.0, 4)
    got, exp = both(ctx, "r", [1e-6, 9.0], d, autocorr=True, periodic=True, box=10.0)
    assert int(got["npairs"].sum()) == d.n * (d.n - 1)
    assert_match(got, exp)
    got, exp = both(ctx, "r", gen.log_edges(0.3, 6.0, 8), d, e, autocorr=False, periodic=True, box=10.0)
    assert_match(got, exp)
    got, exp = both(ctx, "rppi", gen.log_edges(0.3, 6.0, 8), d, autocorr=True, periodic=True, box=10.0,
                    pimax=6.0, npibins=6)
    assert_match(got, exp)
    got, exp = both(ctx, "r", [1e-6, 18.0], d, autocorr=True, periodic=False)
    assert int(got["npairs"].sum()) == d.n * (d.n - 1)


def test_degenerate_inputs(ctx):
    edges = [0.0, 0.5, 1.0, 2.0]
    empty = gen.Catalogue(*(np.zeros(0, np.float32) for _ in range(3)))
    got = gpu_count(ctx, "r", edges, empty, autocorr=True, periodic=True, box=5.0)
    assert got["npairs"].tolist() == [0, 0, 0]
    one = gen.Catalogue(*(np.array([1.0], np.float32) for _ in range(3)))
    got = gpu_count(ctx, "r", edges, one, autocorr=True, periodic=True, box=5.0)
    assert got["npairs"].tolist() == [1, 0, 0]            # its self pair (first edge 0, Appendix B)
    same = gen.Catalogue(*(np.full(300, 2.5, np.float32) for _ in range(3)))
    got, exp = both(ctx, "r", edges, same, autocorr=True, periodic=True, box=5.0)
    assert got["npairs"].tolist() == [300 * 300, 0, 0]
    assert_match(got, exp)
    edge = gen.Catalogue(np.array([0.0, 5.0, 5.0, 2.5], np.float32), np.array([0.0, 0.0, 5.0, 2.5], np.float32),
                         np.array([5.0, 0.0, 0.0, 2.5], np.float32))
    got, exp = both(ctx, "r", edges, edge, autocorr=True, periodic=True, box=5.0)
    assert_match(got, exp)


def test_near_edge_adversarial(ctx):
    """Pairs placed at e_k (1 +- delta) for delta from 1e-9 to 1e-5, and exactly on e_k."""
    edges = gen.log_edges(0.1, 10.0, 8)
    rng = np.random.Generator(np.random.PCG64(9))
    pts = []
    L = 100.0
    for k, e in enumerate(edges):
        for delta in (0.0, 1e-9, -1e-9, 1e-7, -1e-7, 1e-6, -1e-6, 1e-5, -1e-5):
            c = rng.uniform(15, 85, 3)
            v = rng.normal(size=3)
            v /= np.linalg.norm(v)
            pts.append(c)
            pts.append(c + v * e * (1 + delta))
    a = np.array(pts)
    for dt in (np.float32, np.float64):
        d = gen.Catalogue(*(a[:, i].astype(dt) for i in range(3)))
        got, exp = both(ctx, "r", edges, d, autocorr=True, periodic=True, box=L)
        assert_match(got, exp)
        got, exp = both(ctx, "rppi", edges, d, autocorr=True, periodic=True, box=L, pimax=5.0, npibins=5)
        assert_match(got, exp)


def test_auto_equals_cross_gpu(ctx):
    d = _catalogue("r", 40, 21)
    edges = gen.log_edges(0.0 + 0.05, 7.0, 10)
    a = gpu_count(ctx, "r", edges, d, autocorr=True, periodic=True, box=40.0)
    c = gpu_count(ctx, "r", edges, d, d, autocorr=False, periodic=True, box=40.0)
    assert np.array_equal(a["npairs"], c["npairs"])
    e0 = np.concatenate([[0.0], edges])
    a = gpu_count(ctx, "r", e0, d, autocorr=True, periodic=True, box=40.0)
    c = gpu_count(ctx, "r", e0, d, d, autocorr=False, periodic=True, box=40.0)
    assert np.array_equal(a["npairs"], c["npairs"])


def test_host_inputs_equal_device_inputs(ctx):
    d = _catalogue("r", 40, 31)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 32)
    edges = gen.log_edges(0.05, 7.0, 12)
    kw = dict(autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
    a = gpu_count(ctx, "r", edges, d, device=True, **kw)
    b = gpu_count(ctx, "r", edges, d, device=False, **kw)
    assert np.array_equal(a["npairs"], b["npairs"])
    np.testing.assert_allclose(a["wsum"], b["wsum"], rtol=TOL)


def test_lattice_on_the_edges(ctx):
    """A 40^3 integer lattice in a periodic box with integer edges: about an eighth of the pairs
    in range lie exactly on an edge (lattice vectors of integer length: axes, (2,2,1), (4,3,0),
    (4,4,2)), so millions of pairs go to the FP64 recheck.  With the queue started at 4096 entries
    it must grow; counts and sums still equal the oracle's."""
    import paper_1911_03545_gb300 as cf
    g = np.arange(40, dtype=np.float32)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    d = gen.Catalogue(X.ravel(), Y.ravel(), Z.ravel(), gen.uniform_weights(X.size, 0.5, 1.5, 71))
    edges = np.arange(1.0, 7.0)
    kw = dict(autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
    cf.cf_set_option(ctx, cf.CF_OPT_QUEUE, 4096)
    try:
        got = gpu_count(ctx, "r", edges, d, **kw)
        st = cf.cf_get_stats(ctx)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_QUEUE, 0)
    assert st["rechecked_pairs"] > 1_000_000
    assert_match(got, oracle.count("r", edges, d, **kw), True, True)


def test_options_do_not_change_results(ctx):
    import paper_1911_03545_gb300 as cf
    d = _catalogue("r", 60, 41)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 42)
    edges = gen.log_edges(0.05, 7.0, 12)
    kw = dict(autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
    exp = oracle.count("r", edges, d, **kw)
    for opt, val in ((cf.CF_OPT_TILE, 64), (cf.CF_OPT_JCHUNK, 37), (cf.CF_OPT_WARPS, 2), (cf.CF_OPT_CTAS_PER_SM, 1),
                     (cf.CF_OPT_QUEUE, 1), (cf.CF_OPT_VARIANT, 2), (cf.CF_OPT_VARIANT, 1), (cf.CF_OPT_CELL_ORDER, 1),
                     (cf.CF_OPT_CELL_ORDER, 2), (cf.CF_OPT_CELL_ORDER, 4), (cf.CF_OPT_CELL_PRUNE, 1)):
        cf.cf_set_option(ctx, opt, val)
        try:
            got = gpu_count(ctx, "r", edges, d, **kw)
        finally:
            cf.cf_set_option(ctx, opt, 0)
        assert_match(got, exp, True, True)


def test_batch_equals_single(ctx):
    import paper_1911_03545_gb300 as cf
    import torch
    edges = gen.log_edges(0.1, 8.0, 10)
    cats = [gen.batch_catalogue(i, n, L=60.0, members=20) for i, n in enumerate([900, 3000, 50, 1700])]
    p = cf.params(kind="rppi", edges=edges, autocorr=True, periodic=True, box=60.0, pimax=10.0, npibins=10)
    pts = [cf.points(*to_dev(c, "cuda:0")) for c in cats]
    outs = cf.cf_batch_count(ctx, p, pts)
    for c, o in zip(cats, outs):
        single = cf.cf_count(ctx, p, cf.points(*to_dev(c, "cuda:0")))
        assert np.array_equal(o["npairs"], single["npairs"])
        exp = oracle.count("rppi", edges, c, autocorr=True, periodic=True, box=60.0, pimax=10.0, npibins=10)
        assert np.array_equal(o["npairs"], exp["npairs"])
    torch.cuda.synchronize()


def test_errors_leave_context_usable(ctx):
    import paper_1911_03545_gb300 as cf
    edges = gen.log_edges(0.1, 5.0, 6)
    bad = gen.uniform_box(100, 10.0, 1)
    bad.x[3] = 10.5
    with pytest.raises(cf.CfError) as ei:
        gpu_count(ctx, "r", edges, bad, autocorr=True, periodic=True, box=10.0)
    assert ei.value.status == -1
    nan = gen.uniform_box(100, 10.0, 2)
    nan.y[5] = np.nan
    with pytest.raises(cf.CfError):
        gpu_count(ctx, "r", edges, nan, autocorr=True, periodic=False)
    # a periodic call checks its inputs after the count (its bounding-box pass runs beside the
    # build): a NaN, an infinite weight or a point past L still fails the call, and the next works
    for bad_w in (False, True):
        bad = gen.uniform_box(3000, 10.0, 5)
        bad.w = gen.uniform_weights(bad.n, 0.5, 1.5, 6)
        if bad_w:
            bad.w[17] = np.inf
        else:
            bad.z[2999] = np.nan
        with pytest.raises(cf.CfError) as ei:
            gpu_count(ctx, "r", edges, bad, autocorr=True, periodic=True, box=10.0, weighted=True)
        assert ei.value.status == -1
        good = gen.uniform_box(3000, 10.0, 7)
        got, exp = both(ctx, "r", edges, good, autocorr=True, periodic=True, box=10.0)
        assert_match(got, exp)
    with pytest.raises(cf.CfError):
        gpu_count(ctx, "r", [1.0, 0.5], nan, autocorr=True, periodic=False)
    import torch
    small = cf.cf_create(0, torch.cuda.current_stream())
    try:
        cf.cf_set_option(small, cf.CF_OPT_MEM_CAP, 1 << 16)
        big = gen.uniform_box(200000, 50.0, 3)
        with pytest.raises(cf.CfError) as ei:
            gpu_count(small, "r", edges, big, autocorr=True, periodic=True, box=50.0)
        assert ei.value.status == -2
        cf.cf_set_option(small, cf.CF_OPT_MEM_CAP, 0)
        good = gen.uniform_box(2000, 10.0, 4)
        got, exp = both(small, "r", edges, good, autocorr=True, periodic=True, box=10.0)
        assert_match(got, exp)
    finally:
        cf.cf_destroy(small)
    good = gen.uniform_box(2000, 10.0, 4)
    got, exp = both(ctx, "r", edges, good, autocorr=True, periodic=True, box=10.0)
    assert_match(got, exp)


@pytest.mark.parametrize("kind,autocorr,periodic,weighted,ravg", CASES[::3])
def test_compacting_variant_parity(ctx, kind, autocorr, periodic, weighted, ravg):
    """The two-phase compacting pair kernel (variant 2) gives the same results."""
    import paper_1911_03545_gb300 as cf
    cf.cf_set_option(ctx, cf.CF_OPT_VARIANT, 2)
    try:
        test_random_parity(ctx, kind, autocorr, periodic, weighted, ravg)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_VARIANT, 0)


@pytest.mark.parametrize("variant", [1, 2])
def test_tile_shapes_wrap_and_diagonal(ctx, variant):
    """Ragged i tiles (1 to 4 slots of 32 points), odd j ranges, cells paired with themselves and the
    explicit minimum image (Rmax = 5 in a box of 12: two cells per axis) together, against the
    oracle, for several tile sizes and j range lengths."""
    import paper_1911_03545_gb300 as cf
    d = gen.clustered_box(30, 37, 0.8, 12.0, 91)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 92)
    edges = gen.log_edges(0.05, 5.0, 9)
    kw_r = dict(autocorr=True, periodic=True, box=12.0, weighted=True, ravg=True)
    kw_p = dict(autocorr=True, periodic=True, box=12.0, pimax=5.0, npibins=5)
    exp_r = oracle.count("r", edges, d, **kw_r)
    exp_p = oracle.count("rppi", edges, d, **kw_p)
    cf.cf_set_option(ctx, cf.CF_OPT_VARIANT, variant)
    try:
        for tile in (32, 96, 128):
            for jchunk in (31, 129, 512):
                cf.cf_set_option(ctx, cf.CF_OPT_TILE, tile)
                cf.cf_set_option(ctx, cf.CF_OPT_JCHUNK, jchunk)
                assert_match(gpu_count(ctx, "r", edges, d, **kw_r), exp_r, True, True)
                assert_match(gpu_count(ctx, "rppi", edges, d, **kw_p), exp_p)
    finally:
        for opt in (cf.CF_OPT_VARIANT, cf.CF_OPT_TILE, cf.CF_OPT_JCHUNK):
            cf.cf_set_option(ctx, opt, 0)


def test_cell_pruning_keeps_results(ctx):
    """Skipping cell pairs by their points' bounding boxes (the default), and inside a kept cell pair
    the 32-point groups of the j cell out of reach of an i tile (CF_OPT_BLOCK_PRUNE), changes
    neither counts nor sums, and on clustered data each removes evaluated pairs."""
    import paper_1911_03545_gb300 as cf
    d = gen.clustered_box(120, 40, 0.7, 60.0, 93)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 94)
    edges = gen.log_edges(0.05, 6.0, 10)
    kw_r = dict(autocorr=True, periodic=True, box=60.0, weighted=True, ravg=True)
    kw_p = dict(autocorr=True, periodic=True, box=60.0, pimax=8.0, npibins=8)
    exp_r = oracle.count("r", edges, d, **kw_r)
    exp_p = oracle.count("rppi", edges, d, **kw_p)
    exp_w = oracle.count("wp", edges, d, **kw_p)
    evaluated = {}
    for prune in (0, 1):
        for block in (0, 1):
            cf.cf_set_option(ctx, cf.CF_OPT_CELL_PRUNE, prune)
            cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, block)
            try:
                assert_match(gpu_count(ctx, "r", edges, d, **kw_r), exp_r, True, True)
                evaluated[prune, block] = cf.cf_get_stats(ctx)["evaluated_pairs"]
                assert_match(gpu_count(ctx, "rppi", edges, d, **kw_p), exp_p)
                assert_match(gpu_count(ctx, "wp", edges, d, **kw_p), exp_w)
            finally:
                cf.cf_set_option(ctx, cf.CF_OPT_CELL_PRUNE, 0)
                cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, 0)
    assert evaluated[0, 0] < evaluated[1, 0]
    # block pruning works from the cells' group boxes, which only cell pruning builds
    assert evaluated[0, 1] < evaluated[0, 0] and evaluated[1, 1] == evaluated[1, 0]


def test_cell_pruning_at_the_largest_edge(ctx):
    """Two tight groups in neighbouring cells at separations just below, at and just above the largest
    edge (10): a pruned cell pair must never hold a pair the oracle counts."""
    pts = []
    for k, delta in enumerate([-1e-4, -1e-5, -2e-6, 0.0, 2e-6, 1e-5, 1e-4]):
        y = 5.0 + 12.0 * k
        for m in range(3):
            pts.append((12.0, y + 0.01 * m, 50.0))
            pts.append((22.0 + delta, y + 0.01 * m, 50.0))
    a = np.array(pts, dtype=np.float64)
    d = gen.Catalogue(a[:, 0].astype(np.float32), a[:, 1].astype(np.float32), a[:, 2].astype(np.float32))
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 95).astype(np.float32)
    edges = np.array([1.0, 5.0, 9.99, 10.0])
    for kind, kw in (("r", {}), ("r", dict(weighted=True, ravg=True)), ("rppi", dict(pimax=10.0, npibins=10)),
                     ("wp", dict(pimax=10.0, npibins=10))):
        wr = kw.get("weighted", False)
        got, exp = both(ctx, kind, edges, d, autocorr=True, periodic=True, box=100.0, **kw)
        assert_match(got, exp, wr, wr)
        got, exp = both(ctx, kind, edges, d, d, autocorr=False, periodic=True, box=100.0, **kw)
        assert_match(got, exp, wr, wr)


def test_maximum_bin_counts(ctx):
    """The largest tables the ABI accepts (252 bins; 252 x 252 rp-pi slots).  An rp-pi or mocks
    histogram that large does not fit in one warp's shared memory: those kinds then add straight
    into the global histograms.  r keeps lane-private histograms (one warp per CTA with weights
    and ravg)."""
    d = gen.clustered_box(40, 40, 1.0, 40.0, 81)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 82)
    edges = gen.log_edges(0.05, 9.0, 252)
    for weighted, ravg in ((False, False), (True, True)):
        kw = dict(autocorr=True, periodic=True, box=40.0, pimax=9.0, npibins=252, weighted=weighted, ravg=ravg)
        assert_match(gpu_count(ctx, "rppi", edges, d, **kw), oracle.count("rppi", edges, d, **kw), weighted, ravg)
    kw = dict(autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
    assert_match(gpu_count(ctx, "r", edges, d, **kw), oracle.count("r", edges, d, **kw), True, True)
    m = gen.survey_cone(3000, 0.0, 30.0, 10.0, 40.0, 100.0, 140.0, 83, members=30, sigma=1.0)
    m.w = gen.uniform_weights(m.n, 0.5, 1.5, 84)
    kw = dict(autocorr=True, periodic=False, pimax=9.0, npibins=252, weighted=True, ravg=True)
    assert_match(gpu_count(ctx, "mocks", edges, m, **kw), oracle.count("mocks", edges, m, **kw), True, True)


@pytest.mark.parametrize("kind", ["r", "rppi", "wp", "theta", "mocks"])
def test_band_audit_agrees(ctx, kind):
    """CF_OPT_AUDIT sends every evaluated pair to the FP64 recheck: its counts must equal the normal
    FP32 path's bit for bit (the band audit) and the oracle's."""
    import paper_1911_03545_gb300 as cf
    if kind == "theta":
        d = gen.sphere_patch(20000, 0.0, 40.0, -10.0, 30.0, 91)
        edges = gen.log_edges(0.01, 2.0, 16)
        kw = dict(autocorr=True, periodic=False)
    elif kind == "mocks":
        d = gen.survey_cone(20000, 0.0, 60.0, 0.0, 40.0, 100.0, 300.0, 92, members=50, sigma=1.5)
        edges = gen.log_edges(0.2, 15.0, 12)
        kw = dict(autocorr=True, periodic=False, pimax=15.0, npibins=15)
    else:
        d = gen.clustered_box(400, 50, 1.0, 100.0, 93)
        edges = gen.log_edges(0.1, 10.0, 16)
        kw = dict(autocorr=True, periodic=True, box=100.0)
        if kind in ("rppi", "wp"):
            kw.update(pimax=12.0, npibins=12)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 94)
    kw.update(weighted=True, ravg=True)
    normal = gpu_count(ctx, kind, edges, d, **kw)
    st = cf.cf_get_stats(ctx)
    cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, 1)
    try:
        assert_match(gpu_count(ctx, kind, edges, d, **kw), normal, True, True)
        sp = cf.cf_get_stats(ctx)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, 0)
    cf.cf_set_option(ctx, cf.CF_OPT_AUDIT, 1)
    try:
        audited = gpu_count(ctx, kind, edges, d, **kw)
        sa = cf.cf_get_stats(ctx)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_AUDIT, 0)
    # every pair of the work items is queued: a cell's pairs with itself once (j > i), the rest
    # i x j.  Block pruning evaluates fewer (how many fewer varies a little from call to call: the
    # points of a sub-cell take their places, and so their 32-point groups, by atomic ranks).
    assert sa["evaluated_pairs"] == st["evaluated_pairs"] and sp["evaluated_pairs"] <= st["evaluated_pairs"]
    assert int(np.asarray(audited["npairs"]).sum()) // 2 <= sa["rechecked_pairs"] <= sa["evaluated_pairs"]
    assert_match(normal, audited, True, True)
    assert_match(audited, oracle.count(kind, edges, d, **kw), True, True)


@pytest.mark.parametrize("periodic", [True, False])
def test_points_on_and_beside_cell_boundaries(ctx, periodic):
    """The cell build computes cell coordinates, cell-relative positions and cell-pair gaps in float32
    for float32 inputs, and redoes a coordinate in FP64 within a guard band of a cell boundary.  Here
    the cells are exactly as wide as the largest edge, so a point put in the wrong neighbour cell
    would lose pairs just inside that edge; every coordinate lies on a boundary, 1-3 ulps beside
    one, or half a cell in, on a grid that starts at 0 (periodic) or at -30 (non-periodic)."""
    L, w = 60.0, 6.0
    edges = gen.log_edges(0.5, w, 8)                       # 10 cells of width 6 = the last edge
    lo = 0.0 if periodic else -30.0
    rng = np.random.Generator(np.random.PCG64(404))
    vals = []
    for k in range(11):
        b = np.float32(lo + w * k)
        for d in (-3, -2, -1, 0, 1, 2, 3):
            v = b
            for _ in range(abs(d)):
                v = np.nextafter(v, np.float32(np.inf) if d > 0 else np.float32(-np.inf), dtype=np.float32)
            vals.append(v)
        vals.append(np.float32(lo + w * k + 0.5 * w))
    vals = np.array(sorted(set(float(v) for v in vals)), dtype=np.float32)
    vals = vals[(vals >= lo) & (vals <= lo + L)] if periodic else vals[(vals >= lo) & (vals <= lo + 60.0)]
    if periodic:
        vals = vals[vals < L]                              # x = L is the same place as 0
    n = 3000
    pts = vals[rng.integers(0, len(vals), size=(n, 3))]
    d = gen.Catalogue(pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(),
                      gen.uniform_weights(n, 0.5, 1.5, 405))
    kw = dict(autocorr=True, periodic=periodic, box=L, weighted=True, ravg=True)
    got = gpu_count(ctx, "r", edges, d, **kw)
    exp = oracle.count("r", edges, d, **kw)
    assert_match(got, exp, True, True)
    assert int(np.asarray(exp["npairs"]).sum()) > 10000


def test_work_list_outgrows_the_previous_size(ctx):
    """A repeat call on the same plan writes its work list in one pass, into the previous call's
    size plus a quarter.  A catalogue with many more cell pairs than the one before it overflows
    that capacity; the call then counts again with the size it measured.  Every call equals the
    oracle."""
    import torch
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    try:
        edges = gen.log_edges(0.2, 5.0, 8)
        dense = gen.clustered_box(1, 20000, 0.5, 100.0, 71)     # a few cells
        spread = gen.uniform_box(20000, 100.0, 72)              # every cell
        items = []
        for d in (dense, spread, dense, spread):
            got, exp = both(c, "r", edges, d, autocorr=True, periodic=True, box=100.0)
            assert_match(got, exp)
            items.append(cf.cf_get_stats(c)["work_items"])
        assert items[1] > items[0] + items[0] // 4 + 1024
        assert items[3] == items[1] and items[2] == items[0]
    finally:
        cf.cf_destroy(c)


def test_scan_over_many_tiles(ctx):
    """The cell scan's tile offsets are scanned by the last block in chunks of 4096 tiles: 68^3
    cells with 64 Morton sub-cells each make 2.0e7 keys (4913 tiles), so the second chunk runs.
    The grid has more cells than points, so the work list visits only the listed cells that hold
    points.  Two calls (the second writes its work list in one pass) equal the oracle."""
    import torch
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    try:
        cf.cf_set_option(c, cf.CF_OPT_CELL_ORDER, 4)
        edges = gen.log_edges(0.1, 1.0, 6)
        d = gen.uniform_box(200000, 68.0, 81)
        for _ in range(2):
            got, exp = both(c, "r", edges, d, autocorr=True, periodic=True, box=68.0)
            assert_match(got, exp)
        assert cf.cf_get_stats(c)["cells"] == 68 ** 3
    finally:
        cf.cf_destroy(c)


def test_work_list_in_instance_order(ctx):
    """A work list long enough to be handed to the pair kernel ordered by instance (tiles of up to
    128 points of cells holding from a few to several hundred clustered points, so every tile size
    and cells with themselves; j ranges of 32: tens of thousands of items).  Two calls (the second
    writes its list in one pass) equal the oracle for weighted DD(r) with ravg and for DD(rp, pi)."""
    import torch
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    try:
        cf.cf_set_option(c, cf.CF_OPT_TILE, 128)
        cf.cf_set_option(c, cf.CF_OPT_JCHUNK, 32)
        d = gen.clustered_box(800, 100, 1.0, 40.0, 131)
        d.w = gen.uniform_weights(d.n, 0.5, 1.5, 132)
        edges = gen.log_edges(0.1, 6.0, 12)
        kw_r = dict(autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
        kw_p = dict(autocorr=True, periodic=True, box=40.0, pimax=6.0, npibins=6)
        exp_r, exp_p = oracle.count("r", edges, d, **kw_r), oracle.count("rppi", edges, d, **kw_p)
        for _ in range(2):
            assert_match(gpu_count(c, "r", edges, d, **kw_r), exp_r, True, True)
            assert cf.cf_get_stats(c)["work_items"] >= 40960
            assert_match(gpu_count(c, "rppi", edges, d, **kw_p), exp_p)
    finally:
        cf.cf_destroy(c)


@pytest.mark.parametrize("kind", ["r", "theta", "rppi"])
def test_device_views_not_16_byte_aligned(ctx, kind):
    """Device inputs may be views that start 4 bytes into an allocation (x = t[1:]): the passes that
    read four float32 points per 16-byte load take their per-point path then, with the same
    results (a periodic call, whose input check runs beside the build, and a non-periodic one)."""
    import torch

    import paper_1911_03545_gb300 as cf
    if kind == "theta":
        d = gen.sphere_patch(5001, 0.0, 30.0, -10.0, 20.0, 97)
        edges = gen.log_edges(0.01, 2.0, 10)
        kws = [dict(autocorr=True, periodic=False)]
    else:
        d = gen.clustered_box(50, 100, 1.0, 40.0, 98)
        edges = gen.log_edges(0.1, 6.0, 10)
        kws = [dict(autocorr=True, periodic=True, box=40.0), dict(autocorr=True, periodic=False)]
        if kind == "rppi":
            kws = [dict(k, pimax=8.0, npibins=8) for k in kws]
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 99)
    for kw in kws:
        kw = dict(kw, weighted=True, ravg=True)
        ts = []
        for a in (d.x, d.y, d.z, d.w):
            t = torch.empty(d.n + 1, dtype=torch.float32, device="cuda:0")
            t[1:] = torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")
            ts.append(t[1:])
        assert ts[0].data_ptr() % 16 != 0
        p = cf.params(kind=kind, edges=edges, **{k: v for k, v in kw.items() if k != "ravg"}, ravg=True)
        got = cf.cf_count(ctx, p, cf.points(*ts))
        exp = oracle.count(kind, edges, d, **kw)
        assert_match(got, exp, True, True)
