"""How the pair kernel holds its sums: per-warp fixed point (two 32-bit words per slot) for rp-pi
and mocks where the terms' range allows it, FP64 otherwise, and flushes bounded in pairs so that
no 32-bit count or fixed-point word a warp holds can wrap.

Each case checks which form ran (cf_stats.fixed_sums) and compares with the FP64 oracle: counts
bit-exact, sums within 1e-6 relative (negative weights: within 1e-6 of the sum of |terms|, the
bound that FP32 products allow when a sum may cancel).  The last case puts every pair of 1.5M
points into one (rp, pi) slot on one warp per SM, so that each warp sees several times 2^32
pairs of that slot; the count has the closed form N^2 (ordered pairs plus the N self pairs of a
first edge at 0, Appendix B).
"""
import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import TOL, assert_match, gpu_count

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


def _box(n, seed, w):
    d = gen.clustered_box(max(1, n // 40), 40, 1.0, 60.0, seed)
    d.w = np.asarray(w(d.n, seed + 1)).astype(d.x.dtype)
    return d


def _run(ctx, kind, edges, d, weighted, ravg):
    import paper_1911_03545_gb300 as cf
    if kind == "mocks":
        kw = dict(autocorr=True, periodic=False, pimax=12.0, npibins=6, weighted=weighted, ravg=ravg)
    else:
        kw = dict(autocorr=True, periodic=True, box=60.0, pimax=12.0, npibins=6, weighted=weighted, ravg=ravg)
    got = gpu_count(ctx, kind, edges, d, **kw)
    return got, cf.cf_get_stats(ctx)["fixed_sums"], kw


def _cone(n, seed, w):
    d = gen.survey_cone(n, 0.0, 40.0, 10.0, 40.0, 150.0, 260.0, seed, members=40, sigma=1.0)
    d.w = np.asarray(w(d.n, seed + 1)).astype(d.x.dtype)
    return d


def _narrow(n, s):
    return gen.uniform_weights(n, 0.5, 1.5, s)


def _wide(n, s):
    # log-uniform over six decades: products span 1e12, beyond any fixed-point scale
    r = np.random.Generator(np.random.PCG64(s))
    return np.exp(r.uniform(np.log(1e-3), np.log(1e3), n))


@pytest.mark.parametrize("kind", ["rppi", "mocks"])
@pytest.mark.parametrize("weighted,ravg,want", [(True, False, 1), (False, True, 2), (True, True, 3)])
def test_fixed_point_sums(ctx, kind, weighted, ravg, want):
    d = _box(6000, 11, _narrow) if kind == "rppi" else _cone(6000, 12, _narrow)
    edges = gen.log_edges(0.1, 10.0, 10)
    got, fx, kw = _run(ctx, kind, edges, d, weighted, ravg)
    assert fx == want
    assert_match(got, oracle.count(kind, edges, d, **kw), weighted, ravg)


@pytest.mark.parametrize("kind", ["rppi", "mocks"])
def test_fp64_sums_when_the_range_is_wide(ctx, kind):
    d = _box(6000, 21, _wide) if kind == "rppi" else _cone(6000, 22, _wide)
    edges = gen.log_edges(0.1, 10.0, 10)
    got, fx, kw = _run(ctx, kind, edges, d, True, True)
    assert fx == 0
    assert_match(got, oracle.count(kind, edges, d, **kw), True, True)
    # weights off, ravg over edges spanning 1e2: fixed point again for ravg
    got, fx, kw = _run(ctx, kind, edges, d, False, True)
    assert fx == 2
    assert_match(got, oracle.count(kind, edges, d, **kw), False, True)


@pytest.mark.parametrize("kind", ["rppi", "mocks"])
def test_fp64_ravg_from_a_first_edge_at_zero(ctx, kind):
    """rp may then be arbitrarily small against its bin's sum: with ravg every sum of the call
    stays FP64 (one form per call); weight sums alone do not depend on the edges."""
    d = _box(5000, 31, _narrow) if kind == "rppi" else _cone(5000, 32, _narrow)
    edges = np.concatenate([[0.0], gen.log_edges(0.1, 10.0, 8)])
    for weighted, ravg, want in ((True, True, 0), (False, True, 0), (True, False, 1)):
        got, fx, kw = _run(ctx, kind, edges, d, weighted, ravg)
        assert fx == want
        assert_match(got, oracle.count(kind, edges, d, **kw), weighted, ravg)


@pytest.mark.parametrize("kind", ["rppi", "mocks"])
def test_negative_weights_stay_fp64(ctx, kind):
    def signed(n, s):
        return np.random.Generator(np.random.PCG64(s)).uniform(-1.0, 1.5, n)
    d = _box(5000, 41, signed) if kind == "rppi" else _cone(5000, 42, signed)
    edges = gen.log_edges(0.1, 10.0, 8)
    got, fx, kw = _run(ctx, kind, edges, d, True, False)
    assert fx == 0
    exp = oracle.count(kind, edges, d, **kw)
    assert np.array_equal(np.asarray(got["npairs"]), np.asarray(exp["npairs"]))
    d_abs = gen.Catalogue(d.x, d.y, d.z, np.abs(d.w))
    scale = np.asarray(oracle.count(kind, edges, d_abs, **kw)["wsum"])
    err = np.abs(np.asarray(got["wsum"]) - np.asarray(exp["wsum"]))
    assert np.all(err <= TOL * scale), float(np.max(err / np.maximum(scale, 1e-300)))


def test_captured_batch_keeps_fp64_sums(ctx):
    """A captured graph is replayed on new weights: its sums are FP64 whatever the first call's
    weights allowed."""
    import torch

    import paper_1911_03545_gb300 as cf
    from tests.gpu_util import to_dev
    d = _box(4000, 51, _narrow)
    edges = gen.log_edges(0.1, 10.0, 8)
    kw = dict(autocorr=True, periodic=True, box=60.0, pimax=12.0, npibins=6, weighted=True, ravg=True)
    p = cf.params(kind="rppi", edges=edges, **kw)
    t = to_dev(d, "cuda:0", True)
    cats = [cf.points(*t[:3], t[3])]
    cf.cf_batch_capture(ctx, p, cats)
    w2 = _wide(d.n, 52).astype(d.x.dtype)
    t[3].copy_(torch.from_numpy(w2))
    out = cf.cf_batch_replay(ctx, p, 1)
    assert cf.cf_get_stats(ctx)["fixed_sums"] == 0
    d2 = gen.Catalogue(d.x, d.y, d.z, w2)
    assert_match(out[0], oracle.count("rppi", edges, d2, **kw), True, True)


def test_counts_past_32_bits_per_warp(ctx):
    """1.5M points in a unit cube, one rp bin [0, 2) and one pi bin [0, 2): every ordered pair and
    every self pair lands in slot (0, 0), N^2 = 2.25e12 in all.  With one warp per SM each warp
    evaluates about 7e9 pairs of that slot, past 2^32; the bounded flushes keep its 32-bit counts
    exact."""
    import torch

    import paper_1911_03545_gb300 as cf
    n = 1_500_000
    d = gen.uniform_box(n, 1.0, 61)
    edges = np.array([0.0, 2.0])
    opts = {cf.CF_OPT_CTAS_PER_SM: 1, cf.CF_OPT_WARPS: 1, cf.CF_OPT_QUEUE: 1 << 24}
    for k, v in opts.items():
        cf.cf_set_option(ctx, k, v)
    try:
        got = gpu_count(ctx, "rppi", edges, d, autocorr=True, periodic=False, pimax=2.0, npibins=1)
        st = cf.cf_get_stats(ctx)
    finally:
        for k in opts:
            cf.cf_set_option(ctx, k, 0)
    assert int(np.asarray(got["npairs"]).ravel()[0]) == n * n
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert st["evaluated_pairs"] / sms > 1.5 * 2 ** 32
