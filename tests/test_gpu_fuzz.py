"""Randomised GPU parity: seeded random problems against the FP64 oracle.

Each case draws a kind, auto or cross, periodic or not (mocks and theta: not), the box, how the points
are placed (uniform, clustered, far from the origin), their dtype, the number and spacing of the
edges (log or linear, sometimes starting at 0), weights, ravg, the refinement and the pair-kernel
options, and compares the library with the oracle: counts bit-exact, sums within 1e-6 relative.
The cases are small (the oracle's brute force finishes in milliseconds) but span several cells,
ragged tiles and, with many bins, large tables.
"""
import math

import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import assert_match, gpu_count

pytestmark = pytest.mark.gpu

NCASES = 200


def _case(seed):
    r = np.random.Generator(np.random.PCG64(9000 + seed))
    kind = ["r", "rppi", "wp", "theta", "mocks"][int(r.integers(0, 5))]
    autocorr = bool(r.random() < 0.6)
    periodic = kind in ("r", "rppi", "wp") and bool(r.random() < 0.6)
    if kind == "wp":
        autocorr = True
    dtype = np.float64 if r.random() < 0.3 else np.float32
    n1 = int(r.integers(1, 1500))
    n2 = int(r.integers(1, 1500))
    nb = int(r.choice([1, 2, 5, 12, 30, 80, 252]))
    weighted = bool(r.random() < 0.4)
    ravg = bool(r.random() < 0.4)
    kw = dict(autocorr=autocorr, periodic=periodic, weighted=weighted, ravg=ravg)
    if kind == "theta":
        tmax = float(r.uniform(0.5, 40.0))
        ra0 = float(r.uniform(0, 300))
        dec0 = float(r.uniform(-90, 60))
        span = float(r.uniform(2, 60))

        def cat(n, s):
            return gen.sphere_patch(n, ra0, ra0 + span, dec0, min(90.0, dec0 + span), s)
        lo = tmax * float(r.uniform(0.002, 0.3))
    else:
        L = float(r.uniform(8.0, 300.0))
        rmax = L * float(r.uniform(0.03, 0.45 if periodic else 0.8))
        off = 0.0 if periodic else float(r.choice([0.0, -L / 2, 1000.0, 30000.0]))
        clustered = r.random() < 0.5
        if kind == "mocks":
            off = float(r.choice([0.0, 3.0 * L, 20.0 * L]))   # observer inside or far outside

        def cat(n, s):
            if clustered:
                c = gen.clustered_box(max(1, n // 20), 20, max(0.05, rmax / 8), L, s)
                c = c.subset(slice(0, n)) if c.n > n else c
            else:
                c = gen.uniform_box(n, L, s)
            return gen.Catalogue(*(getattr(c, a).astype(np.float64) + off for a in "xyz"))
        lo = rmax * float(r.uniform(0.001, 0.3))
        kw["box"] = L
        tmax = rmax
        if kind in ("rppi", "wp", "mocks"):
            kw["pimax"] = float(rmax * r.uniform(0.3, 1.2))
            kw["npibins"] = int(r.choice([1, 3, 10, 40]))
    hi = tmax
    if r.random() < 0.5:
        edges = np.exp(np.linspace(math.log(lo), math.log(hi), nb + 1))
    else:
        edges = np.linspace(lo, hi, nb + 1)
    edges[-1] = hi
    if r.random() < 0.2:
        edges[0] = 0.0
    d1 = cat(n1, 9100 + seed)
    d2 = None if autocorr else cat(n2, 9200 + seed)
    for d in (d1, d2):
        if d is None:
            continue
        d.x, d.y, d.z = (v.astype(dtype) for v in (d.x, d.y, d.z))
        if weighted:
            d.w = (gen.uniform_weights(d.n, 0.1, 3.0, 9300 + seed)).astype(dtype)
    opts = dict(refine=(int(r.integers(1, 4)),) * 3)
    knobs = {"variant": int(r.integers(1, 3)), "tile": int(r.choice([128, 64])),
             "jchunk": int(r.choice([512, 128])), "noprune": int(r.integers(0, 2)),
             "thetagrid": int(r.integers(0, 2)), "block": int(r.integers(0, 2))}
    return kind, edges, d1, d2, kw, opts, knobs


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    yield c
    cf.cf_destroy(c)


@pytest.mark.parametrize("seed", range(NCASES))
def test_random_problem(ctx, seed):
    from paper_1911_03545_gb300 import tune
    kind, edges, d1, d2, kw, opts, knobs = _case(seed)
    tune.apply(ctx, knobs)
    try:
        got = gpu_count(ctx, kind, edges, d1, d2, refine=opts["refine"], **kw)
    finally:
        tune.reset(ctx)
    exp = oracle.count(kind, edges, d1, d2, mode="brute", **kw)
    assert_match(got, exp, kw["weighted"], kw["ravg"])
