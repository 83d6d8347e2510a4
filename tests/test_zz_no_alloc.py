"""The allocation-free entry point against the regular one (GPU).

cf_count_noalloc is for callers that cannot allocate device memory (a framework's memory pool,
plugins where allocation is forbidden, code that must not allocate after start-up).  It writes
into the caller's device tensors using only a fixed scratch array inside the library.  Its
results must equal cf_count's: counts bit-exact, weighted sums and ravg within 1e-6 relative,
on two calls in a row (the second call must not see the first call's scratch contents).
"""
import numpy as np
import pytest

import gen
from tests.gpu_util import TOL, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    ctx = cf.cf_create(0, torch.cuda.current_stream())
    yield cf, ctx, torch
    cf.cf_destroy(ctx)


CASES = [
    ("r", True, True, True, True),
    ("rppi", True, True, False, False),
    ("theta", True, False, False, True),
    ("wp", False, True, True, False),
    ("mocks", False, False, True, True),
]


@pytest.mark.parametrize("kind,autocorr,periodic,weighted,ravg", CASES)
def test_noalloc_matches_cf_count_twice(env, kind, autocorr, periodic, weighted, ravg):
    cf, ctx, torch = env
    if kind == "theta":
        d1 = gen.sphere_patch(2500, 0.0, 20.0, 0.0, 20.0, 61)
        d2 = gen.sphere_patch(2000, 0.0, 20.0, 0.0, 20.0, 62)
        edges = gen.log_edges(0.02, 3.0, 12)
    else:
        d1 = gen.clustered_box(40, 60, 1.2, 40.0, 63)
        d2 = gen.clustered_box(30, 60, 1.2, 40.0, 64)
        edges = gen.log_edges(0.05, 7.0, 12)
    d1.w = gen.uniform_weights(d1.n, 0.5, 1.5, 65)
    d2.w = gen.uniform_weights(d2.n, 0.5, 1.5, 66)
    p = cf.params(kind=kind, edges=edges, autocorr=autocorr, periodic=periodic, box=40.0, pimax=9.0, npibins=9,
                  weighted=weighted, ravg=ravg)
    t1 = to_dev(d1, "cuda:0", weighted)
    t2 = to_dev(d2, "cuda:0", weighted)
    P1 = cf.points(*t1[:3], t1[3] if weighted else None)
    P2 = None if autocorr else cf.points(*t2[:3], t2[3] if weighted else None)
    exp = cf.cf_count(ctx, p, P1, P2)
    stream = torch.cuda.current_stream()
    for _ in range(2):
        npairs = torch.full((p.nout,), 12345, dtype=torch.int64, device="cuda:0")
        wsum = torch.full((p.nout,), -1.0, dtype=torch.float64, device="cuda:0")
        rav = torch.full((p.nout,), -1.0, dtype=torch.float64, device="cuda:0")
        cf.cf_count_noalloc(p, P1, P2, npairs, wsum, rav, stream)
        torch.cuda.synchronize()
        got_n = npairs.cpu().numpy().astype(np.uint64)
        assert np.array_equal(got_n, np.asarray(exp["npairs"]).ravel())
        if weighted:
            np.testing.assert_allclose(wsum.cpu().numpy(), np.asarray(exp["wsum"]).ravel(), rtol=TOL, atol=0)
        if ravg:
            np.testing.assert_allclose(rav.cpu().numpy(), np.asarray(exp["ravg"]).ravel(), rtol=TOL, atol=0)


def test_noalloc_rejects_oversized_histogram(env):
    cf, ctx, torch = env
    d = gen.uniform_box(100, 40.0, 1)
    t = to_dev(d, "cuda:0", False)
    p = cf.params(kind="rppi", edges=gen.log_edges(0.1, 5.0, 100), autocorr=True, periodic=True, box=40.0,
                  pimax=30.0, npibins=30)                     # 3000 slots > 2048
    out = torch.zeros(p.nout, dtype=torch.int64, device="cuda:0")
    with pytest.raises(cf.CfError) as ei:
        cf.cf_count_noalloc(p, cf.points(*t[:3]), None, out)
    assert ei.value.status == -1
