"""Full-size parity: the measured workloads at their full sizes, in the launch configuration
bench.py times, against expected histograms the FP64 oracle wrote (tests/golden/make_golden.py).

Counts must be bit-identical; weighted sums and ravg within 1e-6 relative.  A fingerprint of the
generated arrays guards against a generator that produces different inputs on another machine.
"""
import json
import os

import numpy as np
import pytest

import gen
from tests.golden.make_golden import fingerprint, workload
from tests.gpu_util import TOL, to_dev

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
NAMES = sorted(f[5:-5] for f in os.listdir(GOLDEN) if f.startswith("full_") and f.endswith(".json"))


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    yield c
    cf.cf_destroy(c)


BLOCK = ["clustered_r_1m", "clustered_rppi_2m_wr", "clustered_rppi_dr", "mock_dr_rppi"]


@pytest.mark.parametrize("name,block", [(n, 0) for n in NAMES] + [(n, 1) for n in BLOCK if n in NAMES])
def test_full_size_against_oracle(ctx, name, block):
    """Default options, and for some workloads with the work list's group pruning on."""
    import paper_1911_03545_gb300 as cf
    with open(os.path.join(GOLDEN, f"full_{name}.json")) as f:
        gold = json.load(f)
    wl = workload(name)
    if fingerprint(wl.d1, wl.d2) != gold["fingerprint"]:
        pytest.skip("this machine's generator produced different inputs than the golden file's")
    p = cf.params(kind=wl.kind, edges=wl.edges, autocorr=wl.autocorr, periodic=wl.periodic, box=wl.box,
                  pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted, ravg=wl.ravg)

    def pts(c):
        t = to_dev(c, "cuda:0", wl.weighted)
        return cf.points(*t[:3], t[3] if wl.weighted else None)

    cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, block)
    try:
        got = cf.cf_count(ctx, p, pts(wl.d1), None if wl.autocorr else pts(wl.d2))
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_BLOCK_PRUNE, 0)
    if name == "clustered_rppi_2m_wr":
        assert cf.cf_get_stats(ctx)["fixed_sums"] == 3     # weights in [0.5, 1.5): fixed-point sums
    n = np.asarray(got["npairs"]).ravel().astype(np.uint64)
    e = np.asarray(gold["npairs"], dtype=np.uint64)
    assert np.array_equal(n, e), np.argwhere(n != e)[:10]
    if wl.weighted:
        np.testing.assert_allclose(np.asarray(got["wsum"]).ravel(), gold["wsum"], rtol=TOL, atol=0)
    if wl.ravg:
        np.testing.assert_allclose(np.asarray(got["ravg"]).ravel(), gold["ravg"], rtol=TOL, atol=0)


TUNED = ["clustered_r_1m", "clustered_rppi_2m", "sphere_theta_1m", "mock_dr_rppi", "clustered_rppi_2m_wr"]


@pytest.mark.parametrize("name", [n for n in TUNED if n in NAMES])
def test_full_size_in_the_tuned_configuration(ctx, name):
    """The launch configuration bench.py times is the tuner's pick: run the tuner on the workload
    (no cache), then count in that configuration and compare with the oracle's histogram."""
    import torch

    import paper_1911_03545_gb300 as cf
    from paper_1911_03545_gb300 import tune
    with open(os.path.join(GOLDEN, f"full_{name}.json")) as f:
        gold = json.load(f)
    wl = workload(name)
    if fingerprint(wl.d1, wl.d2) != gold["fingerprint"]:
        pytest.skip("this machine's generator produced different inputs than the golden file's")
    p = cf.params(kind=wl.kind, edges=wl.edges, autocorr=wl.autocorr, periodic=wl.periodic, box=wl.box,
                  pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted, ravg=wl.ravg)

    def pts(c):
        t = to_dev(c, "cuda:0", wl.weighted)
        return cf.points(*t[:3], t[3] if wl.weighted else None)

    d1 = pts(wl.d1)
    d2 = None if wl.autocorr else pts(wl.d2)
    cfg = tune.tune(ctx, p, d1, d2, device_name=torch.cuda.get_device_name(0),
                    npoints=wl.d1.n + (0 if wl.autocorr else wl.d2.n), reps=1, passes=1, use_cache=False)
    try:
        got = cf.cf_count(ctx, p, d1, d2)
    finally:
        tune.reset(ctx)
    n = np.asarray(got["npairs"]).ravel().astype(np.uint64)
    assert np.array_equal(n, np.asarray(gold["npairs"], dtype=np.uint64)), (cfg, np.argwhere(n != gold["npairs"])[:10])
    if wl.weighted:
        np.testing.assert_allclose(np.asarray(got["wsum"]).ravel(), gold["wsum"], rtol=TOL, atol=0)
    if wl.ravg:
        np.testing.assert_allclose(np.asarray(got["ravg"]).ravel(), gold["ravg"], rtol=TOL, atol=0)


@pytest.mark.parametrize("name", [n for n in ("clustered_r_1m", "mock_dr_rppi") if n in NAMES])
def test_full_size_band_audit(ctx, name):
    """The band audit at full size: with CF_OPT_AUDIT every evaluated pair is binned by the FP64
    recheck alone, and the result must equal the oracle's histogram (as the FP32 path's does)."""
    import paper_1911_03545_gb300 as cf
    with open(os.path.join(GOLDEN, f"full_{name}.json")) as f:
        gold = json.load(f)
    wl = workload(name)
    if fingerprint(wl.d1, wl.d2) != gold["fingerprint"]:
        pytest.skip("this machine's generator produced different inputs than the golden file's")
    p = cf.params(kind=wl.kind, edges=wl.edges, autocorr=wl.autocorr, periodic=wl.periodic, box=wl.box,
                  pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted, ravg=wl.ravg)

    def pts(c):
        t = to_dev(c, "cuda:0", wl.weighted)
        return cf.points(*t[:3], t[3] if wl.weighted else None)

    cf.cf_set_option(ctx, cf.CF_OPT_AUDIT, 1)
    # refinement 2 keeps the mocks workload's evaluated pairs (4e9 at refinement 1) within the
    # audit's 32-bit queue count
    cf.cf_set_option(ctx, cf.CF_OPT_REFINE, 2 if name == "mock_dr_rppi" else 0)
    try:
        got = cf.cf_count(ctx, p, pts(wl.d1), None if wl.autocorr else pts(wl.d2))
        st = cf.cf_get_stats(ctx)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_AUDIT, 0)
        cf.cf_set_option(ctx, cf.CF_OPT_REFINE, 0)
    # every evaluated pair went to FP64 (a cell's pairs with itself once, j > i): several 1e8 of them
    assert 5 * 10 ** 8 < st["rechecked_pairs"] <= st["evaluated_pairs"]
    if not wl.autocorr:
        assert st["rechecked_pairs"] == st["evaluated_pairs"]
    n = np.asarray(got["npairs"]).ravel().astype(np.uint64)
    assert np.array_equal(n, np.asarray(gold["npairs"], dtype=np.uint64)), np.argwhere(n != gold["npairs"])[:10]
    if wl.weighted:
        np.testing.assert_allclose(np.asarray(got["wsum"]).ravel(), gold["wsum"], rtol=TOL, atol=0)
    if wl.ravg:
        np.testing.assert_allclose(np.asarray(got["ravg"]).ravel(), gold["ravg"], rtol=TOL, atol=0)
