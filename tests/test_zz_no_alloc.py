"""The allocation-free entry point against the regular one (GPU).

cf_count_noalloc is for callers that cannot allocate device memory (a framework's memory pool,
plugins where allocation is forbidden, code that must not allocate after start-up).  It writes
into the caller's device tensors using only a fixed scratch array inside the library.  Its
results must equal cf_count's and the FP64 oracle's: counts bit-exact, weighted sums and ravg
within 1e-6 relative, on two calls in a row (the second call must not see the first call's scratch
contents).  After its first call on a device (which resolves the scratch array's address and may
load the library's device code), further calls must leave the device's free memory unchanged.
"""
import numpy as np
import pytest

import gen
import oracle
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


# kind, autocorr, periodic, weighted, ravg, first edge at 0 (self pairs of Appendix B), float64 inputs
CASES = [
    ("r", True, True, True, True, False, False),
    ("rppi", True, True, False, False, False, False),
    ("theta", True, False, False, True, False, False),
    ("wp", False, True, True, False, False, False),
    ("mocks", False, False, True, True, False, False),
    ("r", True, True, True, True, True, False),        # the w^2 self-pair sum and the N self pairs
    ("rppi", True, True, True, True, True, False),
    ("r", True, True, True, True, False, True),        # float64 inputs
    ("mocks", True, False, True, True, True, True),
]


def _inputs(kind, zero_edge, f64):
    if kind == "theta":
        d1 = gen.sphere_patch(2500, 0.0, 20.0, 0.0, 20.0, 61)
        d2 = gen.sphere_patch(2000, 0.0, 20.0, 0.0, 20.0, 62)
        edges = gen.log_edges(0.02, 3.0, 12)
    elif kind == "mocks":
        d1 = gen.survey_cone(2400, 0.0, 30.0, 10.0, 40.0, 60.0, 90.0, 63, members=30, sigma=1.2)
        d2 = gen.survey_cone(1800, 0.0, 30.0, 10.0, 40.0, 60.0, 90.0, 64, members=30, sigma=1.2)
        edges = gen.log_edges(0.05, 7.0, 12)
    else:
        d1 = gen.clustered_box(40, 60, 1.2, 40.0, 63)
        d2 = gen.clustered_box(30, 60, 1.2, 40.0, 64)
        edges = gen.log_edges(0.05, 7.0, 12)
    if zero_edge:
        edges = np.concatenate([[0.0], edges])
    for i, d in enumerate((d1, d2)):
        d.w = gen.uniform_weights(d.n, 0.5, 1.5, 65 + i)
        if f64:
            for a in ("x", "y", "z", "w"):
                setattr(d, a, getattr(d, a).astype(np.float64))
    return d1, d2, edges


@pytest.mark.parametrize("kind,autocorr,periodic,weighted,ravg,zero_edge,f64", CASES)
def test_noalloc_matches_cf_count_twice(env, kind, autocorr, periodic, weighted, ravg, zero_edge, f64):
    cf, ctx, torch = env
    d1, d2, edges = _inputs(kind, zero_edge, f64)
    p = cf.params(kind=kind, edges=edges, autocorr=autocorr, periodic=periodic, box=40.0, pimax=9.0, npibins=9,
                  weighted=weighted, ravg=ravg)
    t1 = to_dev(d1, "cuda:0", weighted)
    t2 = to_dev(d2, "cuda:0", weighted)
    P1 = cf.points(*t1[:3], t1[3] if weighted else None)
    P2 = None if autocorr else cf.points(*t2[:3], t2[3] if weighted else None)
    exp = cf.cf_count(ctx, p, P1, P2)
    kw = dict(autocorr=autocorr, periodic=periodic, box=40.0, pimax=9.0, npibins=9, weighted=weighted, ravg=ravg)
    orc = oracle.count(kind, edges, d1, None if autocorr else d2, **kw)
    assert np.array_equal(np.asarray(exp["npairs"]).ravel(), np.asarray(orc["npairs"]).ravel())
    if zero_edge:
        assert int(np.asarray(orc["npairs"]).ravel()[0]) >= d1.n      # the self pairs are in bin 0
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
            np.testing.assert_allclose(wsum.cpu().numpy(), np.asarray(orc["wsum"]).ravel(), rtol=TOL, atol=0)
        if ravg:
            np.testing.assert_allclose(rav.cpu().numpy(), np.asarray(exp["ravg"]).ravel(), rtol=TOL, atol=0)
            np.testing.assert_allclose(rav.cpu().numpy(), np.asarray(orc["ravg"]).ravel(), rtol=TOL, atol=0)


def test_noalloc_leaves_device_memory_unchanged(env):
    """The property the entry point exists for: once its first call on the device has resolved the
    scratch address, calls change neither the device's free memory (cudaMemGetInfo) nor what torch
    holds.  The outputs are allocated before the measurement."""
    cf, ctx, torch = env
    d1, _, edges = _inputs("r", True, False)
    p = cf.params(kind="r", edges=edges, autocorr=True, periodic=True, box=40.0, weighted=True, ravg=True)
    t1 = to_dev(d1, "cuda:0", True)
    P1 = cf.points(*t1[:3], t1[3])
    outs = [torch.zeros(p.nout, dtype=torch.int64, device="cuda:0"),
            torch.zeros(p.nout, dtype=torch.float64, device="cuda:0"),
            torch.zeros(p.nout, dtype=torch.float64, device="cuda:0")]
    stream = torch.cuda.current_stream()
    cf.cf_count_noalloc(p, P1, None, *outs, stream)        # first call on this device
    torch.cuda.synchronize()
    first = [o.clone() for o in outs]
    # the device is shared with nothing else in this process; another process changing its free
    # memory between the two readings would show as a mismatch, so take the best of three tries
    same = False
    for _ in range(3):
        free0, _ = torch.cuda.mem_get_info()
        reserved0 = torch.cuda.memory_reserved()
        for _ in range(3):
            cf.cf_count_noalloc(p, P1, None, *outs, stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        if free1 == free0 and torch.cuda.memory_reserved() == reserved0:
            same = True
            break
    assert same, (free0, free1)
    # the same results: counts exactly, FP64 sums (added in a varying order) within the tolerance
    assert torch.equal(first[0], outs[0])
    for a, b in zip(first[1:], outs[1:]):
        np.testing.assert_allclose(b.cpu().numpy(), a.cpu().numpy(), rtol=TOL, atol=0)


def test_noalloc_binding_checks_its_outputs(env):
    """The binding hands raw pointers to the library, which writes p.nout entries: it refuses a
    tensor that is short, of the wrong type, not contiguous or not on the GPU."""
    cf, ctx, torch = env
    d = gen.uniform_box(200, 40.0, 2)
    t = to_dev(d, "cuda:0", False)
    p = cf.params(kind="r", edges=gen.log_edges(0.5, 5.0, 6), autocorr=True, periodic=True, box=40.0,
                  weighted=False, ravg=True)
    P = cf.points(*t[:3])
    good = torch.zeros(p.nout, dtype=torch.int64, device="cuda:0")
    bad = [torch.zeros(p.nout - 1, dtype=torch.int64, device="cuda:0"),
           torch.zeros(p.nout, dtype=torch.int32, device="cuda:0"),
           torch.zeros(2 * p.nout, dtype=torch.int64, device="cuda:0")[::2],
           torch.zeros(p.nout, dtype=torch.int64)]
    for b in bad:
        with pytest.raises(ValueError):
            cf.cf_count_noalloc(p, P, None, b)
    with pytest.raises(ValueError):
        cf.cf_count_noalloc(p, P, None, good, None, torch.zeros(p.nout, dtype=torch.float32, device="cuda:0"))
    cf.cf_count_noalloc(p, P, None, good, None, torch.zeros(p.nout, dtype=torch.float64, device="cuda:0"))
    torch.cuda.synchronize()


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
