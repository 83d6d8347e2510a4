"""DD(rp, pi) of observed positions (Appendix A.2.1, the line of sight of Fisher et al.) on the GPU
against the FP64 oracle: hand-worked pairs, survey cones of clustered mock galaxies and randoms
(auto and data-random cross, refinement 1-3), weights and ravg on float32 and float64 inputs,
catalogues around the observer (the near-observer recheck), pairs on the bin edges, self pairs,
the allocation-free entry point, and what the kind refuses."""
import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import assert_match, gpu_count, to_dev
from tests.test_oracle_mocks import EDGES, HAND, NPI, PIMAX

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


def _cat(pts, w=None, dtype=np.float32):
    pts = np.asarray(pts, dtype=np.float64)
    return gen.Catalogue(*(pts[:, a].astype(dtype) for a in range(3)),
                         None if w is None else np.asarray(w, dtype=dtype))


def _orc(edges, d1, d2=None, **kw):
    kw.setdefault("pimax", PIMAX)
    kw.setdefault("npibins", NPI)
    return oracle.count("mocks", edges, d1, d2, autocorr=d2 is None, periodic=False, **kw)


def _gpu(ctx, edges, d1, d2=None, **kw):
    kw.setdefault("pimax", PIMAX)
    kw.setdefault("npibins", NPI)
    return gpu_count(ctx, "mocks", edges, d1, d2, autocorr=d2 is None, periodic=False, **kw)


def test_hand_pairs(ctx):
    for (a, b, c, d), expect in HAND:
        cat = _cat([(a, b, c), (-a, -b, d)])
        got = np.asarray(_gpu(ctx, EDGES, cat)["npairs"])
        want = np.zeros((len(EDGES) - 1, NPI), dtype=np.uint64)
        if expect is not None:
            want[expect] = 2
        assert np.array_equal(got, want), ((a, b, c, d), got.tolist())


def _cone(scale, seed_shift=0):
    wl = gen.workload("mock_dr_rppi", scale)
    if seed_shift:
        wl.d1 = gen.survey_cone(wl.d1.n, 0.0, 90.0, 0.0, 60.0, 300.0, 300.0 + 700.0 * scale ** (1 / 3),
                                1007 + seed_shift, members=100, sigma=2.0)
    return wl


@pytest.mark.parametrize("refine", [1, 2, 3])
def test_cone_auto_and_data_random(ctx, refine):
    wl = _cone(0.02)
    kw = dict(pimax=wl.pimax, npibins=wl.npibins)
    r = (refine,) * 3
    got = _gpu(ctx, wl.edges, wl.d1, refine=r, **kw)
    assert_match(got, _orc(wl.edges, wl.d1, **kw))
    assert int(np.asarray(got["npairs"]).sum()) > 10000
    got = _gpu(ctx, wl.edges, wl.d1, wl.d2, refine=r, **kw)
    assert_match(got, _orc(wl.edges, wl.d1, wl.d2, **kw))
    assert int(np.asarray(got["npairs"]).sum()) > 10000


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_weights_and_ravg(ctx, dtype):
    wl = _cone(0.01, seed_shift=5)
    d1 = gen.Catalogue(*(getattr(wl.d1, a).astype(dtype) for a in "xyz"),
                       gen.uniform_weights(wl.d1.n, 0.5, 1.5, 901).astype(dtype))
    d2 = gen.Catalogue(*(getattr(wl.d2, a)[:8000].astype(dtype) for a in "xyz"),
                       gen.uniform_weights(8000, 0.5, 1.5, 902).astype(dtype))
    edges = gen.log_edges(0.05, 30.0, 12)
    kw = dict(pimax=35.0, npibins=7, weighted=True, ravg=True)
    assert_match(_gpu(ctx, edges, d1, **kw), _orc(edges, d1, **kw), True, True)
    assert_match(_gpu(ctx, edges, d1, d2, **kw), _orc(edges, d1, d2, **kw), True, True)
    kw["weighted"] = False
    assert_match(_gpu(ctx, edges, d1, **kw), _orc(edges, d1, **kw), False, True)


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_observer_inside_the_catalogue(ctx, dtype):
    """Points all around the observer: midpoints near the origin go to the FP64 recheck; pairs
    symmetric about the origin have l = 0 exactly (pi = 0 by the definition)."""
    r = np.random.Generator(np.random.PCG64(903))
    c = r.uniform(-40, 40, size=(60, 3))
    pts = (c[:, None, :] + r.normal(0, 1.5, size=(60, 40, 3))).reshape(-1, 3)
    sym = r.uniform(-3, 3, size=(200, 3))
    pts = np.concatenate([pts, sym, -sym, [[0.0, 0.0, 0.0]]])
    d = _cat(pts, w=r.uniform(0.5, 1.5, len(pts)), dtype=dtype)
    edges = gen.log_edges(0.2, 8.0, 10)
    kw = dict(pimax=8.0, npibins=8, weighted=True, ravg=True)
    got = _gpu(ctx, edges, d, **kw)
    assert_match(got, _orc(edges, d, **kw), True, True)
    e0 = np.concatenate([[0.0], edges])
    kw = dict(pimax=8.0, npibins=8)
    assert_match(_gpu(ctx, e0, d, **kw), _orc(e0, d, **kw))


def test_pairs_on_the_edges(ctx):
    """A dyadic lattice seen from far along z: separations and line-of-sight components land on
    the rp and pi edges exactly, so many pairs sit inside the FP32 bands and are rechecked."""
    import paper_1911_03545_gb300 as cf
    g = np.arange(-6, 7) * 0.5
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel() + 4096.0], axis=1)
    d = _cat(pts)
    edges = np.array([0.5, 1.0, 1.5, 2.0, 3.0, 4.0])
    kw = dict(pimax=4.0, npibins=8)
    assert_match(_gpu(ctx, edges, d, **kw), _orc(edges, d, **kw))
    assert cf.cf_get_stats(ctx)["rechecked_pairs"] > 0


def test_self_pairs_and_cross_with_itself(ctx):
    wl = _cone(0.005)
    e0 = np.concatenate([[0.0], wl.edges])
    kw = dict(pimax=wl.pimax, npibins=wl.npibins)
    auto = _gpu(ctx, e0, wl.d1, **kw)
    cross = _gpu(ctx, e0, wl.d1, wl.d1, **kw)
    assert np.array_equal(auto["npairs"], cross["npairs"])
    assert_match(auto, _orc(e0, wl.d1, **kw))
    assert int(np.asarray(auto["npairs"])[0, 0]) >= wl.d1.n


def test_host_inputs_and_refused_requests(ctx):
    import paper_1911_03545_gb300 as cf
    wl = _cone(0.005)
    kw = dict(pimax=wl.pimax, npibins=wl.npibins)
    host = _gpu(ctx, wl.edges, wl.d1, device=False, **kw)
    assert_match(host, _orc(wl.edges, wl.d1, **kw))
    # this kind has the direct form only: a request for the compacting form runs it anyway
    cf.cf_set_option(ctx, cf.CF_OPT_VARIANT, 2)
    try:
        again = _gpu(ctx, wl.edges, wl.d1, **kw)
        assert cf.cf_get_stats(ctx)["variant"] == 1
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_VARIANT, 0)
    assert np.array_equal(host["npairs"], again["npairs"])
    with pytest.raises(cf.CfError) as ei:
        gpu_count(ctx, "mocks", wl.edges, wl.d1, autocorr=True, periodic=True, box=2000.0, **kw)
    assert ei.value.status == -1


def test_noalloc_entry_point(ctx):
    import torch

    import paper_1911_03545_gb300 as cf
    wl = _cone(0.003)
    d1 = gen.Catalogue(wl.d1.x, wl.d1.y, wl.d1.z, gen.uniform_weights(wl.d1.n, 0.5, 1.5, 904))
    edges = gen.log_edges(0.5, 30.0, 6)
    p = cf.params(kind="mocks", edges=edges, autocorr=True, periodic=False, pimax=30.0, npibins=10,
                  weighted=True, ravg=True)
    t = to_dev(d1, "cuda:0", True)
    nout = p.nout
    npairs = torch.zeros(nout, dtype=torch.int64, device="cuda:0")
    wsum = torch.zeros(nout, dtype=torch.float64, device="cuda:0")
    ravg = torch.zeros(nout, dtype=torch.float64, device="cuda:0")
    cf.cf_count_noalloc(p, cf.points(*t[:3], t[3]), None, npairs, wsum, ravg, torch.cuda.current_stream())
    torch.cuda.synchronize()
    exp = _orc(edges, d1, pimax=30.0, npibins=10, weighted=True, ravg=True)
    got = {"npairs": npairs.cpu().numpy().reshape(6, 10), "wsum": wsum.cpu().numpy().reshape(6, 10),
           "ravg": ravg.cpu().numpy().reshape(6, 10)}
    assert_match(got, exp, True, True)
