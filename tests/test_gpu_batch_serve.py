"""GPU tests of the batched (graph-captured) path and of the serving loop.

batched == one at a time == oracle (counts bit-exact); a captured graph replays to the same
result; the server returns each catalogue's result identically whether it ran alone or mixed
with other requests (counts bit-exact, sums within 1e-6), rejects requests above its memory
budget, withdraws queued requests but lets a running one finish, and fails only the request of a
bad catalogue in a wave.
"""
import time

import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import TOL, to_dev

pytestmark = pytest.mark.gpu

EDGES = gen.log_edges(0.1, 8.0, 10)
L = 60.0


@pytest.fixture(scope="module")
def cf():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as m
    return m


@pytest.fixture(scope="module")
def cats():
    sizes = [900, 3000, 50, 1700, 2500, 400]
    out = []
    for i, n in enumerate(sizes):
        c = gen.batch_catalogue(i, n, L=L, members=20)
        c.w = gen.uniform_weights(c.n, 0.5, 1.5, 500 + i)
        out.append(c)
    return out


def _params(cf, weighted=False):
    return cf.params(kind="rppi", edges=EDGES, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10,
                     weighted=weighted, ravg=weighted)


def test_graph_capture_replay(cf, cats):
    import torch
    cats = list(cats)                       # the new-data replay below must not change the fixture
    ctx = cf.cf_create(0, torch.cuda.current_stream())
    try:
        p = _params(cf)
        pts = [cf.points(*to_dev(c, "cuda:0", False)) for c in cats]
        cf.cf_batch_capture(ctx, p, pts)
        a = cf.cf_batch_replay(ctx, p, len(cats))
        b = cf.cf_batch_replay(ctx, p, len(cats))
        for c, x, y in zip(cats, a, b):
            exp = oracle.count("rppi", EDGES, c, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10)
            assert np.array_equal(x["npairs"], exp["npairs"])
            assert np.array_equal(y["npairs"], exp["npairs"])
        # new data of the same sizes in the same device buffers: the replay counts the new data
        for i, c in enumerate(cats):
            c2 = gen.batch_catalogue(100 + i, c.n, L=L, members=20)
            for ax, t in zip("xyz", pts[i].keep[:3]):
                t.copy_(torch.from_numpy(getattr(c2, ax)).to(t.device))
            cats[i] = c2
        d = cf.cf_batch_replay(ctx, p, len(cats))
        for c, x in zip(cats, d):
            exp = oracle.count("rppi", EDGES, c, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10)
            assert np.array_equal(x["npairs"], exp["npairs"])
    finally:
        cf.cf_destroy(ctx)


def test_replay_checks_that_new_data_fit_the_plan(cf):
    """A replay re-runs the bounding-box pass.  New data that left the captured box (the plan's grid
    and FP32 error bands were made for it) are counted afresh without the graph, which is then
    dropped; data that no call accepts (outside the periodic box, non-finite) are refused."""
    import torch
    ctx = cf.cf_create(0, torch.cuda.current_stream())
    try:
        kw = dict(autocorr=True, periodic=False, pimax=10.0, npibins=10)
        p = cf.params(kind="rppi", edges=EDGES, **kw)
        cs = [gen.batch_catalogue(40 + i, n, L=L, members=20) for i, n in enumerate((1200, 800))]
        pts = [cf.points(*to_dev(c, "cuda:0", False)) for c in cs]
        cf.cf_batch_capture(ctx, p, pts)
        same = cf.cf_batch_replay(ctx, p, 2)
        assert cf.cf_get_stats(ctx)["ms_build"] == 0          # the graph ran
        for c, x in zip(cs, same):
            assert np.array_equal(x["npairs"], oracle.count("rppi", EDGES, c, **kw)["npairs"])
        big = gen.Catalogue(*(getattr(cs[1], ax) * np.float32(1.5) for ax in "xyz"))
        for ax, t in zip("xyz", pts[1].keep[:3]):
            t.copy_(torch.from_numpy(getattr(big, ax)).to(t.device))
        moved = cf.cf_batch_replay(ctx, p, 2)
        assert cf.cf_get_stats(ctx)["ms_build"] > 0           # counted afresh
        for c, x in zip((cs[0], big), moved):
            assert np.array_equal(x["npairs"], oracle.count("rppi", EDGES, c, **kw)["npairs"])
        with pytest.raises(cf.CfError):
            cf.cf_batch_replay(ctx, p, 2)                      # the graph was dropped

        pp = cf.params(kind="rppi", edges=EDGES, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10)
        pts = [cf.points(*to_dev(c, "cuda:0", False)) for c in cs]
        for bad in (L + 5.0, float("nan")):
            cf.cf_batch_capture(ctx, pp, pts)
            keep = float(pts[0].keep[0][7])
            pts[0].keep[0][7] = bad
            with pytest.raises(cf.CfError) as ei:
                cf.cf_batch_replay(ctx, pp, 2)
            assert ei.value.status == -1
            pts[0].keep[0][7] = keep
    finally:
        cf.cf_destroy(ctx)


def test_server_alone_equals_mixed(cf, cats):
    p = _params(cf, weighted=True)
    srv = cf.cf_server_start(0, p, 1 << 30, 64)
    try:
        alone = []
        for c in cats:
            t = cf.cf_server_submit(srv, p, cf.points(c.x, c.y, c.z, c.w))
            r = None
            while r is None:
                r = cf.cf_server_poll(srv, t, 1000)
            alone.append(r)
        tickets = [cf.cf_server_submit(srv, p, cf.points(c.x, c.y, c.z, c.w)) for c in cats]
        mixed = []
        for t in tickets:
            r = None
            while r is None:
                r = cf.cf_server_poll(srv, t, 1000)
            mixed.append(r)
    finally:
        cf.cf_server_stop(srv)
    for c, a, m in zip(cats, alone, mixed):
        exp = oracle.count("rppi", EDGES, c, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10,
                           weighted=True, ravg=True)
        assert np.array_equal(a["npairs"], exp["npairs"])
        assert np.array_equal(m["npairs"], a["npairs"])
        np.testing.assert_allclose(m["wsum"], a["wsum"], rtol=TOL)
        np.testing.assert_allclose(m["ravg"], exp["ravg"], rtol=TOL)


def test_server_budget_and_cancel(cf, cats):
    p = _params(cf)
    srv = cf.cf_server_start(0, p, 8 << 20, 2)
    try:
        big = gen.uniform_box(200000, L, 9)
        with pytest.raises(cf.CfError) as ei:
            cf.cf_server_submit(srv, p, cf.points(big.x, big.y, big.z))
        assert ei.value.status == -2
        tickets = [cf.cf_server_submit(srv, p, cf.points(c.x, c.y, c.z)) for c in cats for _ in range(3)]
        cf.cf_server_cancel(srv, tickets[-1])
        done = 0
        for t in tickets[:-1]:
            r = None
            deadline = time.time() + 60
            while r is None and time.time() < deadline:
                r = cf.cf_server_poll(srv, t, 500)
            assert r is not None
            done += 1
        try:                      # cancelled while queued, or finished before the cancel landed
            r = None
            deadline = time.time() + 60
            while r is None and time.time() < deadline:
                r = cf.cf_server_poll(srv, tickets[-1], 500)
        except cf.CfError as e:
            assert e.status == -6
    finally:
        cf.cf_server_stop(srv)
    assert done == len(tickets) - 1


def test_server_cancel_running_and_queued(cf, cats):
    """A cancel withdraws a queued request (poll then reports CF_ERR_CANCELLED) but not one whose
    wave is on the GPU: that cancel returns False, the request's buffers stay in use, and poll
    returns its full result.  One slot means one request on the GPU at a time, so most of a quick
    burst is still queued when its cancel arrives."""
    p = _params(cf)
    srv = cf.cf_server_start(0, p, 1 << 30, 1)
    order = [i % len(cats) for i in range(24)]
    try:
        tickets = [cf.cf_server_submit(srv, p, cf.points(cats[k].x, cats[k].y, cats[k].z)) for k in order]
        withdrawn = [cf.cf_server_cancel(srv, t) for t in tickets]
        outcome = []
        for t in tickets:
            try:
                r = None
                deadline = time.time() + 60
                while r is None and time.time() < deadline:
                    r = cf.cf_server_poll(srv, t, 500)
                assert r is not None
                outcome.append(r)
            except cf.CfError as e:
                assert e.status == -6
                outcome.append(None)
    finally:
        cf.cf_server_stop(srv)
    exp = [oracle.count("rppi", EDGES, c, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10)
           for c in cats]
    for k, w, r in zip(order, withdrawn, outcome):
        if not w:                       # on the GPU when cancelled: ran to the end
            assert r is not None
        if r is not None:
            assert np.array_equal(r["npairs"], exp[k]["npairs"])
    assert sum(1 for w, r in zip(withdrawn, outcome) if w and r is None) > 0


def test_server_one_bad_catalogue_fails_alone(cf, cats):
    """A catalogue the library rejects (a periodic position outside [0, L]) fails its own request;
    the requests counted in the same wave still get their results."""
    p = _params(cf)
    bad = gen.Catalogue(cats[0].x.copy(), cats[0].y.copy(), cats[0].z.copy())
    bad.x[3] = np.float32(L * 1.5)
    srv = cf.cf_server_start(0, p, 1 << 30, 16)
    try:
        pts = [cf.points(c.x, c.y, c.z) for c in cats[:3]] + [cf.points(bad.x, bad.y, bad.z)] + \
              [cf.points(c.x, c.y, c.z) for c in cats[3:]]
        tickets = [cf.cf_server_submit(srv, p, q) for q in pts]
        got = []
        for t in tickets:
            try:
                r = None
                while r is None:
                    r = cf.cf_server_poll(srv, t, 1000)
                got.append(r)
            except cf.CfError as e:
                got.append(e.status)
        msg = cf.cf_server_last_error(srv)
    finally:
        cf.cf_server_stop(srv)
    assert got[3] == -1 and "[0, box]" in msg
    for c, r in zip(cats, got[:3] + got[4:]):
        exp = oracle.count("rppi", EDGES, c, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10)
        assert np.array_equal(r["npairs"], exp["npairs"])


def test_mocks_batched_and_served(cf):
    """DD(rp, pi) of mock catalogues (Appendix A.2.1) through the batched launch and the server:
    each catalogue's result equals the oracle's, alone and in the mix."""
    import torch
    mcats = [gen.survey_cone(n, 0.0, 40.0, 10.0, 40.0, 100.0, 160.0, 700 + i, members=10, sigma=1.0)
             for i, n in enumerate([800, 2000, 60, 1500])]
    for i, c in enumerate(mcats):
        c.w = gen.uniform_weights(c.n, 0.5, 1.5, 710 + i)
    edges = gen.log_edges(0.2, 8.0, 8)
    p = cf.params(kind="mocks", edges=edges, autocorr=True, periodic=False, pimax=8.0, npibins=8,
                  weighted=True, ravg=True)
    exp = [oracle.count("mocks", edges, c, autocorr=True, periodic=False, pimax=8.0, npibins=8, weighted=True,
                        ravg=True) for c in mcats]
    ctx = cf.cf_create(0, torch.cuda.current_stream())
    try:
        got = cf.cf_batch_count(ctx, p, [cf.points(*to_dev(c, "cuda:0", True)) for c in mcats])
    finally:
        cf.cf_destroy(ctx)
    srv = cf.cf_server_start(0, p, 1 << 30, 16)
    try:
        tickets = [cf.cf_server_submit(srv, p, cf.points(c.x, c.y, c.z, c.w)) for c in mcats]
        served = []
        for t in tickets:
            r = None
            while r is None:
                r = cf.cf_server_poll(srv, t, 1000)
            served.append(r)
    finally:
        cf.cf_server_stop(srv)
    for e, g, s in zip(exp, got, served):
        for r in (g, s):
            assert np.array_equal(np.asarray(r["npairs"]), e["npairs"])
            np.testing.assert_allclose(r["wsum"], e["wsum"], rtol=TOL)
            np.testing.assert_allclose(r["ravg"], e["ravg"], rtol=TOL)
