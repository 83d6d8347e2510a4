"""GPU tests of the batched (graph-captured) path and of the serving loop.

batched == one at a time == oracle (counts bit-exact); a captured graph replays to the same
result; the server returns each catalogue's result identically whether it ran alone or mixed
with other requests (counts bit-exact, sums within 1e-6), rejects requests above its memory
budget, and cancels queued requests.
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
