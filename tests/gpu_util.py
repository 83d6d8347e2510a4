"""Helpers shared by the GPU tests: run a workload through the C ABI and through the oracle."""
import numpy as np

import oracle

TOL = 1e-6          # relative tolerance for weighted sums and ravg (counts are compared exactly)


def to_dev(cat, dev, with_w=True):
    import torch
    arrs = [cat.x, cat.y, cat.z] + ([cat.w] if (with_w and cat.w is not None) else [])
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrs]


def gpu_count(ctx, kind, edges, d1, d2=None, *, autocorr, periodic, box=0.0, pimax=0.0, npibins=0,
              weighted=False, ravg=False, refine=(0, 0, 0), device=True, dev="cuda:0"):
    import paper_1911_03545_gb300 as cf
    p = cf.params(kind=kind, edges=edges, autocorr=autocorr, periodic=periodic, box=box, pimax=pimax,
                  npibins=npibins, ravg=ravg, weighted=weighted, refine=refine)

    def pts(d):
        if device:
            t = to_dev(d, dev, weighted)
            return cf.points(*t[:3], t[3] if weighted else None)
        return cf.points(d.x, d.y, d.z, d.w if weighted else None)

    return cf.cf_count(ctx, p, pts(d1), None if autocorr else pts(d2))


def oracle_count(kind, edges, d1, d2=None, **kw):
    return oracle.count(kind, edges, d1, d2, **kw)


def assert_match(got, exp, weighted=False, ravg=False, tol=TOL):
    g = np.asarray(got["npairs"]).astype(np.uint64)
    e = np.asarray(exp["npairs"]).astype(np.uint64)
    if not np.array_equal(g, e):
        diff = np.argwhere(g != e)
        raise AssertionError(f"counts differ at {diff[:10].tolist()}: gpu {g[tuple(diff[0])]} oracle {e[tuple(diff[0])]}"
                             f"\n gpu={g.ravel().tolist()}\n orc={e.ravel().tolist()}")
    if weighted:
        np.testing.assert_allclose(got["wsum"], exp["wsum"], rtol=tol, atol=0)
    if ravg:
        np.testing.assert_allclose(got["ravg"], exp["ravg"], rtol=tol, atol=0)
