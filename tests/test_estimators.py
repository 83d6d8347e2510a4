"""Estimators on top of the counts (Sec. 2.1, Eq. 2, Appendix B): closed forms, identities, and
agreement with the oracle's wp formula; one GPU test ties them to the library's wp output."""
import math

import numpy as np
import pytest

import gen
from paper_1911_03545_gb300 import estimators as est


def test_rr_analytic_closed_forms():
    n, box = 1000, 50.0
    edges = np.array([0.0, 1.0, 2.0, 5.0])
    rr = est.rr_analytic("r", edges, n, box)
    # total over bins: the whole sphere of radius 5 at density (N-1)/V, plus N self pairs
    assert rr.sum() == pytest.approx(4.0 / 3.0 * math.pi * 125.0 * n * (n - 1) / box ** 3 + n, rel=1e-12)
    assert rr[1] == pytest.approx(4.0 / 3.0 * math.pi * 7.0 * n * (n - 1) / box ** 3, rel=1e-12)
    rp = np.array([0.5, 1.0, 3.0])
    rr2 = est.rr_analytic("rppi", rp, n, box, pimax=4.0, npibins=4)
    assert rr2.shape == (2, 4)
    # every pi bin of one rp bin has the same volume: annulus x 2 x dpi
    assert np.allclose(rr2[0], math.pi * 0.75 * 2.0 * n * (n - 1) / box ** 3, rtol=1e-12)
    wp = est.rr_analytic("wp", rp, n, box, pimax=4.0)
    assert np.allclose(wp, rr2.sum(axis=1), rtol=1e-12)


def test_xi_theory_of_uniform_box_is_zero(orc):
    import oracle
    n, box = 6000, 40.0
    d = gen.uniform_box(n, box, 11)
    edges = gen.log_edges(1.0, 12.0, 8)
    dd = oracle.count("r", edges, d, autocorr=True, periodic=True, box=box, lib=orc)["npairs"]
    xi = est.xi_theory(dd, n, box, edges)
    rr = est.rr_analytic("r", edges, n, box)
    # ordered counts are twice the unique ones: sigma(xi) = sqrt(2 RR) / RR for Poisson-like bins
    sig = np.sqrt(2.0 * rr) / rr
    assert np.all(np.abs(xi) < 5 * sig)


def test_landy_szalay_identity_when_randoms_are_the_data(orc):
    """With R = D (first edge > 0): DR = cross(D, D) = DD and LS = 2/N exactly."""
    import oracle
    n = 2500
    d = gen.clustered_box(50, 50, 1.0, 40.0, 12)
    edges = gen.log_edges(0.2, 8.0, 8)
    kw = dict(periodic=True, box=40.0, lib=orc)
    dd = oracle.count("r", edges, d, autocorr=True, **kw)["npairs"]
    dr = oracle.count("r", edges, d, d, autocorr=False, **kw)["npairs"]
    assert np.array_equal(dd, dr)
    ls = est.landy_szalay(dd, dr, dd, n, n)
    live = np.asarray(dd) > 0
    assert np.allclose(ls[live], 2.0 / n, rtol=1e-9, atol=0)


def test_landy_szalay_of_uniform_data_is_small(orc):
    import oracle
    d, r = gen.uniform_box(3000, 40.0, 21), gen.uniform_box(6000, 40.0, 22)
    edges = gen.log_edges(2.0, 10.0, 5)
    kw = dict(periodic=True, box=40.0, lib=orc)
    dd = oracle.count("r", edges, d, autocorr=True, **kw)["npairs"]
    dr = oracle.count("r", edges, d, r, autocorr=False, **kw)["npairs"]
    rr = oracle.count("r", edges, r, autocorr=True, **kw)["npairs"]
    ls = est.landy_szalay(dd, dr, rr, d.n, r.n)
    assert np.all(np.abs(ls) < 0.05)


def test_wp_from_xi_equals_oracle_wp_formula(orc):
    """Eq. 2 summed over unit-width pi bins of the natural estimator equals the oracle's closed form
    DD_total / (N(N-1)/V * pi (rp_hi^2 - rp_lo^2)) - 2 pimax."""
    import oracle
    n, box = 4000, 60.0
    d = gen.clustered_box(80, 50, 2.0, box, 13)
    edges = gen.log_edges(0.5, 10.0, 6)
    kw = dict(autocorr=True, periodic=True, box=box, pimax=12.0, npibins=12, lib=orc)
    rppi = oracle.count("rppi", edges, d, **kw)["npairs"]
    rr = est.rr_analytic("rppi", edges, n, box, pimax=12.0, npibins=12)
    wp = est.wp_from_xi(est.xi_natural(rppi, rr, n, n), 12.0, 12)
    dd_wp = np.asarray(rppi).reshape(6, 12).sum(axis=1)
    ref = oracle.wp_from_counts(dd_wp, edges, n, [box] * 3, 12.0)
    assert np.allclose(wp, ref, rtol=1e-10, atol=1e-9)


@pytest.mark.gpu
def test_library_wp_equals_estimator_on_its_counts():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    from tests.gpu_util import gpu_count
    n, box = 20000, 100.0
    d = gen.clustered_box(400, 50, 2.0, box, 14)
    edges = gen.log_edges(0.5, 15.0, 8)
    ctx = cf.cf_create(0, torch.cuda.current_stream())
    try:
        kw = dict(autocorr=True, periodic=True, box=box, pimax=20.0, npibins=20)
        rppi = gpu_count(ctx, "rppi", edges, d, **kw)["npairs"]
        got = gpu_count(ctx, "wp", edges, d, **kw)
    finally:
        cf.cf_destroy(ctx)
    rr = est.rr_analytic("rppi", edges, n, box, pimax=20.0, npibins=20)
    wp = est.wp_from_xi(est.xi_natural(rppi, rr, n, n), 20.0, 20)
    assert np.array_equal(np.asarray(rppi).reshape(8, 20).sum(axis=1), got["npairs"])
    assert np.allclose(got["wp"], wp, rtol=1e-10, atol=1e-9)
