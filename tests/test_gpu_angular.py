"""DD(theta) on the angular grid (declination bands x right-ascension cells, Sec. 4.1.2) against the
FP64 oracle: footprints from a small patch to the full sky and a polar cap, refinement 1-3, a small and
a large largest angle (the large one makes cells near the poles search every RA cell)."""
import numpy as np
import pytest

import gen
import oracle
from tests.gpu_util import assert_match, gpu_count

pytestmark = pytest.mark.gpu

FOOTPRINTS = {
    "patch": (0.0, 25.0, -5.0, 20.0),
    "full_sky": (0.0, 360.0, -90.0, 90.0),
    "polar_cap": (0.0, 360.0, 62.0, 90.0),
    "equatorial_strip": (0.0, 360.0, -1.5, 1.5),
}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_1911_03545_gb300 as cf
    c = cf.cf_create(0, torch.cuda.current_stream())
    cf.cf_set_option(c, cf.CF_OPT_THETA_GRID, 1)
    yield c
    cf.cf_destroy(c)


@pytest.mark.parametrize("refine", [1, 2, 3])
@pytest.mark.parametrize("tmax", [2.5, 20.0])
@pytest.mark.parametrize("name", sorted(FOOTPRINTS))
def test_angular_grid_parity(ctx, name, tmax, refine):
    ra0, ra1, dec0, dec1 = FOOTPRINTS[name]
    n = 2500 if tmax > 10 else 6000
    d = gen.sphere_patch(n, ra0, ra1, dec0, dec1, 300 + refine)
    edges = gen.log_edges(tmax / 200.0, tmax, 12)
    got = gpu_count(ctx, "theta", edges, d, autocorr=True, periodic=False, refine=(refine, refine, refine))
    exp = oracle.count("theta", edges, d, autocorr=True, periodic=False)
    assert_match(got, exp)
    assert int(np.asarray(got["npairs"]).sum()) > 1000


@pytest.mark.parametrize("name", ["full_sky", "polar_cap"])
def test_angular_grid_weights_ravg_cross_float64(ctx, name):
    ra0, ra1, dec0, dec1 = FOOTPRINTS[name]
    d1 = gen.sphere_patch(4000, ra0, ra1, dec0, dec1, 311)
    d2 = gen.sphere_patch(3000, ra0, ra1, dec0, dec1, 312)
    d1.w = gen.uniform_weights(d1.n, 0.5, 1.5, 313)
    d2.w = gen.uniform_weights(d2.n, 0.5, 1.5, 314)
    edges = gen.log_edges(0.05, 6.0, 10)
    kw = dict(periodic=False, weighted=True, ravg=True)
    got = gpu_count(ctx, "theta", edges, d1, d2, autocorr=False, **kw)
    assert_match(got, oracle.count("theta", edges, d1, d2, autocorr=False, **kw), True, True)
    got = gpu_count(ctx, "theta", edges, d1, autocorr=True, **kw)
    assert_match(got, oracle.count("theta", edges, d1, autocorr=True, **kw), True, True)
    f64 = gen.Catalogue(*(getattr(d1, a).astype(np.float64) for a in "xyz"))
    got = gpu_count(ctx, "theta", edges, f64, autocorr=True, periodic=False)
    assert_match(got, oracle.count("theta", edges, f64, autocorr=True, periodic=False))


def test_angular_grid_equals_3d_grid_and_rejects_non_unit(ctx):
    import paper_1911_03545_gb300 as cf
    d = gen.sphere_patch(5000, 0.0, 360.0, 40.0, 90.0, 315)
    edges = gen.log_edges(0.02, 4.0, 10)
    ang = gpu_count(ctx, "theta", edges, d, autocorr=True, periodic=False)
    cf.cf_set_option(ctx, cf.CF_OPT_THETA_GRID, 0)
    try:
        grid3 = gpu_count(ctx, "theta", edges, d, autocorr=True, periodic=False)
    finally:
        cf.cf_set_option(ctx, cf.CF_OPT_THETA_GRID, 1)
    assert np.array_equal(ang["npairs"], grid3["npairs"])
    long = gen.Catalogue(d.x * np.float32(1.01), d.y * np.float32(1.01), d.z * np.float32(1.01))
    with pytest.raises(cf.CfError) as ei:
        gpu_count(ctx, "theta", edges, long, autocorr=True, periodic=False)
    assert ei.value.status == -1
    # the context stays usable
    again = gpu_count(ctx, "theta", edges, d, autocorr=True, periodic=False)
    assert np.array_equal(again["npairs"], ang["npairs"])
