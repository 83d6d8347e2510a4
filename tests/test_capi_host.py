"""Host-side tests of the C ABI (no GPU): the library loads, exports every function that
include/cf.h declares, validates arguments, and plans correctly.

The plan probe exposes the host planner: grid dimensions (Sec. 4.1 Eq. 3, Sec. 4.2), the
neighbour stencil (Sec. 4.3), the FP32 error bands and the bin lookup tables (Sec. 4.7).  The
tables are checked exhaustively around every edge against the definition of the classes, and
the bands are checked against the actual FP32 error of the kernel's arithmetic sequence.
"""
import ctypes
import math

import numpy as np
import pytest

import gen


@pytest.fixture(scope="module")
def cf():
    from paper_1911_03545_gb300 import build
    build.build()
    import paper_1911_03545_gb300 as m
    return m


def test_library_exports_every_declared_function(cf):
    from paper_1911_03545_gb300 import _capi
    names = _capi.header_functions()
    assert len(names) >= 16, names
    L = _capi.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_null_arguments_are_rejected(cf):
    from paper_1911_03545_gb300 import _capi
    L = _capi.lib()
    assert L.cf_set_option(None, 1, 0) == _capi.CF_ERR_ARG
    assert L.cf_get_stats(None, None) == _capi.CF_ERR_ARG
    assert L.cf_destroy(None) == _capi.CF_ERR_ARG
    assert L.cf_count(None, None, None, None, None) == _capi.CF_ERR_ARG
    assert L.cf_last_error(None) == b"null context"
    assert L.cf_server_poll(None, 1, 0) == _capi.CF_ERR_ARG
    assert L.cf_plan_probe(None, None, 0, 0, None, None, None, 0, None, 0, None) == _capi.CF_ERR_ARG


@pytest.mark.parametrize("edges,err", [([1.0, 0.5], "increasing"), ([-1.0, 2.0], ">= 0"),
                                       ([0.1, float("nan")], "finite")])
def test_bad_edges_rejected(cf, edges, err):
    p = cf.params(kind="r", edges=edges, autocorr=True, periodic=True, box=10.0)
    with pytest.raises(cf.CfError):
        cf.cf_plan_probe(p, [0, 0, 0, 10, 10, 10], 100)


def test_bad_params_rejected(cf):
    bb = [0, 0, 0, 10, 10, 10]
    with pytest.raises(cf.CfError):                     # theta is non-periodic
        cf.cf_plan_probe(cf.params(kind="theta", edges=[1, 2], periodic=True, box=1.0), bb, 10)
    with pytest.raises(cf.CfError):                     # pimax required
        cf.cf_plan_probe(cf.params(kind="rppi", edges=[1, 2], periodic=True, box=10.0, npibins=4), bb, 10)
    with pytest.raises(cf.CfError):
        cf.cf_plan_probe(cf.params(kind="r", edges=[1, 2], periodic=True, box=0.0), bb, 10)
    with pytest.raises(cf.CfError):
        cf.cf_plan_probe(cf.params(kind="theta", edges=[1, 190]), bb, 10)


def test_grid_dimensions(cf):
    # Sec. 4.1: n = floor(extent / Rmax) per axis; rp-pi uses Rmax in x, y and pimax in z
    p = cf.params(kind="r", edges=gen.log_edges(0.1, 20.0, 20), autocorr=True, periodic=True, box=420.0)
    info = cf.cf_plan_probe(p, [0, 0, 0, 420, 420, 420], 10 ** 6)
    assert info["grid"] == [21, 21, 21] and info["nstencil"] == 27 and info["wrap"] == [0, 0, 0]
    p = cf.params(kind="rppi", edges=gen.log_edges(0.1, 25.0, 14), autocorr=True, periodic=True, box=1000.0,
                  pimax=40.0, npibins=40)
    info = cf.cf_plan_probe(p, [0, 0, 0, 1000, 1000, 1000], 2 * 10 ** 6)
    assert info["grid"] == [40, 40, 25]
    # Sec. 4.2: k sub-cells per axis, (2k+1)^3 neighbours before pruning by the cell gap
    p = cf.params(kind="r", edges=gen.log_edges(0.1, 20.0, 20), autocorr=True, periodic=True, box=420.0,
                  refine=(2, 2, 2))
    info = cf.cf_plan_probe(p, [0, 0, 0, 420, 420, 420], 10 ** 6)
    assert info["grid"] == [42, 42, 42]
    assert info["nstencil"] == 125                      # the corner gap sqrt(3)*10 < 20: nothing pruned
    p = cf.params(kind="r", edges=gen.log_edges(0.1, 20.0, 20), autocorr=True, periodic=True, box=420.0,
                  refine=(3, 3, 3))
    info = cf.cf_plan_probe(p, [0, 0, 0, 420, 420, 420], 10 ** 6)
    w = 420.0 / 63
    gap2 = [sum((max(0, abs(v) - 1) * w) ** 2 for v in (a, b, c))
            for a in range(-3, 4) for b in range(-3, 4) for c in range(-3, 4)]
    need = sum(1 for g in gap2 if g < 400.0)                 # a pair within Rmax is possible
    allowed = sum(1 for g in gap2 if g <= 400.0 * (1 + 1e-6))  # plus borderline offsets kept by margin
    assert info["grid"] == [63, 63, 63] and need <= info["nstencil"] <= allowed < 343
    # fewer than 2k+1 cells on a periodic axis: explicit minimum image on that axis
    p = cf.params(kind="r", edges=[0.1, 9.0], autocorr=True, periodic=True, box=(10.0, 30.0, 10.0))
    info = cf.cf_plan_probe(p, [0, 0, 0, 10, 30, 10], 1000)
    assert info["wrap"] == [1, 0, 1] and info["grid"] == [1, 3, 1]
    # non-periodic: the grid covers the bounding box
    p = cf.params(kind="theta", edges=gen.log_edges(0.001, 1.0, 20), autocorr=True)
    info = cf.cf_plan_probe(p, [0.0, 0.0, -0.17, 1.0, 1.0, 0.5], 10 ** 6)
    chord = 2 * math.sin(math.radians(1.0) / 2)
    assert info["grid"] == [int(1 / chord), int(1 / chord), int(0.67 / chord)]


def _values_near(e2, stride_far=101, span=3000):
    """float32 bit patterns: every pattern within `span` ulps of each edge, strided elsewhere."""
    lo = np.float32(max(e2[0] * 0.25, 1e-30))
    hi = np.float32(e2[-1] * 4.0)
    b0, b1 = lo.view(np.uint32), hi.view(np.uint32)
    bits = [np.arange(b0, b1, stride_far, dtype=np.uint64)]
    for e in e2:
        if e <= 0:
            continue
        c = int(np.float32(e).view(np.uint32))
        bits.append(np.arange(max(0, c - span), c + span, dtype=np.uint64))
    b = np.unique(np.concatenate(bits)).astype(np.uint32)
    return b.view(np.float32)


def _check_classes(vals, cls, E, B, nbins_out):
    B = np.array(B, dtype=np.float64)
    if E[0] == 0.0:
        B[0] = -np.inf          # no value lies below a first edge of 0: that edge needs no band
    x = vals.astype(np.float64)
    ulp = np.spacing(vals).astype(np.float64)
    dist = np.abs(x[:, None] - E[None, :])
    within = (dist <= B[None, :]).any(axis=1)
    near = (dist <= B[None, :] + 2 * ulp[:, None]).any(axis=1)
    # a value within a band of an edge must be re-evaluated in FP64
    assert np.all(cls[within] == 0xFF), "value within an edge band was not marked ambiguous"
    # an ambiguous value must lie within a band (plus the outward rounding of the band ends)
    assert np.all(near[cls == 0xFF]), "ambiguous region wider than the bands"
    # definite classes must equal the exact bin of the FP32 value
    k = np.searchsorted(E, x, side="right") - 1
    exact = np.where((k >= 0) & (k < len(E) - 1), k, 0xFE)
    if E[0] == 0.0:
        exact = np.where(x < E[-1], np.clip(k, 0, len(E) - 2), 0xFE)
    definite = cls != 0xFF
    assert np.array_equal(cls[definite], exact[definite].astype(np.uint32))
    assert cls.max() <= 0xFF and np.all((cls < nbins_out) | (cls >= 0xFE))


@pytest.mark.parametrize("cut", [0, 2], ids=["clamped", "cut"])
@pytest.mark.parametrize("name", ["clustered_r", "uniform_f64", "theta", "zero_first", "dense_edges"])
def test_lut_matches_band_definition(cf, name, cut):
    import oracle
    box, f64, bbox = 420.0, False, [0, 0, 0, 420, 420, 420]
    if name == "clustered_r":
        kind, edges = "r", gen.log_edges(0.1, 20.0, 20)
    elif name == "uniform_f64":
        kind, edges, f64, box, bbox = "r", gen.log_edges(0.1, 25.0, 20), True, 250.0, [0, 0, 0, 250, 250, 250]
    elif name == "theta":
        kind, edges, bbox = "theta", gen.log_edges(0.001, 1.0, 20), [0.0, 0.0, -0.17, 1.0, 1.0, 0.5]
    elif name == "zero_first":
        kind, edges = "r", np.array([0.0, 0.5, 1.0, 2.0, 4.0, 8.0])
    else:
        kind, edges = "r", np.concatenate([gen.log_edges(1.0, 1.2, 30), [5.0]])
    p = cf.params(kind=kind, edges=edges, autocorr=True, periodic=kind != "theta", box=box)
    E = oracle.squared_edges(kind, edges)
    vals = _values_near(E)
    out = cf.cf_plan_probe(p, bbox, 10 ** 6, f64, which=cut, values=vals)
    _check_classes(vals, out["classes"], E, out["bands_r"], len(edges) - 1)


@pytest.mark.parametrize("cut", [0, 2], ids=["clamped", "cut"])
@pytest.mark.parametrize("kind", ["rppi", "wp"])
def test_pi_lut_matches_band_definition(cf, kind, cut):
    p = cf.params(kind=kind, edges=gen.log_edges(0.1, 25.0, 14), autocorr=True, periodic=True, box=1000.0,
                  pimax=40.0, npibins=40)
    pe = np.arange(41, dtype=np.float64)
    vals = _values_near(pe[1:])
    vals = np.concatenate([vals, np.float32([0.0, 1e-30, 0.5])])
    out = cf.cf_plan_probe(p, [0, 0, 0, 1000, 1000, 1000], 2 * 10 ** 6, which=1 + cut, values=vals)
    if kind == "rppi":
        _check_classes(vals, out["classes"], pe, out["bands_p"], 40)
    else:
        # wp integrates over 0 <= |dz| < pimax: one pi class, banded at pimax only
        _check_classes(vals, out["classes"], pe[[0, 40]], out["bands_p"][[0, 40]], 1)


def _fma32(a, b, c):
    # float32 fused multiply-add emulated in float64: a*b is exact in float64; the sum is
    # correctly rounded except in rare double-rounding cases (one float32 ulp at most)
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(np.float32)


@pytest.mark.parametrize("precise", [False, True])
def test_bands_cover_actual_fp32_error(cf, precise):
    """Replay the kernel's FP32 sequence on random cell-relative pairs of a 420-box grid with
    21 cells per axis and compare with FP64: the error must stay within a quarter of the band
    (the band carries a factor-4 safety margin)."""
    rng = np.random.Generator(np.random.PCG64(3))
    edges = gen.log_edges(0.1, 20.0, 20)
    p = cf.params(kind="r", edges=edges, autocorr=True, periodic=True, box=420.0, ravg=precise)
    info = cf.cf_plan_probe(p, [0, 0, 0, 420, 420, 420], 10 ** 6)
    import oracle
    E = oracle.squared_edges("r", edges)
    w = 20.0
    n = 400000
    xi = rng.uniform(60, 360, size=(n, 3)).astype(np.float32)
    # j within ~25 of i so that most pairs land in the binned range; each point is stored
    # relative to the origin of its own cell, as the scatter kernel does
    xj = (xi.astype(np.float64) + np.clip(rng.normal(0, 8, size=(n, 3)), -50, 50)).astype(np.float32)
    oi = np.floor(xi.astype(np.float64) / w) * w
    oj = np.floor(xj.astype(np.float64) / w) * w
    Xi = (xi.astype(np.float64) - oi).astype(np.float32)
    Xj = (xj.astype(np.float64) - oj).astype(np.float32)
    assert np.array_equal(Xi.astype(np.float64), xi.astype(np.float64) - oi)     # exact
    assert np.array_equal(Xj.astype(np.float64), xj.astype(np.float64) - oj)
    S = (oi - oj)
    Sh = S.astype(np.float32)
    Sl = (S - Sh.astype(np.float64)).astype(np.float32)
    s = (Xi + Sh).astype(np.float32)
    if precise:
        bb = (s - Xi).astype(np.float32)
        e = ((Xi - (s - bb)).astype(np.float32) + (Sh - bb)).astype(np.float32)
        e = (e + Sl).astype(np.float32)
        dx = ((s + (-Xj)).astype(np.float32) + e).astype(np.float32)
    else:
        dx = (s + (-Xj)).astype(np.float32)
    d2 = (dx[:, 0] * dx[:, 0]).astype(np.float32)
    d2 = _fma32(dx[:, 1], dx[:, 1], d2)
    d2 = _fma32(dx[:, 2], dx[:, 2], d2)
    t = xi.astype(np.float64) - xj.astype(np.float64)
    d64 = (t[:, 0] * t[:, 0] + t[:, 1] * t[:, 1]) + t[:, 2] * t[:, 2]
    err = np.abs(d2.astype(np.float64) - d64)
    k = np.clip(np.searchsorted(E, d64), 0, len(E) - 1)
    k2 = np.clip(k - 1, 0, len(E) - 1)
    band = np.minimum(out_band(info, k), out_band(info, k2))
    inr = d64 < E[-1] * 1.2
    assert inr.sum() > 100000
    assert np.all(err[inr] <= band[inr] / 4), float(np.max(err[inr] / band[inr]))


def out_band(info, k):
    return np.asarray(info["bands_r"])[k]


MOCK_EDGES = gen.log_edges(0.1, 40.0, 14)
MOCK_PIMAX, MOCK_NPI = 50.0, 25
MOCK_BBOX = [0.0, 0.0, 0.0, 1100.0, 1100.0, 1100.0]


@pytest.mark.parametrize("which", [0, 1], ids=["rp2", "pi2"])
def test_mocks_luts_match_band_definition(cf, which):
    """DD(rp, pi) of mocks (Appendix A.2.1) bins rp^2 against e^2 and pi^2 against the squared pi
    edges; both tables must follow the band definition like the other kinds'."""
    p = cf.params(kind="mocks", edges=MOCK_EDGES, autocorr=True, periodic=False, pimax=MOCK_PIMAX,
                  npibins=MOCK_NPI)
    if which == 0:
        E = MOCK_EDGES ** 2
        vals = _values_near(E)
    else:
        pe = np.arange(MOCK_NPI + 1, dtype=np.float64) * (MOCK_PIMAX / MOCK_NPI)
        pe[-1] = MOCK_PIMAX
        E = pe * pe
        vals = np.concatenate([_values_near(E[1:]), np.float32([0.0, 1e-30, 0.5])])
    out = cf.cf_plan_probe(p, MOCK_BBOX, 10 ** 6, which=which, values=vals)
    B = out["bands_r"] if which == 0 else out["bands_p"]
    _check_classes(vals, out["classes"], E, B, len(E) - 1)


def test_mocks_bands_cover_actual_fp32_error(cf):
    """Replay the mocks kernel's FP32 sequence on near-edge pairs of clustered points 300-1000 from
    the observer and compare with the oracle's FP64 arithmetic: rp^2 = |s x A_i|^2 / l.l and
    pi^2 = (s.l)^2 / l.l must stay within a quarter of the band of the nearest edge (the bands carry
    a factor-4 margin).  The reciprocal is emulated correctly rounded; its 2-ulp allowance is added
    to the measured error."""
    p = cf.params(kind="mocks", edges=MOCK_EDGES, autocorr=True, periodic=False, pimax=MOCK_PIMAX,
                  npibins=MOCK_NPI)
    info = cf.cf_plan_probe(p, MOCK_BBOX, 10 ** 6)
    assert min(info["width"]) >= 64.0          # the replay's cells below are no wider
    rng = np.random.Generator(np.random.PCG64(5))
    n = 300000
    d = np.cbrt(rng.uniform(300.0 ** 3, 1000.0 ** 3, n))
    u = rng.normal(size=(n, 3))
    u /= np.linalg.norm(u, axis=1)[:, None]
    mid = np.abs(d[:, None] * u) + 100.0      # every coordinate positive: origins below stay exact
    # pairs about the midpoint `mid` at rp and pi near the edges: s across and along its line of sight
    los = mid / np.linalg.norm(mid, axis=1)[:, None]
    perp = np.cross(los, rng.normal(size=(n, 3)))
    perp /= np.linalg.norm(perp, axis=1)[:, None]
    rp_t = rng.choice(MOCK_EDGES, n) * (1 + rng.uniform(-1e-3, 1e-3, n))
    pi_t = rng.uniform(0, MOCK_PIMAX, n)
    sv = perp * rp_t[:, None] + los * pi_t[:, None]
    xi = (mid + 0.5 * sv).astype(np.float32)
    xj = (mid - 0.5 * sv).astype(np.float32)
    # cells of width 64 (origins multiples of 64: cell-relative coordinates exact in float32)
    oi, oj = np.floor(xi / 64.0) * 64.0, np.floor(xj / 64.0) * 64.0
    Xi = (xi.astype(np.float64) - oi).astype(np.float32)
    Xj = (xj.astype(np.float64) - oj).astype(np.float32)
    assert np.array_equal(Xi.astype(np.float64), xi.astype(np.float64) - oi)
    Sh = (oi - oj).astype(np.float32)
    f32 = np.float32
    s = ((Xi + Sh).astype(f32) + (-Xj)).astype(f32)                   # s = v_i - v_j
    A = xi
    l = (s.astype(np.float64) * -0.5 + A.astype(np.float64)).astype(f32)
    sl = (s[:, 0] * l[:, 0]).astype(f32)
    sl = _fma32(s[:, 1], l[:, 1], sl)
    sl = _fma32(s[:, 2], l[:, 2], sl)
    ll = (l[:, 0] * l[:, 0]).astype(f32)
    ll = _fma32(l[:, 1], l[:, 1], ll)
    ll = _fma32(l[:, 2], l[:, 2], ll)
    sl2 = (sl * sl).astype(f32)
    c = np.stack([(s[:, 1] * A[:, 2]).astype(f32) - (s[:, 2] * A[:, 1]).astype(f32),
                  (s[:, 2] * A[:, 0]).astype(f32) - (s[:, 0] * A[:, 2]).astype(f32),
                  (s[:, 0] * A[:, 1]).astype(f32) - (s[:, 1] * A[:, 0]).astype(f32)], axis=1).astype(f32)
    c2 = (c[:, 0] * c[:, 0]).astype(f32)
    c2 = _fma32(c[:, 1], c[:, 1], c2)
    c2 = _fma32(c[:, 2], c[:, 2], c2)
    r = (1.0 / ll.astype(np.float64)).astype(f32)
    pi2 = (sl2 * r).astype(f32).astype(np.float64)
    rp2 = (c2 * r).astype(f32).astype(np.float64)
    # the oracle's FP64 order
    a, b = xi.astype(np.float64), xj.astype(np.float64)
    S, L = a - b, 0.5 * (a + b)
    dot = lambda x, y: (x[:, 0] * y[:, 0] + x[:, 1] * y[:, 1]) + x[:, 2] * y[:, 2]  # noqa: E731
    pi2_64 = dot(S, L) ** 2 / dot(L, L)
    rp2_64 = np.maximum(dot(S, S) - pi2_64, 0.0)
    u = 2.0 ** -24
    E = MOCK_EDGES ** 2
    k = np.argmin(np.abs(rp2_64[:, None] - E[None, :]), axis=1)
    near = np.abs(rp2_64 - E[k]) < 0.01 * E[k]
    err = np.abs(rp2 - rp2_64) + 3 * u * rp2_64
    assert near.sum() > 100000
    band = np.asarray(info["bands_r"])[k]
    assert np.all(err[near] <= band[near] / 4), float(np.max(err[near] / band[near]))
    P = (np.arange(MOCK_NPI + 1) * (MOCK_PIMAX / MOCK_NPI)) ** 2
    m = np.argmin(np.abs(pi2_64[:, None] - P[None, :]), axis=1)
    okm = (m > 0) & (rp2_64 < E[-1] * 1.05)
    err = np.abs(pi2 - pi2_64) + 3 * u * pi2_64
    band = np.asarray(info["bands_p"])[m]
    assert okm.sum() > 100000
    assert np.all(err[okm] <= band[okm] / 4), float(np.max(err[okm] / band[okm]))


@pytest.mark.parametrize("kind", ["rppi", "mocks"])
def test_tables_at_the_largest_sizes(cf, kind):
    """252 rp bins and 252 pi bins: the tables need several hundred fine entries, so a coarse
    entry must address fine entries beyond the first 256 correctly."""
    edges = gen.log_edges(0.05, 9.0, 252)
    p = cf.params(kind=kind, edges=edges, autocorr=True, periodic=kind == "rppi", box=40.0, pimax=9.0, npibins=252)
    bb = [0, 0, 0, 40, 40, 40] if kind == "rppi" else [30, 5, 15, 140, 90, 100]
    E = edges ** 2
    vals = _values_near(E, span=200)
    for which in ((0, 2) if kind == "rppi" else (0,)):
        out = cf.cf_plan_probe(p, bb, 1600, which=which, values=vals)
        _check_classes(vals, out["classes"], E, out["bands_r"], 252)
    assert out["fine_entries"] > 256
    pe = np.arange(253) * (9.0 / 252)
    pe[-1] = 9.0
    P = pe if kind == "rppi" else pe * pe
    vals = np.concatenate([_values_near(P[1:], span=200), np.float32([0.0, 1e-30, 0.01])])
    for which in ((1, 3) if kind == "rppi" else (1,)):
        out = cf.cf_plan_probe(p, bb, 1600, which=which, values=vals)
        _check_classes(vals, out["classes"], P, out["bands_p"], 252)
