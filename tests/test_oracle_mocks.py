"""Pins for the oracle's DD(rp, pi) of observed / mock galaxies (Appendix A.2.1, the line of sight of
Fisher et al.): s = v1 - v2, l = (v1 + v2) / 2, pi = s.l / |l|, rp^2 = s.s - pi^2.

Each check ties the oracle to something other than its own formula:
  * hand-worked pairs whose line of sight is exactly the z axis (v1 = (a, b, c), v2 = (-a, -b, d)
    gives l = (0, 0, (c + d) / 2), so pi = |c - d| and rp = 2 sqrt(a^2 + b^2), exact in binary);
  * the same histogram from an independent formulation, rp^2 = |s x l|^2 / |l|^2 (numpy), equal
    except for pairs within rounding of an edge;
  * invariance under exact rotations, reflections and axis permutations about the observer;
  * the far-field limit: for a cluster far along z the line of sight is the z axis, so the counts
    approach the plane-parallel DD(rp, pi);
  * auto == cross(D, D), all oracle modes agree, self pairs when the first edge is 0.
"""
import numpy as np
import pytest

import gen
import oracle

EDGES = np.array([0.5, 1.0, 2.0, 3.0])
PIMAX, NPI = 4.0, 4

# (a, b, c, d) -> expected (rp bin, pi bin) of the pair, None when it is outside every bin.
#   rp = 2 sqrt(a^2 + b^2), pi = |c - d|; rp bins [0.5,1) [1,2) [2,3); pi bins of width 1 below 4
HAND = [
    ((0.5, 0.0, 10.0, 7.0), (1, 3)),      # rp 1 (tie: upper bin), pi 3 (tie: upper bin)
    ((0.25, 0.0, 10.0, 9.5), (0, 0)),     # rp 0.5 (tie on the first edge), pi 0.5
    ((0.0, 0.75, 8.0, 6.5), (1, 1)),      # rp 1.5, pi 1.5
    ((0.5, 0.5, 20.0, 18.0), (1, 2)),     # rp sqrt(2), pi 2 (tie)
    ((1.5, 0.0, 10.0, 9.0), None),        # rp 3: the last edge is exclusive
    ((0.5, 0.0, 10.0, 6.0), None),        # pi 4 = pimax: excluded
    ((0.125, 0.0, 10.0, 9.0), None),      # rp 0.25: below the first edge
    ((1.0, 0.0, 5.0, 5.0), (2, 0)),       # rp 2 (tie), pi 0
]


def _cat(pts, w=None):
    pts = np.asarray(pts, dtype=np.float64)
    return gen.Catalogue(pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(),
                         None if w is None else np.asarray(w, dtype=np.float64))


def _mocks(lib, d1, d2=None, edges=EDGES, mode="zwin", **kw):
    kw.setdefault("pimax", PIMAX)
    kw.setdefault("npibins", NPI)
    return oracle.count("mocks", edges, d1, d2, autocorr=d2 is None, periodic=False, mode=mode, lib=lib, **kw)


def check_hand_pairs(lib):
    for (a, b, c, d), expect in HAND:
        cat = _cat([(a, b, c), (-a, -b, d)])
        got = _mocks(lib, cat, mode="brute")["npairs"]
        want = np.zeros((len(EDGES) - 1, NPI), dtype=np.uint64)
        if expect is not None:
            want[expect] = 2                  # one unique pair, ordered counts (Sec. 4.3)
        assert np.array_equal(got, want), ((a, b, c, d), got.tolist())


def check_hand_ravg(lib):
    """ravg of the mocks is the mean of rp = sqrt(s.s - pi^2) (Appendix A.2.1, Sec. 6.5): for the
    hand pairs rp = 2 sqrt(a^2 + b^2) exactly, so their ravg is that value; weighted, two pairs in
    one slot average by their weights."""
    for (a, b, c, d), expect in HAND:
        if expect is None:
            continue
        out = _mocks(lib, _cat([(a, b, c), (-a, -b, d)]), mode="brute", ravg=True)
        want = np.zeros((len(EDGES) - 1, NPI))
        want[expect] = 2.0 * np.sqrt(a * a + b * b)
        np.testing.assert_allclose(out["ravg"], want, rtol=1e-15, atol=0)
    # slot (1, 1): P1 rp 1.5 pi 1.5 with weights 1, 2; P2 rp sqrt(2) pi 1.25 with weights 4, 2.
    # Pairs across P1 and P2 are 12 apart along the line of sight (pi > pimax).
    pts = [(0.0, 0.75, 8.0), (0.0, -0.75, 6.5), (0.5, 0.5, 20.0), (-0.5, -0.5, 18.75)]
    out = _mocks(lib, _cat(pts, [1.0, 2.0, 4.0, 2.0]), mode="brute", ravg=True, weighted=True)
    assert out["npairs"][1, 1] == 4 and int(out["npairs"].sum()) == 4
    assert out["wsum"][1, 1] == 20.0
    np.testing.assert_allclose(out["ravg"][1, 1], (2 * 1.5 + 8 * np.sqrt(2.0)) / 10, rtol=1e-15)
    out = _mocks(lib, _cat(pts), mode="brute", ravg=True)
    np.testing.assert_allclose(out["ravg"][1, 1], (1.5 + np.sqrt(2.0)) / 2, rtol=1e-15)


def _numpy_cross_form(d):
    """rp^2 and pi^2 of every unordered pair from the cross product: |s x l|^2 / |l|^2."""
    v = np.stack([d.x, d.y, d.z], axis=1)
    i, j = np.triu_indices(len(v), 1)
    s = v[i] - v[j]
    l = 0.5 * (v[i] + v[j])
    ll = np.einsum("ij,ij->i", l, l)
    rp2 = np.einsum("ij,ij->i", np.cross(s, l), np.cross(s, l)) / ll
    pi2 = np.einsum("ij,ij->i", s, l) ** 2 / ll
    return rp2, pi2


def check_cross_product_form(lib):
    rng = np.random.Generator(np.random.PCG64(41))
    # a clustered shell seen from the observer at distances 40..60
    c = rng.normal(0, 1, size=(30, 3))
    c = c / np.linalg.norm(c, axis=1)[:, None] * rng.uniform(40, 60, size=(30, 1))
    pts = (c[:, None, :] + rng.normal(0, 1.2, size=(30, 20, 3))).reshape(-1, 3)
    d = _cat(pts)
    got = _mocks(lib, d, mode="brute")["npairs"].astype(np.int64)
    rp2, pi2 = _numpy_cross_form(d)
    e2, p2 = EDGES ** 2, (np.arange(NPI + 1) * (PIMAX / NPI)) ** 2
    ok = (pi2 < p2[-1]) & (rp2 >= e2[0]) & (rp2 < e2[-1])
    want = np.zeros((len(EDGES) - 1, NPI), dtype=np.int64)
    k = np.searchsorted(e2, rp2[ok], side="right") - 1
    m = np.searchsorted(p2, pi2[ok], side="right") - 1
    np.add.at(want, (k, m), 2)
    # pairs within rounding of an edge may land on either side
    near = 0
    for edges_sq, vals in ((e2, rp2), (p2, pi2)):
        dist = np.min(np.abs(vals[:, None] - edges_sq[None, :]), axis=1)
        near += int(np.sum(dist <= 1e-9 * (1.0 + np.abs(vals))))
    assert int(want.sum()) > 500
    assert int(np.abs(got - want).sum()) <= 4 * near, (got.tolist(), want.tolist())


def check_exact_symmetries(lib):
    rng = np.random.Generator(np.random.PCG64(42))
    pts = rng.normal(0, 1.5, size=(400, 3)) + np.array([30.0, -20.0, 25.0])
    pts = np.round(pts * 256) / 256            # dyadic: the transforms below are exact
    base = _mocks(lib, _cat(pts), mode="brute")["npairs"]
    for t in (lambda p: np.stack([-p[:, 1], p[:, 0], p[:, 2]], 1),     # 90 deg about z
              lambda p: np.stack([p[:, 1], p[:, 2], p[:, 0]], 1),      # axis permutation
              lambda p: np.stack([-p[:, 0], p[:, 1], p[:, 2]], 1),     # reflection
              lambda p: p[::-1]):                                      # order of the points
        assert np.array_equal(_mocks(lib, _cat(t(pts)), mode="brute")["npairs"], base)


def check_far_field_limit(lib):
    rng = np.random.Generator(np.random.PCG64(43))
    pts = rng.normal(0, 1.0, size=(600, 3)) + np.array([0.0, 0.0, 1.0e5])
    d = _cat(pts)
    mock = _mocks(lib, d, mode="brute")["npairs"].astype(np.int64)
    pp = oracle.count("rppi", EDGES, d, autocorr=True, periodic=False, pimax=PIMAX, npibins=NPI, mode="brute",
                      lib=lib)["npairs"].astype(np.int64)
    assert int(pp.sum()) > 10000
    # the line of sight deviates from z by <= |s| / |l| ~ 1e-4: only pairs that close to an edge move
    assert int(np.abs(mock - pp).sum()) <= 2e-3 * int(pp.sum())


def check_modes_auto_cross_self(lib):
    rng = np.random.Generator(np.random.PCG64(44))
    pts = rng.normal(0, 1.3, size=(300, 3)) + np.array([10.0, 12.0, -8.0])
    d = _cat(pts, w=rng.uniform(0.5, 1.5, 300))
    kw = dict(weighted=True, ravg=True)
    brute = _mocks(lib, d, mode="brute", **kw)
    zwin = _mocks(lib, d, mode="zwin", **kw)
    cross = _mocks(lib, d, d, mode="brute", **kw)
    assert np.array_equal(brute["npairs"], zwin["npairs"])
    assert np.array_equal(brute["npairs"], cross["npairs"])
    assert np.allclose(brute["wsum"], cross["wsum"], rtol=1e-12)
    rows = sum(_mocks(lib, d, rows=(a, min(a + 70, 300)), **kw)["npairs"].astype(np.int64) for a in range(0, 300, 70))
    assert np.array_equal(rows, brute["npairs"].astype(np.int64))
    # self pairs: with a first edge of 0 the N self pairs go to (rp 0, pi 0) once (Appendix B)
    e0 = np.concatenate([[0.0], EDGES])
    with0 = _mocks(lib, d, edges=e0, mode="brute")["npairs"].astype(np.int64)
    cr0 = _mocks(lib, d, d, edges=e0, mode="brute")["npairs"].astype(np.int64)
    assert np.array_equal(with0, cr0)
    assert with0[0, 0] >= 300 and (with0[0, 0] - 300) % 2 == 0


MOCK_CHECKS = [check_hand_pairs, check_hand_ravg, check_cross_product_form, check_exact_symmetries, check_far_field_limit,
               check_modes_auto_cross_self]


@pytest.mark.parametrize("check", MOCK_CHECKS, ids=lambda c: c.__name__)
def test_mocks_pin(orc, check):
    check(orc)


def test_mocks_refuse_periodic(orc):
    d = _cat([(1.0, 2.0, 3.0), (1.5, 2.0, 3.0)])
    with pytest.raises(RuntimeError):
        oracle.count("mocks", EDGES, d, autocorr=True, periodic=True, box=10.0, pimax=PIMAX, npibins=NPI, lib=orc)
