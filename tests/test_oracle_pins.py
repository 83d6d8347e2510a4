"""Pins for the FP64 oracle: facts fixed by the paper and by mathematics, not by the oracle.

Each test ties one part of the oracle to something other than itself:
  * hand-worked lattices whose separations are exact in binary (edge ties included);
  * reductions to an independent library routine (scipy cKDTree count_neighbors, pdist);
  * closed forms: total pair counts, the analytic uniform RR of Appendix B, the shell mean;
  * invariants stated by the paper: auto == cross(D, D) (Sec. 4.3, Appendix B).
"""
import math

import numpy as np
import pytest

import gen
import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")


class Cat:
    def __init__(self, pts, w=None):
        pts = np.asarray(pts, dtype=np.float64)
        self.x, self.y, self.z = pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy()
        self.w = None if w is None else np.asarray(w, dtype=np.float64)


# ------------------------------------------------------------------------------------------
# Hand-worked lattices (golden values derived in the comments; every distance is exact)
# ------------------------------------------------------------------------------------------

LATTICE = [(0, 0, 0), (1, 0, 0), (0, 2, 0), (3, 4, 0)]
# squared separations: 01:1  02:4  03:25  12:5  13:20  23:13
# edges 1,2,3,5,6 -> squared 1,4,9,25,36; bins [1,2) [2,3) [3,5) [5,6), half open (Code
# naivecorr: skip dist < mindist or dist >= maxdist), a tie goes to the upper bin.
#   01 (1)  -> bin 0 (tie on the first edge is included)
#   02 (4)  -> bin 1 (tie on edge 2)
#   12 (5)  -> bin 1
#   13 (20), 23 (13) -> bin 2
#   03 (25) -> bin 3 (tie on edge 5)
# unordered [1,2,2,1]; auto counts are doubled (Sec. 4.3) -> [2,4,4,2]


def test_lattice_r_counts_and_edge_ties(orc):
    d = Cat(LATTICE)
    out = oracle.count("r", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, mode="brute", lib=orc)
    assert out["npairs"].tolist() == [2, 4, 4, 2]
    # the last edge is exclusive: with max 5 the 25 pair drops out
    out = oracle.count("r", [1, 2, 3, 5], d, autocorr=True, periodic=False, mode="brute", lib=orc)
    assert out["npairs"].tolist() == [2, 4, 4]


def test_lattice_r_weights_and_ravg(orc):
    # dyadic weights so that every sum is exact
    d = Cat(LATTICE, w=[1.0, 2.0, 0.5, 4.0])
    out = oracle.count("r", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, weighted=True,
                       ravg=True, mode="brute", lib=orc)
    # pair weights: 01:2 02:0.5 03:4 12:1 13:8 23:2
    assert out["wsum"].tolist() == [4.0, 3.0, 20.0, 8.0]
    exp = [1.0, (0.5 * 2 + 1 * math.sqrt(5)) / 1.5, (8 * math.sqrt(20) + 2 * math.sqrt(13)) / 10, 5.0]
    np.testing.assert_allclose(out["ravg"], exp, rtol=1e-15)
    # unweighted ravg is the plain mean separation
    out = oracle.count("r", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, ravg=True,
                       mode="brute", lib=orc)
    exp = [1.0, (2 + math.sqrt(5)) / 2, (math.sqrt(20) + math.sqrt(13)) / 2, 5.0]
    np.testing.assert_allclose(out["ravg"], exp, rtol=1e-15)


PERIODIC = [(0, 0, 0), (4, 0, 0), (7, 0, 0), (8, 0, 0), (2, 4, 0)]
# L = 8 on every axis, minimum image as Code normal_pbc: d = a-b; if d > 4: d -= 8; if d <= -4: d += 8
#   AB dx=-4 -> +8 -> 4          s=16
#   AC dx=-7 -> 1                s=1
#   AD dx=-8 -> 0  (x = L is the same place as 0)      s=0
#   AE dx=-2, dy=-4 -> 4         s=20
#   BC dx=-3                     s=9
#   BD dx=-4 -> 4                s=16
#   BE dx=2, dy=-4 -> 4          s=20
#   CD dx=-1                     s=1
#   CE dx=5 -> -3, dy=-4 -> 4    s=25
#   DE dx=6 -> -2, dy=-4 -> 4    s=20
# edges 0,1,2,4,5 -> squared 0,1,4,16,25
#   bin0 [0,1): AD ; bin1 [1,4): AC CD ; bin2 [4,16): BC ; bin3 [16,25): AB BD AE BE DE ; CE excluded
# unordered [1,2,1,5] -> doubled [2,4,2,10]; the first edge is 0, so the 5 self pairs are added once
# (Appendix B) -> [7,4,2,10]


def test_periodic_wrap_ties_and_self_pairs(orc):
    d = Cat(PERIODIC)
    kw = dict(periodic=True, box=8.0, lib=orc)
    out = oracle.count("r", [0, 1, 2, 4, 5], d, autocorr=True, mode="brute", **kw)
    assert out["npairs"].tolist() == [7, 4, 2, 10]
    # Appendix B: the auto-correlation equals the cross-correlation of the set with itself
    cross = oracle.count("r", [0, 1, 2, 4, 5], d, d, autocorr=False, mode="brute", **kw)
    assert cross["npairs"].tolist() == [7, 4, 2, 10]
    rows = oracle.count("r", [0, 1, 2, 4, 5], d, autocorr=True, rows=(0, 5), **kw)
    assert rows["npairs"].tolist() == [7, 4, 2, 10]
    # without the zero edge no self pairs appear
    out = oracle.count("r", [0.5, 1, 2, 4, 5], d, autocorr=True, mode="brute", **kw)
    assert out["npairs"].tolist() == [0, 4, 2, 10]


RPPI = [(0, 0, 0), (1, 0, 1), (0, 2, 0.5), (3, 4, 3)]
# rp^2 = dx^2+dy^2, pi = |dz| (Appendix A.1), rp edges 1,2,3,5,6, pimax 3 with unit pi bins
#   AB rp2=1  pi=1   -> (rp0, pi1)
#   AC rp2=4  pi=0.5 -> (rp1, pi0)
#   AD rp2=25 pi=3   -> excluded, pi must be < pimax
#   BC rp2=5  pi=0.5 -> (rp1, pi0)
#   BD rp2=20 pi=2   -> (rp2, pi2)
#   CD rp2=13 pi=2.5 -> (rp2, pi2)
# doubled: (0,1):2 (1,0):4 (2,2):4 ; wp counts per rp bin: [2,4,4,0]


def test_rppi_and_wp_hand(orc):
    d = Cat(RPPI)
    out = oracle.count("rppi", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, pimax=3.0,
                       npibins=3, mode="brute", lib=orc)
    exp = np.zeros((4, 3), dtype=np.uint64)
    exp[0, 1] = 2
    exp[1, 0] = 4
    exp[2, 2] = 4
    assert (out["npairs"] == exp).all()
    wp = oracle.count("wp", [1, 2, 3, 5, 6], d, autocorr=True, periodic=False, pimax=3.0,
                      npibins=3, mode="brute", lib=orc)
    assert wp["npairs"].tolist() == [2, 4, 4, 0]


# ravg of DD(rp, pi) and wp is the mean projected separation rp = sqrt(dx^2 + dy^2) of the pairs of a
# bin (Appendix A.1: rp is the separation across the line of sight; Sec. 6.5: ravg is the mean
# separation of a bin), not the 3-D separation.  On the same lattice (rp^2 exact):
#   (rp0, pi1): AB rp 1                       -> 1
#   (rp1, pi0): AC rp 2, BC rp sqrt(5)        -> (2 + sqrt 5) / 2
#   (rp2, pi2): BD rp sqrt(20), CD rp sqrt(13) -> (sqrt 20 + sqrt 13) / 2
# With dyadic weights w = (1, 2, 0.5, 4): pair weights AB 2, AC 0.5, BC 1, BD 8, CD 2, so
#   wsum (doubled) (0,1): 4, (1,0): 3, (2,2): 20;
#   weighted ravg (0,1): 1, (1,0): (0.5*2 + 1*sqrt 5)/1.5, (2,2): (8 sqrt 20 + 2 sqrt 13)/10.
# wp sums over pi, so its per-rp-bin values are the same means.
RPPI_W = [1.0, 2.0, 0.5, 4.0]


def test_rppi_and_wp_ravg_hand(orc):
    d = Cat(RPPI)
    kw = dict(autocorr=True, periodic=False, pimax=3.0, npibins=3, mode="brute", lib=orc)
    out = oracle.count("rppi", [1, 2, 3, 5, 6], d, ravg=True, **kw)
    exp = np.zeros((4, 3))
    exp[0, 1] = 1.0
    exp[1, 0] = (2 + math.sqrt(5)) / 2
    exp[2, 2] = (math.sqrt(20) + math.sqrt(13)) / 2
    np.testing.assert_allclose(out["ravg"], exp, rtol=1e-15, atol=0)
    wp = oracle.count("wp", [1, 2, 3, 5, 6], d, ravg=True, **kw)
    np.testing.assert_allclose(wp["ravg"], [1.0, exp[1, 0], exp[2, 2], 0.0], rtol=1e-15, atol=0)
    dw = Cat(RPPI, w=RPPI_W)
    out = oracle.count("rppi", [1, 2, 3, 5, 6], dw, ravg=True, weighted=True, **kw)
    wexp = np.zeros((4, 3))
    wexp[0, 1], wexp[1, 0], wexp[2, 2] = 4.0, 3.0, 20.0
    assert (out["wsum"] == wexp).all()
    rexp = np.zeros((4, 3))
    rexp[0, 1] = 1.0
    rexp[1, 0] = (0.5 * 2 + 1 * math.sqrt(5)) / 1.5
    rexp[2, 2] = (8 * math.sqrt(20) + 2 * math.sqrt(13)) / 10
    np.testing.assert_allclose(out["ravg"], rexp, rtol=1e-15, atol=0)
    wp = oracle.count("wp", [1, 2, 3, 5, 6], dw, ravg=True, weighted=True, **kw)
    assert wp["wsum"].tolist() == [4.0, 3.0, 20.0, 0.0]
    np.testing.assert_allclose(wp["ravg"], [1.0, rexp[1, 0], rexp[2, 2], 0.0], rtol=1e-15, atol=0)


# The weighted self pairs of Appendix B (reading S10 of the design notes: a point paired with itself
# has weight w_i^2 and separation 0).  PERIODIC with dyadic weights A 1, B 2, C 0.5, D 4, E 0.25 and
# edges 0, 2, 4, 5 (squared 0, 4, 16, 25):
#   bin0 [0,4):  AD s=0 (w 4), AC s=1 (w 0.5), CD s=1 (w 2) -> doubled: w 13, sum w*r 2*(0 + 0.5 + 2) = 5
#                self pairs: sum w_i^2 = 1 + 4 + 0.25 + 16 + 0.0625 = 21.3125, separation 0
#                -> wsum 34.3125, weighted ravg 5 / 34.3125, count 6 + 5 = 11
#   bin1 [4,16): BC s=9 (w 1)                                 -> wsum 2, ravg 3, count 2
#   bin2 [16,25): AB BD AE BE DE, s 16 16 20 20 20 (w 2 8 0.25 0.5 1)
#                -> wsum 23.5, sum w*r 2*(4*2 + 4*8 + sqrt(20)*1.75) -> ravg (80 + 3.5 sqrt 20)/23.5, count 10
PERIODIC_W = [1.0, 2.0, 0.5, 4.0, 0.25]


def test_weighted_self_pairs_hand(orc):
    d = Cat(PERIODIC, w=PERIODIC_W)
    kw = dict(periodic=True, box=8.0, weighted=True, ravg=True, lib=orc)
    wexp = [34.3125, 2.0, 23.5]
    rexp = [5.0 / 34.3125, 3.0, (80.0 + 3.5 * math.sqrt(20.0)) / 23.5]
    for out in (oracle.count("r", [0, 2, 4, 5], d, autocorr=True, mode="brute", **kw),
                oracle.count("r", [0, 2, 4, 5], d, autocorr=True, mode="zwin", **kw),
                oracle.count("r", [0, 2, 4, 5], d, autocorr=True, rows=(0, 5), **kw)):
        assert out["npairs"].tolist() == [11, 2, 10]
        assert out["wsum"].tolist() == wexp
        np.testing.assert_allclose(out["ravg"], rexp, rtol=1e-15, atol=0)
    # the cross count of the set with itself meets every point's self pair in the pair loop
    cross = oracle.count("r", [0, 2, 4, 5], d, d, autocorr=False, mode="brute", **kw)
    assert cross["npairs"].tolist() == [11, 2, 10]
    assert cross["wsum"].tolist() == wexp


def test_theta_hand(orc):
    # e_x, e_y, e_z, -e_x: five pairs at exactly 90 deg (chord^2 = 2) and one at 180 deg (chord^2 = 4).
    # Chord edges are c = 2 sin(theta pi/360) in FP64: 60 -> 0.9999999999999998, 90 ->
    # 1.9999999999999996, 180 -> 4.0 (squared).  So the 90-degree pairs fall in [90,180), and
    # the 180-degree pair is excluded by the exclusive last edge.
    d = Cat([(1, 0, 0), (0, 1, 0), (0, 0, 1), (-1, 0, 0)])
    out = oracle.count("theta", [60, 90, 180], d, autocorr=True, periodic=False, mode="brute",
                       ravg=True, lib=orc)
    assert out["npairs"].tolist() == [0, 10]
    np.testing.assert_allclose(out["ravg"], [0.0, 90.0], rtol=1e-14)
    e2 = oracle.squared_edges("theta", [60, 90, 180], lib=orc)
    assert e2.tolist() == [0.9999999999999998, 1.9999999999999996, 4.0]


# ------------------------------------------------------------------------------------------
# Reductions to an independent library routine (scipy cKDTree)
# ------------------------------------------------------------------------------------------

def _cum_to_bins(cum):
    return np.diff(np.asarray(cum, dtype=np.float64))


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("autocorr", [True, False])
def test_r_vs_ckdtree(orc, periodic, autocorr):
    L = 50.0
    d1 = gen.uniform_box(1500, L, 11, dtype=np.float64)
    d2 = gen.uniform_box(1200, L, 12, dtype=np.float32)
    w1 = gen.uniform_weights(d1.n, 0.5, 1.5, 13).astype(np.float64)
    w2 = gen.uniform_weights(d2.n, 0.5, 1.5, 14).astype(np.float64)
    d1.w, d2.w = w1, w2
    edges = gen.log_edges(0.5, 12.0, 9)
    kw = dict(periodic=periodic, box=L, weighted=True, lib=orc)
    a = np.stack([d1.x, d1.y, d1.z], 1).astype(np.float64)
    b = np.stack([d2.x, d2.y, d2.z], 1).astype(np.float64)
    bs = L if periodic else None
    ta = scipy_spatial.cKDTree(a, boxsize=bs)
    if autocorr:
        out = oracle.count("r", edges, d1, autocorr=True, mode="brute", **kw)
        cum = ta.count_neighbors(ta, edges)
        cumw = ta.count_neighbors(ta, edges, weights=(w1, w1))
    else:
        out = oracle.count("r", edges, d1, d2, autocorr=False, mode="brute", **kw)
        tb = scipy_spatial.cKDTree(b, boxsize=bs)
        cum = ta.count_neighbors(tb, edges)
        cumw = ta.count_neighbors(tb, edges, weights=(w1, w2))
    # cKDTree counts ordered pairs with d <= r (self pairs included); random data has no ties
    assert out["npairs"].astype(np.int64).tolist() == _cum_to_bins(cum).astype(np.int64).tolist()
    np.testing.assert_allclose(out["wsum"], _cum_to_bins(cumw), rtol=1e-11)


def test_theta_vs_ckdtree(orc):
    d = gen.sphere_patch(3000, 0.0, 40.0, -10.0, 20.0, 21)
    edges = gen.log_edges(0.05, 4.0, 10)                     # degrees
    out = oracle.count("theta", edges, d, autocorr=True, periodic=False, mode="brute", lib=orc)
    v = np.stack([d.x, d.y, d.z], 1).astype(np.float64)
    t = scipy_spatial.cKDTree(v)
    chords = 2.0 * np.sin(np.deg2rad(edges) / 2.0)           # Euclidean chord = |v1 - v2|
    cum = t.count_neighbors(t, chords)
    assert out["npairs"].astype(np.int64).tolist() == _cum_to_bins(cum).astype(np.int64).tolist()


def test_rppi_marginals_vs_ckdtree(orc):
    L = 40.0
    d = gen.uniform_box(1500, L, 31, dtype=np.float64)     # float64: no exact |dz| ties
    a = np.stack([d.x, d.y, d.z], 1).astype(np.float64)
    # rp marginal: with pimax > L/2 every min-image |dz| passes, so wp counts are 2-D counts on (x, y)
    rp = gen.log_edges(0.5, 10.0, 8)
    wp = oracle.count("wp", rp, d, autocorr=True, periodic=True, box=L, pimax=L, npibins=40,
                      mode="brute", lib=orc)
    t2 = scipy_spatial.cKDTree(a[:, :2], boxsize=L)
    assert wp["npairs"].astype(np.int64).tolist() == _cum_to_bins(t2.count_neighbors(t2, rp)).astype(np.int64).tolist()
    # pi marginal: with rp covering every pair, the pi histogram is the 1-D |dz| histogram
    full = [1e-9, L]
    out = oracle.count("rppi", full, d, autocorr=True, periodic=True, box=L, pimax=10.0,
                       npibins=10, mode="brute", lib=orc)
    t1 = scipy_spatial.cKDTree(a[:, 2:3], boxsize=L)
    pe = np.arange(0, 11, dtype=np.float64)
    cum = t1.count_neighbors(t1, pe)                        # |dz| <= p (self pairs at p=0 cancel)
    # rp >= 1e-9 drops only exact coincidences in (x, y), which random data does not have
    assert out["npairs"][0].astype(np.int64).tolist() == _cum_to_bins(cum).astype(np.int64).tolist()


def test_ravg_vs_pdist(orc):
    d = gen.uniform_box(600, 30.0, 41, dtype=np.float64)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 42).astype(np.float64)
    edges = gen.log_edges(1.0, 20.0, 6)
    out = oracle.count("r", edges, d, autocorr=True, periodic=False, weighted=True, ravg=True,
                       mode="brute", lib=orc)
    from scipy.spatial.distance import pdist
    a = np.stack([d.x, d.y, d.z], 1)
    r = pdist(a)
    iu, ju = np.triu_indices(d.n, 1)
    ww = d.w[iu] * d.w[ju]
    k = np.searchsorted(edges, r, side="right") - 1
    ok = (k >= 0) & (k < len(edges) - 1)
    num = np.bincount(k[ok], weights=(ww * r)[ok], minlength=len(edges) - 1)
    den = np.bincount(k[ok], weights=ww[ok], minlength=len(edges) - 1)
    np.testing.assert_allclose(out["wsum"], 2 * den, rtol=1e-12)
    np.testing.assert_allclose(out["ravg"], num / den, rtol=1e-12)


# ------------------------------------------------------------------------------------------
# Closed forms and invariants
# ------------------------------------------------------------------------------------------

def test_total_count_when_rmax_spans_box(orc):
    L = 10.0
    d = gen.uniform_box(400, L, 51)
    e = gen.uniform_box(300, L, 52)
    # periodic: every min-image separation is <= sqrt(3) L / 2 < 9
    out = oracle.count("r", [1e-6, 9.0], d, autocorr=True, periodic=True, box=L, mode="zwin", lib=orc)
    assert int(out["npairs"].sum()) == d.n * (d.n - 1)
    out = oracle.count("r", [1e-6, 9.0], d, e, autocorr=False, periodic=True, box=L, lib=orc)
    assert int(out["npairs"].sum()) == d.n * e.n
    # non-periodic: the box diagonal is sqrt(3) L < 18
    out = oracle.count("r", [1e-6, 18.0], d, autocorr=True, periodic=False, lib=orc)
    assert int(out["npairs"].sum()) == d.n * (d.n - 1)
    # rp-pi with pimax beyond the largest min-image |dz|
    out = oracle.count("rppi", [1e-6, 9.0], d, autocorr=True, periodic=True, box=L, pimax=6.0,
                       npibins=6, lib=orc)
    assert int(out["npairs"].sum()) == d.n * (d.n - 1)


def _binom_check(counts_unordered, expected, M):
    """5-sigma per bin (E >= 25) and a chi-square over the eligible bins.  For i.i.d. uniform
    points on a torus the pair indicators are pairwise independent, so Var = M p (1-p)."""
    p = expected / M
    var = M * p * (1 - p)
    elig = expected >= 25
    assert elig.sum() >= 3
    z = (counts_unordered[elig] - expected[elig]) / np.sqrt(var[elig])
    assert np.all(np.abs(z) < 5), z
    chi2 = float((z ** 2).sum())
    dof = int(elig.sum())
    assert chi2 < dof + 6 * math.sqrt(2 * dof) + 10, (chi2, dof)


def test_uniform_rr_analytic_r(orc):
    # the correctness workload: N=20000 uniform float64 in a periodic L=250 box, 20 log bins
    wl = gen.workload("uniform_r_20k")
    out = oracle.count("r", wl.edges, wl.d1, autocorr=True, periodic=True, box=wl.box, mode="zwin", lib=orc)
    n = wl.d1.n
    M = n * (n - 1) / 2
    e = wl.edges
    # Appendix B: RR_i = dV_i N (N-1)/V (ordered) -> unordered M * dV_i / V
    Ek = M * (4.0 / 3.0) * math.pi * (e[1:] ** 3 - e[:-1] ** 3) / wl.box ** 3
    _binom_check(out["npairs"].astype(np.float64) / 2, Ek, M)


def test_uniform_rr_analytic_rppi(orc):
    L = 100.0
    d = gen.uniform_box(20000, L, 61)
    rp = gen.log_edges(1.0, 10.0, 6)
    out = oracle.count("rppi", rp, d, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10, lib=orc)
    n = d.n
    M = n * (n - 1) / 2
    area = math.pi * (rp[1:] ** 2 - rp[:-1] ** 2)
    Ek = np.repeat((M * area * 2.0 / L ** 3)[:, None], 10, axis=1)   # pi = |dz|: height 2 per unit bin
    _binom_check(out["npairs"].astype(np.float64).ravel() / 2, Ek.ravel(), M)
    # wp of a uniform set scatters around 0 (Eq. 2 with Appendix B's RR)
    wp = oracle.count("wp", rp, d, autocorr=True, periodic=True, box=L, pimax=10.0, npibins=10, lib=orc)
    dd = wp["npairs"].astype(np.float64)
    rr = n * (n - 1) / L ** 3 * area
    sig = np.sqrt(dd) / rr                                 # Poisson scatter of DD/RR in wp units
    assert np.all(np.abs(wp["wp"]) < 6 * sig + 1e-12), (wp["wp"], sig)


def test_uniform_sphere_theta_analytic(orc):
    d = gen.unit_sphere(6000, 71)
    edges = np.array([2.0, 4.0, 8.0, 16.0, 32.0])
    out = oracle.count("theta", edges, d, autocorr=True, periodic=False, lib=orc)
    n = d.n
    M = n * (n - 1) / 2
    t = np.deg2rad(edges)
    p = (np.cos(t[:-1]) - np.cos(t[1:])) / 2                # cap area fraction of the annulus
    _binom_check(out["npairs"].astype(np.float64) / 2, M * p, M)


def test_uniform_shell_mean_ravg(orc):
    L = 100.0
    d = gen.uniform_box(20000, L, 81)
    e = np.array([2.0, 4.0, 6.0, 8.0, 10.0])
    out = oracle.count("r", e, d, autocorr=True, periodic=True, box=L, ravg=True, lib=orc)
    exp = 0.75 * (e[1:] ** 4 - e[:-1] ** 4) / (e[1:] ** 3 - e[:-1] ** 3)
    np.testing.assert_allclose(out["ravg"], exp, rtol=3e-3)


def test_weights_one_equal_counts(orc):
    d = gen.clustered_box(30, 20, 1.0, 30.0, 91)
    d.w = np.ones(d.n, dtype=np.float32)
    e = gen.log_edges(0.1, 8.0, 12)
    out = oracle.count("r", e, d, autocorr=True, periodic=True, box=30.0, weighted=True, lib=orc)
    assert out["wsum"].tolist() == out["npairs"].astype(np.float64).tolist()


@pytest.mark.parametrize("kind", ["r", "rppi", "wp", "theta"])
def test_modes_agree_and_auto_equals_cross(orc, kind):
    if kind == "theta":
        d = gen.sphere_patch(1500, 0.0, 20.0, 0.0, 20.0, 101)
        e, kw = gen.log_edges(0.05, 3.0, 8), dict(periodic=False)
    else:
        d = gen.clustered_box(20, 50, 1.5, 40.0, 102)
        e, kw = gen.log_edges(0.2, 8.0, 8), dict(periodic=True, box=40.0)
    d.w = gen.uniform_weights(d.n, 0.5, 1.5, 103)
    kw.update(pimax=9.0, npibins=9, weighted=True, ravg=True, lib=orc)
    brute = oracle.count(kind, e, d, autocorr=True, mode="brute", **kw)
    zwin = oracle.count(kind, e, d, autocorr=True, mode="zwin", **kw)
    rows = oracle.count(kind, e, d, autocorr=True, rows=(0, d.n), **kw)
    cross = oracle.count(kind, e, d, d, autocorr=False, mode="zwin", **kw)
    for o in (zwin, rows, cross):
        assert (o["npairs"] == brute["npairs"]).all()
        np.testing.assert_allclose(o["wsum"], brute["wsum"], rtol=1e-12)
        np.testing.assert_allclose(o["ravg"], brute["ravg"], rtol=1e-12)


def test_permutation_invariance(orc):
    d = gen.clustered_box(30, 30, 1.0, 40.0, 111)
    e = gen.log_edges(0.1, 9.0, 10)
    a = oracle.count("r", e, d, autocorr=True, periodic=True, box=40.0, lib=orc)
    p = np.random.Generator(np.random.PCG64(5)).permutation(d.n)
    b = oracle.count("r", e, d.subset(p), autocorr=True, periodic=True, box=40.0, lib=orc)
    assert (a["npairs"] == b["npairs"]).all()


# ------------------------------------------------------------------------------------------
# The z-window on a row sample (the timed CPU baseline) equals brute force on the same rows
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("kind,autocorr,periodic", [("r", True, True), ("r", False, False), ("rppi", True, True),
                                                    ("wp", False, True), ("theta", True, False),
                                                    ("mocks", True, False)])
def test_zwin_rows_equal_brute_rows(orc, kind, autocorr, periodic):
    """Rows i in [r0, r1) against every j: through the z window (mode zwin with rows) and by brute
    force (mode rows) the counts are bit-identical (Sec. 4.6: a pair outside the window has
    |dz| >= zmax, so it is rejected anyway) and the sums equal up to their order of addition; the
    window's rows summed over all rows give the full ordered result."""
    if kind == "theta":
        d1 = gen.sphere_patch(3000, 0.0, 40.0, -10.0, 30.0, 81)
        d2 = gen.sphere_patch(2000, 0.0, 40.0, -10.0, 30.0, 82)
        edges, kw = gen.log_edges(0.01, 2.0, 10), {}
    elif kind == "mocks":
        d1 = gen.survey_cone(3000, 0.0, 30.0, 10.0, 40.0, 60.0, 90.0, 83, members=30, sigma=1.2)
        d2 = gen.survey_cone(2000, 0.0, 30.0, 10.0, 40.0, 60.0, 90.0, 84)
        edges, kw = gen.log_edges(0.1, 6.0, 10), dict(pimax=8.0, npibins=8)
    else:
        d1 = gen.clustered_box(60, 50, 1.5, 80.0, 85, dtype=np.float64)
        d2 = gen.uniform_box(2500, 80.0, 86, dtype=np.float64)
        edges, kw = gen.log_edges(0.1, 9.0, 12), dict(pimax=9.0, npibins=9)
    for d in (d1, d2):
        d.w = gen.uniform_weights(d.n, 0.5, 1.5, 87).astype(np.float64)
    kw.update(autocorr=autocorr, periodic=periodic, box=80.0, weighted=True, ravg=True, lib=orc)
    other = None if autocorr else d2
    for r0, r1 in ((0, 200), (1111, 1500), (d1.n - 150, d1.n)):
        z = oracle.count(kind, edges, d1, other, rows=(r0, r1), mode="zwin", **kw)
        b = oracle.count(kind, edges, d1, other, rows=(r0, r1), mode="rows", **kw)
        assert np.array_equal(z["npairs"], b["npairs"])
        np.testing.assert_allclose(z["wsum"], b["wsum"], rtol=1e-12, atol=0)
        np.testing.assert_allclose(z["rsum"], b["rsum"], rtol=1e-12, atol=0)
    full = oracle.count(kind, edges, d1, other, mode="zwin", **kw)
    allrows = oracle.count(kind, edges, d1, other, rows=(0, d1.n), mode="zwin", **kw)
    assert np.array_equal(full["npairs"], allrows["npairs"])
