"""Correlation-function estimators on top of the pair counts (host arithmetic on count arrays).

The counts come from `cf_count` / `cf_batch_count` / the server and follow the library's
convention: auto-correlations return ORDERED pair counts (every unique pair twice, plus N self
pairs in the first bin when its lower edge is 0, Appendix B), so that auto(D) == cross(D, D).  An
auto count therefore totals N(N-1) (+N), a cross count N1*N2.

  rr_analytic     expected RR of a uniform periodic box, density (N-1)/V (Appendix B)
  xi_natural      1 + xi = DD/RR on normalised counts (Sec. 2.1)
  xi_theory       xi(r) of a periodic box: natural estimator against rr_analytic
  landy_szalay    (DD - 2 DR + RR) / RR on normalised counts (Sec. 2.1, footnote)
  wp_from_xi      wp(rp) = 2 * sum over pi bins of xi(rp, pi) * dpi (Eq. 2)

None of these touch the GPU: they take numpy arrays (the dicts returned by the binding give them).
"""
from __future__ import annotations

import math

import numpy as np


def _norm_auto(counts, n: int) -> np.ndarray:
    """Ordered auto counts as a fraction of all ordered pairs N(N-1)."""
    return np.asarray(counts, dtype=np.float64) / (float(n) * float(n - 1))


def _norm_cross(counts, n1: int, n2: int) -> np.ndarray:
    return np.asarray(counts, dtype=np.float64) / (float(n1) * float(n2))


def shell_volumes(kind: str, edges, pimax: float = 0.0, npibins: int = 0) -> np.ndarray:
    """Volume of each bin: spherical shells for r; for rp-pi the annulus area times 2 * dpi (both
    signs of dz, since pi = |dz|), shape (rp bins, npibins) like the counts; for wp the annulus times
    2 * pimax."""
    e = np.asarray(edges, dtype=np.float64)
    if kind == "r":
        return 4.0 / 3.0 * math.pi * (e[1:] ** 3 - e[:-1] ** 3)
    area = math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    if kind == "wp":
        return area * 2.0 * pimax
    if kind == "rppi":
        dpi = pimax / npibins
        return np.repeat((area * 2.0 * dpi)[:, None], npibins, axis=1)
    raise ValueError(f"no analytic volume for kind {kind!r}")


def rr_analytic(kind: str, edges, n: int, box: float, pimax: float = 0.0, npibins: int = 0) -> np.ndarray:
    """Expected ordered random-random counts for n uniform points in a periodic cube of side box:
    RR_i = dV_i * N * (N-1) / V (Appendix B), plus the N self pairs in the first bin when its lower
    edge is 0 (for rp-pi: the first pi bin of the first rp bin).  Valid while the largest separation
    stays below box / 2 (no bin wraps onto itself)."""
    rr = shell_volumes(kind, edges, pimax, npibins) * float(n) * float(n - 1) / float(box) ** 3
    if float(np.asarray(edges)[0]) == 0.0:
        rr.flat[0] += n
    return rr


def xi_natural(dd, rr, nd: int, nr: int, rr_is_auto: bool = True) -> np.ndarray:
    """1 + xi = DD / RR on normalised counts (Sec. 2.1).  dd: ordered auto counts of nd points;
    rr: ordered auto counts of nr randoms (or analytic RR of nd points: pass nr = nd)."""
    ddn = _norm_auto(dd, nd)
    rrn = _norm_auto(rr, nr) if rr_is_auto else np.asarray(rr, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rrn > 0, ddn / rrn - 1.0, 0.0)


def xi_theory(dd, n: int, box: float, edges) -> np.ndarray:
    """xi(r) of n points in a periodic cube: the natural estimator against the analytic RR."""
    rr = rr_analytic("r", edges, n, box)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rr > 0, np.asarray(dd, dtype=np.float64) / rr - 1.0, 0.0)


def landy_szalay(dd, dr, rr, nd: int, nr: int) -> np.ndarray:
    """(DD - 2 DR + RR) / RR on normalised counts: dd ordered auto counts of the nd data points,
    dr cross counts data x randoms, rr ordered auto counts of the nr randoms."""
    ddn = _norm_auto(dd, nd)
    drn = _norm_cross(dr, nd, nr)
    rrn = _norm_auto(rr, nr)
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(rrn > 0, (ddn - 2.0 * drn + rrn) / rrn, 0.0)


def wp_from_xi(xi_rppi, pimax: float, npibins: int) -> np.ndarray:
    """wp(rp) = 2 * sum_m xi(rp, pi_m) * dpi over 0 <= pi < pimax (Eq. 2); xi_rppi holds nbins rows
    of npibins values (the layout of the rp-pi counts)."""
    x = np.asarray(xi_rppi, dtype=np.float64).reshape(-1, npibins)
    return 2.0 * x.sum(axis=1) * (pimax / npibins)
