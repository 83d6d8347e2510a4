"""FP64 CPU oracle for binned pair counts (test infrastructure).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may import this package.
It is built from `cf_oracle.c` with gcc (-O2 -ffp-contract=off -fopenmp) and loaded with
ctypes.  It shares no code with the CUDA library.

`count()` returns a dict with the paper's outputs (Sec. 2.1, Code naivecorr; Appendix B):
  npairs  uint64, ordered-pair convention (auto counts doubled, plus N self pairs when the
          first edge is 0)
  wsum    sum of w_i*w_j per bin (1 per pair when unweighted)
  rsum    sum of (w_i*w_j*) separation per bin, only when ravg is requested
  ravg    rsum / wsum (weighted) or rsum / npairs, 0 for empty bins
  wp      (kind "wp" with a periodic box) the projected correlation function, Eq. (2) with the
          analytic RR of Appendix B.
Shapes are (nbins,) or, for "rppi", (nbins, npibins).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cf_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

KINDS = {"r": 0, "rppi": 1, "wp": 2, "theta": 3, "mocks": 4}
MODES = {"brute": 0, "zwin": 1, "rows": 2, "zrows": 3}


class _Params(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("autocorr", ctypes.c_int),
        ("periodic", ctypes.c_int),
        ("box", ctypes.c_double * 3),
        ("edges", ctypes.POINTER(ctypes.c_double)),
        ("nbins", ctypes.c_int),
        ("pimax", ctypes.c_double),
        ("npibins", ctypes.c_int),
        ("weighted", ctypes.c_int),
        ("ravg", ctypes.c_int),
    ]


def build(extra_flags=(), out=None, force=False) -> str:
    """Compile the oracle into a shared library; returns its path."""
    out = out or _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if (not force and os.path.exists(out)
            and os.path.getmtime(out) >= os.path.getmtime(_SRC) and not extra_flags):
        return out
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           *extra_flags, _SRC, "-o", out + ".tmp", "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(out + ".tmp", out)
    return out


def _setup(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    lib.or_count.restype = ctypes.c_int
    lib.or_count.argtypes = [ctypes.POINTER(_Params), ctypes.c_int64, dp, dp, dp, dp,
                             ctypes.c_int64, dp, dp, dp, dp, ctypes.c_int, ctypes.c_int,
                             ctypes.c_int64, ctypes.c_int64,
                             ctypes.POINTER(ctypes.c_uint64), dp, dp]
    lib.or_squared_edges.restype = ctypes.c_int
    lib.or_squared_edges.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp]
    return lib


def load(path=None):
    """Load (building if needed) the oracle library.  `path` loads a specific build."""
    global _lib
    if path is not None:
        return _setup(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _setup(ctypes.CDLL(build()))
        return _lib


def _f64(a):
    if a is None:
        return None
    return np.ascontiguousarray(np.asarray(a), dtype=np.float64)   # float32 -> float64 is exact


def _ptr(a):
    if a is None:
        return ctypes.POINTER(ctypes.c_double)()
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def squared_edges(kind: str, edges, lib=None) -> np.ndarray:
    lib = lib or load()
    e = _f64(edges)
    out = np.empty_like(e)
    lib.or_squared_edges(KINDS[kind], _ptr(e), len(e) - 1, _ptr(out))
    return out


def count(kind: str, edges, d1, d2=None, *, autocorr: bool, periodic: bool, box=0.0,
          pimax: float = 0.0, npibins: int = 0, weighted: bool = False, ravg: bool = False,
          mode: str = "zwin", nthreads: int = 0, rows=None, lib=None) -> dict:
    """Count pairs.  d1/d2 are objects with x, y, z (and w) arrays (e.g. gen.Catalogue)."""
    lib = lib or load()
    e = _f64(edges)
    nb = len(e) - 1
    b = (float(box),) * 3 if np.isscalar(box) else tuple(float(v) for v in box)
    p = _Params(KINDS[kind], int(bool(autocorr)), int(bool(periodic)), (ctypes.c_double * 3)(*b),
                _ptr(e), nb, float(pimax), int(npibins), int(bool(weighted)), int(bool(ravg)))
    a1 = [_f64(getattr(d1, c)) for c in "xyz"]
    w1 = _f64(d1.w) if weighted and d1.w is not None else None
    if autocorr or d2 is None:
        a2, w2, n2 = a1, w1, len(a1[0])
    else:
        a2 = [_f64(getattr(d2, c)) for c in "xyz"]
        w2 = _f64(d2.w) if weighted and d2.w is not None else None
        n2 = len(a2[0])
    nout = nb * (npibins if kind in ("rppi", "mocks") else 1)
    npairs = np.zeros(nout, dtype=np.uint64)
    wsum = np.zeros(nout)
    rsum = np.zeros(nout)
    if rows is None:
        r0, r1 = 0, len(a1[0])
        md = MODES[mode]
    else:
        # a row range: every ordered pair of those rows, by brute force or through the z window
        r0, r1 = rows
        md = MODES["zrows"] if mode == "zwin" else MODES["rows"]
    rc = lib.or_count(ctypes.byref(p), len(a1[0]), *[_ptr(a) for a in a1], _ptr(w1),
                      n2, *[_ptr(a) for a in a2], _ptr(w2), md, int(nthreads), int(r0), int(r1),
                      npairs.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), _ptr(wsum), _ptr(rsum))
    if rc != 0:
        raise RuntimeError(f"oracle failed with status {rc}")
    out = {"npairs": npairs, "wsum": wsum}
    if ravg:
        den = wsum if weighted else npairs.astype(np.float64)
        with np.errstate(invalid="ignore", divide="ignore"):
            out["ravg"] = np.where(den > 0, rsum / np.where(den > 0, den, 1), 0.0)
        out["rsum"] = rsum
    if kind == "wp" and periodic and autocorr and rows is None:
        out["wp"] = wp_from_counts(npairs, e, len(a1[0]), b, pimax)
    if kind in ("rppi", "mocks"):
        for k in list(out):
            out[k] = out[k].reshape(nb, npibins)
    return out


def wp_from_counts(npairs, edges, n, box, pimax) -> np.ndarray:
    """Eq. (2) with the natural estimator 1+xi = DD/RR (Sec. 2.1) and the analytic RR of
    Appendix B (density (N-1)/V).  With unit-width pi bins of equal RR,
    wp = 2*sum_m [DD_m/RR_m - 1]*dpi = DD_tot/(N(N-1)/V * pi*(rp_hi^2 - rp_lo^2)) - 2*pimax."""
    e = np.asarray(edges, dtype=np.float64)
    V = float(box[0]) * float(box[1]) * float(box[2])
    area = math.pi * (e[1:] ** 2 - e[:-1] ** 2)
    rr_per_unit_pi = n * (n - 1) / V * area          # ordered pairs per unit line-of-sight length, both signs
    return np.asarray(npairs, dtype=np.float64) / rr_per_unit_pi - 2.0 * pimax
