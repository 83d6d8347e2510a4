"""Seeded synthetic catalogues with the shapes of the paper's workloads.

The paper measures on a ~1.2M-galaxy mock in a periodic L=420 Mpc/h cube (Sec. 5) and on an
Abacus halo catalogue (Sec. 6); neither is available here, so these generators stand in for
them.  Every array is drawn from numpy's PCG64 with a fixed seed, so the same call yields
the same bytes on every machine.

Recipes (float32 unless stated):
  * uniform box: x,y,z ~ U[0, L)                                (float64 kept for the
    small correctness workload).
  * clustered box: ncentres centres ~ U[0, L)^3, each with `members` points offset by
    isotropic N(0, sigma^2); wrapped into [0, L) in float64, then cast to float32; a value
    that rounds up to L is mapped to 0, so every coordinate lies in [0, L).
  * weights ~ U[lo, hi) float32.
  * sphere patch: RA ~ U[ra0, ra1) deg, sin(DEC) ~ U[sin dec0, sin dec1), converted to a unit
    vector in float64, then each component rounded to float32.
  * survey cone (observed galaxies, observer at the origin): RA ~ U[ra0, ra1) deg, sin(DEC) ~
    U[sin dec0, sin dec1), comoving distance d with d^3 ~ U[d0^3, d1^3) (uniform in volume),
    converted to Cartesian in float64; clustered: that recipe for the centres, each with
    `members` points offset by isotropic N(0, sigma^2); every component rounded to float32.
  * edges: log-spaced in float64 with the end points set exactly.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

GEN_VERSION = 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


@dataclasses.dataclass
class Catalogue:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    w: Optional[np.ndarray] = None

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def dtype(self):
        return self.x.dtype

    def subset(self, idx) -> "Catalogue":
        return Catalogue(self.x[idx], self.y[idx], self.z[idx],
                         None if self.w is None else self.w[idx])


def log_edges(lo: float, hi: float, nbins: int) -> np.ndarray:
    e = np.logspace(math.log10(lo), math.log10(hi), nbins + 1, dtype=np.float64)
    e[0] = lo
    e[-1] = hi
    return e


def _wrap_cast(v: np.ndarray, L: float, dtype) -> np.ndarray:
    v = np.mod(v, L)                      # float64, in [0, L]
    out = v.astype(dtype)
    out[out >= dtype(L)] = 0              # a value that rounded up to L goes to 0
    out[out < 0] = 0
    return out


def uniform_box(n: int, L: float, seed: int, dtype=np.float32) -> Catalogue:
    r = _rng(seed)
    p = r.uniform(0.0, L, size=(3, n))
    return Catalogue(*(_wrap_cast(p[a], L, dtype) for a in range(3)))


def clustered_box(ncentres: int, members: int, sigma: float, L: float, seed: int,
                  dtype=np.float32) -> Catalogue:
    r = _rng(seed)
    c = r.uniform(0.0, L, size=(3, ncentres))
    off = r.normal(0.0, sigma, size=(3, ncentres, members))
    p = (c[:, :, None] + off).reshape(3, ncentres * members)
    return Catalogue(*(_wrap_cast(p[a], L, dtype) for a in range(3)))


def uniform_weights(n: int, lo: float, hi: float, seed: int) -> np.ndarray:
    return _rng(seed).uniform(lo, hi, size=n).astype(np.float32)


def sphere_patch(n: int, ra0: float, ra1: float, dec0: float, dec1: float, seed: int) -> Catalogue:
    r = _rng(seed)
    ra = np.deg2rad(r.uniform(ra0, ra1, size=n))
    sdec = r.uniform(math.sin(math.radians(dec0)), math.sin(math.radians(dec1)), size=n)
    cdec = np.sqrt(np.maximum(0.0, 1.0 - sdec * sdec))
    return Catalogue((cdec * np.cos(ra)).astype(np.float32),
                     (cdec * np.sin(ra)).astype(np.float32),
                     sdec.astype(np.float32))


def survey_cone(n: int, ra0: float, ra1: float, dec0: float, dec1: float, d0: float, d1: float, seed: int,
                members: int = 1, sigma: float = 0.0) -> Catalogue:
    """Positions of observed galaxies (or randoms with members = 1) in a survey cone seen from
    the origin; n points in total (n // members centres, the remainder dropped)."""
    r = _rng(seed)
    nc = max(1, n // members)
    ra = np.deg2rad(r.uniform(ra0, ra1, size=nc))
    sdec = r.uniform(math.sin(math.radians(dec0)), math.sin(math.radians(dec1)), size=nc)
    cdec = np.sqrt(np.maximum(0.0, 1.0 - sdec * sdec))
    d = np.cbrt(r.uniform(d0 ** 3, d1 ** 3, size=nc))
    c = np.stack([d * cdec * np.cos(ra), d * cdec * np.sin(ra), d * sdec], axis=1)
    if members > 1:
        c = (c[:, None, :] + r.normal(0.0, sigma, size=(nc, members, 3))).reshape(-1, 3)
    return Catalogue(c[:, 0].astype(np.float32), c[:, 1].astype(np.float32), c[:, 2].astype(np.float32))


def unit_sphere(n: int, seed: int) -> Catalogue:
    """Uniform on the full sphere (for the analytic angular pin)."""
    return sphere_patch(n, 0.0, 360.0, -90.0, 90.0, seed)


# ---------------------------------------------------------------------------------------------
# Named workloads (the five measurement configurations and their scaled-down parity variants)
# ---------------------------------------------------------------------------------------------

@dataclasses.dataclass
class Workload:
    name: str
    kind: str                      # "r", "rppi", "wp", "theta", "mocks"
    autocorr: bool
    periodic: bool
    box: float
    edges: np.ndarray              # r / rp edges, or theta edges in degrees
    d1: Catalogue
    d2: Optional[Catalogue] = None
    pimax: float = 0.0
    npibins: int = 0
    weighted: bool = False
    ravg: bool = False
    extra: dict = dataclasses.field(default_factory=dict)


def batch_sizes(ncat: int = 256, lo: float = 5e4, hi: float = 8e5, seed: int = 4000) -> List[int]:
    r = _rng(seed)
    u = r.uniform(math.log(lo), math.log(hi), size=ncat)
    return [int(round(math.exp(v))) for v in u]


def batch_catalogue(i: int, n: int, L: float = 250.0, members: int = 50, sigma: float = 1.0,
                    seed_base: int = 4100) -> Catalogue:
    nc = max(1, n // members)
    cat = clustered_box(nc, members, sigma, L, seed_base + i)
    if cat.n > n:
        cat = cat.subset(slice(0, n))
    elif cat.n < n:                     # top up with uniform points so N is exact
        extra = uniform_box(n - cat.n, L, seed_base + 100000 + i)
        cat = Catalogue(*(np.concatenate([getattr(cat, a), getattr(extra, a)]) for a in "xyz"))
    return cat


def workload(name: str, scale: float = 1.0) -> Workload:
    """Build a named workload.  `scale` < 1 shrinks the point counts (same recipe and density
    profile per cluster) for parity runs that the oracle finishes in seconds."""
    if name == "uniform_r_20k":
        n = max(8, int(20000 * scale))
        return Workload(name, "r", True, True, 250.0, log_edges(0.1, 25.0, 20),
                        uniform_box(n, 250.0, 1000, dtype=np.float64))
    if name == "clustered_r_1m":
        nc = max(1, int(10000 * scale))
        L = 420.0 * (nc / 10000) ** (1.0 / 3.0) if scale != 1.0 else 420.0
        d = clustered_box(nc, 100, 1.0, L, 1001)
        d.w = uniform_weights(d.n, 0.5, 1.5, 1002)
        return Workload(name, "r", True, True, L, log_edges(0.1, 20.0, 20), d,
                        weighted=True, ravg=True)
    if name in ("clustered_rppi_2m", "clustered_wp_2m", "clustered_rppi_dr", "clustered_rppi_2m_wr"):
        nc = max(1, int(20000 * scale))
        L = 1000.0 * (nc / 20000) ** (1.0 / 3.0) if scale != 1.0 else 1000.0
        d = clustered_box(nc, 100, 2.0, L, 1003)
        kind = "wp" if name == "clustered_wp_2m" else "rppi"
        if name == "clustered_rppi_2m_wr":
            # the same catalogue with pair-product weights and ravg
            d.w = uniform_weights(d.n, 0.5, 1.5, 1009)
            return Workload(name, "rppi", True, True, L, log_edges(0.1, 25.0, 14), d,
                            pimax=40.0, npibins=40, weighted=True, ravg=True)
        if name == "clustered_rppi_dr":
            rn = max(8, int(4000000 * scale))
            rr = uniform_box(rn, L, 1004)
            return Workload(name, "rppi", False, True, L, log_edges(0.1, 25.0, 14), d, rr,
                            pimax=40.0, npibins=40)
        return Workload(name, kind, True, True, L, log_edges(0.1, 25.0, 14), d,
                        pimax=40.0, npibins=40)
    if name == "mock_dr_rppi":
        # DR(rp, pi) of mock galaxies against randoms at 10x their density (the paper's mocks
        # scaling workload, Sec. 5.2), in a 90 x 60 deg cone from 300 to 1000 Mpc/h
        nd = max(8, int(200000 * scale))
        d0, d1 = 300.0, 300.0 + 700.0 * (scale ** (1.0 / 3.0) if scale != 1.0 else 1.0)
        d = survey_cone(nd, 0.0, 90.0, 0.0, 60.0, d0, d1, 1007, members=100, sigma=2.0)
        rr = survey_cone(10 * nd, 0.0, 90.0, 0.0, 60.0, d0, d1, 1008)
        return Workload(name, "mocks", False, False, 0.0, log_edges(0.5, 42.0, 14), d, rr,
                        pimax=42.0, npibins=42)
    if name == "polar_theta_1m":
        n = max(8, int(1000000 * scale))
        return Workload(name, "theta", True, False, 0.0, log_edges(0.001, 1.0, 20),
                        sphere_patch(n, 0.0, 360.0, 60.0, 90.0, 1006))
    if name == "sphere_theta_1m":
        n = max(8, int(1000000 * scale))
        return Workload(name, "theta", True, False, 0.0, log_edges(0.001, 1.0, 20),
                        sphere_patch(n, 0.0, 90.0, -10.0, 30.0, 1005))
    raise KeyError(name)
