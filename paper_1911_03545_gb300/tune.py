"""Autotuner for the pair-counting launch configuration.

Knobs (all results are identical across them; only speed changes):
  variant pair-kernel form: 1 bins every pair where it is formed, 2 compacts the candidates
          of each lane into a per-warp ring first
  refine  sub-cells per Rmax cell (Sec. 4.2): 1, 2, 3
  warps   warps per CTA of the persistent pair kernel (CTA shape; occupancy follows from the
          shared-memory histograms): 0 (as many as fit), 12, 8, 6, 4
  tile    i-tile size (i points held in registers per warp item): 64, 128
  jchunk  j range per work item (staging depth of the j stream): 128, 256, 512
  noprune 1 visits every stencil neighbour; 0 skips cell pairs whose points' bounding boxes are
          farther apart than the largest edge (costs one pass over the points)
  block   1 gives the pair kernel only the 32-point groups of a j cell that may come within the
          largest edge of the i tile; 0 whole cells.  Searched only with tune(..., block=True): it
          lowers the evaluated-pair count, so evaluated-pair rates with and without it differ
  thetagrid DD(theta) only: 0 the 3-D grid over unit vectors, 1 declination bands x RA cells

The tuner times `cf_count` on the caller's own catalogue (coordinate descent from the default,
repeated while a pass still improves, at most twice). Each candidate runs alternately with the
current best, 5 times each, and replaces it only if its median is more than 1 % faster. The
result is cached in a JSON file keyed by device name,
kind, options and an occupancy class (log2 of the mean number of points per Rmax cell).  The cache
path is $CF_TUNE_CACHE, else ~/.cache/cf_gb300_tune.json.
"""
from __future__ import annotations

import json
import math
import os
import time

from . import (CF_DD_RPPI_MOCKS, CF_DD_THETA, CF_OPT_BLOCK_PRUNE, CF_OPT_CELL_PRUNE, CF_OPT_JCHUNK, CF_OPT_REFINE,
               CF_OPT_THETA_GRID, CF_OPT_TILE, CF_OPT_VARIANT, CF_OPT_WARPS, cf_count, cf_get_stats, cf_set_option)

KNOBS = {"variant": [1, 2], "refine": [1, 2, 3], "warps": [0, 12, 8, 6, 4], "tile": [128, 64],
         "jchunk": [512, 256, 128], "noprune": [0, 1], "thetagrid": [0, 1]}
OPT = {"variant": CF_OPT_VARIANT, "refine": CF_OPT_REFINE, "warps": CF_OPT_WARPS, "tile": CF_OPT_TILE,
       "jchunk": CF_OPT_JCHUNK, "noprune": CF_OPT_CELL_PRUNE, "block": CF_OPT_BLOCK_PRUNE,
       "thetagrid": CF_OPT_THETA_GRID}
DEFAULT = {"variant": 1, "refine": 1, "warps": 0, "tile": 128, "jchunk": 512, "noprune": 0, "block": 0,
           "thetagrid": 0}
MARGIN = 0.01


def knobs_for(p, block: bool = False) -> dict:
    """The knobs that can change anything for this kind: the angular grid exists for DD(theta)
    only, and the mocks kind has the direct form only."""
    k = dict(KNOBS)
    if p.kind != CF_DD_THETA:
        k.pop("thetagrid")
    if p.kind == CF_DD_RPPI_MOCKS:
        k.pop("variant")
    if block:
        k["block"] = [0, 1]
    return k


def cache_path() -> str:
    return os.environ.get("CF_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "cf_gb300_tune.json"))


def occupancy_class(p, npoints: int) -> int:
    """log2 of the mean points per cell of the unrefined grid (Sec. 4.1)."""
    from . import cf_plan_probe
    import numpy as np
    box = list(p.c.box) if p.c.periodic else [1.0, 1.0, 1.0]
    bb = [0.0, 0.0, 0.0] + box
    info = cf_plan_probe(p, bb, max(1, npoints))
    cells = max(1, int(np.prod(info["grid"])))
    return int(round(math.log2(max(1.0, npoints / cells))))


def _key(device_name: str, p, npoints: int) -> str:
    return "|".join([device_name, str(p.kind), f"w{p.c.weight}", f"r{p.c.output_ravg}", f"p{p.c.periodic}",
                     f"n{len(p.edges) - 1}", f"occ{occupancy_class(p, npoints)}"])


def apply(ctx, cfg: dict) -> None:
    for k, v in cfg.items():
        cf_set_option(ctx, OPT[k], int(v))


def reset(ctx) -> None:
    apply(ctx, {k: 0 for k in OPT})


def _time(ctx, p, d1, d2, reps: int, timer=None) -> float:
    if timer is not None:
        return min(timer() for _ in range(reps))
    best = float("inf")
    for _ in range(reps):
        t0 = time.perf_counter()
        cf_count(ctx, p, d1, d2)
        st = cf_get_stats(ctx)
        wall = time.perf_counter() - t0
        best = min(best, (st["ms_build"] + st["ms_pair"] + st["ms_recheck"]) / 1e3 or wall)
    return best


def _duel(ctx, p, d1, d2, a: dict, b: dict, reps: int, timer=None):
    """Median times of configurations a and b, measured alternately (a, b, a, b, ...) so that
    drift and noise fall on both alike."""
    ta, tb = [], []
    for _ in range(reps):
        apply(ctx, a)
        ta.append(_time(ctx, p, d1, d2, 1, timer))
        apply(ctx, b)
        tb.append(_time(ctx, p, d1, d2, 1, timer))
    return sorted(ta)[len(ta) // 2], sorted(tb)[len(tb) // 2]


def tune(ctx, p, d1, d2=None, *, device_name: str = "gpu", npoints: int = 0, reps: int = 5,
         passes: int = 2, use_cache: bool = True, log=None, timer=None, block: bool = False) -> dict:
    """Return the best configuration for this workload (and leave it applied on ctx).  timer:
    optional callable that runs one count on ctx and returns its time in seconds (so that the
    tuner ranks configurations by the caller's own measurement); by default the library's event
    times of build, pair kernel and recheck.  block: also search the group pruning knob."""
    key = (_key(device_name, p, npoints or 1) + ("|block" if block else "")) if use_cache else ""
    path = cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    if use_cache and key in cache:
        cfg = cache[key]["cfg"]
        apply(ctx, cfg)
        return cfg
    cfg = dict(DEFAULT)
    apply(ctx, cfg)
    _time(ctx, p, d1, d2, 1, timer)               # warm up
    best_t = _time(ctx, p, d1, d2, reps, timer)
    trials = [(dict(cfg), best_t)]
    # coordinate descent, repeated: a knob's best value can change once later knobs have moved
    for _ in range(passes):
        moved = False
        for knob, values in knobs_for(p, block).items():
            for v in values:
                if v == cfg[knob]:
                    continue
                cand = dict(cfg)
                cand[knob] = v
                # the candidate against the current best, measured alternately; a move must win
                # by a margin (a marginal win of a few repetitions is often noise)
                tc, tb = _duel(ctx, p, d1, d2, cand, cfg, reps, timer)
                trials.append((dict(cand), tc))
                if log:
                    log(f"tune {cand} {tc * 1e3:.3f} ms against {tb * 1e3:.3f} ms")
                if tc < tb * (1.0 - MARGIN):
                    best_t, cfg, moved = tc, cand, True
        if not moved:
            break
    apply(ctx, cfg)
    if use_cache:
        cache[key] = {"cfg": cfg, "ms": best_t * 1e3,
                      "trials": [{"cfg": c, "ms": t * 1e3} for c, t in trials]}
        os.makedirs(os.path.dirname(path), exist_ok=True)
        with open(path + ".tmp", "w") as f:
            json.dump(cache, f, indent=1)
        os.replace(path + ".tmp", path)
    return cfg
