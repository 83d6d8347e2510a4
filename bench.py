"""Benchmark of the GB300 pair counter (one JSON line on rank 0).

Default workload (the headline configuration): DD(r) auto-correlation, periodic L=420 box,
N = 1,000,000 clustered float32 points (10,000 centres x 100 members, Gaussian sigma = 1),
20 log bins 0.1-20, pair-product weights and ravg.  A step is one cf_count of the whole
workload with inputs already resident in HBM; the metric is pair-distance evaluations per
second (separations the pair kernel computes), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl gb300|reference]

Multi-GPU runs (torchrun) are independent replicas: the path of one catalogue does not shard
across GPUs in this build; each rank counts its own copy and `value` sums the ranks' work
over the slowest rank's time.  `--impl reference` times the FP64 CPU oracle instead (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "pair-distance evals/s"
UNIT = "pairs/s"
FP32_INSTR_PER_PAIR = 6          # 3 FADD (dx, dy, dz) + 1 FMUL + 2 FFMA: the algorithmic minimum
# the mocks kind's division-free candidate cut (Appendix A.2.1): s (3), s.s (3), s.A_i (3),
# s.l = s.A_i - s.s/2 (1), l.l = A_i.A_i - s.A_i + s.s/4 (2), (s.l)^2 (1), the two cut products (2)
FP32_INSTR_PER_PAIR_KIND = {"mocks": 15}
L2_FLUSH_BYTES = 512 << 20       # > 129 MB L2

WORKLOADS = {
    "clustered_r_1m": "DD(r) auto, periodic L=420, N=1,000,000 clustered float32 (10,000 centres x 100, "
                      "sigma=1), 20 log bins 0.1-20, pair-product weights U[0.5,1.5) + ravg",
    "uniform_r_20k": "DD(r) auto, periodic L=250, N=20,000 uniform float64, 20 log bins 0.1-25",
    "clustered_rppi_2m": "DD(rp,pi) auto, periodic L=1000, N=2,000,000 clustered float32 (20,000 x 100, "
                         "sigma=2), 14 log rp bins 0.1-25, pimax=40 with 40 pi bins",
    "clustered_rppi_2m_wr": "DD(rp,pi) auto, the clustered_rppi_2m catalogue with pair-product weights U[0.5,1.5) "
                            "+ ravg",
    "clustered_wp_2m": "wp(rp) auto, periodic L=1000, N=2,000,000 clustered float32, 14 log rp bins 0.1-25, pimax=40",
    "clustered_rppi_dr": "DR(rp,pi) cross, periodic L=1000, D=2,000,000 clustered x R=4,000,000 uniform float32, "
                         "14 log rp bins 0.1-25, pimax=40 with 40 pi bins",
    "sphere_theta_1m": "DD(theta) auto, non-periodic, N=1,000,000 unit vectors (RA 0-90, DEC -10..30 deg) float32, "
                       "20 log bins 0.001-1 deg",
    "polar_theta_1m": "DD(theta) auto, non-periodic, N=1,000,000 unit vectors uniform on the polar cap DEC 60..90 deg "
                      "float32, 20 log bins 0.001-1 deg",
    "mock_dr_rppi": "DR(rp,pi) of mocks (Fisher et al. line of sight), non-periodic, D=200,000 clustered (2,000 x 100, "
                    "sigma=2) x R=2,000,000 uniform float32 in a cone RA 0-90, DEC 0-60 deg, 300-1000 Mpc/h from "
                    "the observer, 14 log rp bins 0.5-42, pimax=42 with 42 pi bins",
}


def _env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _parse_config(text: str) -> dict:
    from paper_1911_03545_gb300 import tune
    cfg = {}
    for part in filter(None, text.split(",")):
        k, v = part.split("=")
        if k not in tune.OPT:
            raise SystemExit(f"unknown knob {k!r}; knobs: {sorted(tune.OPT)}")
        cfg[k] = int(v)
    return cfg


def _kernel_sha() -> str:
    h = hashlib.sha256()
    for name in ("cf_pair.cuh", "cf_device.cuh", "cf_internal.h"):
        with open(os.path.join(ROOT, "paper_1911_03545_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(workload: str):
    """DRAM bytes per pair-kernel launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "pair_kernel_traffic.txt")
    try:
        with open(p) as f:
            for line in f:
                parts = line.split()
                if len(parts) >= 3 and not line.startswith("#") and parts[0] == workload:
                    if parts[1] == _kernel_sha():
                        return float(parts[2])
    except OSError:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.index)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            c = [x.strip() for x in line.split(",")]
            if len(c) < 9:
                continue
            try:
                sm.append(float(c[1]))
                mx.append(float(c[2]))
            except ValueError:
                continue
            for n, v in zip(names, c[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.f.name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    world = _env_int("WORLD_SIZE", 1)
    rank = _env_int("RANK", 0)
    local = _env_int("LOCAL_RANK", 0)
    return world, rank, local


def _barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(world, v: float, dev) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(world, v: float, dev) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _wl_params(wl, cf):
    return cf.params(kind=wl.kind, edges=wl.edges, autocorr=wl.autocorr, periodic=wl.periodic, box=wl.box,
                     pimax=wl.pimax, npibins=wl.npibins, ravg=wl.ravg, weighted=wl.weighted)


def _points(cat, weighted, cf, dev=None, pinned=False):
    """Device tensors (dev), pinned host tensors (pinned: the library copies them in every call), or
    pageable numpy arrays."""
    import numpy as np
    import torch
    arrs = [cat.x, cat.y, cat.z] + ([cat.w] if weighted else [])
    if dev is None and not pinned:
        return cf.points(*[np.ascontiguousarray(a) for a in arrs[:3]], arrs[3] if weighted else None)
    t = [torch.from_numpy(np.ascontiguousarray(a)) for a in arrs]
    t = [x.pin_memory() for x in t] if dev is None else [x.to(dev) for x in t]
    return cf.points(*t[:3], t[3] if weighted else None)


# the other configurations, measured in the same run as the headline (each tuned, L2 flushed)
EXTRA_WORKLOADS = ["uniform_r_20k", "clustered_rppi_2m", "clustered_wp_2m", "clustered_rppi_dr", "sphere_theta_1m",
                   "clustered_rppi_2m_wr", "mock_dr_rppi"]
GOLDEN = os.path.join(ROOT, "tests", "golden")


def _fingerprint(*cats) -> str:
    """sha256 of the generated arrays, in the stored histograms' format (x, y, z, w per set)."""
    import numpy as np
    h = hashlib.sha256()
    for c in cats:
        if c is None:
            continue
        for a in (c.x, c.y, c.z, c.w):
            if a is not None:
                h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()


def _parity(name, got, cats) -> dict:
    """The result against the FP64 oracle's stored histogram of the same seeded inputs
    (tests/golden/full_<name>.json, written by tests/golden/make_golden.py): counts bit-exact,
    weighted sums and ravg within 1e-6 relative."""
    import numpy as np
    try:
        with open(os.path.join(GOLDEN, f"full_{name}.json")) as f:
            gold = json.load(f)
    except (OSError, ValueError):
        return {"ok": None, "why": "no stored oracle histogram"}
    if gold.get("fingerprint") != _fingerprint(*cats):
        return {"ok": None, "why": "the generated inputs differ from the stored histogram's"}
    counts = bool(np.array_equal(np.asarray(got["npairs"]).ravel().astype(np.uint64),
                                 np.asarray(gold["npairs"], dtype=np.uint64)))
    worst = 0.0
    for k in ("wsum", "ravg"):
        if k in gold and k in got:
            g = np.asarray(got[k], dtype=np.float64).ravel()
            e = np.asarray(gold[k], dtype=np.float64)
            nz = e != 0
            worst = max(worst, float(np.max(np.abs(g[nz] - e[nz]) / np.abs(e[nz]), initial=0.0)),
                        float(np.max(np.abs(g[~nz]), initial=0.0)))
    return {"ok": counts and worst <= 1e-6, "counts_equal": counts, "max_rel_err_sums": worst,
            "against": f"tests/golden/full_{name}.json"}


def _peak_pairs(dev, kind) -> float:
    """R* in pairs/s: SMs x 128 FP32 lanes x the measured maximum SM clock / FP32 operations per pair."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(_peaks().get("sm_max_mhz", 2070.0))
    return props.multi_processor_count * 128 * sm_max * 1e6 / FP32_INSTR_PER_PAIR_KIND.get(kind, FP32_INSTR_PER_PAIR)


def _measure_workload(args, cf, tune, ctx, name, dev, flush, force: dict | None = None) -> dict:
    """One more configuration on the headline's context: tuned (cache honoured; `force` then
    overrides knobs), 2 untimed calls, then args.extra_steps calls with the L2 flushed before each,
    device-resident inputs."""
    import numpy as np
    import torch

    import gen
    stream = torch.cuda.current_stream(dev)
    wl = gen.workload(name)
    p = _wl_params(wl, cf)
    d1 = _points(wl.d1, wl.weighted, cf, dev)
    d2 = None if wl.autocorr else _points(wl.d2, wl.weighted, cf, dev)
    npts = wl.d1.n + (0 if wl.autocorr else wl.d2.n)

    def step_time():
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        cf.cf_count(ctx, p, d1, d2)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / 1e3

    tune.reset(ctx)
    tuned = tune.tune(ctx, p, d1, d2, device_name=torch.cuda.get_device_name(dev), npoints=npts, reps=3, passes=1,
                      use_cache=not args.no_tune_cache, timer=step_time)
    if force:
        tuned = dict(tuned, **force)
        tune.apply(ctx, tuned)
    for _ in range(2):
        out = cf.cf_count(ctx, p, d1, d2)
    step_ms, pair_ms = [], []
    for _ in range(args.extra_steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = cf.cf_count(ctx, p, d1, d2)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        pair_ms.append(cf.cf_get_stats(ctx)["ms_pair"])
    st = cf.cf_get_stats(ctx)
    tune.reset(ctx)
    ev = int(st["evaluated_pairs"])
    step, pair = statistics.fmean(step_ms), statistics.fmean(pair_ms)
    in_range = int(np.asarray(out["npairs"], dtype=np.float64).sum())
    rec = {
        "workload": WORKLOADS[name], "steps": args.extra_steps, "step_ms": step, "pair_kernel_ms": pair,
        "evaluated_pairs_per_step": ev, "evaluated_pairs_per_s": ev / (step / 1e3),
        "in_range_pairs_per_step": in_range, "in_range_pairs_per_s": in_range / (step / 1e3),
        "roofline_frac": ev / (pair / 1e3) / _peak_pairs(dev, wl.kind),
        "roofline_basis": f"{FP32_INSTR_PER_PAIR_KIND.get(wl.kind, FP32_INSTR_PER_PAIR)} FP32 operations per pair",
        "rechecked_pairs_per_step": int(st["rechecked_pairs"]), "fixed_sums": int(st["fixed_sums"]),
        "tuned": tuned, "parity_vs_golden": _parity(name, out, (wl.d1, None if wl.autocorr else wl.d2)),
    }
    del d1, d2
    return rec


def _extras(args, cf, tune, ctx, dev, local, flush) -> dict:
    """Every configuration besides the headline: the other single-catalogue workloads, and the
    256-catalogue batch counted one at a time, batched, graph-replayed and served."""
    import numpy as np
    out = {"workloads": {name: _measure_workload(args, cf, tune, ctx, name, dev, flush) for name in EXTRA_WORKLOADS}}
    # the same workloads with the pair kernel given only the 32-point groups within reach (an
    # option the line's other figures leave off: it lowers the evaluated-pair count they measure)
    out["block_prune"] = {name: _measure_workload(args, cf, tune, ctx, name, dev, flush, force={"block": 1})
                          for name in ("clustered_r_1m", "clustered_rppi_2m", "clustered_rppi_dr")}
    sizes, cats = _batch_setup(256)
    b = _batch_measure(args, cf, tune, dev, local, sizes, cats, 2)
    r = _serve_measure(args, cf, dev, local, cats, args.extra_requests)
    lat = r["lat"]
    n = b["ncat"]
    out["batch256"] = {
        "workload": BATCH_DESC, "catalogues_per_s_batched": n / b["best"],
        "catalogues_per_s_one_at_a_time": n / b["t_single"], "speedup_vs_one_at_a_time": b["t_single"] / b["best"],
        "seconds_batched": b["t_batch"], "seconds_graph_replay": b["t_graph"], "seconds_one_at_a_time": b["t_single"],
        "pair_kernel_ms": b["pair_ms"], "roofline_frac": b["achieved"] / b["peak"],
        "evaluated_pairs": int(b["st"]["evaluated_pairs"]), "tuned": b["tuned"],
        "parity_batched_vs_single": b["same"], "parity_vs_golden": b["golden"],
    }
    out["serve"] = {
        "workload": BATCH_DESC, "arrivals": "Poisson", "load": args.serve_load, "requests": r["nreq"],
        "capacity_catalogues_per_s": r["capacity"], "served_catalogues_per_s": r["nreq"] / r["t_total"],
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "max": float(np.max(lat))},
        "results_equal_batched": r["ok"], "inputs": "host numpy arrays (copied by the server)",
    }
    return out


# ---------------------------------------------------------------------------------------------
# CPU oracle legs
# ---------------------------------------------------------------------------------------------

def _oracle_rows(wl, seconds: float, seed: int = 0, mode: str = "rows"):
    """Time the oracle (as it stands) on a bounded random sample of rows of the workload: each
    row is every ordered pair (i, j) of one point i, by brute force (mode "rows") or through the
    z window (mode "zwin", pinned equal to brute force on the same rows).  The sample grows until
    its rows take about `seconds` beyond the call's fixed cost.  Returns (rows, seconds, cores,
    fixed seconds of one call)."""
    import numpy as np

    import oracle
    lib = oracle.load()
    cores = os.cpu_count() or 1
    n1 = wl.d1.n
    rng = np.random.Generator(np.random.PCG64(seed))

    def run(rows):
        start = int(rng.integers(0, max(1, n1 - rows)))
        t0 = time.perf_counter()
        oracle.count(wl.kind, wl.edges, wl.d1, None if wl.autocorr else wl.d2, autocorr=wl.autocorr,
                     periodic=wl.periodic, box=wl.box, pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted,
                     ravg=wl.ravg, rows=(start, start + rows), mode=mode, nthreads=cores, lib=lib)
        return time.perf_counter() - t0

    # the fixed cost of a call (loading, threads, the z window's sort of the second set), paid once
    # by a whole-workload run as well
    t_fix = min(run(1), run(1))
    rows = 16
    t = run(rows)
    while t - t_fix < 0.2 and rows < n1:
        rows = min(n1, rows * 4)
        t = run(rows)
    for _ in range(2):      # twice: a short calibration run understates the per-row rate
        rows = int(min(n1, max(1, rows * seconds / max(t - t_fix, 1e-6))))
        t = run(rows)
    return rows, t, cores, t_fix


def _oracle_rows_rate(wl, seconds: float, seed: int = 0):
    """Brute-force oracle rate on a row sample, in evaluated pairs per second.  Returns
    (evals/s, cores, sample text, seconds)."""
    rows, t, cores, _ = _oracle_rows(wl, seconds, seed, "rows")
    n2 = wl.d1.n if wl.autocorr else wl.d2.n
    evals = rows * (n2 - (1 if wl.autocorr else 0))
    sample = (f"{rows} consecutive rows (random start) of the workload, each against all {n2} points, "
              f"brute-force FP64 oracle, {cores} threads, {t:.1f} s")
    return evals / t, cores, sample, t


def _zwin_estimate(wl, seconds: float, seed: int = 1) -> dict:
    """The z-window oracle's time for the whole workload, extrapolated from row samples.  The cost
    of a row is the slope between a sample of R rows and one of 2R rows (each call also pays a fixed
    cost: converting the arrays and the z sort, which the slope cancels); the whole run is that
    fixed cost plus n1 rows.  A row of an auto-correlation scans its full window but bins only
    j > i: between half and all of an ordered row's cost, so the estimate is a range."""
    import numpy as np

    import oracle
    lib = oracle.load()
    cores = os.cpu_count() or 1
    n1 = wl.d1.n
    rng = np.random.Generator(np.random.PCG64(seed + 100))

    def run(rows):
        start = int(rng.integers(0, max(1, n1 - rows)))
        t0 = time.perf_counter()
        oracle.count(wl.kind, wl.edges, wl.d1, None if wl.autocorr else wl.d2, autocorr=wl.autocorr,
                     periodic=wl.periodic, box=wl.box, pimax=wl.pimax, npibins=wl.npibins, weighted=wl.weighted,
                     ravg=wl.ravg, rows=(start, start + rows), mode="zwin", nthreads=cores, lib=lib)
        return time.perf_counter() - t0

    # the oracle hands rows to its threads 64 at a time: a sample of fewer than a few chunks per
    # thread would time one thread's work; grow it while the rows take under `seconds`
    r1 = max(1, min(n1 // 2, 128 * cores))
    t1, t2 = run(r1), run(2 * r1)
    while t2 - t1 < 0.25 * seconds and 4 * r1 <= n1:
        r1 *= 2
        t1, t2 = t2, run(2 * r1)
    per_row = max(t2 - t1, 1e-9) / r1
    fix = max(0.0, t1 - per_row * r1)
    rows_t = per_row * n1
    lo, hi = (fix + 0.5 * rows_t, fix + rows_t) if wl.autocorr else (fix + rows_t, fix + rows_t)
    return {"zwin_seconds_full_est": 0.5 * (lo + hi), "zwin_seconds_full_range": [lo, hi],
            "zwin_sample": f"{r1} and {2 * r1} consecutive rows (random starts) through the z window, {cores} "
                           f"threads, {t1:.2f} s and {t2:.2f} s: {1e3 * per_row:.4f} ms per row, {fix:.2f} s per "
                           f"call; scaled to {n1} rows" + ("; the whole auto-correlation bins only j > i of each "
                                                          "row's window, so its time lies in the range given"
                                                          if wl.autocorr else "")}


def _cpu_baseline(wl, seconds: float) -> dict:
    """The oracle beside the GPU on the box's own cores: its brute-force rate on a row sample (the
    line's unit), and the z-window oracle's time for the whole workload, extrapolated from a row
    sample."""
    rate, cores, sample, _ = _oracle_rows_rate(wl, 0.5 * seconds)
    out = {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample}
    out.update(_zwin_estimate(wl, 0.5 * seconds))
    return out


def _oracle_beside(seconds: float) -> dict:
    """The oracle's time for every other configuration on the same cores: the 20,000-point one run
    whole (brute force and z window), the others through the z window extrapolated from row samples,
    and the 256-catalogue batch from row samples of four of its catalogues, scaled by the sum of
    N^2 (a catalogue's pairs within the window grow as N^2 at a fixed box)."""
    import gen
    import oracle
    lib = oracle.load()
    cores = os.cpu_count() or 1
    out = {}
    for name in EXTRA_WORKLOADS:
        wl = gen.workload(name)
        if name == "uniform_r_20k":
            kw = dict(autocorr=wl.autocorr, periodic=wl.periodic, box=wl.box, weighted=wl.weighted, ravg=wl.ravg,
                      nthreads=cores, lib=lib)
            t = {}
            for mode in ("brute", "zwin"):
                t0 = time.perf_counter()
                oracle.count(wl.kind, wl.edges, wl.d1, None, mode=mode, **kw)
                t[mode] = time.perf_counter() - t0
            n = wl.d1.n
            out[name] = {"brute_seconds": t["brute"], "brute_pairs_per_s": n * (n - 1) / t["brute"],
                         "zwin_seconds": t["zwin"], "sample": f"the whole workload, {cores} threads"}
            continue
        out[name] = _zwin_estimate(wl, seconds)
    sizes, cats = _batch_setup(256)
    per_n2 = []
    for i in (0, 64, 128, 192):
        wl = gen.Workload(f"batch_{i}", "rppi", True, True, 250.0, gen.log_edges(0.1, 20.0, 14), cats[i],
                          pimax=40.0, npibins=40)
        e = _zwin_estimate(wl, 0.25 * seconds, seed=2)
        per_n2.append([x / sizes[i] ** 2 for x in e["zwin_seconds_full_range"]])
    sn2 = float(sum(n * n for n in sizes))
    lo = sn2 * statistics.fmean(r[0] for r in per_n2)
    hi = sn2 * statistics.fmean(r[1] for r in per_n2)
    out["batch256"] = {"zwin_seconds_full_est": 0.5 * (lo + hi), "zwin_seconds_full_range": [lo, hi],
                       "zwin_sample": f"row samples of catalogues 0, 64, 128 and 192 through the z window, {cores} "
                                      f"threads; seconds per N^2 averaged and scaled by the batch's sum of N^2"}
    return out


def _line_config(args, world) -> dict:
    """The workload's description, the same in the GPU line and the reference arm's line (the launch
    shape the GPU arm tuned goes under "launch")."""
    return {"workload": WORKLOADS[args.workload], "name": args.workload,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "flushed between timed steps (512 MB write outside the step events)"}


def run_reference(args, wl, world, rank):
    if rank != 0:
        return 0
    per_step = max(0.05, args.ref_seconds / max(1, args.steps + args.warmup))
    rates = []
    cores, sample = os.cpu_count() or 1, ""
    t_all = 0.0
    for s in range(args.warmup + args.steps):
        rate, cores, sample, t = _oracle_rows_rate(wl, per_step, seed=s)
        if s >= args.warmup:
            rates.append(rate)
            t_all += t
    value = statistics.fmean(rates)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_all / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _line_config(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# GPU leg
# ---------------------------------------------------------------------------------------------

def run_gpu(args, wl, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03545_gb300 as cf

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    stream = torch.cuda.current_stream(dev)
    ctx = cf.cf_create(local, stream)
    p = _wl_params(wl, cf)
    d1 = _points(wl.d1, wl.weighted, cf, dev)
    d2 = None if wl.autocorr else _points(wl.d2, wl.weighted, cf, dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    from paper_1911_03545_gb300 import tune
    npts = wl.d1.n + (0 if wl.autocorr else wl.d2.n)
    if args.config:
        tuned = dict(tune.DEFAULT, **_parse_config(args.config))
        tune.apply(ctx, tuned)
    elif args.no_tune:
        tuned = dict(tune.DEFAULT)
        tune.apply(ctx, tuned)
    else:
        def step_time():
            # the timed step's own measurement: L2 flushed, CUDA events around the call
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            cf.cf_count(ctx, p, d1, d2)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1) / 1e3
        tuned = tune.tune(ctx, p, d1, d2, device_name=torch.cuda.get_device_name(dev), npoints=npts,
                          use_cache=not args.no_tune_cache, timer=step_time)

    for _ in range(args.warmup):
        cf.cf_count(ctx, p, d1, d2)
    torch.cuda.synchronize(dev)

    # ---- timed steps, device-resident inputs ----
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    _barrier(world)
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    with Clocks(local) as clk:
        for k in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps (outside the events)
            evs[k][0].record(stream)
            out = cf.cf_count(ctx, p, d1, d2)
            evs[k][1].record(stream)
            stats.append(cf.cf_get_stats(ctx))
        torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    _barrier(world)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_dev = sum(step_ms) / 1e3
    evaluated = stats[-1]["evaluated_pairs"]
    t_max = _max_over_ranks(world, t_dev, dev)
    total_evals = _sum_over_ranks(world, float(evaluated) * args.steps, dev)
    value = total_evals / t_max
    in_range = int(np.asarray(out["npairs"], dtype=np.float64).sum())
    pair_ms = [s["ms_pair"] for s in stats]
    launches = sum(s["kernel_launches"] for s in stats)

    # ---- e2e through the public API with pinned host buffers (H2D of inputs, D2H of results inside) ----
    h1 = _points(wl.d1, wl.weighted, cf, pinned=True)
    h2 = None if wl.autocorr else _points(wl.d2, wl.weighted, cf, pinned=True)
    cf.cf_count(ctx, p, h1, h2)
    e2e_steps = max(3, min(args.steps, 50))
    torch.cuda.synchronize(dev)
    _barrier(world)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        res = cf.cf_count(ctx, p, h1, h2)
    torch.cuda.synchronize(dev)
    t_e2e = _max_over_ranks(world, time.perf_counter() - t0, dev)
    e2e_value = _sum_over_ranks(world, float(evaluated) * e2e_steps, dev) / t_e2e
    es = 8 if wl.d1.dtype == np.float64 else 4
    h2d = (wl.d1.n * (4 if wl.weighted else 3) +
           (0 if wl.autocorr else wl.d2.n * (4 if wl.weighted else 3))) * es
    d2h = sum(v.nbytes for v in res.values())

    # ---- roofline of the pair kernel (events on the launching stream, inside the library) ----
    peaks = _peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    ipp = FP32_INSTR_PER_PAIR_KIND.get(wl.kind, FP32_INSTR_PER_PAIR)
    peak = props.multi_processor_count * 128 * sm_max * 1e6 / ipp
    achieved = evaluated / (statistics.fmean(pair_ms) / 1e3)
    clocks = clk.summary()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": _line_config(args, world),
        "launch": {"grid": stats[-1]["grid"], "refine": stats[-1]["refine"], "tuned": tuned},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "steps": e2e_steps},
        "gpu_launches": int(launches),
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
                     "frac": achieved / peak, "traffic": _traffic(args.workload),
                     "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x {sm_max:.0f} MHz / "
                                   f"{ipp} instr per pair"},
        "clocks": clocks,
        "pair_kernel_ms": statistics.fmean(pair_ms),
        "evaluated_pairs_per_step": int(evaluated),
        "in_range_pairs_per_step": in_range,
        "in_range_pairs_per_s": in_range * args.steps / t_dev,
        "rechecked_pairs_per_step": int(stats[-1]["rechecked_pairs"]),
        "work_items": int(stats[-1]["work_items"]),
        "wall_s_timed_region": wall,
    }
    line["parity_vs_golden"] = _parity(args.workload, out, (wl.d1, None if wl.autocorr else wl.d2))
    if rank == 0 and world == 1 and not args.no_extras:
        line.update(_extras(args, cf, tune, ctx, dev, local, flush))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(wl, args.cpu_seconds)
        if not args.no_extras:
            line["cpu_baseline"]["other_configs"] = _oracle_beside(args.cpu_seconds / 6)
    if rank == 0:
        print(json.dumps(line), flush=True)
    cf.cf_destroy(ctx)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------------------
# batched and served forms (256 mock catalogues)
# ---------------------------------------------------------------------------------------------

BATCH_DESC = ("256 mock catalogues, periodic L=250, N log-uniform in [5e4, 8e5] (sum 7.4e7), 50-member clusters "
              "sigma=1, DD(rp,pi) auto, 14 log rp bins 0.1-20, pimax=40 with 40 pi bins, float32")


def _batch_setup(ncat, lo=5e4, hi=8e5):
    import gen
    # the first 256 sizes of a range are the same for any ncat (one seeded sequence)
    sizes = gen.batch_sizes(max(256, ncat), lo, hi)[:ncat]
    cats = [gen.batch_catalogue(i, n) for i, n in enumerate(sizes)]
    return sizes, cats


def _batch_desc(args, sizes):
    if args.ncat == 256 and (args.batch_min, args.batch_max) == (5e4, 8e5):
        return BATCH_DESC
    return BATCH_DESC.replace("256", str(args.ncat)).replace(
        "[5e4, 8e5] (sum 7.4e7)", f"[{args.batch_min:g}, {args.batch_max:g}] (sum {sum(sizes):.2g})")


def _batch_params(cf):
    import gen
    return cf.params(kind="rppi", edges=gen.log_edges(0.1, 20.0, 14), autocorr=True, periodic=True, box=250.0,
                     pimax=40.0, npibins=40)


def _batch_measure(args, cf, tune, dev, local, sizes, cats, steps) -> dict:
    """Config 4 counted one catalogue at a time (one cf_count each), batched (one cell build and one
    persistent pair kernel over all catalogues), and graph-replayed; device-resident inputs."""
    import numpy as np
    import torch

    stream = torch.cuda.current_stream(dev)
    p = _batch_params(cf)
    pts = [_points(c, False, cf, dev) for c in cats]
    ctx = cf.cf_create(local, stream)
    med = int(np.argsort(sizes)[len(sizes) // 2])
    tuned = tune.tune(ctx, p, pts[med], None, device_name=torch.cuda.get_device_name(dev), npoints=sizes[med],
                      use_cache=not args.no_tune_cache)
    # one at a time (the plain path: one cf_count per catalogue)
    singles = [cf.cf_count(ctx, p, q) for q in pts[:4]]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    singles = [cf.cf_count(ctx, p, q) for q in pts]
    t_single = time.perf_counter() - t0
    # batched: one cell build + one persistent pair kernel over all catalogues
    outs = cf.cf_batch_count(ctx, p, pts)
    times, pair_ms = [], []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        outs = cf.cf_batch_count(ctx, p, pts)
        times.append(time.perf_counter() - t0)
        pair_ms.append(cf.cf_get_stats(ctx)["ms_pair"])
    st = cf.cf_get_stats(ctx)
    # graph-captured replay of the same batch
    cf.cf_batch_capture(ctx, p, pts)
    gtimes = []
    for _ in range(max(1, steps)):
        t0 = time.perf_counter()
        gouts = cf.cf_batch_replay(ctx, p, len(pts))
        gtimes.append(time.perf_counter() - t0)
    same = all(np.array_equal(a["npairs"], b["npairs"]) and np.array_equal(a["npairs"], g["npairs"])
               for a, b, g in zip(singles, outs, gouts))
    # the catalogues whose oracle histograms are stored
    checked = {}
    for i, c in enumerate(cats):
        par = _parity(f"batch_{i}", outs[i], (c,))
        if par["ok"] is not None:
            checked[f"batch_{i}"] = par["ok"]
    cf.cf_destroy(ctx)
    t_batch, t_graph = min(times), min(gtimes)
    best = min(t_batch, t_graph)
    peak = _peak_pairs(dev, "rppi")
    achieved = st["evaluated_pairs"] / (min(pair_ms) / 1e3)
    return {"ncat": len(pts), "points": int(sum(sizes)), "tuned": tuned, "t_single": t_single, "t_batch": t_batch,
            "t_graph": t_graph, "best": best, "same": same, "golden": checked, "st": st, "pair_ms": min(pair_ms),
            "achieved": achieved, "peak": peak}


def run_batch(args, world, rank, local):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03545_gb300 as cf
    from paper_1911_03545_gb300 import tune

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    sizes, cats = _batch_setup(args.ncat, args.batch_min, args.batch_max)
    b = _batch_measure(args, cf, tune, dev, local, sizes, cats, args.steps)
    n, st = b["ncat"], b["st"]
    line = {
        "metric": "batched catalogues/s", "value": n / b["best"], "unit": "catalogues/s", "n_gpus": 1,
        "steps": args.steps, "warmup": 1, "ms_per_step": 1e3 * b["best"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": _batch_desc(args, sizes), "name": "batch", "ncat": n, "points": b["points"],
                   "tuned": b["tuned"]},
        "one_at_a_time": {"value": n / b["t_single"], "unit": "catalogues/s", "seconds": b["t_single"]},
        "batched": {"value": n / b["t_batch"], "seconds": b["t_batch"]},
        "graph_replay": {"value": n / b["t_graph"], "seconds": b["t_graph"]},
        "speedup_vs_one_at_a_time": b["t_single"] / b["best"],
        "parity_batched_vs_single": b["same"], "parity_vs_golden": b["golden"],
        "evaluated_pairs": int(st["evaluated_pairs"]), "work_items": int(st["work_items"]),
        "roofline": {"bound": "alu", "achieved": b["achieved"] / 1e9, "peak": b["peak"] / 1e9, "unit": "Gpair/s",
                     "frac": b["achieved"] / b["peak"], "traffic": None},
        "pair_kernel_ms": b["pair_ms"], "gpu_launches": int(st["kernel_launches"]),
    }
    print(json.dumps(line), flush=True)
    return 0


def _serve_measure(args, cf, dev, local, cats, nreq) -> dict:
    """Poisson arrivals at args.serve_load of the capacity measured in the same session (everything
    submitted at once); p50 / p99 latency from submit to the poll that returns the result."""
    import threading

    import numpy as np
    import torch

    p = _batch_params(cf)
    hosts = [cf.points(c.x, c.y, c.z) for c in cats]
    srv = cf.cf_server_start(local, p, args.serve_budget << 30, args.serve_slots)

    def drain(tickets, done):
        pending = dict(tickets)
        while pending:
            for tk in list(pending):
                r = cf.cf_server_poll(srv, tk, 0)
                if r is not None:
                    done[pending.pop(tk)] = (time.perf_counter(), r)
            time.sleep(0.0002)

    # capacity: everything submitted at once (the server batches continuously)
    for _ in range(2):
        t0 = time.perf_counter()
        tks = {cf.cf_server_submit(srv, p, h): i for i, h in enumerate(hosts)}
        done = {}
        drain(tks, done)
        cap_s = time.perf_counter() - t0
    capacity = len(hosts) / cap_s
    rate = args.serve_load * capacity
    rng = np.random.Generator(np.random.PCG64(7))
    arrivals = np.cumsum(rng.exponential(1.0 / rate, size=nreq))
    order = rng.integers(0, len(hosts), size=nreq)
    submit_t, tickets, finished = {}, {}, {}
    lock = threading.Lock()
    stop = threading.Event()

    def poller():
        while not stop.is_set() or tickets:
            with lock:
                items = list(tickets.items())
            for tk, k in items:
                r = cf.cf_server_poll(srv, tk, 0)
                if r is not None:
                    finished[k] = (time.perf_counter(), r)
                    with lock:
                        tickets.pop(tk, None)
            time.sleep(0.0002)

    th = threading.Thread(target=poller)
    th.start()
    t_start = time.perf_counter()
    for k in range(nreq):
        now = time.perf_counter() - t_start
        if arrivals[k] > now:
            time.sleep(arrivals[k] - now)
        ts = time.perf_counter()
        tk = cf.cf_server_submit(srv, p, hosts[int(order[k])])
        with lock:
            tickets[tk] = k
            submit_t[k] = ts
    stop.set()
    th.join()
    t_total = time.perf_counter() - t_start
    cf.cf_server_stop(srv)
    lat = np.array([finished[k][0] - submit_t[k] for k in range(nreq)]) * 1e3
    # every served result equals the batched result of the same catalogue
    ctx = cf.cf_create(local, torch.cuda.current_stream(dev))
    ref = cf.cf_batch_count(ctx, p, [_points(c, False, cf, dev) for c in cats])
    cf.cf_destroy(ctx)
    ok = all(np.array_equal(finished[k][1]["npairs"], ref[int(order[k])]["npairs"]) for k in range(nreq))
    return {"nreq": nreq, "t_total": t_total, "capacity": capacity, "lat": lat, "ok": ok}


def run_serve(args, world, rank, local):
    """Poisson arrivals at a fraction of the measured capacity; p50 / p99 latency."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_1911_03545_gb300 as cf

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    sizes, cats = _batch_setup(args.ncat)
    r = _serve_measure(args, cf, dev, local, cats, args.serve_requests)
    lat = r["lat"]
    line = {
        "metric": "served catalogues/s", "value": r["nreq"] / r["t_total"], "unit": "catalogues/s", "n_gpus": 1,
        "steps": r["nreq"], "warmup": 2, "ms_per_step": float(np.mean(lat)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_DESC, "name": "serve", "arrivals": "Poisson", "load": args.serve_load,
                   "capacity_catalogues_per_s": r["capacity"], "budget_gib": args.serve_budget,
                   "slots": args.serve_slots, "inputs": "host numpy arrays (copied by the server)"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p90": float(np.percentile(lat, 90)),
                       "p99": float(np.percentile(lat, 99)), "mean": float(np.mean(lat)), "max": float(np.max(lat))},
        "results_equal_batched": r["ok"],
    }
    print(json.dumps(line), flush=True)
    return 0


def run_sweep(args, world, rank, local):
    """Scaling with particle number and with Rmax, each for refinement factors k = 1, 2, 3 (Sec. 4.2
    and the scaling study of Sec. 5): DD(r) auto on the clustered L=420 catalogue (random subsamples for
    the N series, the full 1e6 points for the Rmax series), 20 log bins from 0.1 to Rmax."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import gen
    import paper_1911_03545_gb300 as cf

    dev = torch.device(f"cuda:{local}")
    torch.cuda.set_device(dev)
    ctx = cf.cf_create(local, torch.cuda.current_stream(dev))
    wl = gen.workload("clustered_r_1m")
    full, L = wl.d1, wl.box
    perm = np.random.Generator(np.random.PCG64(77)).permutation(full.n)

    def sub(n):
        idx = np.sort(perm[:n])
        return gen.Catalogue(full.x[idx], full.y[idx], full.z[idx])

    rows, same = [], True

    def measure(cat, rmax, series):
        nonlocal same
        edges = gen.log_edges(0.1, rmax, 20)
        pts = _points(cat, False, cf, dev)
        ref = None
        for k in (1, 2, 3):
            p = cf.params(kind="r", edges=edges, autocorr=True, periodic=True, box=L, refine=(k, k, k))
            res = cf.cf_count(ctx, p, pts)
            pair, tot = [], []
            for _ in range(args.sweep_reps):
                res = cf.cf_count(ctx, p, pts)
                st = cf.cf_get_stats(ctx)
                pair.append(st["ms_pair"])
                tot.append(st["ms_build"] + st["ms_pair"] + st["ms_recheck"])
            counts = np.asarray(res["npairs"])
            if ref is None:
                ref = counts
            same = same and np.array_equal(ref, counts)
            rows.append({"series": series, "n": int(cat.n), "rmax": rmax, "refine": k,
                         "pair_ms": float(np.median(pair)), "device_ms": float(np.median(tot)),
                         "evaluated_pairs": int(st["evaluated_pairs"]), "in_range_pairs": int(counts.sum()),
                         "cells": int(st["cells"])})

    for n in (10_000, 30_000, 100_000, 300_000, 1_000_000):
        measure(sub(n) if n < full.n else full, 20.0, "N")
    for rmax in (5.0, 10.0, 40.0, 80.0):
        measure(full, rmax, "Rmax")
    if rank == 0:
        print(json.dumps({"metric": "scaling sweep", "workload": "clustered_r_1m recipe, DD(r) auto, periodic L=420, "
                          "20 log bins 0.1-Rmax, float32, unweighted", "rows": rows,
                          "counts_identical_across_refine": bool(same),
                          "refine_model": "evaluated pairs relative to k=1: ((k+1)/(2k))^3 for cubic sub-cells"}),
              flush=True)
    cf.cf_destroy(ctx)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="clustered_r_1m", choices=sorted(WORKLOADS) + ["batch256", "serve", "sweep"])
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-seconds", type=float, default=150.0,
                    help="oracle time of the whole --impl reference run (split over its steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-tune-cache", action="store_true")
    ap.add_argument("--config", default="", help="pin the launch configuration instead of tuning, "
                    "e.g. variant=2,warps=8 (knobs of paper_1911_03545_gb300.tune)")
    ap.add_argument("--ncat", type=int, default=256)
    ap.add_argument("--batch-min", type=float, default=5e4, help="smallest catalogue of the batch workload")
    ap.add_argument("--batch-max", type=float, default=8e5, help="largest catalogue of the batch workload")
    ap.add_argument("--sweep-reps", type=int, default=3)
    ap.add_argument("--serve-load", type=float, default=0.8)
    ap.add_argument("--serve-requests", type=int, default=1024)
    ap.add_argument("--serve-budget", type=int, default=16, help="GiB")
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--no-extras", action="store_true",
                    help="measure the headline workload only (not the other configurations, batch and serving)")
    ap.add_argument("--extra-steps", type=int, default=5, help="timed steps of each other workload")
    ap.add_argument("--extra-requests", type=int, default=1024, help="Poisson requests of the serving run")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = _dist()
    if args.workload == "batch256":
        return run_batch(args, world, rank, local)
    if args.workload == "serve":
        return run_serve(args, world, rank, local)
    if args.workload == "sweep":
        return run_sweep(args, world, rank, local)
    import gen
    wl = gen.workload(args.workload)
    if args.impl == "reference":
        return run_reference(args, wl, world, rank)
    return run_gpu(args, wl, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
