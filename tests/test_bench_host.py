"""Host-side checks of bench.py's workload plumbing (no GPU): the batch workload's catalogue sizes
with default options are exactly the 256 catalogues the golden files and the batch tests use, a
larger batch extends the same seeded sequence, and the JSON line's description names the sizes it
ran."""
import argparse

import gen


def _args(**kw):
    a = dict(ncat=256, batch_min=5e4, batch_max=8e5)
    a.update(kw)
    return argparse.Namespace(**a)


def test_default_batch_sizes_are_the_measured_workload():
    assert gen.batch_sizes(1024, 5e4, 8e5)[:256] == gen.batch_sizes()
    s = gen.batch_sizes()
    assert len(s) == 256 and min(s) >= 5e4 and max(s) <= 8e5
    assert abs(sum(s) - 7.42e7) < 0.01 * 7.42e7    # the seeded draw (its expectation is 6.9e7)


def test_batch_description_follows_the_options():
    import bench
    sizes = gen.batch_sizes()
    assert bench._batch_desc(_args(), sizes) == bench.BATCH_DESC
    small = gen.batch_sizes(1024, 1e3, 2e4)
    assert min(small) >= 1e3 and max(small) <= 2e4
    d = bench._batch_desc(_args(ncat=1024, batch_min=1e3, batch_max=2e4), small)
    assert d.startswith("1024 mock catalogues") and "[1000, 20000]" in d and "5e4" not in d


def test_parity_flag_against_the_stored_histograms():
    """bench.py's parity flag: the stored oracle histogram itself passes, a count off by one or a
    sum off by 2e-6 fails, and inputs that differ from the stored ones get no flag (None)."""
    import json
    import os

    import numpy as np

    import bench
    from tests.golden.make_golden import fingerprint
    wl = gen.workload("uniform_r_20k")
    assert bench._fingerprint(wl.d1) == fingerprint(wl.d1)
    with open(os.path.join(bench.GOLDEN, "full_uniform_r_20k.json")) as f:
        gold = json.load(f)
    got = {"npairs": np.asarray(gold["npairs"], dtype=np.uint64), "wsum": np.asarray(gold["wsum"])}
    assert bench._parity("uniform_r_20k", got, (wl.d1,))["ok"] is True
    bad = dict(got, npairs=got["npairs"].copy())
    bad["npairs"][5] += 1
    assert bench._parity("uniform_r_20k", bad, (wl.d1,))["ok"] is False
    off = dict(got, wsum=got["wsum"] * (1 + 2e-6))
    assert bench._parity("uniform_r_20k", off, (wl.d1,))["ok"] is False
    other = gen.uniform_box(100, 250.0, 1, dtype=np.float64)
    assert bench._parity("uniform_r_20k", got, (other,))["ok"] is None
    assert bench._parity("no_such_workload", got, (wl.d1,))["ok"] is None


def test_zwin_estimate_brackets_a_whole_run():
    """The CPU baseline's z-window estimate (slope between two row samples plus the call's fixed
    cost) on a scaled-down clustered workload: a range with lo <= hi, within a factor 4 of the time
    of the whole run it stands for."""
    import time

    import bench
    import oracle
    wl = gen.workload("clustered_r_1m", scale=0.05)
    est = bench._zwin_estimate(wl, 0.5)
    lo, hi = est["zwin_seconds_full_range"]
    assert 0.0 < lo <= hi and lo <= est["zwin_seconds_full_est"] <= hi
    t0 = time.perf_counter()
    oracle.count(wl.kind, wl.edges, wl.d1, None, autocorr=True, periodic=True, box=wl.box, weighted=True, ravg=True,
                 mode="zwin")
    t = time.perf_counter() - t0
    assert hi >= t / 4 and lo <= 4 * t, (lo, hi, t)
