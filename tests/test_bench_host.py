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
