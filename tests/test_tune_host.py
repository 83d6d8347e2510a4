"""The autotuner's decisions on the CPU: a fake timer stands in for the GPU (each configuration gets
a known time plus noise), and the option setter is replaced, so only the search logic runs."""
import numpy as np
import pytest

pytest.importorskip("ctypes")


def _fake(monkeypatch, times, noise=0.0, seed=0):
    from paper_1911_03545_gb300 import tune
    state = {}
    monkeypatch.setattr(tune, "apply", lambda ctx, cfg: state.update(cfg=dict(cfg)))
    rng = np.random.Generator(np.random.PCG64(seed))

    def timer():
        return times(state["cfg"]) * (1.0 + noise * rng.standard_normal())
    return tune, timer


class _P:
    kind = 0


def test_tuner_finds_the_fastest_configuration(monkeypatch):
    # a separable landscape: the best values are jchunk 128, tile 64, warps 8, refine 2
    def times(c):
        t = 1.0
        t *= {512: 1.10, 256: 1.05, 128: 1.0}[c["jchunk"]]
        t *= {128: 1.04, 64: 1.0}[c["tile"]]
        t *= {0: 1.06, 12: 1.03, 8: 1.0, 6: 1.02, 4: 1.08}[c["warps"]]
        t *= {1: 1.2, 2: 1.0, 3: 1.1}[c["refine"]]
        t *= {1: 1.0, 2: 1.3}[c["variant"]]
        t *= {0: 1.0, 1: 1.02}[c["noprune"]]
        return t
    tune, timer = _fake(monkeypatch, times, noise=0.002)
    cfg = tune.tune(None, _P(), None, use_cache=False, timer=timer)
    assert (cfg["jchunk"], cfg["tile"], cfg["warps"], cfg["refine"], cfg["variant"], cfg["noprune"],
            cfg["block"]) == (128, 64, 8, 2, 1, 0, 0)


def test_tuner_keeps_the_default_within_the_margin(monkeypatch):
    # every alternative is within 0.5 % of the default: noise must not move the configuration
    def times(c):
        return 1.0 - 0.005 * (c["jchunk"] == 256)
    tune, timer = _fake(monkeypatch, times, noise=0.003, seed=3)
    cfg = tune.tune(None, _P(), None, use_cache=False, timer=timer)
    assert cfg == tune.DEFAULT


def test_tuner_knobs_follow_the_kind():
    from paper_1911_03545_gb300 import CF_DD_RPPI_MOCKS, CF_DD_THETA, tune

    class K:
        def __init__(self, kind):
            self.kind = kind
    assert "thetagrid" in tune.knobs_for(K(CF_DD_THETA)) and "variant" in tune.knobs_for(K(CF_DD_THETA))
    assert "thetagrid" not in tune.knobs_for(K(0))
    assert "variant" not in tune.knobs_for(K(CF_DD_RPPI_MOCKS))
    assert all("block" not in tune.knobs_for(K(k)) for k in range(5))      # searched only on request
    assert tune.knobs_for(K(0), block=True)["block"] == [0, 1]


def test_tuner_searches_group_pruning_on_request(monkeypatch):
    # group pruning 10 % faster: found only when the caller asks for it
    def times(c):
        return 1.0 * (0.9 if c["block"] else 1.0)
    tune, timer = _fake(monkeypatch, times, noise=0.002, seed=5)
    assert tune.tune(None, _P(), None, use_cache=False, timer=timer)["block"] == 0
    assert tune.tune(None, _P(), None, use_cache=False, timer=timer, block=True)["block"] == 1
