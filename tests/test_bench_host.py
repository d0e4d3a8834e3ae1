"""Host logic of the benchmark: when the committed ncu counters may be
reported as the pair kernel's DRAM traffic (CPU only)."""
import types

import pytest


def _args(**kw):
    a = dict(workload="lognormal-n1e6-s5e5", skin_abs=100.0, skin_s=0.02, densify=6000, warmup=3, steps=20,
             iters_per_step=100)
    a.update(kw)
    return types.SimpleNamespace(**a)


def test_traffic_is_reported_for_the_captured_library_and_state():
    import bench
    t, pairs = bench.pair_traffic(_args(), 0)
    assert t is not None and t > 0 and pairs > 0


@pytest.mark.parametrize("kw", [dict(skin_abs=20.0), dict(skin_s=0.1), dict(steps=21),
                                dict(workload="powerlaw-n1e5-s20")])
def test_traffic_is_withheld_for_another_state(kw):
    import bench
    assert bench.pair_traffic(_args(**kw), 0) == (None, None)


def test_traffic_is_withheld_for_another_library(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "library_sha", lambda: "0" * 64)
    assert bench.pair_traffic(_args(), 0) == (None, None)
