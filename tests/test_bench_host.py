"""Host logic of the benchmark (CPU only): when the committed ncu counters may
be reported as the pair kernel's DRAM traffic, and that the oracle leg runs
without loading anything of the CUDA library."""
import os
import subprocess
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _args(**kw):
    a = dict(workload="lognormal-n1e6-s5e5", skin_abs=100.0, skin_s=0.02, densify=6000, warmup=3, steps=20,
             iters_per_step=100)
    a.update(kw)
    return types.SimpleNamespace(**a)


def _captured_pairs():
    import bench
    import re
    with open(os.path.join(ROOT, "profiles", "k_pair_mixed-lognormal-n1e6-s5e5.md")) as f:
        return int(re.search(r"traffic_pairs: (\d+)", f.read()).group(1))


def _captured_sha():
    import re
    with open(os.path.join(ROOT, "profiles", "k_pair_mixed-lognormal-n1e6-s5e5.md")) as f:
        return re.search(r"sha256 prefix `([0-9a-f]+)`", f.read()).group(1)


def test_traffic_is_reported_for_the_captured_library_and_state(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "library_sha", lambda: _captured_sha() + "0" * 48)
    P = _captured_pairs()
    for Pn in (P, int(P * 1.02), int(P * 0.98)):
        t, pairs = bench.pair_traffic(_args(), Pn)
        assert t is not None and t > 0 and pairs == P


@pytest.mark.parametrize("kw,scale", [(dict(skin_abs=20.0), 1.0), (dict(skin_s=0.1), 1.0), ({}, 1.05), ({}, 0.9),
                                      (dict(workload="powerlaw-n1e5-s20"), 1.0)])
def test_traffic_is_withheld_for_another_state(kw, scale, monkeypatch):
    import bench
    monkeypatch.setattr(bench, "library_sha", lambda: _captured_sha() + "0" * 48)
    assert bench.pair_traffic(_args(**kw), int(_captured_pairs() * scale)) == (None, None)


def test_traffic_is_withheld_for_another_library(monkeypatch):
    import bench
    monkeypatch.setattr(bench, "library_sha", lambda: "0" * 64)
    assert bench.pair_traffic(_args(), _captured_pairs()) == (None, None)


def test_oracle_leg_loads_nothing_of_the_cuda_library():
    """The CPU baseline and the reference arm take their constants from the
    oracle: after a sample, neither the binding module nor librcp.so is
    loaded in the process."""
    code = (
        "import sys, numpy as np, bench\n"
        "from paper_2608_12235_b300 import inputs\n"
        "D0 = inputs.lognormal(3000, 0.5, 10.0)\n"
        "r = bench.cpu_baseline(D0, 3, 0.6, threads=2)\n"
        "assert r[0] > 0 and r[2] >= 1\n"
        "maps = open('/proc/self/maps').read()\n"
        "assert 'librcp.so' not in maps, 'librcp.so loaded'\n"
        "assert 'paper_2608_12235_b300.rcp' not in sys.modules\n"
        "print('ok')\n")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "ok" in r.stdout, r.stderr


def test_bounded_box_options_map_to_the_configuration():
    """--walls / --container become rcp_config keys; a container starts from
    the non-overlapping placement (a uniform draw leaves spheres outside)."""
    import bench
    assert bench.bounds_of(types.SimpleNamespace(walls=0, container=0)) == {}
    assert bench.bounds_of(types.SimpleNamespace(walls=7, container=0)) == {"walls": 7}
    assert bench.bounds_of(types.SimpleNamespace(walls=0, container=1)) == {"container": 1, "placement": 1}
    assert bench.bounds_of(types.SimpleNamespace(walls=4, container=2)) == {"walls": 4, "container": 2,
                                                                             "placement": 1}
