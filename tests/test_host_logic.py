"""Host logic around the kernels, on the CPU: the autotuner's cache and key,
the bench's bandwidth sets and its workload record."""
import importlib.util
import json
import os

import numpy as np
import pytest

from paper_1206_6857_gb300 import autotune
from workloads import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench", os.path.join(ROOT, "bench.py"))
    b = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(b)
    return b


def test_autotune_cache_roundtrip(tmp_path):
    p = str(tmp_path / "tuned.json")
    key = autotune.key_for(3, 1_000_000, [0.002, 1.7], 1.73)
    assert key == "D3_N1e6_h-3..0"
    assert autotune.cache(p, key) is None
    best = {"leaf_size": 64, "plimit": 0, "cost_weight": [512.0, 512.0, 1.0, 1.0], "seconds": 0.7}
    autotune.cache(p, key, best)
    assert autotune.cache(p, key) == best
    autotune.cache(p, "D5_N1e5_h-2..0", dict(best, leaf_size=128))
    data = json.load(open(p))
    assert set(data) == {key, "D5_N1e5_h-2..0"}


def test_autotune_candidates_are_valid_options():
    for leaf in autotune.DEFAULT_LEAVES:
        assert 2 <= leaf <= 128
    for cw in autotune.DEFAULT_COSTS:
        assert len(cw) == 4 and all(v > 0 for v in cw)


def test_bench_bandwidth_sets():
    b = _bench()
    wl = synth.config2(0.001)
    h = wl.h
    lscv = b.sum_bandwidths(wl, "lscv")
    assert lscv.size == 2 * h.size
    assert np.allclose(np.sort(lscv), np.sort(np.concatenate([h, h * np.sqrt(2.0)])))
    assert np.array_equal(b.sum_bandwidths(wl, "sum"), h)
    s = b.sum_bandwidths(wl, "search")
    assert s.size == 2 * b.SEARCH_ROUNDS * b.SEARCH_PER_ROUND


def test_bench_workload_record():
    b = _bench()
    wl = synth.config2(0.001)
    cfg = b.wl_config(wl, "lscv", 1e-2)
    assert cfg["gaussian_sums"] == 2 * cfg["nh"] and cfg["mode"] == "lscv" and cfg["eps"] == 1e-2
    assert cfg["parallelism"] == "replicas"


def test_autotuner_plimit_candidates():
    """PLIMIT is searched (2..8, even) where series orders are affordable."""
    from paper_1206_6857_gb300 import autotune
    assert autotune.default_plimits(5) == (0, 2, 4, 6, 8)
    assert autotune.default_plimits(16) == (0,)
