"""Autotuner selection and caching logic on CPU (timings injected)."""
import json

from paper_2311_13798_gb300.autotune import Autotuner, shape_key


def test_picks_fastest_and_caches(tmp_path):
    calls = []

    def timer(h, k, p):
        calls.append(dict(p))
        return 10.0 + (p["split_min"] == 128) * -5.0 + (p["t_max"] == 1) * 3.0 + (p["width_min"] == 4) * -1.0

    path = str(tmp_path / "tune.json")
    t = Autotuner(cache_path=path, timer=timer, device_name="GB300")
    info = {"m": 10_000_000, "tau": 246}
    best = t.tune(object(), 7, info)
    assert best == {"t_max": 0, "split_min": 128, "width_min": 4, "warps_per_block": 0}
    assert t.choice(object(), 7, info) == {"t_max": 0, "split_min": 128, "width_min": 4}
    n = len(calls)
    assert t.tune(object(), 7, info) == best and len(calls) == n  # cached, not re-measured
    d = json.load(open(path))
    assert shape_key(info, 7, "GB300") in d
    # a new tuner reads the cache from disk
    t2 = Autotuner(cache_path=path, timer=lambda *a: 1 / 0, device_name="GB300")
    assert t2.tune(object(), 7, info) == best


def test_small_k_does_not_sweep_split():
    seen = set()

    def timer(h, k, p):
        seen.add(p["split_min"])
        return 1.0

    Autotuner(timer=timer, device_name="x").tune(object(), 5, {"m": 100, "tau": 3})
    assert len(seen) == 1


def test_short_queries_keep_the_defaults():
    calls = []

    def timer(h, k, p):
        calls.append(p)
        return 0.2 - (p["t_max"] == 3) * 0.1   # launch-bound: not searched

    best = Autotuner(timer=timer, device_name="x").tune(object(), 8, {"m": 100, "tau": 9})
    assert best["t_max"] == 0 and len(calls) == 2


def test_keeps_defaults_within_the_margin():
    def timer(h, k, p):
        return 10.0 - (p["t_max"] == 3) * 0.1   # 1 %: below the 3 % margin

    best = Autotuner(timer=timer, device_name="x").tune(object(), 8, {"m": 100, "tau": 9})
    assert best["t_max"] == 0
