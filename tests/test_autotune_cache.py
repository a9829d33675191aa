"""The binding's autotune cache (MDK_AUTOTUNE_CACHE): entries are keyed by
device model, precision and workload key, survive a rewrite, and malformed
entries or files are ignored (host logic, no GPU)."""
import json

from paper_2511_22951_gb300 import mdk


def test_cache_round_trip(tmp_path):
    p = str(tmp_path / "tune.json")
    k1 = mdk.autotune_cache_key("lj_argon_8388608", "mixed", "NVIDIA GB300")
    k2 = mdk.autotune_cache_key("lj_argon_8388608", "fp64", "NVIDIA GB300")
    assert k1 != k2
    assert mdk.autotune_cache_get(p, k1) is None          # no file yet
    mdk.autotune_cache_put(p, k1, {"tpa": 1, "block": 128, "list": "full", "ms": 1.1})
    mdk.autotune_cache_put(p, k2, {"tpa": 1, "block": 256, "list": "half", "ms": 25.0})
    assert mdk.autotune_cache_get(p, k1)["block"] == 128
    assert mdk.autotune_cache_get(p, k2)["list"] == "half"
    assert sorted(json.load(open(p))) == sorted([k1, k2])


def test_cache_ignores_bad_entries(tmp_path):
    p = str(tmp_path / "tune.json")
    k = mdk.autotune_cache_key("w", 1, "dev")
    open(p, "w").write("{not json")
    assert mdk.autotune_cache_get(p, k) is None
    mdk.autotune_cache_put(p, k, {"tpa": 3, "block": 128, "list": "full"})   # bad tpa
    assert mdk.autotune_cache_get(p, k) is None
    mdk.autotune_cache_put(p, k, {"tpa": 2, "block": 128, "list": "sideways"})
    assert mdk.autotune_cache_get(p, k) is None
    mdk.autotune_cache_put(p, k, {"tpa": 2, "block": 512, "list": "cells"})
    assert mdk.autotune_cache_get(p, k)["tpa"] == 2
