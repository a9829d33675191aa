"""The bench's roofline numerators follow the documented per-unit models
(host arithmetic only, no GPU): algorithmic bytes per atom-step of each list
kind, the BPNN FLOP count, and when a recorded DRAM-traffic figure applies."""
import os
import sys

import pytest

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402
from paper_2511_22951_gb300 import workloads as W  # noqa: E402


def test_algorithmic_bytes_per_atom():
    lj = W.config2(n=4)
    # own record 16 + list 4 n + count 4 + x, v read and written 96 + build-time offset 16
    # (mixed; x_ref 24 in FP64) + cell 4 + next 16
    assert bench.algorithmic_bytes_per_atom(lj, "mixed", 78.0, "full") == 464
    assert bench.algorithmic_bytes_per_atom(lj, "mixed", 39.0, "half") == 464 - 156 + 48
    assert bench.algorithmic_bytes_per_atom(lj, "mixed", 0.0, "cells") == 148
    assert bench.algorithmic_bytes_per_atom(lj, "fp64", 78.0, "full") == 464 + 8 + 32
    eam = W.config3(ncx=4, ncyz=2)
    assert bench.algorithmic_bytes_per_atom(eam, "mixed", 54.0, "full") == 188 + 8 * 54


def test_bpnn_flops_per_atom():
    m = W.maise_like_bpnn(0)
    f = bench.bpnn_flops_per_atom(m, 54)
    pairs = 54 * 53 / 2
    per_pair = (21 + 7 * 6 + 12 * 4 + 2 * 43) + (50 + 30 * 6 + 8 * 4 + 16 * 43)
    assert f == pytest.approx(pairs * per_pair, rel=0.01)
    assert 1.5e6 < f < 1.8e6


def test_traffic_applies_only_to_the_captured_shape():
    lj = W.config2(n=4)
    t = bench.TRAFFIC[("lj", "mixed", "full")]
    ok = bench.traffic_per_launch(lj, "mixed", 1000, "full", t["neighbors_per_atom"],
                                  t["threads_per_atom"])
    if t["sources_sha256"] == bench.sources_sha256("full"):
        assert ok == pytest.approx(1000 * t["bytes_per_atom"])
    else:
        assert ok is None
    assert bench.traffic_per_launch(lj, "mixed", 1000, "full", 138.25, 1) is None
    assert bench.traffic_per_launch(lj, "mixed", 1000, "full", 78.0, 2) is None
    assert bench.traffic_per_launch(lj, "mixed", 1000, "half") is None
