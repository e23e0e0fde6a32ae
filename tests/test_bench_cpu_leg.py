"""The one-pair bench line's CPU leg (``bench.pair_cpu_leg``), which needs no
GPU: the oracle timing sample and the error of a result against the oracle
value (computed, or stored for the 1e5-point w2 pair)."""
import json
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2007_16135_gb300 import workloads as W  # noqa: E402


def test_small_pair_is_timed_whole_and_checked_against_the_oracle():
    a, ta, b, tb = W.pair_w1(300, 200)
    want = oracle.twed(a, ta, b, tb, 1.0, 1.0, 2)
    cpu, err = bench.pair_cpu_leg(a, ta, b, tb, 1.0, 1.0, 2, "f64", want, 5.0)
    assert cpu["kind"] == "oracle" and cpu["cores"] == 1 and cpu["value"] > 0
    assert cpu["sample"].startswith("the whole pair (300 x 200")
    assert err["rel"] == 0.0 and err["bound"] == 1e-12
    _, err = bench.pair_cpu_leg(a, ta, b, tb, 1.0, 1.0, 2, "f64", want * (1 + 1e-9), 5.0)
    assert err["rel"] == pytest.approx(1e-9, rel=1e-6)


def test_w2_pair_uses_the_stored_oracle_value():
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "w2_oracle.json")))
    a, ta, b, tb = W.pair_w2(g["n"])
    cpu, err = bench.pair_cpu_leg(a, ta, b, tb, g["nu"], g["lambda"], g["p"], "f32",
                                  g["f32_rounded_inputs"], 0.02)
    assert "rows against all" in cpu["sample"]
    assert err["rel"] == 0.0 and err["bound"] == 1e-5
    assert "stored" in err["how"]


def test_large_pair_without_a_stored_value_says_so():
    a, ta, b, tb = W.pair_w2(3000)
    cpu, err = bench.pair_cpu_leg(a, ta, b, tb, 0.001, 1.0, 2, "f64", 1.0, 0.001)
    assert "rows against all 3000 columns" in cpu["sample"]
    assert "note" in err and "rel" not in err
