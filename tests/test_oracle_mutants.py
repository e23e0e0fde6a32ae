"""Pin strength: the oracle's pins must reject plausible mistakes.

Each planted mistake is compiled into a private copy of the oracle (a
textual patch of ``oracle/twed_oracle.c`` from ``tests/mutants.py``) and run
through the same independent pins that ``test_oracle.py`` applies to the
real oracle.  A mistake that no pin rejects
would mean the pins do not pin that part of the definition.
"""
import json
import os

import numpy as np
import pytest

import oracle
from tests import mutants
from tests.bruteforce import lp, twed_bruteforce

MUTANTS = {
    1: "match term drops c(i-1,j-1)",
    2: "match time term indexes b by the row (the printed typo)",
    3: "lambda missing from the deletion costs",
    4: "left border D(i,0) = 0 instead of infinity",
    5: "deletion in a uses dA(i-1) instead of dA(i)",
    6: "p = 2 norm without the square root",
    7: "nu missing from the match time term",
    8: "c(i-1,j-1) subtracted instead of added",
    9: "second match cost taken at (i-1, j) instead of (i-1, j-1)",
}


def _pins(twed):
    """Return the name of the first pin that `twed` fails, or None."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        got = twed(np.array(c["a"]), c["ta"], np.array(c["b"]), c["tb"], c["nu"], c["lam"], c["p"])
        if got != pytest.approx(c["expected"], rel=1e-12, abs=1e-12):
            return "hand:" + c["name"]
    rng = np.random.default_rng(0)
    for _ in range(40):
        n, m = rng.integers(1, 6, size=2)
        dim, p = int(rng.integers(1, 4)), int(rng.choice([1, 2, 3]))
        a, b = rng.normal(size=(n, dim)), rng.normal(size=(m, dim))
        ta, tb = np.cumsum(rng.exponential(1, n)), np.cumsum(rng.exponential(1, m))
        nu, lam = float(rng.uniform(0.01, 2)), float(rng.uniform(0, 2))
        if twed(a, ta, b, tb, nu, lam, p) != pytest.approx(
                twed_bruteforce(a, ta, b, tb, nu, lam, p), rel=1e-12, abs=1e-12):
            return "bruteforce"
    for _ in range(10):
        m, dim = int(rng.integers(2, 20)), int(rng.integers(1, 4))
        a, b = rng.normal(size=(1, dim)), rng.normal(size=(m, dim))
        ta, tb = np.cumsum(rng.exponential(1, 1)), np.cumsum(rng.exponential(1, m))
        row = lp(a[0], b[0], 2) + 0.5 * abs(ta[0] - tb[0]) + sum(
            lp(b[j], b[j - 1], 2) + 0.5 * abs(tb[j] - tb[j - 1]) + 0.3 for j in range(1, m))
        if twed(a, ta, b, tb, 0.5, 0.3, 2) != pytest.approx(row, rel=1e-12) or \
                twed(b, tb, a, ta, 0.5, 0.3, 2) != pytest.approx(row, rel=1e-12):
            return "closed-form"
    return None


def test_real_oracle_passes_every_pin():
    assert _pins(oracle.twed) is None


@pytest.mark.parametrize("k", sorted(MUTANTS), ids=lambda k: MUTANTS[k])
def test_planted_mistake_is_caught(k, tmp_path):
    mutant = oracle.twed_of(mutants.build(str(tmp_path), k))
    assert _pins(mutant) is not None, f"no pin rejects: {MUTANTS[k]}"
