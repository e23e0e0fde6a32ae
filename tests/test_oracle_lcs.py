"""Pins of the LCS oracle (``oracle.lcs_length``, ``lcs_length_rolling``,
``lcs_pairs``): the paper's first named extension of its diagonal band
(section "Generalized Dynamic Programming Extensions", "Direct Extension:
LCS").  Pinned by hand-worked cases (one is the standard textbook example),
brute-force enumeration of subsequences, and closed forms."""
import itertools
import json
import os

import numpy as np
import pytest

import oracle
from tests import mutants

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def codes(s):
    return [ord(c) for c in s]


def is_subsequence(sub, seq):
    it = iter(seq)
    return all(any(c == d for d in it) for c in sub)


def brute_lcs(x, y):
    """Longest subsequence of x that is also one of y, by enumeration."""
    for k in range(min(len(x), len(y)), 0, -1):
        for idx in itertools.combinations(range(len(x)), k):
            if is_subsequence([x[i] for i in idx], y):
                return k
    return 0


def test_hand_worked_cases():
    for c in json.load(open(os.path.join(GOLDEN, "lcs_hand_worked.json")))["cases"]:
        x, y = codes(c["x"]), codes(c["y"])
        assert oracle.lcs_length(x, y) == c["length"], c["name"]
        assert oracle.lcs_length_rolling(x, y) == c["length"], c["name"]
        xi, yj = oracle.lcs_pairs(x, y)
        assert xi.tolist() == c["xi"] and yj.tolist() == c["yj"], c["name"]
        assert "".join(c["x"][i] for i in xi) == c["subsequence"]


@pytest.mark.parametrize("seed", range(60))
def test_against_brute_force(seed):
    rng = np.random.default_rng(seed)
    alphabet = int(rng.integers(2, 5))
    x = rng.integers(0, alphabet, int(rng.integers(0, 11))).tolist()
    y = rng.integers(0, alphabet, int(rng.integers(0, 11))).tolist()
    want = brute_lcs(x, y)
    assert oracle.lcs_length(x, y) == want
    assert oracle.lcs_length_rolling(x, y) == want
    xi, yj = oracle.lcs_pairs(x, y)
    assert len(xi) == len(yj) == want
    assert np.all(np.diff(xi) > 0) and np.all(np.diff(yj) > 0)
    assert all(x[i] == y[j] for i, j in zip(xi, yj))


def test_closed_forms():
    rng = np.random.default_rng(9)
    x = rng.integers(0, 6, 300).tolist()
    assert oracle.lcs_length(x, x) == 300                     # identity
    assert oracle.lcs_length(x, []) == 0 and oracle.lcs_length([], x) == 0
    assert oracle.lcs_length([7] * 40, [7] * 25) == 25          # min(n, m)
    assert oracle.lcs_length(x, [v + 10 for v in x]) == 0       # disjoint alphabets
    sub = x[::3]
    assert oracle.lcs_length(sub, x) == len(sub)               # a subsequence of x
    y = rng.integers(0, 6, 250).tolist()
    assert oracle.lcs_length(x, y) == oracle.lcs_length(y, x)  # symmetry
    # indel distance: n + m - 2 LCS is at least |n - m| and at most n + m
    d = len(x) + len(y) - 2 * oracle.lcs_length(x, y)
    assert abs(len(x) - len(y)) <= d <= len(x) + len(y)


@pytest.mark.parametrize("n,m,alphabet", [(2000, 1500, 4), (1000, 3000, 20), (777, 777, 2)])
def test_rolling_equals_full(n, m, alphabet):
    rng = np.random.default_rng(n + m + alphabet)
    x = rng.integers(0, alphabet, n)
    y = rng.integers(0, alphabet, m)
    full = oracle.lcs_length(x, y)
    assert oracle.lcs_length_rolling(x, y) == full
    xi, yj = oracle.lcs_pairs(x, y)
    assert len(xi) == full and np.array_equal(x[xi], y[yj])


# ------------------------------------------------------------ pin strength
LCS_MUTANTS = {
    20: "walk goes left on ties",
    21: "equal symbols extend the cell above instead of the diagonal",
    22: "rolling rows read the up-left cell for the up cell",
}


def _lcs_pins(lib):
    """Name of the first LCS pin that the variant `lib` fails, or None."""
    for c in json.load(open(os.path.join(GOLDEN, "lcs_hand_worked.json")))["cases"]:
        x, y = codes(c["x"]), codes(c["y"])
        if oracle.lcs_length(x, y, lib) != c["length"] or \
                oracle.lcs_length_rolling(x, y, lib) != c["length"]:
            return "hand-length:" + c["name"]
        xi, yj = oracle.lcs_pairs(x, y, lib)
        if xi.tolist() != c["xi"] or yj.tolist() != c["yj"]:
            return "hand-walk:" + c["name"]
    rng = np.random.default_rng(123)
    for _ in range(40):
        x = rng.integers(0, 3, int(rng.integers(0, 9))).tolist()
        y = rng.integers(0, 3, int(rng.integers(0, 9))).tolist()
        want = brute_lcs(x, y)
        if oracle.lcs_length(x, y, lib) != want or oracle.lcs_length_rolling(x, y, lib) != want:
            return "bruteforce"
    return None


def test_real_lcs_oracle_passes_every_pin(tmp_path):
    assert _lcs_pins(mutants.build(str(tmp_path), 0)) is None


@pytest.mark.parametrize("k", sorted(LCS_MUTANTS), ids=lambda k: LCS_MUTANTS[k])
def test_planted_lcs_mistake_is_caught(k, tmp_path):
    lib = mutants.build(str(tmp_path), k)
    assert _lcs_pins(lib) is not None, f"no pin rejects: {LCS_MUTANTS[k]}"
