"""Pins of the edit-path oracle (``oracle.twed_path``): an optimal alignment
(paper: the introduction names the edit path as a by-product of the dynamic
program; it is the first of the widening rows).

Pinned against things other than the oracle itself: hand-derived paths of
the hand-worked cases, a case built so that only the tie-break order decides,
and brute-force enumeration of every monotone path on tiny inputs with an
independent restatement of the step costs (``tests/bruteforce.py``)."""
import json
import os

import numpy as np
import pytest

import oracle
from tests import mutants
from bruteforce import all_paths, step_costs, twed_bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def path_cost(moves, a, ta, b, tb, nu, lam, p):
    """Cost of a move string under the brute-force module's step costs."""
    n, m, c, del_a, del_b = step_costs(a, ta, b, tb, nu, lam, p)
    i, j = 1, 1
    cost = c(1, 1) + c(0, 0)
    for mv in moves:
        if mv == "M":
            i += 1
            j += 1
            cost += c(i, j) + c(i - 1, j - 1)
        elif mv == "A":
            i += 1
            cost += del_a(i)
        else:
            j += 1
            cost += del_b(j)
    assert (i, j) == (n, m), "the path must end at (n, m)"
    return cost


def valid(moves, n, m):
    return (set(moves) <= set("MAB") and moves.count("M") + moves.count("A") == n - 1
            and moves.count("M") + moves.count("B") == m - 1)


def test_hand_worked_paths():
    cases = {c["name"]: c for c in json.load(open(os.path.join(GOLDEN, "hand_worked.json")))["cases"]}
    paths = json.load(open(os.path.join(GOLDEN, "hand_worked_paths.json")))["cases"]
    assert {p["name"] for p in paths} == set(cases)
    for p in paths:
        c = cases[p["name"]]
        value, moves = oracle.twed_path(c["a"], c["ta"], c["b"], c["tb"], c["nu"], c["lam"], c["p"])
        assert moves == p["path"], p["name"]
        assert value == pytest.approx(c["expected"], rel=1e-15, abs=1e-15), p["name"]


def test_tie_break_takes_delete_in_a_before_delete_in_b():
    # a = (0, 0), b = (10, 10), nu = lambda = 0: the match path costs
    # 10 + 10 + 10 = 30, and both delete paths (A then B, B then A) cost 10.
    # Walking back from (2,2), delete in a is tried before delete in b, so
    # the cell before (2,2) is (1,2): the forward path is B, A.
    value, moves = oracle.twed_path([[0.0], [0.0]], [1.0, 2.0], [[10.0], [10.0]], [1.0, 2.0],
                                    0.0, 0.0, 2)
    assert value == 10.0
    assert moves == "BA"


# Every cost zero (zero values, nu = lambda = 0): every path costs 0 and all
# finite candidates tie, so the walk-back rule alone fixes the path.  By hand:
# 2 x 2: at (2,2) the match is tried first -> "M".  4 x 2: (4,2) match from
# (3,1); at (3,1) the match would come from the infinite border, so delete in
# a from (2,1), then again from (1,1) -> forward "AAM".  2 x 4: (2,4) match
# from (1,3); in row 1 only deletes in b are finite -> "BBM".
ALL_TIES = [((2, 2), "M"), ((4, 2), "AAM"), ((2, 4), "BBM")]


def _all_ties_path(twed_path, n, m):
    return twed_path(np.zeros((n, 1)), np.arange(1.0, n + 1), np.zeros((m, 1)),
                     np.arange(1.0, m + 1), 0.0, 0.0, 2)


@pytest.mark.parametrize("shape,path", ALL_TIES)
def test_all_ties_follow_the_walk_back_order(shape, path):
    value, moves = _all_ties_path(oracle.twed_path, *shape)
    assert value == 0.0 and moves == path


def test_identical_series_align_point_to_point():
    rng = np.random.default_rng(5)
    a = np.cumsum(rng.normal(size=(17, 3)), axis=0)
    t = np.cumsum(rng.exponential(1.0, 17))
    value, moves = oracle.twed_path(a, t, a, t, 0.3, 0.7, 2)
    assert value == 0.0
    assert moves == "M" * 16


@pytest.mark.parametrize("seed", range(40))
def test_path_is_optimal_against_every_path(seed):
    rng = np.random.default_rng(1000 + seed)
    n, m = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    dim = int(rng.integers(1, 4))
    p = int(rng.choice([1, 2, 3]))
    a = rng.normal(size=(n, dim))
    b = rng.normal(size=(m, dim))
    ta = np.cumsum(rng.exponential(1.0, n))
    tb = np.cumsum(rng.exponential(1.0, m))
    nu, lam = float(rng.uniform(0, 1)), float(rng.uniform(0, 1))
    value, moves = oracle.twed_path(a, ta, b, tb, nu, lam, p)
    assert valid(moves, n, m)
    best = twed_bruteforce(a, ta, b, tb, nu, lam, p)
    # the path's own cost, summed independently, is the minimum over all paths
    assert path_cost(moves, a, ta, b, tb, nu, lam, p) == pytest.approx(best, rel=1e-12)
    assert value == pytest.approx(best, rel=1e-12)
    assert value == oracle.twed(a, ta, b, tb, nu, lam, p)
    # and no enumerated path is cheaper than it
    costs = [path_cost("".join(q), a, ta, b, tb, nu, lam, p) for q in all_paths(n, m)]
    assert min(costs) >= value * (1 - 1e-12) - 1e-300


@pytest.mark.parametrize("n,m,dim,p", [(60, 45, 1, 2), (33, 90, 4, 2), (70, 70, 2, 1)])
def test_longer_paths_cost_the_distance(n, m, dim, p):
    rng = np.random.default_rng(n * m + dim)
    a = np.cumsum(rng.normal(size=(n, dim)), axis=0)
    b = np.cumsum(rng.normal(size=(m, dim)), axis=0)
    ta = np.cumsum(rng.exponential(1.0, n))
    tb = np.cumsum(rng.exponential(1.0, m))
    value, moves = oracle.twed_path(a, ta, b, tb, 0.5, 1.0, p)
    assert valid(moves, n, m)
    assert value == oracle.twed(a, ta, b, tb, 0.5, 1.0, p)
    assert path_cost(moves, a, ta, b, tb, 0.5, 1.0, p) == pytest.approx(value, rel=1e-12)


def test_path_rejects_bad_arguments():
    with pytest.raises(oracle.OracleError):
        oracle.twed_path([[0.0]], [0.0], [[1.0]], [0.0], -1.0, 0.0, 2)


# ------------------------------------------------------------ pin strength
PATH_MUTANTS = {
    10: "walk tries delete in b before delete in a",
    11: "walk tries delete in a before the match",
    12: "moves returned in walk (reverse) order",
}


def _path_pins(twed_path):
    """Name of the first path pin that `twed_path` fails, or None."""
    cases = {c["name"]: c for c in json.load(open(os.path.join(GOLDEN, "hand_worked.json")))["cases"]}
    for p in json.load(open(os.path.join(GOLDEN, "hand_worked_paths.json")))["cases"]:
        c = cases[p["name"]]
        if twed_path(c["a"], c["ta"], c["b"], c["tb"], c["nu"], c["lam"], c["p"])[1] != p["path"]:
            return "hand:" + p["name"]
    if twed_path([[0.0], [0.0]], [1.0, 2.0], [[10.0], [10.0]], [1.0, 2.0], 0.0, 0.0, 2)[1] != "BA":
        return "tie-break"
    for shape, path in ALL_TIES:
        if _all_ties_path(twed_path, *shape)[1] != path:
            return "all-ties"
    rng = np.random.default_rng(77)
    for _ in range(30):
        n, m = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        a, b = rng.normal(size=(n, 2)), rng.normal(size=(m, 2))
        ta, tb = np.cumsum(rng.exponential(1.0, n)), np.cumsum(rng.exponential(1.0, m))
        _, moves = twed_path(a, ta, b, tb, 0.4, 0.6, 2)
        if not valid(moves, n, m):
            return "validity"
        try:
            cost = path_cost(moves, a, ta, b, tb, 0.4, 0.6, 2)
        except AssertionError:
            return "validity"
        if cost != pytest.approx(twed_bruteforce(a, ta, b, tb, 0.4, 0.6, 2), rel=1e-12):
            return "bruteforce"
    return None


def test_real_path_oracle_passes_every_path_pin():
    assert _path_pins(oracle.twed_path) is None


@pytest.mark.parametrize("k", sorted(PATH_MUTANTS), ids=lambda k: PATH_MUTANTS[k])
def test_planted_path_mistake_is_caught(k, tmp_path):
    mutant = oracle.twed_path_of(mutants.build(str(tmp_path), k))
    assert _path_pins(mutant) is not None, f"no pin rejects: {PATH_MUTANTS[k]}"
