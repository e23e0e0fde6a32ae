"""Pins for the CPU oracle (no GPU).

The oracle is only trusted after it agrees with things that do not come from
itself: hand-worked values, closed forms that the infinite border and the
recurrence imply, exact invariants of the metric (paper, "Background": TWED is
a proper metric), and an explicit minimum over all edit paths on short inputs.
Each plausible slip (a dropped match term, a wrong time index, a missing nu or
lambda, a border error, an off-by-one in the deletion costs, a wrong lp norm)
changes at least one of these.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from tests.bruteforce import all_paths, delannoy, lp, twed_bruteforce

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "hand_worked.json")


def _cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c["name"])
def test_hand_worked(case):
    a, b = np.array(case["a"]), np.array(case["b"])
    args = (a, case["ta"], b, case["tb"], case["nu"], case["lam"], case["p"])
    want = case["expected"]
    assert oracle.twed(*args) == pytest.approx(want, rel=1e-13, abs=1e-13)
    assert oracle.twed_rolling(*args) == oracle.twed(*args)
    assert twed_bruteforce(*args) == pytest.approx(want, rel=1e-13, abs=1e-13)


def test_path_count_is_delannoy():
    # enumeration sanity: paths from (1,1) to (n,m) = Delannoy(n-1, m-1)
    for n, m in [(1, 1), (2, 3), (4, 4), (6, 6), (5, 2)]:
        assert len(all_paths(n, m)) == delannoy(n - 1, m - 1)
    assert delannoy(6, 6) == 8989


def _rand_series(rng, n, dim, increasing=True):
    v = rng.normal(size=(n, dim))
    t = np.cumsum(rng.exponential(1.0, n)) if increasing else rng.uniform(0, 10, n)
    return v, t


@pytest.mark.parametrize("seed", range(60))
def test_bruteforce_agreement(seed):
    rng = np.random.default_rng(seed)
    n, m = rng.integers(1, 7, size=2)
    dim = int(rng.integers(1, 4))
    p = int(rng.choice([1, 2, 3]))
    nu = float(rng.uniform(0.01, 2.0))
    lam = float(rng.choice([0.0, rng.uniform(0.0, 2.0)]))
    a, ta = _rand_series(rng, n, dim, increasing=bool(seed % 3))
    b, tb = _rand_series(rng, m, dim, increasing=bool(seed % 3))
    got = oracle.twed(a, ta, b, tb, nu, lam, p)
    want = twed_bruteforce(a, ta, b, tb, nu, lam, p)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-12)


@pytest.mark.parametrize("seed", range(20))
def test_one_row_and_one_column_closed_forms(seed):
    # Step 3's infinite border leaves one finite path through a 1 x m matrix:
    # D(1,m) = c(1,1) + sum_{j=2..m} dB(j); the n x 1 case mirrors it.
    rng = np.random.default_rng(100 + seed)
    dim = int(rng.integers(1, 5))
    p = int(rng.choice([1, 2, 3]))
    nu, lam = float(rng.uniform(0, 2)), float(rng.uniform(0, 2))
    m = int(rng.integers(1, 40))
    a, ta = _rand_series(rng, 1, dim)
    b, tb = _rand_series(rng, m, dim)
    c11 = lp(a[0], b[0], p) + nu * abs(ta[0] - tb[0])
    row = c11 + sum(lp(b[j], b[j - 1], p) + nu * abs(tb[j] - tb[j - 1]) + lam for j in range(1, m))
    assert oracle.twed(a, ta, b, tb, nu, lam, p) == pytest.approx(row, rel=1e-12)
    assert oracle.twed(b, tb, a, ta, nu, lam, p) == pytest.approx(row, rel=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_diagonal_path_when_lambda_dominates(seed):
    # n = m and lambda larger than the whole diagonal path: every other path
    # uses at least two deletions, so TWED = c(n,n) + 2 sum_{i<n} c(i,i).
    rng = np.random.default_rng(200 + seed)
    n, dim = int(rng.integers(2, 30)), int(rng.integers(1, 4))
    a, ta = _rand_series(rng, n, dim)
    b, tb = _rand_series(rng, n, dim)
    nu = float(rng.uniform(0.1, 1.0))
    c = [lp(a[i], b[i], 2) + nu * abs(ta[i] - tb[i]) for i in range(n)]
    diag = c[-1] + 2.0 * sum(c[:-1])
    assert oracle.twed(a, ta, b, tb, nu, 10.0 * diag + 1.0, 2) == pytest.approx(diag, rel=1e-12)


def test_zero_values_no_time_penalty():
    # nu = 0 and all values 0: matches are free, at least |n-m| deletions.
    for n, m in [(1, 1), (1, 9), (7, 3), (20, 20), (33, 5)]:
        for lam in (0.0, 0.25, 3.0):
            a, b = np.zeros((n, 2)), np.zeros((m, 2))
            got = oracle.twed(a, np.arange(n) * 1.7, b, np.arange(m) * 0.3, 0.0, lam, 2)
            assert got == lam * abs(n - m)


@pytest.mark.parametrize("seed", range(12))
def test_identity_symmetry_nonnegativity(seed):
    rng = np.random.default_rng(300 + seed)
    dim, p = int(rng.integers(1, 5)), int(rng.choice([1, 2, 3]))
    nu, lam = float(rng.uniform(0, 2)), float(rng.uniform(0, 2))
    a, ta = _rand_series(rng, int(rng.integers(1, 60)), dim)
    b, tb = _rand_series(rng, int(rng.integers(1, 60)), dim)
    assert oracle.twed(a, ta, a, ta, nu, lam, p) == 0.0
    ab = oracle.twed(a, ta, b, tb, nu, lam, p)
    assert ab == oracle.twed(b, tb, a, ta, nu, lam, p)  # bitwise: mirrored operations
    assert ab >= 0.0


@pytest.mark.parametrize("seed", range(25))
def test_triangle_inequality(seed):
    rng = np.random.default_rng(400 + seed)
    dim, p = int(rng.integers(1, 4)), int(rng.choice([1, 2, 3]))
    nu, lam = float(rng.uniform(1e-3, 2)), float(rng.uniform(0, 2))
    s = [_rand_series(rng, int(rng.integers(1, 25)), dim) for _ in range(3)]
    d = lambda x, y: oracle.twed(x[0], x[1], y[0], y[1], nu, lam, p)
    ac, ab, bc = d(s[0], s[2]), d(s[0], s[1]), d(s[1], s[2])
    assert ac <= (ab + bc) * (1 + 1e-12) + 1e-12


@pytest.mark.parametrize("p", [1, 2, 3])
def test_time_shift_and_scaling(p):
    rng = np.random.default_rng(7)
    a, ta = _rand_series(rng, 31, 3)
    b, tb = _rand_series(rng, 17, 3)
    nu, lam = 0.7, 0.4
    base = oracle.twed(a, ta, b, tb, nu, lam, p)
    # shifting every timestamp of both series changes no |dt|
    assert oracle.twed(a, ta + 12.5, b, tb + 12.5, nu, lam, p) == pytest.approx(base, rel=1e-12)
    # scaling values, times and lambda by 2 scales every cost by 2 exactly
    # (binary scaling commutes with correctly rounded +, *, sqrt)
    s2 = oracle.twed(2 * a, 2 * ta, 2 * b, 2 * tb, nu, 2 * lam, p)
    if p in (1, 2):
        assert s2 == 2 * base
    else:
        assert s2 == pytest.approx(2 * base, rel=1e-12)
    s3 = oracle.twed(3 * a, 3 * ta, 3 * b, 3 * tb, nu, 3 * lam, p)
    assert s3 == pytest.approx(3 * base, rel=1e-12)


@pytest.mark.parametrize("seed", range(6))
def test_rolling_is_bitwise_full(seed):
    rng = np.random.default_rng(500 + seed)
    dim, p = int(rng.integers(1, 9)), int(rng.choice([1, 2, 3]))
    a, ta = _rand_series(rng, int(rng.integers(1, 400)), dim)
    b, tb = _rand_series(rng, int(rng.integers(1, 400)), dim)
    args = (a, ta, b, tb, 0.3, 0.9, p)
    assert oracle.twed_rolling(*args) == oracle.twed(*args)


def test_delete_costs_match_definition():
    rng = np.random.default_rng(11)
    a, ta = _rand_series(rng, 9, 3)
    got = oracle.delete_costs(a, ta, 0.5, 0.25, 2)
    # first entry uses the zero padding a_0 = 0, t_0 = 0 (never read by the DP)
    want = [lp(a[0], np.zeros(3), 2) + 0.5 * abs(ta[0]) + 0.25]
    want += [lp(a[i], a[i - 1], 2) + 0.5 * abs(ta[i] - ta[i - 1]) + 0.25 for i in range(1, 9)]
    np.testing.assert_allclose(got, want, rtol=1e-14)


def test_pairs_threads_match_single_calls():
    from paper_2007_16135_gb300 import workloads as W
    S = W.set_w3(nseries=12, len_lo=5, len_hi=40)
    pairs = W.sample_upper_pairs(S.n, 30, 3)
    got = oracle.twed_pairs(S.as_tuple(), S.as_tuple(), pairs, 0.5, 0.5, 2, nthreads=4)
    for k, (i, j) in enumerate(pairs):
        a, ta = S.series(i)
        b, tb = S.series(j)
        assert got[k] == oracle.twed(a, ta, b, tb, 0.5, 0.5, 2)


def test_rejects_invalid_arguments():
    a, t = np.zeros((3, 1)), np.arange(3.0)
    with pytest.raises(oracle.OracleError):
        oracle.twed(a[:0], t[:0], a, t, 1.0, 1.0, 2)  # empty series
    with pytest.raises(oracle.OracleError):
        oracle.twed(a, t, a, t, -1.0, 1.0, 2)
    with pytest.raises(oracle.OracleError):
        oracle.twed(a, t, a, t, 1.0, math.nan, 2)
    with pytest.raises(oracle.OracleError):
        oracle.twed(a, t, a, t, 1.0, 1.0, 0)
