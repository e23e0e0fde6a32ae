"""CPU model of the short-pair kernel's wavefront schedule (the recurrence of
the paper's section "Improved Time Warp Edit Distance", Eq. 2), checked
against the oracle's full-matrix evaluation.

The kernel first fills a cost tile, then runs 32 lanes in lockstep: at step
s lane i (row i+1) works on column s - i; a lane outside [0, m) takes cost
+inf and column delete cost 0, lane 0 sees D(0, j) = +inf above it, and the
step count is rounded up to a multiple of 4.  The claims this pins:

* a lane before its first column computes +inf;
* a lane past its last column keeps D(i, m) exactly (its own value plus 0 is
  the least candidate, since D(i, m) <= D(i-1, m) + dA(i));
* so lane n-1 ends on D(n, m) whatever the extra steps,

all in FP64, compared bit for bit with the oracle's D(n, m) (same operation
order per cell).  The model is numpy on the host; it shares nothing with the
CUDA sources.
"""
import numpy as np
import pytest

import oracle


def cell_costs(a, ta, b, tb, nu):
    """c(i, j) for 1 <= i <= n, 1 <= j <= m (p = 2), the oracle's order per
    cell: s = 0; s = s + d_k^2 in component order; sqrt; + nu |t_i - t'_j|."""
    n, m = len(a), len(b)
    c = np.empty((n, m))
    for i in range(n):
        for j in range(m):
            s = 0.0
            for k in range(a.shape[1]):
                d = a[i, k] - b[j, k]
                s = s + d * d
            c[i, j] = np.sqrt(s) + nu * abs(ta[i] - tb[j])
    return c


def delete_costs(x, tx, nu, lam):
    out = np.empty(len(x))
    prev, tprev = np.zeros(x.shape[1]), 0.0
    for i in range(len(x)):
        s = 0.0
        for k in range(x.shape[1]):
            d = x[i, k] - prev[k]
            s = s + d * d
        out[i] = (np.sqrt(s) + nu * abs(tx[i] - tprev)) + lam
        prev, tprev = x[i], tx[i]
    return out


def wavefront_model(c, dA, dB):
    """The kernel's phase 2 for one pair: returns lane n-1's value after the
    rounded-up step count, and every lane's value after each step."""
    n, m = c.shape
    INF = np.inf
    Dl = np.full(32, INF)
    cl = np.zeros(32)
    diagD = np.full(32, INF)
    diagD[0] = 0.0
    diagC = np.zeros(32)
    rows = np.minimum(np.arange(32), n - 1)  # lanes past the last row repeat it
    steps = n + m - 1
    steps4 = (steps + 3) // 4 * 4
    trace = []
    for s in range(steps4):
        upD = np.concatenate([[INF], Dl[:-1]])  # shuffle up; lane 0 sees +inf
        upC = np.concatenate([[cl[0]], cl[:-1]])
        j = s - np.arange(32)
        inside = (j >= 0) & (j < m)
        cc = np.where(inside, c[rows, np.clip(j, 0, m - 1)], INF)
        db = np.where(inside, dB[np.clip(j, 0, m - 1)], 0.0)
        tb = Dl + db
        tm = (diagD + cc) + diagC
        ta = upD + dA[rows]
        Dl = np.minimum(np.minimum(ta, tb), tm)
        cl = cc
        diagD = upD
        diagC = upC
        trace.append(Dl.copy())
    return Dl[n - 1], np.array(trace)


def random_pair(rng, n, m, dim):
    a = np.cumsum(rng.normal(size=(n, dim)), axis=0)
    b = np.cumsum(rng.normal(size=(m, dim)), axis=0)
    ta = np.cumsum(rng.exponential(1.0, n))
    tb = np.cumsum(rng.exponential(1.0, m))
    return a, ta, b, tb


@pytest.mark.parametrize("n,m", [(1, 1), (1, 7), (7, 1), (2, 2), (5, 9), (28, 28), (31, 32), (32, 32), (32, 1),
                                 (17, 30)])
def test_wavefront_model_equals_oracle_bitwise(n, m):
    rng = np.random.default_rng(1000 * n + m)
    a, ta, b, tb = random_pair(rng, n, m, 3)
    nu, lam = 0.5, 0.25
    got, _ = wavefront_model(cell_costs(a, ta, b, tb, nu), delete_costs(a, ta, nu, lam),
                             delete_costs(b, tb, nu, lam))
    want = oracle.twed(a, ta, b, tb, nu, lam, 2)
    assert got == want


def test_lanes_freeze_after_their_last_column():
    # after lane i's last column (step i + m - 1) its value never changes,
    # and before its first column (step i) it is +inf
    rng = np.random.default_rng(7)
    n, m = 20, 11
    a, ta, b, tb = random_pair(rng, n, m, 2)
    _, trace = wavefront_model(cell_costs(a, ta, b, tb, 1.0), delete_costs(a, ta, 1.0, 1.0),
                               delete_costs(b, tb, 1.0, 1.0))
    for i in range(n):
        assert np.all(np.isinf(trace[:i, i]))
        last = trace[i + m - 1, i]
        assert np.all(trace[i + m - 1:, i] == last)
        assert np.isfinite(last)


def test_frozen_row_value_is_the_matrix_last_column():
    # every lane's frozen value is D(i, m) of the full matrix
    rng = np.random.default_rng(8)
    n, m = 13, 9
    a, ta, b, tb = random_pair(rng, n, m, 4)
    nu, lam = 0.3, 0.7
    _, trace = wavefront_model(cell_costs(a, ta, b, tb, nu), delete_costs(a, ta, nu, lam),
                               delete_costs(b, tb, nu, lam))
    for i in range(1, n + 1):
        a_i, ta_i = a[:i], ta[:i]
        assert trace[-1, i - 1] == oracle.twed(a_i, ta_i, b, tb, nu, lam, 2)
