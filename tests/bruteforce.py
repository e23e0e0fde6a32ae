"""Independent restatement of TWED as a minimum over edit paths.

TWED is the cheapest monotone path from (0,0) to (n,m) whose steps are a
match (1,1), a deletion in a (1,0) or a deletion in b (0,1), with the costs of
the paper's section "Time Warp Edit Distance".  The infinite border (step 3)
removes every path that touches row 0 or column 0 after (0,0), so every finite
path starts with the match (0,0) -> (1,1).  This module enumerates all such
paths explicitly (no dynamic program, no shared code with the oracle) and uses
numpy's own lp norm; it is only usable for lengths up to about 7.
"""
import numpy as np


def lp(x, y, p):
    x = np.asarray(x, dtype=np.float64).ravel()
    y = np.asarray(y, dtype=np.float64).ravel()
    if x.size == 1:
        return abs(float(x[0]) - float(y[0]))
    return float(np.linalg.norm(x - y, ord=p))


def step_costs(a, ta, b, tb, nu, lam, p):
    a = np.asarray(a, dtype=np.float64).reshape(len(ta), -1)
    b = np.asarray(b, dtype=np.float64).reshape(len(tb), -1)
    n, m = a.shape[0], b.shape[0]
    zero = np.zeros(a.shape[1])
    pa = [zero] + list(a)
    pb = [zero] + list(b)
    qa = [0.0] + [float(t) for t in ta]
    qb = [0.0] + [float(t) for t in tb]

    def c(i, j):
        return lp(pa[i], pb[j], p) + nu * abs(qa[i] - qb[j])

    def del_a(i):
        return lp(pa[i], pa[i - 1], p) + nu * abs(qa[i] - qa[i - 1]) + lam

    def del_b(j):
        return lp(pb[j], pb[j - 1], p) + nu * abs(qb[j] - qb[j - 1]) + lam

    return n, m, c, del_a, del_b


def all_paths(n, m):
    """Every monotone step sequence from (1,1) to (n,m) (lists of moves)."""
    out = []

    def rec(i, j, moves):
        if i == n and j == m:
            out.append(list(moves))
            return
        if i < n and j < m:
            moves.append("M"); rec(i + 1, j + 1, moves); moves.pop()
        if i < n:
            moves.append("A"); rec(i + 1, j, moves); moves.pop()
        if j < m:
            moves.append("B"); rec(i, j + 1, moves); moves.pop()

    rec(1, 1, [])
    return out


def twed_bruteforce(a, ta, b, tb, nu, lam, p=2):
    n, m, c, del_a, del_b = step_costs(a, ta, b, tb, nu, lam, p)
    best = np.inf
    for moves in all_paths(n, m):
        i, j = 1, 1
        cost = c(1, 1) + c(0, 0)  # the forced first match (0,0) -> (1,1)
        for mv in moves:
            if mv == "M":
                i += 1; j += 1
                cost += c(i, j) + c(i - 1, j - 1)
            elif mv == "A":
                i += 1
                cost += del_a(i)
            else:
                j += 1
                cost += del_b(j)
        best = min(best, cost)
    return best


def delannoy(n, m):
    """Number of monotone (1,0)/(0,1)/(1,1) paths across an n x m grid."""
    from math import comb
    return sum(comb(n, k) * comb(m, k) * 2 ** k for k in range(min(n, m) + 1))
