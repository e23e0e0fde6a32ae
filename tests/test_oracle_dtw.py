"""Pins of the DTW oracle (``oracle.dtw``): the related time-warp distance of
the paper's introduction, the second problem for a generic diagonal band.
Pinned by a hand-worked case, enumeration of every warping path on tiny
inputs with numpy's own lp norm, and closed forms."""
import numpy as np
import pytest

import oracle
from tests import mutants
from bruteforce import all_paths, lp


def brute_dtw(a, b, p):
    """Minimum over all warping paths (steps (1,1), (1,0), (0,1) from (1,1)
    to (n,m)) of the summed point distances of the visited cells."""
    a = np.asarray(a, dtype=np.float64).reshape(len(a), -1)
    b = np.asarray(b, dtype=np.float64).reshape(len(b), -1)
    best = np.inf
    for moves in all_paths(len(a), len(b)):
        i, j = 0, 0
        cost = lp(a[0], b[0], p)
        for mv in moves:
            i += mv in "MA"
            j += mv in "MB"
            cost += lp(a[i], b[j], p)
        best = min(best, cost)
    return best


def test_hand_worked():
    # a = (0, 1, 2), b = (0, 2): point distances rows (0 2), (1 1), (2 0);
    # D(1,1)=0, D(1,2)=2, D(2,1)=1, D(2,2)=1+min(0,2,1)=1, D(3,1)=3,
    # D(3,2)=0+min(D(2,1)=1, D(2,2)=1, D(3,1)=3)=1
    assert oracle.dtw([0.0, 1.0, 2.0], [0.0, 2.0]) == 1.0


@pytest.mark.parametrize("seed", range(40))
def test_against_every_warping_path(seed):
    rng = np.random.default_rng(500 + seed)
    n, m = int(rng.integers(1, 7)), int(rng.integers(1, 7))
    dim = int(rng.integers(1, 4))
    p = int(rng.choice([1, 2, 3]))
    a, b = rng.normal(size=(n, dim)), rng.normal(size=(m, dim))
    assert oracle.dtw(a, b, p) == pytest.approx(brute_dtw(a, b, p), rel=1e-12)


def test_closed_forms():
    rng = np.random.default_rng(3)
    a = np.cumsum(rng.normal(size=(50, 3)), axis=0)
    b = np.cumsum(rng.normal(size=(35, 3)), axis=0)
    assert oracle.dtw(a, a) == 0.0                                   # identity
    assert oracle.dtw(a, b) == oracle.dtw(b, a)                      # symmetry
    # one point against a series: every cell of the single row is visited
    one = a[:1]
    want = sum(np.linalg.norm(one[0] - x) for x in b)
    assert oracle.dtw(one, b) == pytest.approx(want, rel=1e-12)
    # two constant series: a shortest path visits max(n, m) cells
    assert oracle.dtw(np.full(7, 1.5), np.full(4, -0.5)) == pytest.approx(7 * 2.0)
    # a stretched copy: repeating points costs nothing
    assert oracle.dtw(np.repeat(a, 2, axis=0), a) == 0.0


# ------------------------------------------------------------ pin strength
DTW_MUTANTS = {
    30: "the left neighbour is left out of the minimum",
    31: "the best predecessor is halved",
    32: "the 1-D point distance is squared",
}


def _dtw_pins(lib):
    """Name of the first DTW pin that the variant `lib` fails, or None."""
    if oracle.dtw([0.0, 1.0, 2.0], [0.0, 2.0], lib=lib) != 1.0:
        return "hand"
    rng = np.random.default_rng(321)
    for _ in range(30):
        n, m = int(rng.integers(1, 6)), int(rng.integers(1, 6))
        dim, p = int(rng.integers(1, 3)), int(rng.choice([1, 2]))
        a, b = rng.normal(size=(n, dim)), rng.normal(size=(m, dim))
        if oracle.dtw(a, b, p, lib=lib) != pytest.approx(brute_dtw(a, b, p), rel=1e-12):
            return "bruteforce"
    return None


def test_real_dtw_oracle_passes_every_pin(tmp_path):
    assert _dtw_pins(mutants.build(str(tmp_path), 0)) is None


@pytest.mark.parametrize("k", sorted(DTW_MUTANTS), ids=lambda k: DTW_MUTANTS[k])
def test_planted_dtw_mistake_is_caught(k, tmp_path):
    lib = mutants.build(str(tmp_path), k)
    assert _dtw_pins(lib) is not None, f"no pin rejects: {DTW_MUTANTS[k]}"
