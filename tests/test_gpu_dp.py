"""GPU parity of the dynamic programs beside TWED's value: TWED edit paths,
LCS lengths and subsequences, DTW (paper, sections "Introduction" and
"Generalized Dynamic Programming Extensions").

Every case compares the CUDA path with the CPU oracle on the same seeded
inputs: integer results and FP64 results for p = 1, 2 bit for bit, edit
paths move for move (the walk-back order is part of the definition), FP32
within the 1e-5 bound against FP64 on the same FP32-rounded inputs.  Lengths
straddle the strips (32 lanes x 4 or 8 rows) and the 16-column choice words.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


def walk_set(seed, lengths, dim):
    rng = np.random.default_rng(seed)
    return W.pack([(np.cumsum(rng.normal(size=(n, dim)), axis=0), np.cumsum(rng.exponential(1.0, n)))
                   for n in lengths])


# ------------------------------------------------------------- edit paths
def test_paths_of_the_hand_worked_cases(tw):
    cases = {c["name"]: c for c in json.load(open(os.path.join(GOLDEN, "hand_worked.json")))["cases"]}
    for pth in json.load(open(os.path.join(GOLDEN, "hand_worked_paths.json")))["cases"]:
        c = cases[pth["name"]]
        value, moves = tw.twed_path(c["a"], c["ta"], c["b"], c["tb"], c["nu"], c["lam"], c["p"])
        assert moves == pth["path"], pth["name"]
        assert value == oracle.twed(c["a"], c["ta"], c["b"], c["tb"], c["nu"], c["lam"], c["p"])


@pytest.mark.parametrize("n,m,path", [(2, 2, "M"), (4, 2, "AAM"), (2, 4, "BBM"), (40, 3, None), (3, 40, None)])
def test_all_ties_follow_the_walk_back_order(tw, n, m, path):
    # every cost zero: all candidates tie and the tie order alone fixes the path
    args = (np.zeros((n, 1)), np.arange(1.0, n + 1), np.zeros((m, 1)), np.arange(1.0, m + 1), 0.0, 0.0, 2)
    value, moves = tw.twed_path(*args)
    want = oracle.twed_path(*args)
    assert (value, moves) == want
    if path is not None:
        assert moves == path


@pytest.mark.parametrize("seed", range(12))
def test_paths_equal_the_oracle_move_for_move(tw, seed):
    rng = np.random.default_rng(500 + seed)
    n, m = int(rng.integers(1, 300)), int(rng.integers(1, 300))
    dim = int(rng.choice([1, 2, 3, 5, 9]))
    p = int(rng.choice([1, 2]))
    a, b = np.cumsum(rng.normal(size=(n, dim)), 0), np.cumsum(rng.normal(size=(m, dim)), 0)
    ta, tb = np.cumsum(rng.exponential(1.0, n)), np.cumsum(rng.exponential(1.0, m))
    nu, lam = float(rng.uniform(0, 1)), float(rng.uniform(0, 2))
    got = tw.twed_path(a, ta, b, tb, nu, lam, p)
    assert got == oracle.twed_path(a, ta, b, tb, nu, lam, p)


def test_path_batch_at_w3_lengths(tw):
    # 24 pairs of dim-8 sinusoid mixtures, lengths up to 2048 (the batched
    # workload's length range), FP64: moves equal the oracle's, distances bitwise
    import torch
    S = W.set_w3(nseries=16, len_lo=64, len_hi=2048, stream=7)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float64)
    rng = np.random.default_rng(9)
    pairs = np.stack([rng.integers(0, S.n, 24), rng.integers(0, S.n, 24)], 1)
    dist, moves, offs, lens = tw.twed_path_batch(D, D, torch.as_tensor(pairs).cuda(), 0.5, 0.5, 2)
    tw.default_handle().sync_status()
    dist, moves, offs, lens = (x.cpu().numpy() for x in (dist, moves, offs, lens))
    for k, (x, y) in enumerate(pairs):
        (av, at), (bv, bt) = S.series(x), S.series(y)
        value, want = oracle.twed_path(av, at, bv, bt, 0.5, 0.5, 2)
        got = "".join(tw.MOVE_CHARS[v] for v in moves[offs[k]:offs[k] + lens[k]])
        assert dist[k] == value and got == want, k


def test_path_f32_is_an_optimal_path_within_the_bound(tw):
    rng = np.random.default_rng(33)
    a, b = np.cumsum(rng.normal(size=(150, 3)), 0), np.cumsum(rng.normal(size=(170, 3)), 0)
    ta, tb = np.arange(1.0, 151), np.arange(1.0, 171)
    value, moves = tw.twed_path(a, ta, b, tb, 0.5, 1.0, 2, dtype="f32")
    a32, b32 = (x.astype(np.float32).astype(np.float64) for x in (a, b))
    want = oracle.twed(a32, ta, b32, tb, 0.5, 1.0, 2)
    assert abs(value - want) <= 1e-5 * want
    assert moves.count("M") + moves.count("A") == 149 and moves.count("M") + moves.count("B") == 169
    # the FP32 path, priced in FP64 by the oracle's definition, is optimal within the bound
    from tests.test_oracle_path import path_cost
    assert abs(path_cost(moves, a32, ta, b32, tb, 0.5, 1.0, 2) - want) <= 1e-5 * want


# ------------------------------------------------------------- LCS
def test_lcs_hand_worked(tw):
    for c in json.load(open(os.path.join(GOLDEN, "lcs_hand_worked.json")))["cases"]:
        x = [ord(ch) for ch in c["x"]]
        y = [ord(ch) for ch in c["y"]]
        xi, yj = tw.lcs_pairs(x, y)
        assert xi.tolist() == c["xi"] and yj.tolist() == c["yj"], c["name"]


@pytest.mark.parametrize("alphabet", [2, 4, 26])
def test_lcs_batch_equals_the_oracle(tw, alphabet):
    import torch
    rng = np.random.default_rng(alphabet)
    lens = [0, 1, 15, 16, 17, 255, 256, 257, 700, 1300] + [int(v) for v in rng.integers(0, 900, 14)]
    seqs = [rng.integers(0, alphabet, n) for n in lens]
    X = tw.DeviceSeqs.from_lists(seqs)
    pairs = np.stack([rng.integers(0, len(seqs), 300), rng.integers(0, len(seqs), 300)], 1)
    got = tw.lcs_batch(X, X, torch.as_tensor(pairs).cuda()).cpu().numpy()
    tw.default_handle().sync_status()
    want = [oracle.lcs_length_rolling(seqs[x], seqs[y]) for x, y in pairs]
    assert got.tolist() == want


@pytest.mark.parametrize("n,m,alphabet", [(1, 1, 2), (7, 300, 3), (257, 33, 4), (600, 900, 8), (2000, 1500, 20)])
def test_lcs_subsequence_equals_the_oracle(tw, n, m, alphabet):
    rng = np.random.default_rng(n + m)
    x, y = rng.integers(0, alphabet, n), rng.integers(0, alphabet, m)
    xi, yj = tw.lcs_pairs(x, y)
    wx, wy = oracle.lcs_pairs(x, y)
    assert np.array_equal(xi, wx) and np.array_equal(yj, wy)


def test_lcs_of_identical_and_disjoint_sequences(tw):
    x = np.arange(500) % 37
    xi, yj = tw.lcs_pairs(x, x)
    assert np.array_equal(xi, np.arange(500)) and np.array_equal(yj, np.arange(500))
    xi, yj = tw.lcs_pairs(np.zeros(300, dtype=np.int32), np.ones(200, dtype=np.int32))
    assert xi.size == 0 and yj.size == 0
    xi, yj = tw.lcs_pairs([], [1, 2, 3])
    assert xi.size == 0


# ------------------------------------------------------------- DTW
@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (3, 2), (5, 2), (9, 2), (4, 3)])
def test_dtw_batch_f64_equals_the_oracle(tw, dim, p):
    import torch
    rng = np.random.default_rng(dim * 10 + p)
    lens = [1, 2, 127, 128, 129, 300, 511] + [int(v) for v in rng.integers(1, 700, 9)]
    S = walk_set(dim + p, lens, dim)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float64)
    pairs = np.stack([rng.integers(0, S.n, 60), rng.integers(0, S.n, 60)], 1)
    got = tw.dtw_batch(D, D, torch.as_tensor(pairs).cuda(), p).cpu().numpy()
    tw.default_handle().sync_status()
    want = np.array([oracle.dtw(S.series(x)[0], S.series(y)[0], p) for x, y in pairs])
    if p in (1, 2):
        assert np.array_equal(got, want)
    else:  # pow is not correctly rounded: 1e-12 (DTW(a, a) = 0 exactly)
        assert np.all(got[want == 0] == 0)
        nz = want > 0
        assert np.max(np.abs(got[nz] - want[nz]) / want[nz]) <= 1e-12


def test_dtw_f32_within_the_bound(tw):
    import torch
    rng = np.random.default_rng(77)
    S = walk_set(78, [int(v) for v in rng.integers(50, 1200, 12)], 3).astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    pairs = np.array([(i, j) for i in range(S.n) for j in range(S.n)])
    got = tw.dtw_batch(D, D, torch.as_tensor(pairs).cuda(), 2).cpu().numpy().astype(np.float64)
    S64 = S.astype(np.float64)
    want = np.array([oracle.dtw(S64.series(x)[0], S64.series(y)[0], 2) for x, y in pairs])
    diag = pairs[:, 0] == pairs[:, 1]
    assert np.all(got[diag] == 0.0)
    assert np.max(np.abs(got[~diag] - want[~diag]) / want[~diag]) <= 1e-5


def test_dtw_one_pair_from_host(tw):
    rng = np.random.default_rng(5)
    a, b = np.cumsum(rng.normal(size=(400, 2)), 0), np.cumsum(rng.normal(size=(333, 2)), 0)
    assert tw.dtw(a, b, 2) == oracle.dtw(a, b, 2)
    assert tw.dtw(a, a, 1) == 0.0


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (2, 2), (4, 2), (5, 2), (8, 1), (8, 2)])
def test_dtw_batch_f32_staged_layouts(tw, dim, p):
    # FP32 compiled layouts run DTW on the staged engine: lengths straddle its
    # 256-row strips and 32-column staging chunks
    import torch
    rng = np.random.default_rng(900 + 10 * dim + p)
    lens = [1, 2, 31, 32, 33, 255, 256, 257, 600] + [int(v) for v in rng.integers(1, 800, 7)]
    S = walk_set(dim * 3 + p, lens, dim).astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    pairs = np.stack([rng.integers(0, S.n, 80), rng.integers(0, S.n, 80)], 1)
    got = tw.dtw_batch(D, D, torch.as_tensor(pairs).cuda(), p).cpu().numpy().astype(np.float64)
    tw.default_handle().sync_status()
    S64 = S.astype(np.float64)
    want = np.array([oracle.dtw(S64.series(x)[0], S64.series(y)[0], p) for x, y in pairs])
    same = pairs[:, 0] == pairs[:, 1]
    assert np.all(got[same] == 0.0)
    assert np.max(np.abs(got[~same] - want[~same]) / want[~same]) <= 1e-5


@pytest.mark.parametrize("dim,p", [(1, 2), (2, 1), (3, 2), (4, 2), (8, 1), (8, 2)])
def test_path_batch_f32_staged_layouts(tw, dim, p):
    # FP32 compiled layouts record the choices on the staged engine (words of
    # 16 steps, strips of up to 256 rows): every path is a valid monotone path
    # whose cost, priced in FP64 on the same FP32-rounded inputs, is optimal
    # within the 1e-5 bound, and the distance is within it too
    import torch
    from tests.test_oracle_path import path_cost
    rng = np.random.default_rng(700 + 10 * dim + p)
    lens = [1, 2, 15, 16, 17, 255, 256, 257, 513] + [int(v) for v in rng.integers(1, 700, 7)]
    S = walk_set(40 + dim + p, lens, dim).astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    pairs = np.stack([rng.integers(0, S.n, 40), rng.integers(0, S.n, 40)], 1)
    dist, moves, offs, lens_ = tw.twed_path_batch(D, D, torch.as_tensor(pairs).cuda(), 0.5, 0.75, p)
    tw.default_handle().sync_status()
    dist, moves, offs, lens_ = (x.cpu().numpy() for x in (dist, moves, offs, lens_))
    S64 = S.astype(np.float64)
    for k, (x, y) in enumerate(pairs):
        (av, at), (bv, bt) = S64.series(x), S64.series(y)
        want = oracle.twed(av, at, bv, bt, 0.5, 0.75, p)
        got = "".join(tw.MOVE_CHARS[v] for v in moves[offs[k]:offs[k] + lens_[k]])
        assert got.count("M") + got.count("A") == len(at) - 1, k
        assert got.count("M") + got.count("B") == len(bt) - 1, k
        tol = 1e-5 * max(want, 1e-30)
        assert abs(float(dist[k]) - want) <= tol, k
        assert abs(path_cost(got, av, at, bv, bt, 0.5, 0.75, p) - want) <= tol, k
