"""GPU parity of the compiled wide-point strips (FP32, p = 2, dims 16, 28 and
64; paper, section "Higher Dimensions") against the oracle.

The many-pairs kernel runs them for all-pairs plans and explicit pair lists;
lengths straddle the strips (32 lanes x 8, 4 or 2 rows) and the 32-column
chunks of the 96-column staging ring.  FP32 results are compared with the
FP64 oracle on the same FP32-rounded inputs, within the 1e-5 relative bound.
"""
import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu
DIMS = [16, 28, 64]


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
    out = [(np.cumsum(rng.normal(size=(n, dim)), axis=0) / np.sqrt(dim), np.cumsum(rng.exponential(1.0, n)))
           for n in lengths]
    return W.pack(out).astype(np.float32)


def oracle_pairs(SA, SB, nu, lam, pairs):
    return oracle.twed_pairs(SA.astype(np.float64).as_tuple(), SB.astype(np.float64).as_tuple(), pairs,
                             nu, lam, 2)


def rel(got, want):
    return np.abs(got - want) / np.maximum(np.abs(want), 1e-300)


@pytest.mark.parametrize("dim", DIMS)
def test_wide_allpairs_symmetric(tw, dim):
    import torch
    rng = np.random.default_rng(dim)
    lens = [1, 2, 31, 32, 33, 63, 64, 65, 95, 96, 97, 255, 256, 257] + [int(v) for v in rng.integers(1, 700, 10)]
    S = walk_set(dim, lens, dim)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    plan = tw.Plan(D, None, 0.5, 0.5, 2)
    M = plan.execute().cpu().numpy()
    plan.status()
    n = S.n
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, n)])
    ref = oracle_pairs(S, S, 0.5, 0.5, pairs)
    assert rel(M[pairs[:, 0], pairs[:, 1]], ref).max() <= 1e-5
    assert np.array_equal(M, M.T)
    assert np.all(np.diag(M) == 0)


@pytest.mark.parametrize("dim", DIMS)
def test_wide_block_plan(tw, dim):
    import torch
    rng = np.random.default_rng(100 + dim)
    SA = walk_set(200 + dim, [int(v) for v in rng.integers(1, 600, 9)], dim)
    SB = walk_set(300 + dim, [int(v) for v in rng.integers(1, 900, 11)], dim)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    plan = tw.Plan(A, B, 1.0, 1.0, 2)
    M = plan.execute().cpu().numpy()
    plan.status()
    pairs = np.array([(i, j) for i in range(SA.n) for j in range(SB.n)])
    ref = oracle_pairs(SA, SB, 1.0, 1.0, pairs).reshape(SA.n, SB.n)
    assert rel(M, ref).max() <= 1e-5


@pytest.mark.parametrize("dim", DIMS)
def test_wide_explicit_pairs(tw, dim):
    import torch
    rng = np.random.default_rng(400 + dim)
    S = walk_set(500 + dim, [int(v) for v in rng.integers(1, 500, 20)], dim)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    pairs = np.stack([rng.integers(0, S.n, 150), rng.integers(0, S.n, 150)], 1)
    got = tw.twed_batch(D, D, torch.as_tensor(pairs).cuda(), 0.25, 2.0, 2).cpu().numpy()
    tw.default_handle().sync_status()
    want = oracle_pairs(S, S, 0.25, 2.0, pairs)
    same = pairs[:, 0] == pairs[:, 1]
    assert np.all(got[same] == 0.0)
    assert rel(got[~same], want[~same]).max() <= 1e-5


def test_wide_dim64_agrees_with_w4_recipe(tw):
    # the dim-64 CUDA-core arm on the smoothed N(0, 1) recipe of the dim-64
    # block workload, 40 x 40 series, against the oracle on sampled pairs
    import torch
    SA = W.set_w4(nseries=40, stream=0).astype(np.float32)
    SB = W.set_w4(nseries=40, stream=1).astype(np.float32)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    plan = tw.Plan(A, B, 1.0, 1.0, 2, opts=tw.make_opts(xterm=tw.XTERM_OFF))
    M = plan.execute().cpu().numpy()
    plan.status()
    rng = np.random.default_rng(7)
    pairs = np.stack([rng.integers(0, 40, 60), rng.integers(0, 40, 60)], 1)
    ref = oracle_pairs(SA, SB, 1.0, 1.0, pairs)
    assert rel(M[pairs[:, 0], pairs[:, 1]], ref).max() <= 1e-5
