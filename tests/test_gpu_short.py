"""GPU parity of the short-pair kernel (every series of both sets at most 32
points; p = 2, dims 16 and 28 in FP32 and FP64, 64 in FP32) against the
oracle: the cost tile of one pair per warp, then the wavefront over it
(paper, section "Improved Time Warp Edit Distance", Eq. 2; the image shape
of section "Experiments").

FP64 results are compared bit for bit (the kernel forms every cost and
candidate with the oracle's operations in the oracle's order); FP32 within
the 1e-5 relative bound against the FP64 oracle on the same FP32-rounded
inputs.  Lengths cover 1, 2, 31 and 32 points; sets whose longest series has
33 points, and values that are not 16-byte aligned, take the strip kernels
and must agree as well.
"""
import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


def walk_set(seed, lengths, dim, dtype=np.float64):
    rng = np.random.default_rng(seed)
    out = [(np.cumsum(rng.normal(size=(n, dim)), axis=0) / np.sqrt(dim), np.cumsum(rng.exponential(1.0, n)))
           for n in lengths]
    S = W.pack(out)
    return S.astype(np.float32) if dtype == np.float32 else S


def short_lengths(rng, k, hi=32):
    return [1, 2, 31, hi] + [int(v) for v in rng.integers(1, hi + 1, k - 4)]


def oracle_pairs(SA, SB, nu, lam, pairs):
    return oracle.twed_pairs(SA.astype(np.float64).as_tuple(), SB.astype(np.float64).as_tuple(), pairs,
                             nu, lam, 2)


def rel(got, want):
    return np.abs(got - want) / np.maximum(np.abs(want), 1e-300)


CASES = [("f64", 16), ("f64", 28), ("f32", 16), ("f32", 28), ("f32", 64)]


def torch_dtype(dt):
    import torch
    return torch.float64 if dt == "f64" else torch.float32


def check(dt, got, want):
    if dt == "f64":
        np.testing.assert_array_equal(got, want)
    else:
        assert rel(got, want).max() <= 1e-5


@pytest.mark.parametrize("dt,dim", CASES)
def test_short_allpairs_symmetric(tw, dt, dim):
    rng = np.random.default_rng(dim + (0 if dt == "f64" else 1000))
    S = walk_set(dim, short_lengths(rng, 40), dim, np.float64 if dt == "f64" else np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch_dtype(dt))
    plan = tw.Plan(D, None, 0.5, 0.75, 2)
    M = plan.execute().cpu().numpy()
    plan.status()
    n = S.n
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, n)])
    want = oracle_pairs(S, S, 0.5, 0.75, pairs)
    check(dt, M[pairs[:, 0], pairs[:, 1]], want)
    assert np.array_equal(M, M.T)
    assert np.all(np.diag(M) == 0)


@pytest.mark.parametrize("dt,dim", CASES)
def test_short_block_plan(tw, dt, dim):
    rng = np.random.default_rng(100 + dim)
    npdt = np.float64 if dt == "f64" else np.float32
    SA = walk_set(200 + dim, short_lengths(rng, 23), dim, npdt)
    SB = walk_set(300 + dim, short_lengths(rng, 37), dim, npdt)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch_dtype(dt))
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch_dtype(dt))
    plan = tw.Plan(A, B, 1.0, 1.0, 2)
    M = plan.execute().cpu().numpy()
    plan.status()
    pairs = np.array([(i, j) for i in range(SA.n) for j in range(SB.n)])
    want = oracle_pairs(SA, SB, 1.0, 1.0, pairs).reshape(SA.n, SB.n)
    check(dt, M, want)


@pytest.mark.parametrize("dt,dim", CASES)
@pytest.mark.parametrize("order", ["list", "longest"])
def test_short_explicit_pairs(tw, dt, dim, order):
    import torch
    rng = np.random.default_rng(400 + dim)
    npdt = np.float64 if dt == "f64" else np.float32
    SA = walk_set(500 + dim, short_lengths(rng, 30), dim, npdt)
    SB = walk_set(600 + dim, short_lengths(rng, 20), dim, npdt)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch_dtype(dt))
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch_dtype(dt))
    # 203 pairs: a ragged last grab of the 8-pair schedule, repeated pairs
    pairs = np.stack([rng.integers(0, SA.n, 203), rng.integers(0, SB.n, 203)], 1)
    pairs[:5] = pairs[5]
    od = tw.ORDER_LONGEST_FIRST if order == "longest" else tw.ORDER_LIST
    got = tw.twed_batch(A, B, torch.as_tensor(pairs).cuda(), 0.25, 2.0, 2, order=od).cpu().numpy()
    tw.default_handle().sync_status()
    check(dt, got, oracle_pairs(SA, SB, 0.25, 2.0, pairs))


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_short_same_series_is_zero(tw, dt):
    import torch
    S = walk_set(9, [1, 5, 28, 32], 28, np.float64 if dt == "f64" else np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch_dtype(dt))
    pairs = torch.as_tensor(np.array([[k, k] for k in range(S.n)])).cuda()
    got = tw.twed_batch(D, D, pairs, 1.0, 1.0, 2).cpu().numpy()
    tw.default_handle().sync_status()
    assert np.all(got == 0.0)


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_33_points_takes_the_strips_and_agrees(tw, dt):
    # one 33-point series moves the whole set off the short kernel
    import torch
    rng = np.random.default_rng(33)
    npdt = np.float64 if dt == "f64" else np.float32
    S = walk_set(33, short_lengths(rng, 20) + [33], 28, npdt)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch_dtype(dt))
    M = tw.Plan(D, None, 1.0, 1.0, 2).execute().cpu().numpy()
    pairs = np.array([(i, j) for i in range(S.n) for j in range(i + 1, S.n)])
    want = oracle_pairs(S, S, 1.0, 1.0, pairs)
    got = M[pairs[:, 0], pairs[:, 1]]
    assert rel(got, want).max() <= (1e-12 if dt == "f64" else 1e-5)


def test_unaligned_values_take_the_scalar_path(tw):
    # values 4 bytes past a 16-byte boundary: neither the short kernel nor
    # the wide strips (both copy points in 16-byte pieces) may run
    import torch
    rng = np.random.default_rng(5)
    for lens in (short_lengths(rng, 12), [40, 70, 3, 33]):
        S = walk_set(5, lens, 28, np.float32)
        base = torch.zeros(S.vals.size + 1, dtype=torch.float32, device="cuda")
        base[1:] = torch.as_tensor(S.vals.reshape(-1)).cuda()
        vals = base[1:].view(S.vals.shape)
        assert vals.data_ptr() % 16 == 4
        D = tw.DeviceSet(vals, torch.as_tensor(S.ts).cuda(), torch.as_tensor(S.offs).cuda(),
                         np.ascontiguousarray(S.offs, dtype=np.int64))
        plan = tw.Plan(D, None, 1.0, 1.0, 2)
        M = plan.execute().cpu().numpy()
        plan.status()
        pairs = np.array([(i, j) for i in range(S.n) for j in range(i + 1, S.n)])
        assert rel(M[pairs[:, 0], pairs[:, 1]], oracle_pairs(S, S, 1.0, 1.0, pairs)).max() <= 1e-5


@pytest.mark.parametrize("dt", ["f64", "f32"])
def test_u3_block_bitwise_or_bounded(tw, dt):
    # the image recipe (28 x 28 strokes) through the short kernel
    import torch
    SA, SB = W.set_u3(48, stream=4), W.set_u3(56, stream=5)
    if dt == "f32":
        SA, SB = SA.astype(np.float32), SB.astype(np.float32)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch_dtype(dt))
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch_dtype(dt))
    plan = tw.Plan(A, B, 1.0, 1.0, 2)
    M = plan.execute().cpu().numpy()
    plan.status()
    pairs = np.array([(i, j) for i in range(SA.n) for j in range(SB.n)])
    check(dt, M, oracle_pairs(SA, SB, 1.0, 1.0, pairs).reshape(SA.n, SB.n))
