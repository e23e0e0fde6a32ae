"""GPU parity of the batched and all-pairs entry points against the oracle."""
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


def oracle_matrix(SA, SB, nu, lam, p, pairs):
    A64 = SA.astype(np.float64)
    B64 = SB.astype(np.float64)
    return oracle.twed_pairs(A64.as_tuple(), B64.as_tuple(), pairs, nu, lam, p)


def ragged_set(seed, nseries, lo, hi, dim, dtype):
    rng = np.random.default_rng(seed)
    out = []
    for n in rng.integers(lo, hi + 1, size=nseries):
        v = np.cumsum(rng.normal(size=(n, dim)), axis=0)
        t = np.cumsum(rng.exponential(1.0, n))
        out.append((v, t))
    return W.pack(out).astype(dtype)


def rel(got, want):
    return np.abs(got - want) / np.maximum(np.abs(want), 1e-300)


@pytest.mark.parametrize("dim,p", [(8, 2), (1, 2), (3, 1), (5, 2)])
def test_allpairs_symmetric_f32(tw, dim, p):
    import torch
    S = ragged_set(dim * 10 + p, 37, 1, 700, dim, np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    plan = tw.Plan(D, None, 0.5, 0.5, p)
    M = plan.execute().cpu().numpy()
    n = S.n
    pairs = np.array([(i, j) for i in range(n) for j in range(i + 1, n)])
    ref = oracle_matrix(S, S, 0.5, 0.5, p, pairs)
    assert rel(M[pairs[:, 0], pairs[:, 1]], ref).max() <= 1e-5
    assert np.array_equal(M, M.T)
    assert np.all(np.diag(M) == 0)
    assert plan.pairs == n * (n - 1) // 2
    L = S.lengths.astype(np.int64)
    assert plan.cells == int((L.sum() ** 2 - (L ** 2).sum()) // 2)


@pytest.mark.parametrize("dim,p", [(8, 2), (2, 1), (4, 3)])
def test_allpairs_block_f64_bitwise(tw, dim, p):
    import torch
    SA = ragged_set(100 + dim, 19, 1, 600, dim, np.float64)
    SB = ragged_set(200 + dim, 23, 1, 900, dim, np.float64)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float64)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float64)
    plan = tw.Plan(A, B, 0.75, 0.3, p)
    M = plan.execute().cpu().numpy()
    pairs = np.array([(i, j) for i in range(SA.n) for j in range(SB.n)])
    ref = oracle_matrix(SA, SB, 0.75, 0.3, p, pairs).reshape(SA.n, SB.n)
    if p in (1, 2):
        assert np.array_equal(M, ref)
    else:
        assert rel(M, ref).max() <= 1e-12


def test_plan_reexecute_and_new_output(tw):
    import torch
    S = ragged_set(5, 16, 30, 300, 3, np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    plan = tw.Plan(D, None, 1.0, 1.0, 2)
    m1 = plan.execute().clone()
    out = torch.full_like(m1, -1.0)
    m2 = plan.execute(out)
    m3 = plan.execute(out)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(m2, m3)


def test_explicit_pairs_match_oracle(tw):
    import torch
    SA = ragged_set(31, 25, 1, 1200, 4, np.float32)
    SB = ragged_set(32, 17, 1, 1500, 4, np.float32)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    rng = np.random.default_rng(0)
    pairs = np.stack([rng.integers(0, SA.n, 300), rng.integers(0, SB.n, 300)], axis=1)
    out = tw.twed_batch(A, B, torch.as_tensor(pairs).cuda(), 1.0, 1.0, 2)
    got = out.cpu().numpy()
    ref = oracle_matrix(SA, SB, 1.0, 1.0, 2, pairs)
    assert rel(got, ref).max() <= 1e-5


def test_host_allpairs_equals_plan(tw):
    import torch
    S = W.set_w3(nseries=40, len_lo=64, len_hi=512).astype(np.float32)
    host = tw.twed_allpairs_host_f32(S.vals, S.ts, S.offs, None, 0.5, 0.5, 2)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    dev = tw.Plan(D, None, 0.5, 0.5, 2).execute().cpu().numpy()
    assert np.array_equal(host, dev)


def test_w3_recipe_small_matches_oracle(tw):
    # the 4096-series dim-8 recipe at 64 series, all pairs against the oracle
    import torch
    S = W.set_w3(nseries=64).astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    M = tw.Plan(D, None, 0.5, 0.5, 2).execute().cpu().numpy()
    pairs = W.sample_upper_pairs(S.n, 400, 3)
    ref = oracle_matrix(S, S, 0.5, 0.5, 2, pairs)
    assert rel(M[pairs[:, 0], pairs[:, 1]], ref).max() <= 1e-5


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_autotuned_plan_matches_default_plan(tw, dtype):
    # the autotuner only changes the schedule (rows per lane, blocks per SM):
    # FP64 stays bit-identical, FP32 within rounding of the reordered strips
    import torch
    S = W.set_w3(nseries=40, len_lo=20, len_hi=700)
    td = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        S = S.astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, td)
    base = tw.Plan(D, None, 0.5, 0.5, 2).execute().cpu().numpy()
    tuned_plan = tw.Plan(D, None, 0.5, 0.5, 2, opts=tw.make_opts(autotune=1))
    tuned = tuned_plan.execute().cpu().numpy()
    assert "autotuned" in tuned_plan.describe()
    if dtype == "f64":
        np.testing.assert_array_equal(tuned, base)
    else:
        np.testing.assert_allclose(tuned, base, rtol=1e-6)


def _mixed_set(seed, nshort, nlong, dim=3):
    rng = np.random.default_rng(seed)
    lens = list(rng.integers(20, 80, size=nshort)) + list(rng.integers(3000, 4000, size=nlong))
    rng.shuffle(lens)
    series = [(np.cumsum(rng.normal(size=(n, dim)), axis=0), np.cumsum(rng.exponential(1.0, n)))
              for n in lens]
    return W.pack(series)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_plan_cutover_for_long_pairs(tw, dtype):
    # a few long series among short ones: their pairs exceed a warp's share of
    # the plan and run on the one-pair block-cooperative schedule
    import torch
    S = _mixed_set(21, 46, 4)
    SB = _mixed_set(22, 20, 3)
    td = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        S, SB = S.astype(np.float32), SB.astype(np.float32)
    for B in (None, SB):
        D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, td)
        DB = None if B is None else tw.DeviceSet.from_numpy(B.vals, B.ts, B.offs, td)
        plan = tw.Plan(D, DB, 0.3, 0.7, 2)
        assert "cut-over" in plan.describe(), plan.describe()
        M = plan.execute().cpu().numpy()
        Bo = S if B is None else B
        pairs = np.array([(i, j) for i in range(S.n) for j in range(Bo.n) if B is not None or i < j])
        want = oracle.twed_pairs(S.astype(np.float64).as_tuple(), Bo.astype(np.float64).as_tuple(),
                                 pairs, 0.3, 0.7, 2)
        got = M[pairs[:, 0], pairs[:, 1]].astype(np.float64)
        if dtype == "f64":
            np.testing.assert_array_equal(got, want)
        else:
            np.testing.assert_allclose(got, want, rtol=1e-5)
        if B is None:
            assert np.all(M == M.T) and np.all(np.diag(M) == 0)
        plan.close()


@pytest.mark.parametrize("dtype,dim,p,order", [(np.float64, 1, 2, 1), (np.float64, 3, 1, 1),
                                               (np.float32, 4, 2, 1), (np.float32, 2, 2, 1),
                                               (np.float32, 3, 2, 0)])
def test_explicit_pairs_run_orders(tw, dtype, dim, p, order):
    """More pairs than resident warps, so the longest-first order goes
    through the device counting sort; every result must still land at its
    own pair's position (FP64: bit-exact with the oracle).  The list holds
    repeated pairs, 1-point series and cell counts from 1 to 4e5, so many
    size classes are populated."""
    import torch
    rng = np.random.default_rng(dim * 7 + p)

    def series(n):
        return np.cumsum(rng.normal(size=(n, dim)), axis=0), np.cumsum(rng.exponential(1.0, n))

    # series 0 of each set has one point
    SA = W.pack([series(1)] + [series(int(n)) for n in rng.integers(2, 641, 59)]).astype(dtype)
    SB = W.pack([series(1)] + [series(int(n)) for n in rng.integers(2, 641, 44)]).astype(dtype)
    tdt = torch.float64 if dtype == np.float64 else torch.float32
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, tdt)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, tdt)
    npairs = 9000
    pairs = np.stack([rng.integers(0, SA.n, npairs), rng.integers(0, SB.n, npairs)], axis=1)
    pairs[:50] = pairs[50:100]  # repeated pairs
    pairs[100:140, 0] = 0       # 1-point rows
    pairs[140:150] = 0          # 1 x 1
    out = tw.twed_batch(A, B, torch.as_tensor(pairs).cuda(), 0.7, 0.3, p, order=order)
    got = out.cpu().numpy()
    cells = SA.lengths[pairs[:, 0]].astype(np.int64) * SB.lengths[pairs[:, 1]]
    assert cells.min() == 1 and cells.max() > 100000
    ref = oracle_matrix(SA, SB, 0.7, 0.3, p, pairs)
    if dtype == np.float64:
        if p in (1, 2):
            assert np.array_equal(got, ref)
        else:
            assert rel(got, ref).max() <= 1e-12
    else:
        assert rel(got, ref).max() <= 1e-5
    assert np.array_equal(got[:50], got[50:100])


def test_explicit_pairs_unknown_order_rejected(tw):
    import torch
    S = ragged_set(5, 4, 3, 9, 2, np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    pairs = torch.zeros((3, 2), dtype=torch.int64, device="cuda")
    with pytest.raises(RuntimeError, match="unknown pair order"):
        tw.twed_batch(D, D, pairs, 1.0, 1.0, 2, order=2)
