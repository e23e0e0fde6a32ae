"""Tensor-core cross term (dim 64, p = 2, TF32 inputs, FP32 accumulation).

The cell cost uses |a_i - b_j|^2 = |a_i|^2 + |b_j|^2 - 2 a_i . b_j with the
dot products on the tensor cores.  TF32 keeps 10 mantissa bits of each
input, so every cost carries about 1e-4 relative error; the test bounds the
TWED error at 2e-3 relative and checks that the CUDA-core FP32 path on the
same inputs stays within the 1e-5 FP32 bound.  Lengths straddle the 64-row
strips (two rows per lane) and the 16-column tiles (1, 15, 16, 17, 63, 64,
65, 127, 128, 129, ...); further cases cover more row series than one work
item holds (64), the symmetric plan's per-chunk items, and column series
longer than 1024 points (the boundary rows stream through global memory).
"""
import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LENGTHS_A = [1, 15, 16, 17, 63, 64, 65, 127, 128, 129, 300, 257]
LENGTHS_B = [1, 16, 33, 128, 200, 255, 256, 513]


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


def smoothed_set(seed, lengths):
    rng = np.random.default_rng(seed)
    out = []
    for n in lengths:
        raw = rng.standard_normal((n + 4, 64))
        c = np.cumsum(np.vstack([np.zeros((1, 64)), raw]), axis=0)
        out.append(((c[5:] - c[:-5]) / 5.0, np.arange(1, n + 1, dtype=np.float64)))
    return W.pack(out).astype(np.float32)


def matrix(tw, SA, SB, xterm, nu=1.0, lam=1.0):
    import torch
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32) if SB is not None else None
    plan = tw.Plan(A, B, nu, lam, 2, opts=tw.make_opts(xterm=xterm))
    M = plan.execute().cpu().numpy()
    plan.status()
    return M, plan.describe()


def oracle_block(SA, SB):
    pairs = np.array([(i, j) for i in range(SA.n) for j in range(SB.n)])
    A64, B64 = SA.astype(np.float64), SB.astype(np.float64)
    return oracle.twed_pairs(A64.as_tuple(), B64.as_tuple(), pairs, 1.0, 1.0, 2).reshape(SA.n, SB.n)


def test_tensor_core_block_matches_oracle(tw):
    SA, SB = smoothed_set(1, LENGTHS_A), smoothed_set(2, LENGTHS_B)
    ref = oracle_block(SA, SB)
    Mx, desc = matrix(tw, SA, SB, tw.XTERM_TF32)
    assert "tensor-core" in desc
    rel = np.abs(Mx - ref) / ref
    print(f"tensor-core cross term: max rel err {rel.max():.3e}, mean {rel.mean():.3e}")
    assert rel.max() <= 2e-3
    Mc, _ = matrix(tw, SA, SB, tw.XTERM_OFF)
    assert (np.abs(Mc - ref) / ref).max() <= 1e-5


def test_tensor_core_symmetric_plan(tw):
    S = smoothed_set(3, [40, 129, 1, 256, 17, 90, 300])
    Mx, _ = matrix(tw, S, None, tw.XTERM_TF32)
    ref = oracle_block(S, S)
    iu = np.triu_indices(S.n, 1)
    assert (np.abs(Mx[iu] - ref[iu]) / ref[iu]).max() <= 2e-3
    assert np.array_equal(Mx, Mx.T) and np.all(np.diag(Mx) == 0)


def test_tensor_core_refuses_other_shapes(tw):
    import torch
    S = smoothed_set(4, [20, 30])
    V = S.vals[:, :32].copy()
    D = tw.DeviceSet.from_numpy(V, S.ts, S.offs, torch.float32)
    with pytest.raises(tw.TwedError) as ei:
        tw.Plan(D, None, 1.0, 1.0, 2, opts=tw.make_opts(xterm=tw.XTERM_TF32))
    assert ei.value.status == tw.TWED_ERR_UNSUPPORTED


def test_w4_full_size_sampled(tw):
    # 2048 x 2048 series, dim 64, lengths U[256, 1024]: the bench's launch
    # configuration; 64 sampled pairs against the FP64 oracle
    import torch
    SA = W.set_w4(stream=0).astype(np.float32)
    SB = W.set_w4(stream=1).astype(np.float32)
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    plan = tw.Plan(A, B, 1.0, 1.0, 2, opts=tw.make_opts(xterm=tw.XTERM_TF32))
    M = plan.execute()
    plan.status()
    pairs = W.sample_block_pairs(SA.n, SB.n, 64, 4)
    got = M[torch.as_tensor(pairs[:, 0]).cuda(), torch.as_tensor(pairs[:, 1]).cuda()].cpu().numpy()
    A64, B64 = SA.astype(np.float64), SB.astype(np.float64)
    ref = oracle.twed_pairs(A64.as_tuple(), B64.as_tuple(), pairs, 1.0, 1.0, 2)
    rel = np.abs(got - ref) / ref
    print(f"w4 full size, 64 sampled pairs: max rel err {rel.max():.3e}")
    assert rel.max() <= 2e-3


def test_tensor_core_many_rows_long_columns(tw):
    # 150 row series (three work items per column series, uneven strip
    # counts per consumer warp) against columns of 1 .. 2100 points
    rng = np.random.default_rng(11)
    SA = smoothed_set(5, [int(v) for v in rng.integers(1, 200, 150)])
    SB = smoothed_set(6, [1, 17, 1100, 2100, 64, 1025])
    ref = oracle_block(SA, SB)
    Mx, _ = matrix(tw, SA, SB, tw.XTERM_TF32)
    rel = np.abs(Mx - ref) / ref
    print(f"many rows, long columns: max rel err {rel.max():.3e}")
    assert np.all(np.isfinite(Mx)) and rel.max() <= 2e-3


def test_tensor_core_symmetric_several_chunks(tw):
    # 140 series: three chunks of rows, including the items on the diagonal
    # of the triangle whose rows are only part of a chunk
    rng = np.random.default_rng(12)
    S = smoothed_set(7, [int(v) for v in rng.integers(1, 160, 140)])
    Mx, _ = matrix(tw, S, None, tw.XTERM_TF32)
    ref = oracle_block(S, S)
    iu = np.triu_indices(S.n, 1)
    rel = np.abs(Mx[iu] - ref[iu]) / ref[iu]
    print(f"symmetric, 140 series: max rel err {rel.max():.3e}")
    assert rel.max() <= 2e-3
    assert np.array_equal(Mx, Mx.T) and np.all(np.diag(Mx) == 0)


def test_tensor_core_reexecute_is_stable(tw):
    # the kernel keeps no state between executes: the same plan twice gives
    # the same matrix bit for bit
    import torch
    SA, SB = smoothed_set(8, [90, 33, 200]), smoothed_set(9, [70, 5, 400])
    A = tw.DeviceSet.from_numpy(SA.vals, SA.ts, SA.offs, torch.float32)
    B = tw.DeviceSet.from_numpy(SB.vals, SB.ts, SB.offs, torch.float32)
    plan = tw.Plan(A, B, 1.0, 1.0, 2, opts=tw.make_opts(xterm=tw.XTERM_TF32))
    M1 = plan.execute().cpu().numpy()
    plan.status()
    M2 = plan.execute().cpu().numpy()
    plan.status()
    assert np.array_equal(M1, M2)


# BF16 inputs (TWED_XTERM_BF16): 8 significant bits, so a rounded point is
# within 2^-9 of each component; d^2 of the rounded points (exact up to FP32
# summation, the norms being those of the rounded points) differs from the
# true d^2 by at most 2 |a - b| |da - db|, about 2^-7 d^2 when |a - b| is of the
# order of |a| and |b| -- a cost within about 0.4%; the bound on the TWED is
# 1e-2 relative.
def test_bf16_block_matches_oracle(tw):
    SA, SB = smoothed_set(1, LENGTHS_A), smoothed_set(2, LENGTHS_B)
    ref = oracle_block(SA, SB)
    Mb, desc = matrix(tw, SA, SB, tw.XTERM_BF16)
    assert "tensor-core" in desc
    rel = np.abs(Mb - ref) / ref
    print(f"BF16 cross term: max rel err {rel.max():.3e}, mean {rel.mean():.3e}")
    assert rel.max() <= 1e-2
    Mt, _ = matrix(tw, SA, SB, tw.XTERM_TF32)
    assert (np.abs(Mt - ref) / ref).max() <= 2e-3


def test_bf16_symmetric_plan(tw):
    S = smoothed_set(3, [40, 129, 1, 256, 17, 90, 300, 1100])
    Mb, _ = matrix(tw, S, None, tw.XTERM_BF16)
    ref = oracle_block(S, S)
    iu = np.triu_indices(S.n, 1)
    assert (np.abs(Mb[iu] - ref[iu]) / ref[iu]).max() <= 1e-2
    assert np.array_equal(Mb, Mb.T) and np.all(np.diag(Mb) == 0)
