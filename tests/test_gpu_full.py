"""Full-size GPU parity in the launch configurations bench.py times.

* w2 (one 3-D pair, n = m = 1e5): FP64 must equal the stored FP64 oracle
  value bit for bit; compensated FP32 must be within 1e-6 of the oracle on
  the same FP32-rounded inputs; plain FP32 is reported and bounded by 1e-4
  (its sums along ~2e5-step paths drift, which is why long pairs default to
  the compensated mode).  The stored values come from
  tests/golden/make_w2_expected.py, which calls only the oracle.
* w3 (4096 series, dim 8, all 8.4M pairs in one plan execute): 300 sampled
  pairs against the oracle, plus symmetry and the zero diagonal.
* w5 (1e5-series database, 1000 queries, the bench's training and search
  configuration): the exact batched k-NN's distances against the oracle on
  sampled (query, result) pairs, the filtered search's recall@10 at 1600
  candidates against that exact k-NN, and its returned distances against
  the oracle on sampled pairs.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2007_16135_gb300 import workloads as W

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(__file__), "golden", "w2_oracle.json")


@pytest.fixture(scope="module")
def tw():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a GPU")
    from paper_2007_16135_gb300 import twed
    twed.load()
    return twed


@pytest.fixture(scope="module")
def w2():
    with open(GOLD) as f:
        gold = json.load(f)
    return gold, W.pair_w2(gold["n"])


def _dev(x, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x)).to(dtype).cuda()


def test_w2_full_f64_bitwise(tw, w2):
    import torch
    gold, (a, ta, b, tb) = w2
    out = tw.twed_dev(_dev(a, torch.float64), _dev(ta, torch.float64), _dev(b, torch.float64),
                      _dev(tb, torch.float64), 0.001, 1.0, 2)
    torch.cuda.synchronize()
    tw.default_handle().sync_status()
    assert out.item() == gold["f64_inputs"]


@pytest.mark.parametrize("accum,bound", [("kahan", 1e-6), ("f32", 1e-4)])
def test_w2_full_f32(tw, w2, accum, bound):
    import torch
    gold, (a, ta, b, tb) = w2
    acc = tw.ACCUM_KAHAN if accum == "kahan" else tw.ACCUM_F32
    out = tw.twed_dev(_dev(a, torch.float32), _dev(ta, torch.float32), _dev(b, torch.float32),
                      _dev(tb, torch.float32), 0.001, 1.0, 2, opts=tw.make_opts(accum=acc))
    torch.cuda.synchronize()
    tw.default_handle().sync_status()
    want = gold["f32_rounded_inputs"]
    err = abs(out.item() - want) / want
    print(f"w2 1e5 FP32 {accum}: rel err {err:.3e}")
    assert err <= bound


def test_w3_full_size_sampled(tw):
    import torch
    S = W.set_w3(nseries=4096).astype(np.float32)
    D = tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)
    plan = tw.Plan(D, None, 0.5, 0.5, 2)
    M = plan.execute()
    torch.cuda.synchronize()
    pairs = W.sample_upper_pairs(S.n, 300, 3)
    got = M[torch.as_tensor(pairs[:, 0]).cuda(), torch.as_tensor(pairs[:, 1]).cuda()].cpu().numpy()
    S64 = S.astype(np.float64)
    ref = oracle.twed_pairs(S64.as_tuple(), S64.as_tuple(), pairs, 0.5, 0.5, 2)
    rel = np.abs(got - ref) / ref
    assert rel.max() <= 1e-5, rel.max()
    idx = torch.arange(0, S.n, 97, device="cuda")
    sub = M[idx][:, idx]
    assert torch.equal(sub, sub.T)
    assert torch.all(torch.diagonal(M) == 0)


def test_w5_full_size_knn(tw):
    import torch
    db = W.set_w5(100_000, stream=1).astype(np.float32)
    qs = W.set_w5(1000, stream=0).astype(np.float32)
    D = tw.DeviceSet.from_numpy(db.vals, db.ts, db.offs, torch.float32)
    Q = tw.DeviceSet.from_numpy(qs.vals, qs.ts, qs.offs, torch.float32)
    index = tw.KnnIndex(D, 1.0, 1.0, 2, config=tw.knn_config())
    index.train()
    ex_idx, ex_dist = index.exact(Q, k=10)
    idx, dist = index.search(Q, k=10, n_candidates=1600)
    torch.cuda.synchronize()
    ex_idx, ex_dist = ex_idx.cpu().numpy(), ex_dist.cpu().numpy()
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    kth = ex_dist[:, 9]
    recall = np.minimum((dist <= kth[:, None]).sum(axis=1), 10).mean() / 10
    assert recall >= 0.99, recall
    # sampled distances of both paths against the oracle
    rng = np.random.default_rng(55)
    qsel = rng.choice(qs.n, size=12, replace=False)
    pairs, got = [], []
    for q in qsel:
        for r in (0, 9):
            pairs.append((q, ex_idx[q, r]))
            got.append(ex_dist[q, r])
            pairs.append((q, idx[q, r]))
            got.append(dist[q, r])
    want = oracle.twed_pairs(qs.astype(np.float64).as_tuple(), db.astype(np.float64).as_tuple(),
                             np.array(pairs, dtype=np.int64), 1.0, 1.0, 2)
    rel = np.abs(np.array(got, dtype=np.float64) - want) / want
    assert rel.max() <= 1e-5, rel.max()
    # the exact path's top-10 are no worse than the filtered ones, rank by rank
    assert np.all(ex_dist <= dist * (1 + 1e-6))
    index.close()
