"""GPU parity of the learned k-NN filter against the oracle in oracle/knn.py.

Tolerances (FP32 kernels against the float64 oracle on the same FP32 inputs):
* feature statistics: 1e-5 relative (FP64 sums of FP32 features);
* embeddings: 2e-4 of the series' largest |e| -- each convolution output sums
  320 FP32 products (worst-case relative error 320 u = 1.9e-5 of the summed
  magnitudes), three layers and a pool over up to 513 rows add up to about
  1e-4 of the magnitudes; 2e-4 leaves a factor of two;
* loss: 1e-4 relative; gradient blocks: 2e-3 of the block's largest |g| (the
  same sums, plus the adjoint and weight-gradient sums over every row);
* Adam: 1e-5 relative;
* row top-k and candidate search: bit-exact indices where the inputs fix the
  order (top-k of given values); for the search, every returned row lies
  within 1e-5 of the oracle's k-th distance and every row clearly inside it
  is returned.
Shapes span several 128-row convolution tiles with ragged tails, series of
length 1-3 (all 'same' padding) and input widths 8 and 16 (dim 4 and 8).
"""
import numpy as np
import pytest

import oracle
from oracle import knn as K
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


def make_set(rng, lens, dim):
    series = [(np.cumsum(rng.normal(size=(n, dim)), axis=0), np.arange(1, n + 1, dtype=np.float64))
              for n in lens]
    return W.pack(series).astype(np.float32)


def oracle_features(S, nu, lam, p):
    out = []
    for s in range(S.n):
        v, t = S.series(s)
        out.append(K.features(v.astype(np.float64), t.astype(np.float64), nu, lam, p))
    return out


def dev_set(tw, S):
    import torch
    return tw.DeviceSet.from_numpy(S.vals, S.ts, S.offs, torch.float32)


def rand_params(rng, dim, scale=0.15):
    return (rng.uniform(-1, 1, size=K.param_count(dim)) * scale).astype(np.float32)


LENS = [1, 2, 3, 5, 64, 127, 128, 129, 300, 513, 17, 255]


@pytest.mark.parametrize("dim,p", [(4, 2), (1, 2), (3, 1), (8, 2)])
def test_feature_stats(tw, dim, p):
    rng = np.random.default_rng(10 + dim + p)
    S = make_set(rng, LENS, dim)
    mu, sd = tw.encoder_stats(dev_set(tw, S), 0.7, 1.3, p)
    omu, osd = K.feature_stats(oracle_features(S, 0.7, 1.3, p))
    np.testing.assert_allclose(mu.cpu().numpy(), omu, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(sd.cpu().numpy(), osd, rtol=1e-5)


def forward_pair(tw, rng, dim, p, lens, mean_len=200.0):
    import torch
    S = make_set(rng, lens, dim)
    feats = oracle_features(S, 1.0, 1.0, p)
    omu, osd = K.feature_stats(feats)
    mu32, sd32 = omu.astype(np.float32), osd.astype(np.float32)
    w = rand_params(rng, dim)
    e = tw.encoder_forward(dev_set(tw, S), 1.0, 1.0, p, torch.as_tensor(w).cuda(),
                           torch.as_tensor(mu32).cuda(), torch.as_tensor(sd32).cuda(), mean_len)
    P = K.unpack(w.astype(np.float64), dim)
    want = np.array([K.forward(P, K.normalise(f, mu32.astype(np.float64), sd32.astype(np.float64)),
                               np.float32(mean_len))[0] for f in feats])
    return e.cpu().numpy(), want


@pytest.mark.parametrize("dim,p", [(4, 2), (1, 2), (8, 2), (3, 1)])
def test_encoder_forward(tw, dim, p):
    rng = np.random.default_rng(20 + dim)
    got, want = forward_pair(tw, rng, dim, p, LENS)
    for s in range(len(LENS)):
        scale = max(np.abs(want[s]).max(), 1e-3)
        assert np.abs(got[s] - want[s]).max() <= 2e-4 * scale, (s, LENS[s])


def test_encoder_forward_many_chunks(tw):
    # enough rows that the forward runs in more than one 2^22-row chunk
    rng = np.random.default_rng(5)
    lens = list(rng.integers(400, 513, size=12000))
    import torch
    S = make_set(rng, lens, 4)
    w = rand_params(rng, 4)
    mu = torch.zeros(6, device="cuda")
    sd = torch.ones(6, device="cuda")
    e = tw.encoder_forward(dev_set(tw, S), 1.0, 1.0, 2, torch.as_tensor(w).cuda(), mu, sd, 300.0)
    e = e.cpu().numpy()
    P = K.unpack(w.astype(np.float64), 4)
    for s in [0, 1, 4000, 9000, 9100, 9200, 11999]:
        v, t = S.series(s)
        f = K.features(v.astype(np.float64), t.astype(np.float64), 1.0, 1.0, 2)
        want = K.forward(P, f, 300.0)[0]
        assert np.abs(e[s] - want).max() <= 2e-4 * max(np.abs(want).max(), 1e-3), s


@pytest.mark.parametrize("gsize,ngroups", [(4, 3), (2, 5), (32, 1)])
def test_loss_and_gradient(tw, gsize, ngroups):
    import torch
    rng = np.random.default_rng(30 + gsize)
    nser = max(gsize * ngroups, 12)
    lens = list(rng.integers(1, 300, size=nser))
    lens[0], lens[1] = 1, 129
    S = make_set(rng, lens, 4)
    feats = oracle_features(S, 1.0, 1.0, 2)
    omu, osd = K.feature_stats(feats)
    mu32, sd32 = omu.astype(np.float32), osd.astype(np.float32)
    w = rand_params(rng, 4, scale=0.1)
    groups = rng.permutation(nser)[:gsize * ngroups].reshape(ngroups, gsize)
    npg = gsize * (gsize - 1) // 2
    labels = rng.uniform(0.5, 2.0, size=(ngroups, npg)).astype(np.float32)
    inv_sigma = np.float32(0.8)
    mean_len = np.float32(150.0)
    loss, grad = tw.encoder_loss_grad(dev_set(tw, S), 1.0, 1.0, 2, torch.as_tensor(w).cuda(),
                                      torch.as_tensor(mu32).cuda(), torch.as_tensor(sd32).cuda(),
                                      mean_len, groups, torch.as_tensor(labels).cuda(), inv_sigma)
    xs = [K.normalise(f, mu32.astype(np.float64), sd32.astype(np.float64)) for f in feats]
    P = K.unpack(w.astype(np.float64), 4)
    oloss, og = K.loss_and_grad(P, xs, groups, labels.astype(np.float64), float(inv_sigma),
                                float(mean_len))
    assert abs(loss.item() - oloss) <= 1e-4 * abs(oloss)
    got = K.unpack(grad.cpu().numpy().astype(np.float64), 4)
    for name in og:
        scale = np.abs(og[name]).max()
        assert np.abs(got[name] - og[name]).max() <= 2e-3 * scale, name


def test_adam(tw):
    import torch
    rng = np.random.default_rng(40)
    n = 1000
    th = rng.normal(size=n).astype(np.float32)
    m = np.zeros(n)
    v = np.zeros(n)
    tht, mt, vt = (torch.as_tensor(x, dtype=torch.float32).cuda() for x in (th, m, v))
    oth = th.astype(np.float64)
    for step in (1, 2, 3):
        g = rng.normal(size=n).astype(np.float32)
        tw.adam_step(tht, torch.as_tensor(g).cuda(), mt, vt, step, 1e-2)
        oth, m, v = K.adam(oth, g.astype(np.float64), m, v, step, 1e-2)
    np.testing.assert_allclose(tht.cpu().numpy(), oth, rtol=1e-5, atol=1e-6)


@pytest.mark.parametrize("rows,cols,k", [(5, 1, 1), (3, 31, 7), (4, 1024, 200), (2, 1025, 1025),
                                         (3, 5000, 4096), (2, 100000, 10), (1, 100000, 200),
                                         (40, 2000, 33)])
def test_topk_rows_bitexact_with_ties(tw, rows, cols, k):
    import torch
    rng = np.random.default_rng(rows * 7 + cols + k)
    # few distinct values -> many ties; negative and positive, no -0.0
    D = (rng.integers(-50, 50, size=(rows, cols)) * 0.25).astype(np.float32)
    D[D == 0] = 0.0
    idx, val = tw.topk_rows(torch.as_tensor(D).cuda(), k)
    want_i, want_v = K.topk_rows(D, k)
    np.testing.assert_array_equal(idx.cpu().numpy(), want_i)
    np.testing.assert_array_equal(val.cpu().numpy(), want_v.astype(np.float32))


def test_topk_rows_with_leading_dimension(tw):
    import torch
    rng = np.random.default_rng(3)
    D = rng.normal(size=(6, 700)).astype(np.float32)
    idx, val = tw.topk_rows(torch.as_tensor(D).cuda(), 50, cols=500)
    want_i, want_v = K.topk_rows(D[:, :500], 50)
    np.testing.assert_array_equal(idx.cpu().numpy(), want_i)
    np.testing.assert_array_equal(val.cpu().numpy(), want_v)


@pytest.mark.parametrize("ndb,nq,k", [(5000, 7, 200), (300, 3, 300), (1000, 40, 1)])
def test_embed_search(tw, ndb, nq, k):
    import torch
    rng = np.random.default_rng(ndb + nq + k)
    db = rng.normal(size=(ndb, 32)).astype(np.float32)
    q = rng.normal(size=(nq, 32)).astype(np.float32)
    idx, val = tw.embed_search(torch.as_tensor(db).cuda(), torch.as_tensor(q).cuda(), k)
    idx, val = idx.cpu().numpy(), val.cpu().numpy()
    sdb, sq = K.search_rows(db, q)
    D = K.sq_l2(sq, sdb)
    for i in range(nq):
        order = np.sort(D[i])
        kth = order[k - 1]
        tol = 1e-5 * max(kth, 1.0)
        assert len(set(idx[i].tolist())) == k
        assert np.all(D[i, idx[i]] <= kth + tol)
        inside = np.nonzero(D[i] < kth - tol)[0]
        assert set(inside.tolist()) <= set(idx[i].tolist())
        np.testing.assert_allclose(val[i], D[i, idx[i]], rtol=1e-5, atol=1e-5)
        assert np.all(np.diff(val[i]) >= 0)


# ---------------------------------------------------------------- the index
@pytest.fixture(scope="module")
def small_index(tw):
    import torch
    db = W.set_w5(600, stream=1).astype(np.float32)
    qs = W.set_w5(8, stream=0).astype(np.float32)
    cfg = tw.knn_config(group_size=16, groups_per_step=8, epochs=4, train_pairs=12000, seed=7)
    D = dev_set(tw, db)
    index = tw.KnnIndex(D, 1.0, 1.0, 2, config=cfg)
    stats = index.train()
    # exact distances from the oracle for every (query, database) pair
    pairs = np.array([(q, x) for q in range(qs.n) for x in range(db.n)], dtype=np.int64)
    want = oracle.twed_pairs((qs.vals, qs.ts, qs.offs), (db.vals, db.ts, db.offs), pairs, 1.0, 1.0,
                             2).reshape(qs.n, db.n)
    return index, db, qs, dev_set(tw, qs), stats, want


def test_training_reduces_loss(small_index):
    _, _, _, _, stats, _ = small_index
    assert stats["steps"] > 0
    assert stats["label_pairs"] >= 12000
    assert stats["last_loss"] < stats["first_loss"]


def test_index_embeddings_match_oracle_forward(tw, small_index):
    index, db, _, _, _, _ = small_index
    w = index.params().astype(np.float64)
    e = index.embeddings().cpu().numpy()
    feats = oracle_features(db, 1.0, 1.0, 2)
    omu, osd = K.feature_stats(feats)
    P = K.unpack(w, 4)
    mean_len = np.float32(db.lengths.mean())
    for s in [0, 17, 599]:
        x = K.normalise(feats[s], omu.astype(np.float32).astype(np.float64),
                        osd.astype(np.float32).astype(np.float64))
        want = K.forward(P, x, float(mean_len))[0]
        assert np.abs(e[s] - want).max() <= 2e-4 * max(np.abs(want).max(), 1e-3), s


def test_exact_knn_matches_oracle(tw, small_index):
    index, db, qs, Q, _, want = small_index
    idx, dist = index.exact(Q, k=10)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    for q in range(qs.n):
        kth = np.sort(want[q])[9]
        np.testing.assert_allclose(dist[q], want[q, idx[q]], rtol=1e-5)
        assert np.all(want[q, idx[q]] <= kth * (1 + 1e-5))
        inside = np.nonzero(want[q] < kth * (1 - 1e-5))[0]
        assert set(inside.tolist()) <= set(idx[q].tolist())


def test_search_distances_are_exact_and_bounded_by_exact_knn(tw, small_index):
    index, db, qs, Q, _, want = small_index
    idx, dist = index.search(Q, k=10, n_candidates=100)
    ex_idx, ex_dist = index.exact(Q, k=10)
    idx, dist, ex_dist = idx.cpu().numpy(), dist.cpu().numpy(), ex_dist.cpu().numpy()
    for q in range(qs.n):
        np.testing.assert_allclose(dist[q], want[q, idx[q]], rtol=1e-5)
        assert np.all(np.diff(dist[q]) >= 0)
        assert np.all(dist[q] >= ex_dist[q] * (1 - 1e-6))


def test_search_with_every_candidate_equals_exact(tw, small_index):
    # all database rows as candidates: the re-rank sees every pair, so it
    # must find the exact k-NN (the explicit-pair and all-pairs launches may
    # round the last FP32 bit differently, hence the 1e-6 band)
    index, db, _, Q, _, _ = small_index
    idx, dist = index.search(Q, k=10, n_candidates=db.n)
    ex_idx, ex_dist = index.exact(Q, k=10)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    ex_idx, ex_dist = ex_idx.cpu().numpy(), ex_dist.cpu().numpy()
    np.testing.assert_allclose(dist, ex_dist, rtol=1e-6)
    for q in range(idx.shape[0]):
        clear = np.abs(dist[q] - ex_dist[q][-1]) > 1e-6 * ex_dist[q][-1]
        assert set(idx[q][clear].tolist()) <= set(ex_idx[q].tolist())


def test_rerank_launch_shape_is_timed(tw, small_index):
    _, _, _, _, stats, _ = small_index
    assert stats["rerank_rows_per_lane"] in (2, 4, 6, 8)
    assert stats["rerank_blocks_per_sm"] >= 1
    assert stats["tune_ms"] > 0


def test_fresh_index_from_params_searches_alike(tw, small_index):
    # set_params on an untrained index embeds the database and times the
    # re-rank shape itself; the search must give the trained index's answer
    # (the value of a pair does not depend on the launch shape)
    index, db, _, Q, _, _ = small_index
    cfg = tw.knn_config(group_size=16, groups_per_step=8, epochs=4, train_pairs=12000, seed=7)
    other = tw.KnnIndex(dev_set(tw, db), 1.0, 1.0, 2, config=cfg)
    other.set_params(index.params())
    st = other.stats()
    assert st["rerank_rows_per_lane"] in (2, 4, 6, 8) and st["tune_ms"] > 0
    i0, d0 = index.search(Q, k=10, n_candidates=64)
    i1, d1 = other.search(Q, k=10, n_candidates=64)
    np.testing.assert_array_equal(i0.cpu().numpy(), i1.cpu().numpy())
    np.testing.assert_allclose(d0.cpu().numpy(), d1.cpu().numpy(), rtol=1e-6)
    other.close()


def test_set_params_reembeds(tw, small_index):
    index, db, _, _, _, _ = small_index
    w = index.params()
    e0 = index.embeddings().cpu().numpy()
    index.set_params(w)
    e1 = index.embeddings().cpu().numpy()
    np.testing.assert_array_equal(e0, e1)


@pytest.mark.parametrize("bad", ["k0", "k_gt_c", "c_gt_n"])
def test_search_rejects_bad_sizes(tw, small_index, bad):
    index, db, _, Q, _, _ = small_index
    k, c = {"k0": (0, 10), "k_gt_c": (20, 10), "c_gt_n": (10, db.n + 1)}[bad]
    with pytest.raises(tw.TwedError) as ei:
        index.search(Q, k=max(k, 1) if bad != "k0" else 0, n_candidates=c)
    assert ei.value.status == tw.TWED_ERR_INVALID_ARG


def test_search_host_matches_device_search(tw, small_index):
    index, db, qs, Q, _, _ = small_index
    idx, dist = index.search(Q, k=5, n_candidates=64)
    hidx, hdist = index.search_host(qs.vals, qs.ts, qs.offs, k=5, n_candidates=64)
    np.testing.assert_array_equal(hidx, idx.cpu().numpy())
    np.testing.assert_array_equal(hdist, dist.cpu().numpy())


def test_search_profile_counts_rerank_cells(tw, small_index):
    index, db, qs, Q, _, _ = small_index
    index.search(Q, k=3, n_candidates=db.n)
    ms, cells = index.search_profile()
    assert cells == int(qs.lengths.sum()) * int(db.lengths.sum())
    assert all(m >= 0 for m in ms) and ms[2] > 0


def test_pipe_peaks_are_plausible(tw):
    import torch
    props = torch.cuda.get_device_properties(0)
    nominal = props.multi_processor_count * 128 * 2.1e9  # FFMA lanes x a clock above max
    f32 = tw.pipe_peak(tw.PEAK_FFMA32)
    f64 = tw.pipe_peak(tw.PEAK_DFMA64)
    assert 0.2 * nominal < f32 < nominal
    assert 0 < f64 < f32


def test_training_with_mined_groups(tw):
    # half of the labelled pairs from mined groups (an anchor and its nearest
    # series under the half-trained model): every pair is labelled exactly and
    # the index still searches correctly
    import torch
    db = W.set_w5(400, stream=1).astype(np.float32)
    qs = W.set_w5(4, stream=0).astype(np.float32)
    cfg = tw.knn_config(group_size=8, groups_per_step=8, epochs=4, train_pairs=4000,
                        mine_fraction=0.5, seed=3)
    index = tw.KnnIndex(dev_set(tw, db), 1.0, 1.0, 2, config=cfg)
    stats = index.train()
    assert stats["mined_pairs"] > 0 and stats["label_pairs"] > stats["mined_pairs"]
    idx, dist = index.search(dev_set(tw, qs), k=3, n_candidates=50)
    idx, dist = idx.cpu().numpy(), dist.cpu().numpy()
    pairs = np.array([(q, int(x)) for q in range(qs.n) for x in idx[q]])
    want = oracle.twed_pairs(qs.astype(np.float64).as_tuple(), db.astype(np.float64).as_tuple(),
                             pairs, 1.0, 1.0, 2).reshape(qs.n, 3)
    np.testing.assert_allclose(dist, want, rtol=1e-5)
    index.close()
