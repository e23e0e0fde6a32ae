"""Pins for the learned k-NN oracle (``oracle/knn.py``).

Each check ties the oracle to something other than itself: PyTorch's own
conv1d / autograd / Adam in float64 (independent library implementations of
the same definitions), the C TWED oracle's delete costs, adjoint identities,
finite differences, closed forms and hand-worked selections with ties.
"""
import numpy as np
import pytest

import oracle
from oracle import knn as K

torch = pytest.importorskip("torch")


def rand_params(rng, dim, scale=0.2):
    p = {}
    for name, shape in K.param_shapes(dim):
        p[name] = rng.normal(scale=scale, size=shape)
    return p


def torch_forward(params, x, mean_len):
    """Independent float64 statement with torch's conv1d (padding 2)."""
    F = torch.nn.functional
    t = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    h = torch.tensor(x.T[None], dtype=torch.float64)
    for i in (1, 2, 3):
        h = F.relu(F.conv1d(h, t[f"W{i}"], t[f"b{i}"], padding=2))
    e = t["Wl"] @ (h[0].sum(dim=1) / mean_len) + t["bl"]
    return e, t


def test_conv_same_matches_torch_conv1d():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(37, 6))
    W = rng.normal(size=(64, 6, 5))
    b = rng.normal(size=64)
    got = K.conv_same(x, W, b)
    want = torch.nn.functional.conv1d(torch.tensor(x.T[None]), torch.tensor(W), torch.tensor(b),
                                      padding=2)[0].numpy().T
    np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3, 5, 40])
def test_forward_matches_torch(L):
    rng = np.random.default_rng(L)
    params = rand_params(rng, 4)
    x = rng.normal(size=(L, 6))
    e, _ = K.forward(params, x, 17.0)
    want, _ = torch_forward(params, x, 17.0)
    np.testing.assert_allclose(e, want.detach().numpy(), rtol=1e-11, atol=1e-12)


def test_transpose_is_the_adjoint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(23, 64))
    y = rng.normal(size=(23, 64))
    W = rng.normal(size=(64, 64, 5))
    lhs = np.sum(K.conv_same(x, W, np.zeros(64)) * y)
    rhs = np.sum(x * K.conv_same_transpose(y, W))
    assert abs(lhs - rhs) <= 1e-10 * abs(lhs)


def test_wgrad_is_the_derivative_of_the_inner_product():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(19, 6))
    y = rng.normal(size=(19, 64))
    W = rng.normal(size=(64, 6, 5))
    g = K.conv_same_wgrad(x, y)
    # <conv(x, W), y> is linear in W, so its gradient is exact under any step
    f = lambda W_: np.sum(K.conv_same(x, W_, np.zeros(64)) * y)
    for (o, c, k) in [(0, 0, 0), (5, 3, 4), (63, 5, 2)]:
        E = np.zeros_like(W)
        E[o, c, k] = 1.0
        assert abs((f(W + E) - f(W)) - g[o, c, k]) <= 1e-9 * (1 + abs(g[o, c, k]))


def make_series(rng, lens, dim=4):
    xs = []
    for n in lens:
        v = np.cumsum(rng.normal(size=(n, dim)), axis=0)
        t = np.arange(1, n + 1, dtype=np.float64)
        xs.append(K.features(v, t, 1.0, 1.0, 2))
    mu, sd = K.feature_stats(xs)
    return [K.normalise(f, mu, sd) for f in xs]


def torch_group_loss(params, xs, groups, labels, inv_sigma, mean_len):
    ts = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in params.items()}
    F = torch.nn.functional
    emb = {}
    for s in sorted(set(np.asarray(groups).ravel().tolist())):
        h = torch.tensor(xs[s].T[None], dtype=torch.float64)
        for i in (1, 2, 3):
            h = F.relu(F.conv1d(h, ts[f"W{i}"], ts[f"b{i}"], padding=2))
        emb[s] = ts["Wl"] @ (h[0].sum(dim=1) / mean_len) + ts["bl"]
    loss, n = 0.0, 0
    for gi, grp in enumerate(groups):
        for pi, (a, b) in enumerate(K.group_pairs(len(grp))):
            ea, eb = emb[int(grp[a])], emb[int(grp[b])]
            model = ((ea[:31] - eb[:31]) ** 2).sum() + ea[31] + eb[31]
            loss = loss + (model - labels[gi][pi] * inv_sigma) ** 2
            n += 1
    loss = loss / n
    loss.backward()
    return loss.item(), {k: v.grad.numpy() for k, v in ts.items()}


def test_loss_and_grad_match_torch_autograd():
    rng = np.random.default_rng(3)
    xs = make_series(rng, [7, 12, 5, 30, 9, 16])
    params = rand_params(rng, 4, scale=0.3)
    groups = [[0, 3, 5], [1, 2, 4]]
    labels = rng.uniform(1, 3, size=(2, 3))
    loss, grad = K.loss_and_grad(params, xs, groups, labels, 0.7, 12.0)
    tl, tg = torch_group_loss(params, xs, groups, labels, 0.7, 12.0)
    assert abs(loss - tl) <= 1e-11 * abs(tl)
    for name in grad:
        scale = np.abs(tg[name]).max()
        np.testing.assert_allclose(grad[name], tg[name], rtol=0, atol=1e-10 * scale, err_msg=name)


def test_gradient_finite_differences():
    rng = np.random.default_rng(4)
    xs = make_series(rng, [6, 9, 11])
    params = rand_params(rng, 4, scale=0.3)
    groups = [[0, 1, 2]]
    labels = [[1.0, 2.0, 1.5]]
    _, grad = K.loss_and_grad(params, xs, groups, labels, 1.0, 8.0)
    for name, idx in [("W1", (3, 5, 1)), ("b2", (7,)), ("W3", (10, 20, 4)), ("Wl", (31, 2)),
                      ("bl", (0,))]:
        h = 1e-6
        p1 = {k: v.copy() for k, v in params.items()}
        p2 = {k: v.copy() for k, v in params.items()}
        p1[name][idx] += h
        p2[name][idx] -= h
        fd = (K.loss_and_grad(p1, xs, groups, labels, 1.0, 8.0)[0] -
              K.loss_and_grad(p2, xs, groups, labels, 1.0, 8.0)[0]) / (2 * h)
        assert abs(fd - grad[name][idx]) <= 1e-5 * (1 + abs(fd)), (name, fd, grad[name][idx])


def test_delete_cost_channel_matches_twed_oracle():
    rng = np.random.default_rng(5)
    v = np.cumsum(rng.normal(size=(50, 3)), axis=0)
    t = np.cumsum(rng.exponential(1.0, 50))
    f = K.features(v, t, 0.3, 0.7, 2)
    np.testing.assert_array_equal(f[:, :3], v)
    np.testing.assert_array_equal(f[:, 3], t)
    want = oracle.delete_costs(v, t, 0.3, 0.7, 2)
    np.testing.assert_allclose(f[:, 4], want, rtol=1e-15, atol=0)


def test_feature_stats_small_example():
    f = [np.array([[1.0, 5.0], [3.0, 5.0]]), np.array([[5.0, 5.0]])]
    mu, sd = K.feature_stats(f)
    np.testing.assert_allclose(mu, [3.0, 5.0])
    np.testing.assert_allclose(sd, [np.sqrt(8.0 / 3.0), 1.0])  # constant channel -> 1


def test_adam_matches_torch_and_first_step_closed_form():
    rng = np.random.default_rng(6)
    theta = rng.normal(size=20)
    grads = [rng.normal(size=20) for _ in range(3)]
    m = np.zeros(20)
    v = np.zeros(20)
    th = theta.copy()
    for s, g in enumerate(grads, start=1):
        th, m, v = K.adam(th, g, m, v, s, 1e-2)
        if s == 1:
            # m_hat = g, v_hat = g^2  ->  step = lr * g / (|g| + eps)
            np.testing.assert_allclose(th, theta - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-14)
    tp = torch.tensor(theta, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    for g in grads:
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(th, tp.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_pair_model_closed_form():
    ea = np.zeros(32)
    eb = np.zeros(32)
    ea[0], eb[0] = 3.0, 0.0
    ea[1], eb[1] = 0.0, 4.0
    ea[31], eb[31] = 2.0, -0.5
    assert K.pair_model(ea, eb) == 25.0 + 1.5


def test_search_rows_rank_like_the_pair_model():
    rng = np.random.default_rng(7)
    db = rng.normal(size=(300, 32))
    q = rng.normal(size=(5, 32))
    sdb, sq = K.search_rows(db, q)
    D = K.sq_l2(sq, sdb)
    zmin = db[:, 31].min()
    for i in range(5):
        model = np.array([K.pair_model(q[i], db[j]) for j in range(300)])
        np.testing.assert_allclose(D[i], model - q[i, 31] - zmin, rtol=1e-12, atol=1e-12)
        assert (np.argsort(D[i], kind="stable") == np.argsort(model, kind="stable")).mean() > 0.99


def test_topk_rows_ties_by_index():
    D = np.array([[3.0, 1.0, 2.0, 1.0, 0.5, 2.0],
                  [7.0, 7.0, 7.0, 7.0, 7.0, 7.0]])
    idx, val = K.topk_rows(D, 4)
    assert idx.tolist() == [[4, 1, 3, 2], [0, 1, 2, 3]]
    assert val.tolist() == [[0.5, 1.0, 1.0, 2.0], [7.0] * 4]


def test_recall_counts_ties():
    found = np.array([[1.0, 2.0, 3.0], [1.0, 5.0, 3.0]])
    true_kth = np.array([3.0, 3.0])
    assert K.recall_at_k(found, true_kth) == pytest.approx((3 + 2) / 6)


def test_param_count():
    assert K.param_count(4) == 64 * 6 * 5 + 64 + 2 * (64 * 64 * 5 + 64) + 32 * 64 + 32
