"""CPU oracle for the learned k-NN filter -- TEST INFRASTRUCTURE ONLY.

Plain float64 numpy statement of the learned candidate filter that sits in
front of exact TWED re-ranking.  The paper itself has no learned component;
what is restated here is the design the library implements, written as the
textbook definitions of each piece, with no blocking, fusion or reordering:

* ``features``      -- per point: the values a_i, the timestamp t_i and the
                       TWED delete cost dA(i) = d(a_i, a_{i-1}) + nu|t_i -
                       t_{i-1}| + lambda with the paper's padding a_0 = 0,
                       t_0 = 0 (section "Time Warp Edit Distance").
* ``feature_stats`` -- per-channel mean and population standard deviation
                       over every point of a set.
* ``forward``       -- three 1-D convolutions (64 channels, 5 taps, zero
                       'same' padding, ReLU), a length-weighted mean pool
                       (sum over time / mean length of the database) and a
                       linear map 64 -> 32.
* ``pair_model``    -- the additive distance model for two embeddings
                       e = (psi in R^31, z): |psi_a - psi_b|^2 + z_a + z_b.
* ``loss_and_grad`` -- mean squared error of the pair model against TWED
                       labels scaled by 1/sigma over all pairs inside groups
                       of series, with hand-derived gradients.
* ``adam``          -- one Adam step (Kingma and Ba, 2015, Algorithm 1).
* ``search_rows``   -- the database search vector (psi, sqrt(z - z_min)) and
                       the query vector (psi, 0): their squared L2 distance is
                       the pair model minus (z_q + z_min), so it ranks the
                       database exactly as the pair model does.
* ``topk_rows``     -- the k smallest entries of each row, ties broken by the
                       smaller column index.
* ``recall_at_k``   -- the fraction of true k nearest neighbours found, an
                       item counting as found when its exact distance is not
                       above the true k-th distance (ties).

Parameter layout (one flat float array, row-major blocks in this order):
W1[64][C0][5], b1[64], W2[64][64][5], b2[64], W3[64][64][5], b3[64],
Wl[32][64], bl[32], with C0 = dim + 2 input channels.  Convolution:
y[t][o] = b[o] + sum_k sum_c W[o][c][k] x[t + k - 2][c], x = 0 outside the
series.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this module; the library never does.  Parity pins for
these functions are in ``tests/test_oracle_knn.py``.
"""
from __future__ import annotations

import numpy as np

CH = 64
TAPS = 5
EMB = 32
PSI = EMB - 1


def n_inputs(dim: int) -> int:
    return dim + 2


def param_shapes(dim: int):
    c0 = n_inputs(dim)
    return [("W1", (CH, c0, TAPS)), ("b1", (CH,)), ("W2", (CH, CH, TAPS)), ("b2", (CH,)),
            ("W3", (CH, CH, TAPS)), ("b3", (CH,)), ("Wl", (EMB, CH)), ("bl", (EMB,))]


def param_count(dim: int) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(dim)))


def unpack(flat, dim: int) -> dict:
    flat = np.asarray(flat, dtype=np.float64)
    out, o = {}, 0
    for name, shape in param_shapes(dim):
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    assert o == flat.size, (o, flat.size)
    return out


def pack(params: dict, dim: int) -> np.ndarray:
    return np.concatenate([np.asarray(params[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes(dim)])


# ------------------------------------------------------------------ inputs
def lp_dist(x, y, p):
    """d(x, y) = (sum_k |x_k - y_k|^p)^(1/p) row by row; |x - y| for dim 1."""
    diff = np.abs(np.asarray(x, np.float64) - np.asarray(y, np.float64))
    if diff.ndim == 1:
        return diff
    if diff.shape[1] == 1:
        return diff[:, 0]
    if p == 1:
        return diff.sum(axis=1)
    if p == 2:
        return np.sqrt((diff * diff).sum(axis=1))
    return (diff ** p).sum(axis=1) ** (1.0 / p)


def features(vals, ts, nu, lam, p=2):
    """Raw per-point inputs of one series: [a_i (dim values), t_i, dA(i)]."""
    a = np.asarray(vals, np.float64)
    if a.ndim == 1:
        a = a[:, None]
    t = np.asarray(ts, np.float64)
    prev_a = np.vstack([np.zeros((1, a.shape[1])), a[:-1]])
    prev_t = np.concatenate([[0.0], t[:-1]])
    delete = lp_dist(a, prev_a, p) + nu * np.abs(t - prev_t) + lam
    return np.hstack([a, t[:, None], delete[:, None]])


def feature_stats(feature_list):
    """Mean and population standard deviation of every channel over all
    points; a channel with zero spread gets scale 1."""
    allf = np.vstack(feature_list)
    mu = allf.mean(axis=0)
    sd = np.sqrt(((allf - mu) ** 2).mean(axis=0))
    sd[sd == 0] = 1.0
    return mu, sd


def normalise(f, mu, sd):
    return (f - mu) / sd


# ----------------------------------------------------------------- forward
def conv_same(x, W, b):
    """y[t][o] = b[o] + sum_k sum_c W[o][c][k] x[t+k-2][c], zero outside."""
    L = x.shape[0]
    xp = np.vstack([np.zeros((2, x.shape[1])), x, np.zeros((2, x.shape[1]))])
    y = np.tile(b, (L, 1))
    for k in range(TAPS):
        y = y + xp[k:k + L] @ W[:, :, k].T
    return y


def conv_same_transpose(dy, W):
    """Adjoint of conv_same in x: dx[t][c] = sum_k sum_o W[o][c][k] dy[t-k+2][o]."""
    L = dy.shape[0]
    dyp = np.vstack([np.zeros((2, dy.shape[1])), dy, np.zeros((2, dy.shape[1]))])
    dx = np.zeros((L, W.shape[1]))
    for k in range(TAPS):
        # dy[t - k + 2] = dyp[t - k + 4]
        dx = dx + dyp[4 - k:4 - k + L] @ W[:, :, k]
    return dx


def conv_same_wgrad(x, dy):
    """dW[o][c][k] = sum_t dy[t][o] x[t+k-2][c]."""
    L = x.shape[0]
    xp = np.vstack([np.zeros((2, x.shape[1])), x, np.zeros((2, x.shape[1]))])
    dW = np.zeros((dy.shape[1], x.shape[1], TAPS))
    for k in range(TAPS):
        dW[:, :, k] = dy.T @ xp[k:k + L]
    return dW


def forward(params: dict, x, mean_len: float):
    """Embedding of one normalised series x [L][C0]; returns (e, cache)."""
    h1 = np.maximum(conv_same(x, params["W1"], params["b1"]), 0.0)
    h2 = np.maximum(conv_same(h1, params["W2"], params["b2"]), 0.0)
    h3 = np.maximum(conv_same(h2, params["W3"], params["b3"]), 0.0)
    pooled = h3.sum(axis=0) / mean_len
    e = params["Wl"] @ pooled + params["bl"]
    return e, (x, h1, h2, h3, pooled)


def backward(params: dict, cache, de, mean_len: float) -> dict:
    """Gradients of a scalar loss with dL/de = de, for one series."""
    x, h1, h2, h3, pooled = cache
    g = {"Wl": np.outer(de, pooled), "bl": de.copy()}
    dpooled = params["Wl"].T @ de
    d3 = np.tile(dpooled / mean_len, (h3.shape[0], 1)) * (h3 > 0)
    g["W3"] = conv_same_wgrad(h2, d3)
    g["b3"] = d3.sum(axis=0)
    d2 = conv_same_transpose(d3, params["W3"]) * (h2 > 0)
    g["W2"] = conv_same_wgrad(h1, d2)
    g["b2"] = d2.sum(axis=0)
    d1 = conv_same_transpose(d2, params["W2"]) * (h1 > 0)
    g["W1"] = conv_same_wgrad(x, d1)
    g["b1"] = d1.sum(axis=0)
    return g


# -------------------------------------------------------------- pair model
def pair_model(ea, eb):
    """|psi_a - psi_b|^2 + z_a + z_b for embeddings e = (psi, z)."""
    d = ea[:PSI] - eb[:PSI]
    return float(d @ d) + ea[PSI] + eb[PSI]


def group_pairs(g: int):
    """The pairs (a, b), a < b, of a group of g series in row-major order."""
    return [(a, b) for a in range(g) for b in range(a + 1, g)]


def loss_and_grad(params: dict, xs, groups, labels, inv_sigma: float, mean_len: float):
    """Loss = (1/npairs) sum over every group and pair (a < b) of
    (pair_model(e_a, e_b) - y * inv_sigma)^2, and its parameter gradient.

    ``xs``: normalised series; ``groups``: [ngroups][g] indices into xs;
    ``labels``: [ngroups][g(g-1)/2] TWED values in group_pairs order.
    """
    groups = np.asarray(groups)
    ng, g = groups.shape
    pairs = group_pairs(g)
    npairs = ng * len(pairs)
    used = sorted(set(groups.ravel().tolist()))
    emb, caches = {}, {}
    for s in used:
        emb[s], caches[s] = forward(params, xs[s], mean_len)
    de = {s: np.zeros(EMB) for s in used}
    loss = 0.0
    for gi in range(ng):
        for pi, (a, b) in enumerate(pairs):
            sa, sb = int(groups[gi, a]), int(groups[gi, b])
            r = pair_model(emb[sa], emb[sb]) - labels[gi][pi] * inv_sigma
            loss += r * r
            # d r / d psi_a = 2 (psi_a - psi_b), d r / d z_a = 1
            c = 2.0 * r / npairs
            diff = emb[sa][:PSI] - emb[sb][:PSI]
            de[sa][:PSI] += c * 2.0 * diff
            de[sb][:PSI] -= c * 2.0 * diff
            de[sa][PSI] += c
            de[sb][PSI] += c
    grad = {name: np.zeros(shape) for name, shape in param_shapes(params["W1"].shape[1] - 2)}
    for s in used:
        gs = backward(params, caches[s], de[s], mean_len)
        for name in grad:
            grad[name] += gs[name]
    return loss / npairs, grad


def adam(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step number ``step`` (1-based); returns new
    (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


# ------------------------------------------------------------------ search
def search_rows(emb_db, emb_q):
    """Search vectors: database (psi, sqrt(z - z_min)), query (psi, 0)."""
    emb_db = np.asarray(emb_db, np.float64)
    emb_q = np.asarray(emb_q, np.float64)
    zmin = emb_db[:, PSI].min()
    db = emb_db.copy()
    db[:, PSI] = np.sqrt(emb_db[:, PSI] - zmin)
    q = emb_q.copy()
    q[:, PSI] = 0.0
    return db, q


def sq_l2(q, db):
    """D[i][j] = |q_i - db_j|^2, summed over components in order."""
    q = np.asarray(q, np.float64)
    db = np.asarray(db, np.float64)
    D = np.zeros((q.shape[0], db.shape[0]))
    for c in range(q.shape[1]):
        diff = q[:, c:c + 1] - db[None, :, c]
        D += diff * diff
    return D


def topk_rows(D, k: int):
    """Indices and values of the k smallest entries of every row, ascending,
    ties broken by the smaller column index."""
    D = np.asarray(D)
    idx = np.argsort(D, axis=1, kind="stable")[:, :k]
    return idx, np.take_along_axis(D, idx, axis=1)


def recall_at_k(found_dist, true_kth):
    """Mean over queries of |{found items with exact distance <= the true
    k-th distance}| / k."""
    found_dist = np.asarray(found_dist, np.float64)
    k = found_dist.shape[1]
    hits = (found_dist <= np.asarray(true_kth, np.float64)[:, None]).sum(axis=1)
    return float(np.minimum(hits, k).mean() / k)
