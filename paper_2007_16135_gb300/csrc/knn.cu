// Learned k-NN candidate filter: host orchestration (include/twed.h, section
// "learned k-NN candidate filter").  Labels come from the library's own
// exact batch path; every arithmetic step runs in the kernels of encoder.cu
// and of the TWED engine.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/twed.h"
#include "encoder.h"
#include "handle.h"

using namespace twed::enc;
using twed::detail::set_error;

namespace {

// ------------------------------------------------------------------ helpers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    cudaError_t ensure(size_t b) {
        if (b <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, b);
        if (e == cudaSuccess) bytes = b;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
    template <typename T>
    T* as() const { return static_cast<T*>(p); }
    ~DevBuf() { release(); }
};

uint64_t splitmix64(uint64_t& s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
// Uniform integer in [0, n) (multiply-shift on the top 64 bits).
uint64_t below(uint64_t& s, uint64_t n) {
    return (uint64_t)(((unsigned __int128)splitmix64(s) * n) >> 64);
}
// Uniform float in [-b, b).
float symmetric_uniform(uint64_t& s, float b) {
    const double u = (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0);
    return (float)((2.0 * u - 1.0) * b);
}
template <typename T>
void shuffle(std::vector<T>& v, uint64_t& s) {
    for (size_t i = v.size(); i > 1; --i) std::swap(v[i - 1], v[below(s, i)]);
}

twed_status_t err(twed_handle_t h, twed_status_t st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    return set_error(h, st, buf);
}

#define KNN_CUDA(h, call)                                                                   \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            cudaGetLastError();                                                             \
            return err((h), e_ == cudaErrorMemoryAllocation ? TWED_ERR_ALLOC : TWED_ERR_CUDA, \
                       "%s: %s", #call, cudaGetErrorString(e_));                            \
        }                                                                                   \
    } while (0)

twed_status_t check_set_host(twed_handle_t h, const twed_set_f32_t* s, const char* name,
                             int64_t* maxlen) {
    if (!s || !s->vals || !s->ts || !s->offs || !s->offs_host || s->n < 1)
        return err(h, TWED_ERR_INVALID_ARG, "set %s: null pointer or no series", name);
    if (s->offs_host[0] != 0) return err(h, TWED_ERR_INVALID_ARG, "set %s: offs[0] != 0", name);
    int64_t mx = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        const int64_t len = s->offs_host[i + 1] - s->offs_host[i];
        if (len < 1) return err(h, TWED_ERR_INVALID_ARG, "set %s: series %lld is empty", name, (long long)i);
        if (len > (1 << 24)) return err(h, TWED_ERR_INVALID_ARG, "set %s: series too long", name);
        mx = std::max(mx, len);
    }
    *maxlen = mx;
    return TWED_OK;
}

twed_status_t check_params(twed_handle_t h, int dim, float nu, float lambda, int p) {
    if (dim < 1 || dim + 2 > MAX_C0) return err(h, TWED_ERR_INVALID_ARG, "encoder needs 1 <= dim <= %d", MAX_C0 - 2);
    if (p < 1) return err(h, TWED_ERR_INVALID_ARG, "p must be >= 1");
    if (!std::isfinite(nu) || nu < 0.f) return err(h, TWED_ERR_INVALID_ARG, "nu must be finite and >= 0");
    if (!std::isfinite(lambda) || lambda < 0.f)
        return err(h, TWED_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    return TWED_OK;
}

// --------------------------------------------------------------- encoder run
// Device buffers and launch shapes for encoder passes over batches of series.
constexpr int64_t kMaxRows = (int64_t)1 << 22;  // rows per forward chunk

struct Encoder {
    twed_handle_t h = nullptr;
    int dim = 0, p = 2, cin = 8, sms = 0;
    float nu = 1.f, lambda = 1.f;
    float rel_floor = 0.f;  // loss weighting (twed_knn_config_t::rel_floor)
    Layout L;
    int conv_grid = 0, conv_in_grid = 0, wg_grid64 = 0, wg_grid_in = 0;
    DevBuf x0, rser, h1, h2, h3, da, db, part, wv, pooled, emb, de, dpooled, gloss, meta;

    twed_status_t init(twed_handle_t hh, int dim_, int p_, float nu_, float lambda_) {
        h = hh;
        dim = dim_;
        p = p_;
        nu = nu_;
        lambda = lambda_;
        L = layout(dim);
        cin = cin_pad(L.c0);
        sms = twed::detail::handle_sms(h);
        KNN_CUDA(h, prepare_attributes());
        conv_grid = sms * std::max(1, conv_blocks_per_sm(64));
        conv_in_grid = sms * std::max(1, conv_blocks_per_sm(cin));
        wg_grid64 = sms * std::max(1, wgrad_blocks_per_sm(64));
        wg_grid_in = sms * std::max(1, wgrad_blocks_per_sm(cin));
        KNN_CUDA(h, wv.ensure(sizeof(float) * weight_views_floats(cin)));
        const size_t parts = std::max((size_t)wgrad_parts(64, wg_grid64) * (CH * 64 * TAPS + CH),
                                      (size_t)wgrad_parts(cin, wg_grid_in) * (CH * cin * TAPS + CH));
        KNN_CUDA(h, part.ensure(sizeof(float) * parts));
        return TWED_OK;
    }

    WeightViews views() {
        WeightViews w;
        carve_weight_views(wv.as<float>(), cin, &w);
        return w;
    }

    twed_status_t reserve(int64_t rows, int64_t nser, int64_t ngroups, bool train) {
        const int64_t r = std::max<int64_t>(rows, TM);
        const int64_t ns = std::max<int64_t>(nser, 1), ng = std::max<int64_t>(ngroups, 1);
        KNN_CUDA(h, x0.ensure(sizeof(float) * r * cin));
        KNN_CUDA(h, rser.ensure(sizeof(int32_t) * r));
        KNN_CUDA(h, h1.ensure(sizeof(float) * r * CH));
        KNN_CUDA(h, h2.ensure(sizeof(float) * r * CH));
        if (train) {
            KNN_CUDA(h, h3.ensure(sizeof(float) * r * CH));
            KNN_CUDA(h, da.ensure(sizeof(float) * r * CH));
            KNN_CUDA(h, db.ensure(sizeof(float) * r * CH));
        }
        KNN_CUDA(h, pooled.ensure(sizeof(float) * ns * CH));
        KNN_CUDA(h, emb.ensure(sizeof(float) * ns * EMB));
        KNN_CUDA(h, de.ensure(sizeof(float) * ns * EMB));
        KNN_CUDA(h, dpooled.ensure(sizeof(float) * ns * CH));
        KNN_CUDA(h, gloss.ensure(sizeof(float) * ng));
        KNN_CUDA(h, meta.ensure(sizeof(int64_t) * (2 * ns + 1 + ng)));
        return TWED_OK;
    }

    // Appends the gapped-row bases of series ids[0..n) to `base` (n + 1
    // entries, starting at 2); returns the batch's row count.
    static int64_t batch_rows(const int64_t* offs_host, const int64_t* ids, int64_t n,
                              std::vector<int64_t>& base) {
        const size_t b0 = base.size();
        base.resize(b0 + n + 1);
        base[b0] = 2;
        for (int64_t s = 0; s < n; ++s)
            base[b0 + s + 1] = base[b0 + s] + (offs_host[ids[s] + 1] - offs_host[ids[s]]) + 2;
        return base[b0 + n];
    }

    // Forward of one batch already described on the device (d_ids[nser],
    // d_base[nser + 1], P rows).  Activations stay in x0/h1/h2/h3 (h3 aliases
    // h1 when not training).
    twed_status_t forward_batch(const twed_set_f32_t* set, const int64_t* d_ids,
                                const int64_t* d_base, int64_t nser, int64_t P,
                                const float* d_params, const float* mu, const float* sd,
                                float inv_mean_len, bool train, float* emb_out, cudaStream_t st) {
        KNN_CUDA(h, cudaMemsetAsync(x0.p, 0, sizeof(float) * P * cin, st));
        KNN_CUDA(h, cudaMemsetAsync(rser.p, 0xFF, sizeof(int32_t) * P, st));
        KNN_CUDA(h, gather_features(set->vals, set->ts, set->offs, d_ids, d_base, nser, dim, p, nu,
                                    lambda, mu, sd, cin, x0.as<float>(), rser.as<int32_t>(), st));
        const WeightViews w = views();
        float* H3 = train ? h3.as<float>() : h1.as<float>();
        KNN_CUDA(h, conv_forward(cin, x0.as<float>(), P, w.wt1, d_params + L.b1, rser.as<int32_t>(),
                                 h1.as<float>(), conv_in_grid, st));
        KNN_CUDA(h, conv_forward(64, h1.as<float>(), P, w.wt2, d_params + L.b2, rser.as<int32_t>(),
                                 h2.as<float>(), conv_grid, st));
        KNN_CUDA(h, conv_forward(64, h2.as<float>(), P, w.wt3, d_params + L.b3, rser.as<int32_t>(),
                                 H3, conv_grid, st));
        KNN_CUDA(h, pool_forward(H3, d_base, nser, inv_mean_len, d_params + L.wl, d_params + L.bl,
                                 pooled.as<float>(), emb_out, st));
        return TWED_OK;
    }

    // Embeddings of series ids[0..n) into d_emb[n][32], in row-bounded chunks.
    twed_status_t embed(const twed_set_f32_t* set, const std::vector<int64_t>& ids_all,
                        const float* d_params, const float* mu, const float* sd,
                        float inv_mean_len, float* d_emb, cudaStream_t st) {
        KNN_CUDA(h, transform_weights(d_params, L, cin, views(), st));
        const int64_t n = (int64_t)ids_all.size();
        std::vector<int64_t> base;
        int64_t s0 = 0;
        while (s0 < n) {
            int64_t rows = 2, s1 = s0;
            while (s1 < n) {
                const int64_t len = set->offs_host[ids_all[s1] + 1] - set->offs_host[ids_all[s1]];
                if (s1 > s0 && rows + len + 2 > kMaxRows) break;
                rows += len + 2;
                ++s1;
            }
            const int64_t ns = s1 - s0;
            base.clear();
            const int64_t P = batch_rows(set->offs_host, ids_all.data() + s0, ns, base);
            // the previous chunk must be done before its buffers are resized
            // or its metadata overwritten
            KNN_CUDA(h, cudaStreamSynchronize(st));
            twed_status_t s = reserve(P, ns, 1, false);
            if (s != TWED_OK) return s;
            int64_t* d_base = meta.as<int64_t>();
            int64_t* d_ids = d_base + ns + 1;
            KNN_CUDA(h, cudaMemcpyAsync(d_base, base.data(), sizeof(int64_t) * (ns + 1), cudaMemcpyHostToDevice, st));
            KNN_CUDA(h, cudaMemcpyAsync(d_ids, ids_all.data() + s0, sizeof(int64_t) * ns, cudaMemcpyHostToDevice, st));
            s = forward_batch(set, d_ids, d_base, ns, P, d_params, mu, sd, inv_mean_len, false,
                              d_emb + s0 * EMB, st);
            if (s != TWED_OK) return s;
            s0 = s1;
        }
        return TWED_OK;
    }

    // Loss and gradient of one batch of ngroups groups whose series ids
    // (group-major), gapped-row bases and group ids are already on the device;
    // buffers must have been reserved for P rows.
    twed_status_t loss_grad(const twed_set_f32_t* set, const int64_t* d_ids, const int64_t* d_base,
                            int64_t P, int64_t ngroups, int gsize, const int64_t* d_gids,
                            const float* d_labels, const float* d_inv_sigma, const float* d_params,
                            const float* mu, const float* sd, float inv_mean_len, float* d_grad,
                            float* d_loss, cudaStream_t st) {
        const int64_t nser = ngroups * gsize;
        twed_status_t s = forward_batch(set, d_ids, d_base, nser, P, d_params, mu, sd, inv_mean_len,
                                        true, emb.as<float>(), st);
        if (s != TWED_OK) return s;
        const int64_t npairs = ngroups * (int64_t)gsize * (gsize - 1) / 2;
        KNN_CUDA(h, group_loss(emb.as<float>(), ngroups, gsize, d_gids, d_labels, d_inv_sigma,
                               (float)(1.0 / (double)npairs), rel_floor, d_params + L.wl, de.as<float>(),
                               dpooled.as<float>(), gloss.as<float>(), st));
        KNN_CUDA(h, sum_scaled(gloss.as<float>(), ngroups, 1.0 / (double)npairs, d_loss, st));
        const WeightViews w = views();
        const int32_t* rs = rser.as<int32_t>();
        float* dA = da.as<float>();
        float* dB = db.as<float>();
        KNN_CUDA(h, pool_backward(h3.as<float>(), rs, dpooled.as<float>(), inv_mean_len, P, dA, st));
        KNN_CUDA(h, linear_grad(de.as<float>(), pooled.as<float>(), nser, d_grad + L.wl, d_grad + L.bl, st));
        KNN_CUDA(h, conv_wgrad(64, h2.as<float>(), dA, P, part.as<float>(), wg_grid64, st));
        KNN_CUDA(h, wgrad_reduce(part.as<float>(), wgrad_parts(64, wg_grid64), 64, 64, d_grad + L.w3, d_grad + L.b3, st));
        KNN_CUDA(h, conv_backward_data(dA, P, w.wb3, h2.as<float>(), dB, conv_grid, st));
        KNN_CUDA(h, conv_wgrad(64, h1.as<float>(), dB, P, part.as<float>(), wg_grid64, st));
        KNN_CUDA(h, wgrad_reduce(part.as<float>(), wgrad_parts(64, wg_grid64), 64, 64, d_grad + L.w2, d_grad + L.b2, st));
        KNN_CUDA(h, conv_backward_data(dB, P, w.wb2, h1.as<float>(), dA, conv_grid, st));
        KNN_CUDA(h, conv_wgrad(cin, x0.as<float>(), dA, P, part.as<float>(), wg_grid_in, st));
        KNN_CUDA(h, wgrad_reduce(part.as<float>(), wgrad_parts(cin, wg_grid_in), cin, L.c0, d_grad + L.w1, d_grad + L.b1, st));
        return TWED_OK;
    }
};

}  // namespace

// ===================================================================== index
struct twed_knn_s {
    twed_handle_t h = nullptr;
    twed_set_f32_t db{};
    std::vector<int64_t> db_offs;  // host copy of the database offsets
    int dim = 0, p = 2;
    float nu = 1.f, lambda = 1.f;
    twed_knn_config_t cfg{};
    Encoder enc;
    DevBuf params, grad, m, v, mu, sd, stat_part, labels, lpairs, scalars, emb_db, svec_db, losses, sched;
    DevBuf sbuf, cand, candval, qpairs, rr, pos, qemb, cells;
    DevBuf hq_vals, hq_ts, hq_offs, hq_idx, hq_dist;  // staging of twed_knn_search_host
    double mean_len = 0.0;
    bool trained = false;
    bool searched = false;
    int rr_rmax = 0, rr_per_sm = 0;  // re-rank launch shape (0: defaults)
    twed_knn_stats_t stats{};
    cudaEvent_t ev[5] = {};  // search phase boundaries
    cudaStream_t host_stream = nullptr;
    ~twed_knn_s() {
        for (cudaEvent_t& e : ev)
            if (e) cudaEventDestroy(e);
        if (host_stream) cudaStreamDestroy(host_stream);
    }
};

namespace {

twed_status_t embed_database(twed_knn_t k, cudaStream_t st) {
    std::vector<int64_t> all(k->db.n);
    for (int64_t i = 0; i < k->db.n; ++i) all[i] = i;
    twed_status_t s = k->enc.embed(&k->db, all, k->params.as<float>(), k->mu.as<float>(),
                                   k->sd.as<float>(), (float)(1.0 / k->mean_len),
                                   k->emb_db.as<float>(), st);
    if (s != TWED_OK) return s;
    KNN_CUDA(k->h, search_vectors(k->emb_db.as<float>(), k->db.n, k->scalars.as<float>() + 1,
                                  k->svec_db.as<float>(), st));
    KNN_CUDA(k->h, cudaStreamSynchronize(st));
    return TWED_OK;
}

// The re-rank runs the many-pairs kernel on (query, candidate) pairs, longest
// first.  Its launch shape -- rows-per-lane cap x resident blocks per SM --
// is timed on random database pairs (the length mix of queries drawn like
// the database; about 1e10 cells, at most 2^20 pairs) in the same order, and
// the fastest is kept.  CUDA events on `st`: one warm-up and the best of two
// runs per shape.
twed_status_t tune_rerank(twed_knn_t k, cudaStream_t st) {
    twed_handle_t h = k->h;
    const int64_t N = k->db.n;
    uint64_t rng = k->cfg.seed * 0xD1B54A32D192ED03ull + 0x5bd1e995ull;
    std::vector<int64_t> pr;
    double cells = 0.0;
    while (cells < 1e10 && (int64_t)pr.size() < 2 * ((int64_t)1 << 20)) {
        const int64_t i = (int64_t)below(rng, (uint64_t)N), j = (int64_t)below(rng, (uint64_t)N);
        pr.push_back(i);
        pr.push_back(j);
        cells += (double)(k->db_offs[i + 1] - k->db_offs[i]) * (double)(k->db_offs[j + 1] - k->db_offs[j]);
    }
    const int64_t ns = (int64_t)pr.size() / 2;
    DevBuf dpairs, dout;
    KNN_CUDA(h, dpairs.ensure(sizeof(int64_t) * pr.size()));
    KNN_CUDA(h, dout.ensure(sizeof(float) * ns));
    KNN_CUDA(h, cudaMemcpyAsync(dpairs.p, pr.data(), sizeof(int64_t) * pr.size(), cudaMemcpyHostToDevice, st));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    KNN_CUDA(h, cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) {
        cudaEventDestroy(e0);
        KNN_CUDA(h, ce);
    }
    struct Events {
        cudaEvent_t a, b;
        ~Events() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } guard{e0, e1};
    const int lim = twed::detail::batch_f32_rmax_limit();
    const int occ = twed::detail::batch_f32_max_blocks_per_sm(k->dim, k->p);
    float best = 1e30f;
    int best_r = 0, best_b = 0;
    for (int r : {2, 4, 6, 8}) {
        if (r > lim) continue;
        for (int b = 1; b <= occ; ++b) {
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
                KNN_CUDA(h, cudaEventRecord(e0, st));
                twed_status_t s = twed::detail::batch_f32_shaped(
                    h, &k->db, &k->db, dpairs.as<int64_t>(), ns, k->dim, k->nu, k->lambda, k->p,
                    dout.as<float>(), st, TWED_ORDER_LONGEST_FIRST, r, b);
                if (s != TWED_OK) return s;
                KNN_CUDA(h, cudaEventRecord(e1, st));
                KNN_CUDA(h, cudaEventSynchronize(e1));
                float ms = 0.f;
                KNN_CUDA(h, cudaEventElapsedTime(&ms, e0, e1));
                if (rep > 0) t = std::min(t, ms);
            }
            if (t < best) {
                best = t;
                best_r = r;
                best_b = b;
            }
        }
    }
    k->rr_rmax = best_r;
    k->rr_per_sm = best_b;
    k->stats.rerank_rows_per_lane = best_r;
    k->stats.rerank_blocks_per_sm = best_b;
    return TWED_OK;
}

void init_params(std::vector<float>& w, const Layout& L, uint64_t seed) {
    w.assign(L.total, 0.f);
    uint64_t s = seed * 0x2545F4914F6CDD1Dull + 17;
    auto fill = [&](int64_t off, int64_t n, int fan_in) {
        const float b = 1.0f / std::sqrt((float)fan_in);
        for (int64_t i = 0; i < n; ++i) w[off + i] = symmetric_uniform(s, b);
    };
    fill(L.w1, L.b1 - L.w1, L.c0 * TAPS);
    fill(L.b1, CH, L.c0 * TAPS);
    fill(L.w2, L.b2 - L.w2, CH * TAPS);
    fill(L.b2, CH, CH * TAPS);
    fill(L.w3, L.b3 - L.w3, CH * TAPS);
    fill(L.b3, CH, CH * TAPS);
    fill(L.wl, L.bl - L.wl, CH);
    fill(L.bl, EMB, CH);
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

extern "C" void twed_knn_config_default(twed_knn_config_t* c) {
    if (!c) return;
    c->group_size = 32;
    c->groups_per_step = 32;
    c->epochs = 40;
    c->train_pairs = 1000000;
    c->lr = 2e-3f;
    c->seed = 1;
    c->mine_fraction = 0.0f;
    c->rel_floor = 0.0f;
}

extern "C" twed_status_t twed_knn_create(twed_handle_t h, const twed_set_f32_t* db, int dim,
                                         float nu, float lambda, int p,
                                         const twed_knn_config_t* cfg, twed_knn_t* out) {
    if (!h || !out) return TWED_ERR_INVALID_ARG;
    *out = nullptr;
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, db, "db", &maxlen);
    if (s != TWED_OK) return s;
    if ((s = check_params(h, dim, nu, lambda, p)) != TWED_OK) return s;
    twed_knn_config_t c;
    twed_knn_config_default(&c);
    if (cfg) c = *cfg;
    if (c.group_size < 2 || c.group_size > 64 || c.group_size > db->n)
        return err(h, TWED_ERR_INVALID_ARG, "group_size must be in [2, min(64, ndb)]");
    if (c.groups_per_step < 1 || c.epochs < 0 || c.train_pairs < 1 || !(c.lr > 0.f) ||
        !(c.mine_fraction >= 0.f && c.mine_fraction < 1.f) || !(c.rel_floor >= 0.f && c.rel_floor < 1e30f))
        return err(h, TWED_ERR_INVALID_ARG, "bad training configuration");
    twed_knn_t k = new (std::nothrow) twed_knn_s();
    if (!k) return err(h, TWED_ERR_ALLOC, "index");
    k->h = h;
    k->db = *db;
    k->db_offs.assign(db->offs_host, db->offs_host + db->n + 1);
    k->db.offs_host = k->db_offs.data();
    k->dim = dim;
    k->p = p;
    k->nu = nu;
    k->lambda = lambda;
    k->cfg = c;
    k->mean_len = (double)k->db_offs[db->n] / (double)db->n;
    s = k->enc.init(h, dim, p, nu, lambda);
    const Layout& L = k->enc.L;
    auto alloc = [&](DevBuf& b, size_t bytes) -> bool {
        if (s != TWED_OK) return false;
        cudaError_t e = b.ensure(bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = err(h, TWED_ERR_ALLOC, "index memory (%zu bytes): %s", bytes, cudaGetErrorString(e));
            return false;
        }
        return true;
    };
    alloc(k->params, sizeof(float) * L.total);
    alloc(k->grad, sizeof(float) * L.total);
    alloc(k->m, sizeof(float) * L.total);
    alloc(k->v, sizeof(float) * L.total);
    alloc(k->mu, sizeof(float) * MAX_C0);
    alloc(k->sd, sizeof(float) * MAX_C0);
    alloc(k->stat_part, sizeof(double) * 2 * 1024 * MAX_C0);
    alloc(k->scalars, sizeof(float) * 8);
    alloc(k->emb_db, sizeof(float) * db->n * EMB);
    alloc(k->svec_db, sizeof(float) * db->n * EMB);
    alloc(k->cells, sizeof(unsigned long long));
    for (cudaEvent_t& e : k->ev)
        if (s == TWED_OK && cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            s = err(h, TWED_ERR_CUDA, "event creation");
        }
    if (s == TWED_OK && cudaStreamCreateWithFlags(&k->host_stream, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        s = err(h, TWED_ERR_CUDA, "stream creation");
    }
    if (s != TWED_OK) {
        delete k;
        return s;
    }
    std::vector<float> w;
    init_params(w, L, c.seed);
    if (cudaMemcpy(k->params.p, w.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        delete k;
        return err(h, TWED_ERR_CUDA, "parameter upload");
    }
    *out = k;
    return TWED_OK;
}

extern "C" void twed_knn_destroy(twed_knn_t k) {
    if (!k) return;
    cudaDeviceSynchronize();
    delete k;
}

namespace {

// Pair list (a < b, row-major) of groups [g0, g1) of `members`.
int64_t group_pair_list(const twed_knn_t k, const std::vector<int64_t>& members, int G, int64_t g0,
                        int64_t g1, std::vector<int64_t>& pairs) {
    int64_t cells = 0;
    pairs.clear();
    for (int64_t g = g0; g < g1; ++g)
        for (int a = 0; a < G; ++a)
            for (int b = a + 1; b < G; ++b) {
                const int64_t x = members[g * G + a], y = members[g * G + b];
                pairs.push_back(x);
                pairs.push_back(y);
                cells += (k->db_offs[x + 1] - k->db_offs[x]) * (k->db_offs[y + 1] - k->db_offs[y]);
            }
    return cells;
}

// Exact TWED labels of every pair of groups [g0, g1) into labels[g0 * npg ..].
twed_status_t label_groups(twed_knn_t k, const std::vector<int64_t>& members, int G, int64_t g0,
                           int64_t g1, cudaStream_t st) {
    twed_handle_t h = k->h;
    const int64_t npg = (int64_t)G * (G - 1) / 2;
    std::vector<int64_t> pairs;
    const int64_t cells = group_pair_list(k, members, G, g0, g1, pairs);
    const int64_t n = (g1 - g0) * npg;
    KNN_CUDA(h, k->lpairs.ensure(sizeof(int64_t) * 2 * std::max<int64_t>(n, 1)));
    KNN_CUDA(h, cudaMemcpyAsync(k->lpairs.p, pairs.data(), sizeof(int64_t) * 2 * n, cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaStreamSynchronize(st));
    const auto t0 = std::chrono::steady_clock::now();
    twed_status_t s = twed_batch_f32(h, &k->db, &k->db, k->lpairs.as<int64_t>(), n, k->dim, k->nu,
                                     k->lambda, k->p, k->labels.as<float>() + g0 * npg, st);
    if (s != TWED_OK) return s;
    KNN_CUDA(h, cudaStreamSynchronize(st));
    if ((s = twed_sync_status(h, st)) != TWED_OK) return s;
    k->stats.label_ms += ms_since(t0);
    k->stats.label_pairs += n;
    k->stats.label_cells += cells;
    return TWED_OK;
}

// `epochs` passes over groups [0, ngroups) in seeded shuffled order, one Adam
// step per `groups_per_step` groups, cosine learning rate over total_steps.
twed_status_t run_epochs(twed_knn_t k, const std::vector<int64_t>& members, int G, int64_t ngroups,
                         int epochs, uint64_t& rng, int64_t& step, int64_t total_steps,
                         cudaStream_t st) {
    twed_handle_t h = k->h;
    const twed_knn_config_t& c = k->cfg;
    const Layout& L = k->enc.L;
    const int64_t gps = std::min<int64_t>(c.groups_per_step, ngroups);
    std::vector<int64_t> order(ngroups);
    for (int64_t g = 0; g < ngroups; ++g) order[g] = g;
    // The whole schedule (series ids, gapped-row bases, group ids of every
    // step) is built on the host and uploaded once, so the steps enqueue
    // without host waits.
    std::vector<int64_t> sids, sbase, sgid;
    std::vector<int64_t> step_ng, step_p, step_ids_off, step_base_off, step_gid_off;
    int64_t max_rows = 0, max_ng = 0;
    for (int ep = 0; ep < epochs; ++ep) {
        shuffle(order, rng);
        for (int64_t g0 = 0; g0 < ngroups; g0 += gps) {
            const int64_t ng = std::min(gps, ngroups - g0);
            step_ng.push_back(ng);
            step_ids_off.push_back((int64_t)sids.size());
            step_base_off.push_back((int64_t)sbase.size());
            step_gid_off.push_back((int64_t)sgid.size());
            for (int64_t i = 0; i < ng; ++i) {
                sgid.push_back(order[g0 + i]);
                for (int a = 0; a < G; ++a) sids.push_back(members[order[g0 + i] * G + a]);
            }
            const int64_t P = Encoder::batch_rows(k->db_offs.data(), sids.data() + step_ids_off.back(),
                                                  ng * G, sbase);
            step_p.push_back(P);
            max_rows = std::max(max_rows, P);
            max_ng = std::max(max_ng, ng);
        }
    }
    if (step_ng.empty()) return TWED_OK;
    KNN_CUDA(h, cudaStreamSynchronize(st));
    KNN_CUDA(h, k->sched.ensure(sizeof(int64_t) * (sids.size() + sbase.size() + sgid.size() + 3)));
    int64_t* d_sids = k->sched.as<int64_t>();
    int64_t* d_sbase = d_sids + sids.size();
    int64_t* d_sgid = d_sbase + sbase.size();
    KNN_CUDA(h, cudaMemcpyAsync(d_sids, sids.data(), sizeof(int64_t) * sids.size(), cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaMemcpyAsync(d_sbase, sbase.data(), sizeof(int64_t) * sbase.size(), cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaMemcpyAsync(d_sgid, sgid.data(), sizeof(int64_t) * sgid.size(), cudaMemcpyHostToDevice, st));
    twed_status_t s = k->enc.reserve(max_rows, max_ng * G, max_ng, true);
    if (s != TWED_OK) return s;
    k->enc.rel_floor = k->cfg.rel_floor;
    const float inv_mean_len = (float)(1.0 / k->mean_len);
    const double b1 = 0.9, b2 = 0.999;
    float* sc = k->scalars.as<float>();
    KNN_CUDA(h, transform_weights(k->params.as<float>(), L, k->enc.cin, k->enc.views(), st));
    for (size_t i = 0; i < step_ng.size(); ++i, ++step) {
        s = k->enc.loss_grad(&k->db, d_sids + step_ids_off[i], d_sbase + step_base_off[i], step_p[i],
                             step_ng[i], G, d_sgid + step_gid_off[i], k->labels.as<float>(), sc + 2,
                             k->params.as<float>(), k->mu.as<float>(), k->sd.as<float>(),
                             inv_mean_len, k->grad.as<float>(), k->losses.as<float>() + step, st);
        if (s != TWED_OK) return s;
        const double t = (double)(step + 1);
        const double lr = c.lr * 0.5 * (1.0 + std::cos(M_PI * (double)step / (double)total_steps));
        const float c1 = (float)(1.0 / (1.0 - std::pow(b1, t)));
        const float c2 = (float)(1.0 / (1.0 - std::pow(b2, t)));
        KNN_CUDA(h, adam(k->params.as<float>(), k->grad.as<float>(), k->m.as<float>(),
                         k->v.as<float>(), L.total, (float)lr, (float)b1, (float)b2, 1e-8f, c1, c2, st));
        KNN_CUDA(h, transform_weights(k->params.as<float>(), L, k->enc.cin, k->enc.views(), st));
    }
    KNN_CUDA(h, cudaStreamSynchronize(st));
    return TWED_OK;
}

// Hard groups: an anchor (seeded draw from the database) and the G - 1
// database series nearest to it under the current model (the search
// distance, anchor excluded).  Appends nmine groups to `members`.
twed_status_t mine_groups(twed_knn_t k, int G, int64_t nmine, uint64_t& rng,
                          std::vector<int64_t>& members, cudaStream_t st) {
    twed_handle_t h = k->h;
    const int64_t N = k->db.n;
    twed_status_t s = embed_database(k, st);
    if (s != TWED_OK) return s;
    std::vector<float> emb((size_t)N * EMB);
    KNN_CUDA(h, cudaMemcpy(emb.data(), k->emb_db.p, sizeof(float) * N * EMB, cudaMemcpyDeviceToHost));
    std::vector<int64_t> anchors;
    {
        std::vector<int64_t> perm(N);
        while ((int64_t)anchors.size() < nmine) {
            for (int64_t i = 0; i < N; ++i) perm[i] = i;
            shuffle(perm, rng);
            for (int64_t i = 0; i < N && (int64_t)anchors.size() < nmine; ++i) anchors.push_back(perm[i]);
        }
    }
    const int64_t qc = std::max<int64_t>(1, std::min<int64_t>(nmine, ((int64_t)1 << 28) / N));
    KNN_CUDA(h, k->sbuf.ensure(sizeof(float) * qc * N));
    KNN_CUDA(h, k->qemb.ensure(sizeof(float) * qc * EMB));
    KNN_CUDA(h, k->cand.ensure(sizeof(int64_t) * qc * G));
    KNN_CUDA(h, k->candval.ensure(sizeof(float) * qc * G));
    std::vector<float> qe((size_t)qc * EMB);
    std::vector<int64_t> cand((size_t)qc * G);
    const int topk_grid = twed::detail::handle_sms(h) * 2;
    for (int64_t a0 = 0; a0 < nmine; a0 += qc) {
        const int64_t n = std::min(qc, nmine - a0);
        for (int64_t i = 0; i < n; ++i)
            std::memcpy(&qe[i * EMB], &emb[anchors[a0 + i] * EMB], sizeof(float) * EMB);
        KNN_CUDA(h, cudaMemcpyAsync(k->qemb.p, qe.data(), sizeof(float) * n * EMB, cudaMemcpyHostToDevice, st));
        KNN_CUDA(h, l2_rows(k->qemb.as<float>(), n, k->svec_db.as<float>(), N, k->sbuf.as<float>(), N, st));
        KNN_CUDA(h, topk_rows(k->sbuf.as<float>(), n, N, N, G, k->cand.as<int64_t>(),
                              k->candval.as<float>(), topk_grid, st));
        KNN_CUDA(h, cudaMemcpyAsync(cand.data(), k->cand.p, sizeof(int64_t) * n * G, cudaMemcpyDeviceToHost, st));
        KNN_CUDA(h, cudaStreamSynchronize(st));
        for (int64_t i = 0; i < n; ++i) {
            const int64_t anchor = anchors[a0 + i];
            members.push_back(anchor);
            int taken = 0;
            for (int j = 0; j < G && taken < G - 1; ++j) {
                if (cand[i * G + j] == anchor) continue;
                members.push_back(cand[i * G + j]);
                ++taken;
            }
        }
    }
    return TWED_OK;
}

}  // namespace

extern "C" twed_status_t twed_knn_train(twed_knn_t k) {
    if (!k) return TWED_ERR_INVALID_ARG;
    twed_handle_t h = k->h;
    cudaStream_t st;
    KNN_CUDA(h, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } guard{st};
    const twed_knn_config_t& c = k->cfg;
    const Layout& L = k->enc.L;
    const int64_t N = k->db.n;
    const int G = c.group_size;
    const int64_t npg = (int64_t)G * (G - 1) / 2;
    const double f = std::min(1.0, std::max(0.0, (double)c.mine_fraction));
    const int64_t nmine = f > 0.0 ? (int64_t)std::ceil(f * (double)c.train_pairs / (double)npg) : 0;
    const int64_t nrand = std::max<int64_t>(1, (int64_t)std::ceil((1.0 - f) * (double)c.train_pairs / (double)npg));
    const int e1 = nmine > 0 ? (c.epochs + 1) / 2 : c.epochs;
    const int e2 = c.epochs - e1;
    k->trained = false;
    k->stats = twed_knn_stats_t{};
    // ---- fresh parameters and Adam state
    std::vector<float> w;
    init_params(w, L, c.seed);
    KNN_CUDA(h, cudaMemcpyAsync(k->params.p, w.data(), sizeof(float) * L.total, cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaMemsetAsync(k->m.p, 0, sizeof(float) * L.total, st));
    KNN_CUDA(h, cudaMemsetAsync(k->v.p, 0, sizeof(float) * L.total, st));
    // ---- input statistics
    KNN_CUDA(h, feature_stats(k->db.vals, k->db.ts, k->db.offs, N, k->db_offs[N], k->dim, k->p,
                              k->nu, k->lambda, k->stat_part.as<double>(), k->mu.as<float>(),
                              k->sd.as<float>(), st));
    // ---- random groups: consecutive chunks of seeded permutations
    uint64_t rng = c.seed * 0x9E3779B97F4A7C15ull + 3;
    std::vector<int64_t> members;
    members.reserve((size_t)(nrand + nmine) * G);
    {
        std::vector<int64_t> perm(N);
        int64_t used = N;
        for (int64_t g = 0; g < nrand; ++g) {
            if (used + G > N) {
                for (int64_t i = 0; i < N; ++i) perm[i] = i;
                shuffle(perm, rng);
                used = 0;
            }
            for (int a = 0; a < G; ++a) members.push_back(perm[used + a]);
            used += G;
        }
    }
    KNN_CUDA(h, k->labels.ensure(sizeof(float) * (nrand + nmine) * npg));
    twed_status_t s = label_groups(k, members, G, 0, nrand, st);
    if (s != TWED_OK) return s;
    // ---- sigma = mean label of the random pairs (fixed for all of training)
    float* sc = k->scalars.as<float>();  // [0] mean label, [1] z_min, [2] inv_sigma
    KNN_CUDA(h, sum_scaled(k->labels.as<float>(), nrand * npg, 1.0 / (double)(nrand * npg), sc, st));
    float sigma = 0.f;
    KNN_CUDA(h, cudaMemcpyAsync(&sigma, sc, sizeof(float), cudaMemcpyDeviceToHost, st));
    KNN_CUDA(h, cudaStreamSynchronize(st));
    if (!(sigma > 0.f) || !std::isfinite(sigma))
        return err(h, TWED_ERR_INVALID_ARG, "training labels have no positive scale");
    const float inv_sigma = 1.0f / sigma;
    KNN_CUDA(h, cudaMemcpyAsync(sc + 2, &inv_sigma, sizeof(float), cudaMemcpyHostToDevice, st));
    k->stats.sigma = sigma;
    k->stats.mean_len = k->mean_len;
    // ---- steps: e1 epochs on random groups, then (with mining) e2 on all
    const int64_t gps = std::max<int64_t>(1, c.groups_per_step);
    const int64_t spe1 = (nrand + gps - 1) / gps;
    const int64_t spe2 = (nrand + nmine + gps - 1) / gps;
    const int64_t total_steps = spe1 * e1 + spe2 * e2;
    KNN_CUDA(h, k->losses.ensure(sizeof(float) * std::max<int64_t>(total_steps, 1)));
    int64_t step = 0;
    auto t0 = std::chrono::steady_clock::now();
    if ((s = run_epochs(k, members, G, nrand, e1, rng, step, total_steps, st)) != TWED_OK) return s;
    double train_ms = ms_since(t0);
    if (nmine > 0) {
        if ((s = mine_groups(k, G, nmine, rng, members, st)) != TWED_OK) return s;
        if ((s = label_groups(k, members, G, nrand, nrand + nmine, st)) != TWED_OK) return s;
        k->stats.mined_pairs = nmine * npg;
        t0 = std::chrono::steady_clock::now();
        if ((s = run_epochs(k, members, G, nrand + nmine, e2, rng, step, total_steps, st)) != TWED_OK)
            return s;
        train_ms += ms_since(t0);
    }
    k->stats.train_ms = train_ms;
    k->stats.steps = step;
    if (step > 0) {
        std::vector<float> hist(step);
        KNN_CUDA(h, cudaMemcpy(hist.data(), k->losses.p, sizeof(float) * step, cudaMemcpyDeviceToHost));
        const int64_t n0 = std::min<int64_t>(spe1, step);
        double a = 0, b = 0;
        for (int64_t i = 0; i < n0; ++i) a += hist[i];
        const int64_t n1 = std::min<int64_t>(e2 > 0 ? spe2 : spe1, step);
        for (int64_t i = step - n1; i < step; ++i) b += hist[i];
        k->stats.first_loss = a / n0;
        k->stats.last_loss = b / n1;
    }
    // ---- embed the database
    t0 = std::chrono::steady_clock::now();
    if ((s = embed_database(k, st)) != TWED_OK) return s;
    k->stats.embed_ms = ms_since(t0);
    t0 = std::chrono::steady_clock::now();
    if ((s = tune_rerank(k, st)) != TWED_OK) return s;
    k->stats.tune_ms = ms_since(t0);
    k->trained = true;
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_get_stats(twed_knn_t k, twed_knn_stats_t* out) {
    if (!k || !out) return TWED_ERR_INVALID_ARG;
    *out = k->stats;
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_get_params(twed_knn_t k, float* out, int64_t n) {
    if (!k || !out) return TWED_ERR_INVALID_ARG;
    if (n != k->enc.L.total) return err(k->h, TWED_ERR_INVALID_ARG, "expected %lld parameters", (long long)k->enc.L.total);
    KNN_CUDA(k->h, cudaDeviceSynchronize());
    KNN_CUDA(k->h, cudaMemcpy(out, k->params.p, sizeof(float) * n, cudaMemcpyDeviceToHost));
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_set_params(twed_knn_t k, const float* in, int64_t n) {
    if (!k || !in) return TWED_ERR_INVALID_ARG;
    if (n != k->enc.L.total) return err(k->h, TWED_ERR_INVALID_ARG, "expected %lld parameters", (long long)k->enc.L.total);
    cudaStream_t st;
    KNN_CUDA(k->h, cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    struct StreamGuard {
        cudaStream_t s;
        ~StreamGuard() { cudaStreamSynchronize(s); cudaStreamDestroy(s); }
    } guard{st};
    KNN_CUDA(k->h, cudaMemcpy(k->params.p, in, sizeof(float) * n, cudaMemcpyHostToDevice));
    if (k->stats.mean_len == 0.0) k->stats.mean_len = k->mean_len;
    KNN_CUDA(k->h, feature_stats(k->db.vals, k->db.ts, k->db.offs, k->db.n, k->db_offs[k->db.n],
                                 k->dim, k->p, k->nu, k->lambda, k->stat_part.as<double>(),
                                 k->mu.as<float>(), k->sd.as<float>(), st));
    twed_status_t s = embed_database(k, st);
    if (s != TWED_OK) return s;
    if (k->rr_rmax == 0) {
        const auto t0 = std::chrono::steady_clock::now();
        if ((s = tune_rerank(k, st)) != TWED_OK) return s;
        k->stats.tune_ms = ms_since(t0);
    }
    k->trained = true;
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_get_embeddings(twed_knn_t k, float* d_out, void* stream) {
    if (!k || !d_out) return TWED_ERR_INVALID_ARG;
    if (!k->trained) return err(k->h, TWED_ERR_INVALID_ARG, "index not trained");
    KNN_CUDA(k->h, cudaMemcpyAsync(d_out, k->emb_db.p, sizeof(float) * k->db.n * EMB,
                                   cudaMemcpyDeviceToDevice, (cudaStream_t)stream));
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_search(twed_knn_t k, const twed_set_f32_t* Q, int kk, int C,
                                         int64_t* d_idx, float* d_dist, void* stream) {
    if (!k || !d_idx || !d_dist) return TWED_ERR_INVALID_ARG;
    twed_handle_t h = k->h;
    if (!k->trained) return err(h, TWED_ERR_INVALID_ARG, "index not trained");
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, Q, "queries", &maxlen);
    if (s != TWED_OK) return s;
    const int64_t N = k->db.n, nq = Q->n;
    if (kk < 1 || C < kk || C > N || C > TOPK_MAX)
        return err(h, TWED_ERR_INVALID_ARG, "need 1 <= k <= n_candidates <= min(ndb, %d)", TOPK_MAX);
    cudaStream_t st = (cudaStream_t)stream;
    KNN_CUDA(h, cudaEventRecord(k->ev[0], st));
    // ---- embed the queries (the encoder's buffers are the index's own)
    KNN_CUDA(h, k->qemb.ensure(sizeof(float) * nq * EMB));
    std::vector<int64_t> ids(nq);
    for (int64_t i = 0; i < nq; ++i) ids[i] = i;
    // query statistics: the database's (the encoder was trained on them)
    s = k->enc.embed(Q, ids, k->params.as<float>(), k->mu.as<float>(), k->sd.as<float>(),
                     (float)(1.0 / k->mean_len), k->qemb.as<float>(), st);
    if (s != TWED_OK) return s;
    KNN_CUDA(h, cudaEventRecord(k->ev[1], st));
    // ---- candidates: L2 rows in query chunks, top-C per row
    const int64_t qc = std::max<int64_t>(1, std::min<int64_t>(nq, ((int64_t)1 << 28) / N));
    KNN_CUDA(h, k->sbuf.ensure(sizeof(float) * qc * N));
    KNN_CUDA(h, k->cand.ensure(sizeof(int64_t) * nq * C));
    KNN_CUDA(h, k->candval.ensure(sizeof(float) * nq * C));
    const int topk_grid = twed::detail::handle_sms(h) * 2;
    for (int64_t q0 = 0; q0 < nq; q0 += qc) {
        const int64_t n = std::min(qc, nq - q0);
        KNN_CUDA(h, l2_rows(k->qemb.as<float>() + q0 * EMB, n, k->svec_db.as<float>(), N,
                            k->sbuf.as<float>(), N, st));
        KNN_CUDA(h, topk_rows(k->sbuf.as<float>(), n, N, N, C, k->cand.as<int64_t>() + q0 * C,
                              k->candval.as<float>() + q0 * C, topk_grid, st));
    }
    // ---- exact re-rank of every (query, candidate) pair, then top-k
    KNN_CUDA(h, k->qpairs.ensure(sizeof(int64_t) * 2 * nq * C));
    KNN_CUDA(h, k->rr.ensure(sizeof(float) * nq * C));
    KNN_CUDA(h, k->pos.ensure(sizeof(int64_t) * nq * kk));
    KNN_CUDA(h, make_pairs(k->cand.as<int64_t>(), nq, C, 0, k->qpairs.as<int64_t>(), st));
    KNN_CUDA(h, pair_cells(k->qpairs.as<int64_t>(), nq * C, Q->offs, k->db.offs,
                           k->cells.as<unsigned long long>(), st));
    KNN_CUDA(h, cudaEventRecord(k->ev[2], st));
    s = twed::detail::batch_f32_shaped(h, Q, &k->db, k->qpairs.as<int64_t>(), nq * C, k->dim,
                                       k->nu, k->lambda, k->p, k->rr.as<float>(), st,
                                       TWED_ORDER_LONGEST_FIRST, k->rr_rmax, k->rr_per_sm);
    if (s != TWED_OK) return s;
    KNN_CUDA(h, cudaEventRecord(k->ev[3], st));
    KNN_CUDA(h, topk_rows(k->rr.as<float>(), nq, C, C, kk, k->pos.as<int64_t>(), d_dist, topk_grid, st));
    KNN_CUDA(h, gather_candidates(k->cand.as<int64_t>(), k->pos.as<int64_t>(), nq, C, kk, d_idx, st));
    KNN_CUDA(h, cudaEventRecord(k->ev[4], st));
    k->searched = true;
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_search_profile(twed_knn_t k, double* phase_ms,
                                                 int64_t* rerank_cells) {
    if (!k || !phase_ms || !rerank_cells) return TWED_ERR_INVALID_ARG;
    if (!k->searched) return err(k->h, TWED_ERR_INVALID_ARG, "no search has run");
    KNN_CUDA(k->h, cudaEventSynchronize(k->ev[4]));
    for (int i = 0; i < 4; ++i) {
        float ms = 0.f;
        KNN_CUDA(k->h, cudaEventElapsedTime(&ms, k->ev[i], k->ev[i + 1]));
        phase_ms[i] = ms;
    }
    unsigned long long c = 0;
    KNN_CUDA(k->h, cudaMemcpy(&c, k->cells.p, sizeof c, cudaMemcpyDeviceToHost));
    *rerank_cells = (int64_t)c;
    return TWED_OK;
}

extern "C" twed_status_t twed_knn_search_host(twed_knn_t k, const float* vals, const float* ts,
                                              const int64_t* offs, int64_t nq, int kk, int C,
                                              int64_t* idx, float* dist) {
    if (!k || !vals || !ts || !offs || !idx || !dist || nq < 1) return TWED_ERR_INVALID_ARG;
    twed_handle_t h = k->h;
    if (offs[0] != 0) return err(h, TWED_ERR_INVALID_ARG, "offs[0] != 0");
    const int64_t total = offs[nq];
    for (int64_t i = 0; i < total * k->dim; ++i)
        if (!std::isfinite(vals[i])) return err(h, TWED_ERR_INVALID_ARG, "non-finite query value");
    for (int64_t i = 0; i < total; ++i)
        if (!std::isfinite(ts[i])) return err(h, TWED_ERR_INVALID_ARG, "non-finite query timestamp");
    cudaStream_t st = k->host_stream;
    KNN_CUDA(h, k->hq_vals.ensure(sizeof(float) * std::max<int64_t>(total * k->dim, 1)));
    KNN_CUDA(h, k->hq_ts.ensure(sizeof(float) * std::max<int64_t>(total, 1)));
    KNN_CUDA(h, k->hq_offs.ensure(sizeof(int64_t) * (nq + 1)));
    KNN_CUDA(h, k->hq_idx.ensure(sizeof(int64_t) * nq * std::max(kk, 1)));
    KNN_CUDA(h, k->hq_dist.ensure(sizeof(float) * nq * std::max(kk, 1)));
    KNN_CUDA(h, cudaMemcpyAsync(k->hq_vals.p, vals, sizeof(float) * total * k->dim, cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaMemcpyAsync(k->hq_ts.p, ts, sizeof(float) * total, cudaMemcpyHostToDevice, st));
    KNN_CUDA(h, cudaMemcpyAsync(k->hq_offs.p, offs, sizeof(int64_t) * (nq + 1), cudaMemcpyHostToDevice, st));
    twed_set_f32_t Q{k->hq_vals.as<float>(), k->hq_ts.as<float>(), k->hq_offs.as<int64_t>(), offs, nq};
    twed_status_t s = twed_knn_search(k, &Q, kk, C, k->hq_idx.as<int64_t>(), k->hq_dist.as<float>(), st);
    if (s != TWED_OK) {
        cudaStreamSynchronize(st);
        return s;
    }
    KNN_CUDA(h, cudaMemcpyAsync(idx, k->hq_idx.p, sizeof(int64_t) * nq * kk, cudaMemcpyDeviceToHost, st));
    KNN_CUDA(h, cudaMemcpyAsync(dist, k->hq_dist.p, sizeof(float) * nq * kk, cudaMemcpyDeviceToHost, st));
    KNN_CUDA(h, cudaStreamSynchronize(st));
    return twed_sync_status(h, st);
}

extern "C" twed_status_t twed_knn_exact(twed_knn_t k, const twed_set_f32_t* Q, int kk,
                                        int64_t* d_idx, float* d_dist, void* stream) {
    if (!k || !d_idx || !d_dist) return TWED_ERR_INVALID_ARG;
    twed_handle_t h = k->h;
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, Q, "queries", &maxlen);
    if (s != TWED_OK) return s;
    const int64_t N = k->db.n, nq = Q->n;
    if (kk < 1 || kk > N || kk > TOPK_MAX)
        return err(h, TWED_ERR_INVALID_ARG, "need 1 <= k <= min(ndb, %d)", TOPK_MAX);
    cudaStream_t st = (cudaStream_t)stream;
    KNN_CUDA(h, k->sbuf.ensure(sizeof(float) * nq * N));
    twed_plan_t plan = nullptr;
    s = twed_allpairs_plan_create_f32(h, Q, &k->db, k->dim, k->nu, k->lambda, k->p, nullptr, &plan);
    if (s != TWED_OK) return s;
    s = twed_plan_execute(plan, k->sbuf.p, st);
    if (s == TWED_OK) {
        cudaError_t e = topk_rows(k->sbuf.as<float>(), nq, N, N, kk, d_idx, d_dist,
                                  twed::detail::handle_sms(h) * 2, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            s = err(h, TWED_ERR_CUDA, "exact k-NN: %s", cudaGetErrorString(e));
        }
    }
    if (s == TWED_OK) s = twed_sync_status(h, st);
    cudaStreamSynchronize(st);
    twed_plan_destroy(plan);
    return s;
}

// ======================================================= building blocks
extern "C" int64_t twed_encoder_param_count(int dim) {
    if (dim < 1 || dim + 2 > MAX_C0) return -1;
    return layout(dim).total;
}

extern "C" twed_status_t twed_encoder_stats_f32(twed_handle_t h, const twed_set_f32_t* set, int dim,
                                                float nu, float lambda, int p, float* d_mu,
                                                float* d_sd) {
    if (!h || !d_mu || !d_sd) return TWED_ERR_INVALID_ARG;
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, set, "set", &maxlen);
    if (s != TWED_OK) return s;
    if ((s = check_params(h, dim, nu, lambda, p)) != TWED_OK) return s;
    DevBuf part;
    KNN_CUDA(h, part.ensure(sizeof(double) * 2 * 1024 * MAX_C0));
    KNN_CUDA(h, feature_stats(set->vals, set->ts, set->offs, set->n, set->offs_host[set->n], dim, p,
                              nu, lambda, part.as<double>(), d_mu, d_sd, nullptr));
    KNN_CUDA(h, cudaDeviceSynchronize());
    return TWED_OK;
}

extern "C" twed_status_t twed_encoder_forward_f32(twed_handle_t h, const twed_set_f32_t* set,
                                                  int dim, float nu, float lambda, int p,
                                                  const float* d_params, const float* d_mu,
                                                  const float* d_sd, float mean_len, float* d_emb) {
    if (!h || !d_params || !d_mu || !d_sd || !d_emb) return TWED_ERR_INVALID_ARG;
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, set, "set", &maxlen);
    if (s != TWED_OK) return s;
    if ((s = check_params(h, dim, nu, lambda, p)) != TWED_OK) return s;
    if (!(mean_len > 0.f)) return err(h, TWED_ERR_INVALID_ARG, "mean_len must be > 0");
    Encoder enc;
    if ((s = enc.init(h, dim, p, nu, lambda)) != TWED_OK) return s;
    std::vector<int64_t> ids(set->n);
    for (int64_t i = 0; i < set->n; ++i) ids[i] = i;
    s = enc.embed(set, ids, d_params, d_mu, d_sd, 1.0f / mean_len, d_emb, nullptr);
    if (s != TWED_OK) return s;
    KNN_CUDA(h, cudaDeviceSynchronize());
    return TWED_OK;
}

extern "C" twed_status_t twed_encoder_loss_grad_f32(
    twed_handle_t h, const twed_set_f32_t* set, int dim, float nu, float lambda, int p,
    const float* d_params, const float* d_mu, const float* d_sd, float mean_len,
    const int64_t* groups, int64_t ngroups, int gsize, const float* d_labels, float inv_sigma,
    float* d_grad, float* d_loss) {
    if (!h || !d_params || !d_mu || !d_sd || !groups || !d_labels || !d_grad || !d_loss)
        return TWED_ERR_INVALID_ARG;
    int64_t maxlen = 0;
    twed_status_t s = check_set_host(h, set, "set", &maxlen);
    if (s != TWED_OK) return s;
    if ((s = check_params(h, dim, nu, lambda, p)) != TWED_OK) return s;
    if (gsize < 2 || gsize > 64 || ngroups < 1)
        return err(h, TWED_ERR_INVALID_ARG, "need 2 <= group_size <= 64 and ngroups >= 1");
    if (!(mean_len > 0.f) || !std::isfinite(inv_sigma))
        return err(h, TWED_ERR_INVALID_ARG, "mean_len must be > 0 and inv_sigma finite");
    for (int64_t i = 0; i < ngroups * gsize; ++i)
        if (groups[i] < 0 || groups[i] >= set->n)
            return err(h, TWED_ERR_INVALID_ARG, "group member %lld out of range", (long long)i);
    Encoder enc;
    if ((s = enc.init(h, dim, p, nu, lambda)) != TWED_OK) return s;
    const int64_t nser = ngroups * gsize;
    std::vector<int64_t> gids(ngroups), base;
    for (int64_t g = 0; g < ngroups; ++g) gids[g] = g;
    const int64_t P = Encoder::batch_rows(set->offs_host, groups, nser, base);
    if ((s = enc.reserve(P, nser, ngroups, true)) != TWED_OK) return s;
    DevBuf isg, meta;
    KNN_CUDA(h, isg.ensure(sizeof(float)));
    KNN_CUDA(h, meta.ensure(sizeof(int64_t) * (2 * nser + 1 + ngroups)));
    int64_t* d_ids = meta.as<int64_t>();
    int64_t* d_base = d_ids + nser;
    int64_t* d_gids = d_base + nser + 1;
    KNN_CUDA(h, cudaMemcpy(isg.p, &inv_sigma, sizeof(float), cudaMemcpyHostToDevice));
    KNN_CUDA(h, cudaMemcpy(d_ids, groups, sizeof(int64_t) * nser, cudaMemcpyHostToDevice));
    KNN_CUDA(h, cudaMemcpy(d_base, base.data(), sizeof(int64_t) * (nser + 1), cudaMemcpyHostToDevice));
    KNN_CUDA(h, cudaMemcpy(d_gids, gids.data(), sizeof(int64_t) * ngroups, cudaMemcpyHostToDevice));
    KNN_CUDA(h, transform_weights(d_params, enc.L, enc.cin, enc.views(), nullptr));
    s = enc.loss_grad(set, d_ids, d_base, P, ngroups, gsize, d_gids, d_labels, isg.as<float>(),
                      d_params, d_mu, d_sd, 1.0f / mean_len, d_grad, d_loss, nullptr);
    if (s != TWED_OK) return s;
    KNN_CUDA(h, cudaDeviceSynchronize());
    return TWED_OK;
}

extern "C" twed_status_t twed_adam_f32(twed_handle_t h, float* th, const float* g, float* m,
                                       float* v, int64_t n, int64_t step, float lr, float b1,
                                       float b2, float eps) {
    if (!h || !th || !g || !m || !v || n < 0 || step < 1) return TWED_ERR_INVALID_ARG;
    const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)step)));
    KNN_CUDA(h, adam(th, g, m, v, n, lr, b1, b2, eps, c1, c2, nullptr));
    KNN_CUDA(h, cudaDeviceSynchronize());
    return TWED_OK;
}

extern "C" twed_status_t twed_embed_search_f32(twed_handle_t h, const float* d_db, int64_t ndb,
                                               const float* d_q, int64_t nq, int k, int64_t* d_idx,
                                               float* d_val) {
    if (!h || !d_db || !d_q || !d_idx || !d_val || ndb < 1 || nq < 1) return TWED_ERR_INVALID_ARG;
    if (k < 1 || k > ndb || k > TOPK_MAX)
        return err(h, TWED_ERR_INVALID_ARG, "need 1 <= k <= min(ndb, %d)", TOPK_MAX);
    DevBuf sv, D, zm;
    KNN_CUDA(h, sv.ensure(sizeof(float) * ndb * EMB));
    KNN_CUDA(h, D.ensure(sizeof(float) * nq * ndb));
    KNN_CUDA(h, zm.ensure(sizeof(float)));
    KNN_CUDA(h, search_vectors(d_db, ndb, zm.as<float>(), sv.as<float>(), nullptr));
    KNN_CUDA(h, l2_rows(d_q, nq, sv.as<float>(), ndb, D.as<float>(), ndb, nullptr));
    KNN_CUDA(h, topk_rows(D.as<float>(), nq, ndb, ndb, k, d_idx, d_val,
                          twed::detail::handle_sms(h) * 2, nullptr));
    KNN_CUDA(h, cudaDeviceSynchronize());
    return TWED_OK;
}

extern "C" twed_status_t twed_topk_rows_f32(twed_handle_t h, const float* d_D, int64_t rows,
                                            int64_t cols, int64_t ld, int k, int64_t* d_idx,
                                            float* d_val, void* stream) {
    if (!h || !d_D || !d_idx || !d_val || rows < 0 || cols < 1 || ld < cols) return TWED_ERR_INVALID_ARG;
    if (k < 1 || k > cols || k > TOPK_MAX || cols >= ((int64_t)1 << 31))
        return err(h, TWED_ERR_INVALID_ARG, "need 1 <= k <= min(cols, %d) and cols < 2^31", TOPK_MAX);
    KNN_CUDA(h, topk_rows(d_D, rows, cols, ld, k, d_idx, d_val, twed::detail::handle_sms(h) * 2,
                          (cudaStream_t)stream));
    return TWED_OK;
}
