// Learned k-NN filter kernels: the 1-D convolutional encoder (forward,
// backward, Adam), the embedding search and a row-wise radix top-k.
//
// All arithmetic is FP32 with FP32 accumulation, except the feature
// statistics (FP64 sums).  Every reduction runs in a fixed order (partials
// per block, then one ordered pass), so results do not depend on timing.
// The encoder is a small dense contraction (27 MFLOP per series of 320
// points) that runs on the CUDA cores; the exact TWED re-ranking it feeds
// dominates the query time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "encoder.h"

namespace twed {
namespace enc {

Layout layout(int dim) {
    Layout L;
    L.c0 = dim + 2;
    int64_t o = 0;
    L.w1 = o; o += (int64_t)CH * L.c0 * TAPS;
    L.b1 = o; o += CH;
    L.w2 = o; o += (int64_t)CH * CH * TAPS;
    L.b2 = o; o += CH;
    L.w3 = o; o += (int64_t)CH * CH * TAPS;
    L.b3 = o; o += CH;
    L.wl = o; o += (int64_t)EMB * CH;
    L.bl = o; o += EMB;
    L.total = o;
    return L;
}

size_t weight_views_floats(int cin) {
    return (size_t)cin * TAPS * CH + 4 * (size_t)CH * TAPS * CH;
}

void carve_weight_views(float* base, int cin, WeightViews* w) {
    w->wt1 = base;
    w->wt2 = w->wt1 + (size_t)cin * TAPS * CH;
    w->wt3 = w->wt2 + (size_t)CH * TAPS * CH;
    w->wb2 = w->wt3 + (size_t)CH * TAPS * CH;
    w->wb3 = w->wb2 + (size_t)CH * TAPS * CH;
}

namespace {

// ------------------------------------------------------------ input features
// d(x, y) of two points (|x - y| for dim 1), FP32.
__device__ __forceinline__ float point_dist(const float* x, const float* y, int dim, int p) {
    if (dim == 1) return fabsf(x[0] - y[0]);
    float s = 0.f;
    if (p == 1) {
        for (int k = 0; k < dim; ++k) s += fabsf(x[k] - y[k]);
        return s;
    }
    if (p == 2) {
        for (int k = 0; k < dim; ++k) {
            const float d = x[k] - y[k];
            s += d * d;
        }
        return sqrtf(s);
    }
    for (int k = 0; k < dim; ++k) s += powf(fabsf(x[k] - y[k]), (float)p);
    return powf(s, 1.0f / (float)p);
}

// Raw features of point `row` of a series whose first point is `first`:
// values, timestamp, delete cost with the zero padding before the first point.
__device__ __forceinline__ void point_features(const float* vals, const float* ts, int64_t row,
                                               int64_t first, int dim, int p, float nu,
                                               float lambda, float* f) {
    const float* a = vals + row * dim;
    float zero[MAX_C0];
    const float* prev;
    float tprev;
    if (row == first) {
        for (int k = 0; k < dim; ++k) zero[k] = 0.f;
        prev = zero;
        tprev = 0.f;
    } else {
        prev = a - dim;
        tprev = ts[row - 1];
    }
    for (int k = 0; k < dim; ++k) f[k] = a[k];
    f[dim] = ts[row];
    f[dim + 1] = point_dist(a, prev, dim, p) + nu * fabsf(ts[row] - tprev) + lambda;
}

__global__ void gather_kernel(const float* __restrict__ vals, const float* __restrict__ ts,
                              const int64_t* __restrict__ offs, const int64_t* __restrict__ ids,
                              const int64_t* __restrict__ base, int dim, int p, float nu,
                              float lambda, const float* __restrict__ mu,
                              const float* __restrict__ sd, int cin, float* __restrict__ X0,
                              int32_t* __restrict__ rseries) {
    const int64_t s = blockIdx.x;
    const int64_t src0 = offs[ids[s]];
    const int64_t len = offs[ids[s] + 1] - src0;
    const int64_t dst0 = base[s];
    const int c0 = dim + 2;
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) {
        float f[MAX_C0];
        point_features(vals, ts, src0 + i, src0, dim, p, nu, lambda, f);
        float* out = X0 + (dst0 + i) * cin;
        for (int c = 0; c < cin; ++c) out[c] = c < c0 ? (f[c] - mu[c]) / sd[c] : 0.f;
        rseries[dst0 + i] = (int32_t)s;
    }
}

constexpr int kStatBlocks = 1024;
constexpr int kStatThreads = 256;

// Pass 1 (mode 0): per-block sums of f; pass 2 (mode 1): sums of (f - mean)^2.
__global__ void __launch_bounds__(kStatThreads)
stats_kernel(const float* __restrict__ vals, const float* __restrict__ ts,
             const int64_t* __restrict__ offs, int64_t nser, int dim, int p, float nu,
             float lambda, const double* __restrict__ mean, int mode, double* __restrict__ part) {
    const int c0 = dim + 2;
    double acc[MAX_C0];
    for (int c = 0; c < c0; ++c) acc[c] = 0.0;
    // series-major walk: block b takes series b, b + gridDim.x, ...
    for (int64_t s = blockIdx.x; s < nser; s += gridDim.x) {
        const int64_t lo = offs[s], hi = offs[s + 1];
        for (int64_t r = lo + threadIdx.x; r < hi; r += blockDim.x) {
            float f[MAX_C0];
            point_features(vals, ts, r, lo, dim, p, nu, lambda, f);
            for (int c = 0; c < c0; ++c) {
                const double v = (double)f[c];
                if (mode == 0) {
                    acc[c] += v;
                } else {
                    const double d = v - mean[c];
                    acc[c] += d * d;
                }
            }
        }
    }
    __shared__ double red[kStatThreads];
    for (int c = 0; c < c0; ++c) {
        red[threadIdx.x] = acc[c];
        __syncthreads();
        for (int w = kStatThreads / 2; w > 0; w >>= 1) {
            if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
            __syncthreads();
        }
        if (threadIdx.x == 0) part[(int64_t)blockIdx.x * MAX_C0 + c] = red[0];
        __syncthreads();
    }
}

// One thread per channel sums the block partials in order.
__global__ void stats_finish_kernel(const double* __restrict__ part, int nblocks, int c0,
                                    int64_t npoints, int mode, double* __restrict__ mean,
                                    float* __restrict__ out) {
    const int c = threadIdx.x;
    if (c >= c0) return;
    double s = 0.0;
    for (int b = 0; b < nblocks; ++b) s += part[(int64_t)b * MAX_C0 + c];
    const double m = s / (double)npoints;
    if (mode == 0) {
        mean[c] = m;
        out[c] = (float)m;
    } else {
        const double sd = sqrt(m);
        out[c] = sd > 0.0 ? (float)sd : 1.0f;
    }
}

// ------------------------------------------------------------------ weights
__global__ void transform_kernel(const float* __restrict__ prm, int c0, int cin, int64_t ow1,
                                 int64_t ow2, int64_t ow3, float* __restrict__ wt1,
                                 float* __restrict__ wt2, float* __restrict__ wt3,
                                 float* __restrict__ wb2, float* __restrict__ wb3) {
    const int64_t n1 = (int64_t)cin * TAPS * CH, n2 = (int64_t)CH * TAPS * CH;
    const int64_t total = n1 + 4 * n2;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i < n1) {
            // wt1[ci][k][o] = W1[o][ci][k]
            const int o = (int)(i % CH), k = (int)((i / CH) % TAPS), ci = (int)(i / (CH * TAPS));
            wt1[i] = ci < c0 ? prm[ow1 + ((int64_t)o * c0 + ci) * TAPS + k] : 0.f;
            continue;
        }
        int64_t j = i - n1;
        const int which = (int)(j / n2);
        j -= which * n2;
        const int a = (int)(j / (CH * TAPS)), k = (int)((j / CH) % TAPS), b = (int)(j % CH);
        const int64_t ow = (which == 0 || which == 2) ? ow2 : ow3;
        if (which < 2) {
            // wt[ci=a][k][o=b] = W[o][ci][k]
            (which == 0 ? wt2 : wt3)[j] = prm[ow + ((int64_t)b * CH + a) * TAPS + k];
        } else {
            // wb[o=a][k][ci=b] = W[o][ci][4-k]
            (which == 2 ? wb2 : wb3)[j] = prm[ow + ((int64_t)a * CH + b) * TAPS + (TAPS - 1 - k)];
        }
    }
}

// ------------------------------------------------------------- convolution
// Y[p][o] = sum_ci sum_k wt[ci][k][o] * X[p + k - 2][ci]  over one tile of TM
// output rows; 256 threads, thread = 8 rows x 4 outputs.  The weights stay
// in shared memory across the tiles of a persistent block.
enum { kEpiBiasRelu = 0, kEpiMask = 1 };
constexpr int kConvThreads = 256;
constexpr int kXsLd = TM + 4;

template <int CIN, int EPI>
__global__ void __launch_bounds__(kConvThreads, 1)
conv_kernel(const float* __restrict__ X, int64_t P, const float* __restrict__ wt,
            const float* __restrict__ bias, const float* __restrict__ M,
            const int32_t* __restrict__ rseries, float* __restrict__ Y) {
    extern __shared__ float4 smem4[];
    float* Ws = reinterpret_cast<float*>(smem4);   // [CIN][5][64]
    float* xs = Ws + CIN * TAPS * CH;              // [CIN][kXsLd]
    const int tid = threadIdx.x;
    for (int i = tid; i < CIN * TAPS * CH / 4; i += kConvThreads)
        smem4[i] = reinterpret_cast<const float4*>(wt)[i];
    const int cg = tid & 15, rg = tid >> 4;
    const int o0 = cg * 4, r0 = rg * 8;
    float4 bv = make_float4(0.f, 0.f, 0.f, 0.f);
    if (EPI == kEpiBiasRelu) bv = *reinterpret_cast<const float4*>(bias + o0);
    const int64_t ntiles = (P + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * TM;
        __syncthreads();
        for (int i = tid; i < (TM + 4) * (CIN / 4); i += kConvThreads) {
            const int j = i / (CIN / 4), c4 = i % (CIN / 4);
            const int64_t row = base - 2 + j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row >= 0 && row < P) v = *reinterpret_cast<const float4*>(X + row * CIN + c4 * 4);
            xs[(c4 * 4 + 0) * kXsLd + j] = v.x;
            xs[(c4 * 4 + 1) * kXsLd + j] = v.y;
            xs[(c4 * 4 + 2) * kXsLd + j] = v.z;
            xs[(c4 * 4 + 3) * kXsLd + j] = v.w;
        }
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[r][c] = 0.f;
#pragma unroll 2
        for (int ci = 0; ci < CIN; ++ci) {
            const float4* xp = reinterpret_cast<const float4*>(xs + ci * kXsLd + r0);
            const float4 xa = xp[0], xb = xp[1], xc = xp[2];
            const float x[12] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y,
                                 xb.z, xb.w, xc.x, xc.y, xc.z, xc.w};
#pragma unroll
            for (int k = 0; k < TAPS; ++k) {
                const float4 w = *reinterpret_cast<const float4*>(Ws + (ci * TAPS + k) * CH + o0);
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    acc[r][0] = fmaf(x[r + k], w.x, acc[r][0]);
                    acc[r][1] = fmaf(x[r + k], w.y, acc[r][1]);
                    acc[r][2] = fmaf(x[r + k], w.z, acc[r][2]);
                    acc[r][3] = fmaf(x[r + k], w.w, acc[r][3]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < 8; ++r) {
            const int64_t row = base + r0 + r;
            if (row >= P) break;
            float4 out;
            if (EPI == kEpiBiasRelu) {
                const bool valid = rseries[row] >= 0;
                out.x = valid ? fmaxf(acc[r][0] + bv.x, 0.f) : 0.f;
                out.y = valid ? fmaxf(acc[r][1] + bv.y, 0.f) : 0.f;
                out.z = valid ? fmaxf(acc[r][2] + bv.z, 0.f) : 0.f;
                out.w = valid ? fmaxf(acc[r][3] + bv.w, 0.f) : 0.f;
            } else {
                const float4 m = *reinterpret_cast<const float4*>(M + row * CH + o0);
                out.x = m.x > 0.f ? acc[r][0] : 0.f;
                out.y = m.y > 0.f ? acc[r][1] : 0.f;
                out.z = m.z > 0.f ? acc[r][2] : 0.f;
                out.w = m.w > 0.f ? acc[r][3] : 0.f;
            }
            *reinterpret_cast<float4*>(Y + row * CH + o0) = out;
        }
    }
}

// ----------------------------------------------------------- weight gradient
// part[b][o][ci][k] = sum over the rows this block (and row split) visits of
// dY[p][o] * X[p + k - 2][ci];  part[b][64*CIN*5 + o] = sum of dY[p][o].
// Thread = 4 outputs x 4 input channels x 5 taps; RS row splits share a tile
// when CIN < 64.
template <int CIN>
struct WgradShape {
    static constexpr int CG = CIN / 4;
    static constexpr int RS = 256 / (16 * CG);
    static constexpr int PART = CH * CIN * TAPS + CH;
};

template <int CIN>
__global__ void __launch_bounds__(256, 1)
wgrad_kernel(const float* __restrict__ X, const float* __restrict__ dY, int64_t P,
             float* __restrict__ part) {
    using S = WgradShape<CIN>;
    extern __shared__ float4 smem4[];
    float* dys = reinterpret_cast<float*>(smem4);   // [TM][64]
    float* xs = dys + TM * CH;                      // [TM + 4][CIN]
    const int tid = threadIdx.x;
    const int og = tid & 15, cgi = (tid >> 4) % S::CG, rs = tid / (16 * S::CG);
    float acc[4][4][TAPS];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int k = 0; k < TAPS; ++k) acc[a][b][k] = 0.f;
    float accb[4] = {0.f, 0.f, 0.f, 0.f};
    const int64_t ntiles = (P + TM - 1) / TM;
    for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int64_t base = tile * TM;
        __syncthreads();
        for (int i = tid; i < TM * CH / 4; i += 256) {
            const int j = i / (CH / 4);
            const int64_t row = base + j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row < P) v = reinterpret_cast<const float4*>(dY + row * CH)[i % (CH / 4)];
            smem4[i] = v;
        }
        for (int i = tid; i < (TM + 4) * (CIN / 4); i += 256) {
            const int j = i / (CIN / 4);
            const int64_t row = base - 2 + j;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (row >= 0 && row < P) v = reinterpret_cast<const float4*>(X + row * CIN)[i % (CIN / 4)];
            reinterpret_cast<float4*>(xs)[i] = v;
        }
        __syncthreads();
        if (S::RS == 1) {
            float4 xw[TAPS];
#pragma unroll
            for (int k = 0; k < TAPS - 1; ++k)
                xw[k + 1] = *reinterpret_cast<const float4*>(xs + k * CIN + cgi * 4);
            for (int r = 0; r < TM; ++r) {
#pragma unroll
                for (int k = 0; k < TAPS - 1; ++k) xw[k] = xw[k + 1];
                xw[TAPS - 1] = *reinterpret_cast<const float4*>(xs + (r + TAPS - 1) * CIN + cgi * 4);
                const float4 dy = *reinterpret_cast<const float4*>(dys + r * CH + og * 4);
                const float d[4] = {dy.x, dy.y, dy.z, dy.w};
#pragma unroll
                for (int k = 0; k < TAPS; ++k) {
                    const float x[4] = {xw[k].x, xw[k].y, xw[k].z, xw[k].w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b][k] = fmaf(d[a], x[b], acc[a][b][k]);
                }
                if (cgi == 0)
#pragma unroll
                    for (int a = 0; a < 4; ++a) accb[a] += d[a];
            }
        } else {
            for (int r = rs; r < TM; r += S::RS) {
                const float4 dy = *reinterpret_cast<const float4*>(dys + r * CH + og * 4);
                const float d[4] = {dy.x, dy.y, dy.z, dy.w};
#pragma unroll
                for (int k = 0; k < TAPS; ++k) {
                    const float4 xv = *reinterpret_cast<const float4*>(xs + (r + k) * CIN + cgi * 4);
                    const float x[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                    for (int a = 0; a < 4; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b) acc[a][b][k] = fmaf(d[a], x[b], acc[a][b][k]);
                }
                if (cgi == 0)
#pragma unroll
                    for (int a = 0; a < 4; ++a) accb[a] += d[a];
            }
        }
    }
    float* out = part + ((int64_t)blockIdx.x * S::RS + rs) * S::PART;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b)
#pragma unroll
            for (int k = 0; k < TAPS; ++k)
                out[((og * 4 + a) * CIN + cgi * 4 + b) * TAPS + k] = acc[a][b][k];
    if (cgi == 0)
#pragma unroll
        for (int a = 0; a < 4; ++a) out[CH * CIN * TAPS + og * 4 + a] = accb[a];
}

__global__ void wgrad_reduce_kernel(const float* __restrict__ part, int nparts, int cin, int c0,
                                    float* __restrict__ gW, float* __restrict__ gB) {
    const int64_t nw = (int64_t)CH * c0 * TAPS;
    const int64_t stride = (int64_t)CH * cin * TAPS + CH;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nw + CH;
         i += (int64_t)gridDim.x * blockDim.x) {
        int64_t src;
        if (i < nw) {
            const int64_t o = i / (c0 * TAPS), ci = (i / TAPS) % c0, k = i % TAPS;
            src = (o * cin + ci) * TAPS + k;
        } else {
            src = (int64_t)CH * cin * TAPS + (i - nw);
        }
        float s = 0.f;
        for (int b = 0; b < nparts; ++b) s += part[(int64_t)b * stride + src];
        if (i < nw) gW[i] = s;
        else gB[i - nw] = s;
    }
}

// --------------------------------------------------------- pool and linear
// pooled[s][c] = inv_mean_len * sum_t H3[base_s + t][c];  emb = Wl pooled + bl.
__global__ void __launch_bounds__(256)
pool_kernel(const float* __restrict__ H3, const int64_t* __restrict__ base, float inv_mean_len,
            const float* __restrict__ Wl, const float* __restrict__ bl, float* __restrict__ pooled,
            float* __restrict__ emb) {
    const int64_t s = blockIdx.x;
    const int64_t r0 = base[s], len = base[s + 1] - base[s] - 2;
    const int c = threadIdx.x & 63, g = threadIdx.x >> 6;
    float acc = 0.f;
    for (int64_t t = g; t < len; t += 4) acc += H3[(r0 + t) * CH + c];
    __shared__ float red[4][CH];
    __shared__ float pl[CH];
    red[g][c] = acc;
    __syncthreads();
    if (g == 0) {
        const float v = ((red[0][c] + red[1][c]) + red[2][c]) + red[3][c];
        pl[c] = v * inv_mean_len;
        pooled[s * CH + c] = pl[c];
    }
    __syncthreads();
    if (threadIdx.x < EMB) {
        const int j = threadIdx.x;
        float e = bl[j];
        for (int k = 0; k < CH; ++k) e = fmaf(Wl[j * CH + k], pl[k], e);
        emb[s * EMB + j] = e;
    }
}

// One block per group of G series (batch series gi*G .. gi*G + G - 1):
// r_ab = |psi_a - psi_b|^2 + z_a + z_b - y_ab * inv_sigma for a < b, weight
// w_ab = 1 (rel_floor = 0) or 1 / (y_ab * inv_sigma + rel_floor)^2 (a relative
// error, which weighs near pairs as much as far ones),
// de[a] = inv_npairs * sum_b 2 w_ab r_ab * d(model)/d e_a, dpooled[a] = Wl^T de[a],
// gloss[gi] = sum w_ab r_ab^2.
constexpr int kMaxGroup = 64;
__global__ void __launch_bounds__(256)
group_loss_kernel(const float* __restrict__ emb, int gsize, const int64_t* __restrict__ gids,
                  const float* __restrict__ labels, const float* __restrict__ inv_sigma,
                  float inv_npairs, float rel_floor, const float* __restrict__ Wl, float* __restrict__ de,
                  float* __restrict__ dpooled, float* __restrict__ gloss) {
    __shared__ float e[kMaxGroup][EMB + 1];
    __shared__ float r[kMaxGroup][kMaxGroup];  // w_ab r_ab
    __shared__ float wsum[8];
    __shared__ float dE[kMaxGroup][EMB + 1];
    const int G = gsize;
    const int64_t gi = blockIdx.x;
    const int64_t s0 = gi * G;
    const int npg = G * (G - 1) / 2;
    const float* lab = labels + gids[gi] * npg;
    const float isg = *inv_sigma;
    for (int i = threadIdx.x; i < G * EMB; i += blockDim.x) e[i / EMB][i % EMB] = emb[(s0 + i / EMB) * EMB + i % EMB];
    __syncthreads();
    float lacc = 0.f;
    for (int q = threadIdx.x; q < npg; q += blockDim.x) {
        // invert the row-major triangle index q -> (a, b), a < b
        int a = 0, rem = q;
        while (rem >= G - 1 - a) {
            rem -= G - 1 - a;
            ++a;
        }
        const int b = a + 1 + rem;
        float d2 = 0.f;
        for (int j = 0; j < PSI; ++j) {
            const float d = e[a][j] - e[b][j];
            d2 = fmaf(d, d, d2);
        }
        const float y = lab[q] * isg;
        const float rv = (d2 + e[a][PSI] + e[b][PSI]) - y;
        float w = 1.f;
        if (rel_floor > 0.f) {
            const float iy = 1.f / (y + rel_floor);
            w = iy * iy;
        }
        lacc = fmaf(w * rv, rv, lacc);
        r[a][b] = w * rv;
        r[b][a] = w * rv;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G * EMB; i += blockDim.x) {
        const int a = i / EMB, j = i % EMB;
        float acc = 0.f;
        for (int b = 0; b < G; ++b) {
            if (b == a) continue;
            const float c = 2.f * r[a][b];
            acc += j < PSI ? c * (2.f * (e[a][j] - e[b][j])) : c;
        }
        dE[a][j] = acc * inv_npairs;
        de[(s0 + a) * EMB + j] = dE[a][j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < G * CH; i += blockDim.x) {
        const int a = i / CH, c = i % CH;
        float acc = 0.f;
        for (int j = 0; j < EMB; ++j) acc = fmaf(Wl[j * CH + c], dE[a][j], acc);
        dpooled[(s0 + a) * CH + c] = acc;
    }
    for (int o = 16; o > 0; o >>= 1) lacc += __shfl_down_sync(0xffffffffu, lacc, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = lacc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float acc = 0.f;
        for (int w = 0; w < 8; ++w) acc += wsum[w];
        gloss[gi] = acc;
    }
}

// dPre[p][c] = (H3[p][c] > 0) ? dpooled[rseries[p]][c] * inv_mean_len : 0.
__global__ void pool_backward_kernel(const float* __restrict__ H3, const int32_t* __restrict__ rseries,
                                     const float* __restrict__ dpooled, float inv_mean_len,
                                     int64_t P, float* __restrict__ dPre) {
    const int64_t n4 = P * (CH / 4);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / (CH / 4);
        const int c = (int)(i % (CH / 4)) * 4;
        const int s = rseries[row];
        float4 out = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s >= 0) {
            const float4 h = reinterpret_cast<const float4*>(H3)[i];
            const float4 g = *reinterpret_cast<const float4*>(dpooled + (int64_t)s * CH + c);
            out.x = h.x > 0.f ? g.x * inv_mean_len : 0.f;
            out.y = h.y > 0.f ? g.y * inv_mean_len : 0.f;
            out.z = h.z > 0.f ? g.z * inv_mean_len : 0.f;
            out.w = h.w > 0.f ? g.w * inv_mean_len : 0.f;
        }
        reinterpret_cast<float4*>(dPre)[i] = out;
    }
}

// gWl[j][c] = sum_s de[s][j] pooled[s][c];  gbl[j] = sum_s de[s][j].
__global__ void linear_grad_kernel(const float* __restrict__ de, const float* __restrict__ pooled,
                                   int64_t nser, float* __restrict__ gWl, float* __restrict__ gbl) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < EMB * CH) {
        const int j = i / CH, c = i % CH;
        float acc = 0.f;
        for (int64_t s = 0; s < nser; ++s) acc = fmaf(de[s * EMB + j], pooled[s * CH + c], acc);
        gWl[i] = acc;
    } else if (i < EMB * CH + EMB) {
        const int j = i - EMB * CH;
        float acc = 0.f;
        for (int64_t s = 0; s < nser; ++s) acc += de[s * EMB + j];
        gbl[j] = acc;
    }
}

// Adam (Kingma and Ba, Algorithm 1) with c1 = 1/(1-beta1^t), c2 = 1/(1-beta2^t).
__global__ void adam_kernel(float* __restrict__ th, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, int64_t n, float lr,
                            float b1, float b2, float eps, float c1, float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        th[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
    }
}

__global__ void __launch_bounds__(1024) sum_kernel(const float* __restrict__ x, int64_t n,
                                                   double scale, float* __restrict__ out) {
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += (double)x[i];
    __shared__ double red[1024];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = (float)(red[0] * scale);
}

// -------------------------------------------------------------------- search
__device__ __forceinline__ unsigned ordered_bits(float f) {
    const unsigned u = __float_as_uint(f);
    if (f != f) return 0xFFFFFFFFu;
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_ordered(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void __launch_bounds__(1024) zmin_kernel(const float* __restrict__ emb, int64_t n,
                                                    float* __restrict__ zmin) {
    unsigned best = 0xFFFFFFFFu;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) best = min(best, ordered_bits(emb[i * EMB + PSI]));
    for (int o = 16; o > 0; o >>= 1) best = min(best, __shfl_down_sync(0xffffffffu, best, o));
    __shared__ unsigned wb[32];
    if ((threadIdx.x & 31) == 0) wb[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned b = wb[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) b = min(b, wb[w]);
        zmin[0] = from_ordered(b);
    }
}

__global__ void svec_kernel(const float* __restrict__ emb, int64_t n, const float* __restrict__ zmin,
                            float* __restrict__ svec) {
    const float zm = zmin[0];
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * EMB;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(i % EMB);
        svec[i] = j < PSI ? emb[i] : sqrtf(fmaxf(emb[i] - zm, 0.f));
    }
}

// Tile: 32 queries x 128 database rows; thread = 4 queries x 4 rows.
__global__ void __launch_bounds__(256)
l2_kernel(const float* __restrict__ qemb, int64_t nq, const float* __restrict__ svec, int64_t nx,
          float* __restrict__ D, int64_t ld) {
    __shared__ float qs[32][EMB + 1];
    __shared__ float xs[128][EMB + 1];
    const int64_t q0 = blockIdx.y * 32LL, x0 = blockIdx.x * 128LL;
    for (int i = threadIdx.x; i < 32 * EMB; i += 256) {
        const int r = i / EMB, j = i % EMB;
        qs[r][j] = (q0 + r < nq && j < PSI) ? qemb[(q0 + r) * EMB + j] : 0.f;
    }
    for (int i = threadIdx.x; i < 128 * EMB; i += 256) {
        const int r = i / EMB, j = i % EMB;
        xs[r][j] = (x0 + r < nx) ? svec[(x0 + r) * EMB + j] : 0.f;
    }
    __syncthreads();
    const int tq = threadIdx.x >> 5, tx = threadIdx.x & 31;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
#pragma unroll 8
    for (int j = 0; j < EMB; ++j) {
        float qv[4], xv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) qv[a] = qs[tq * 4 + a][j];
#pragma unroll
        for (int b = 0; b < 4; ++b) xv[b] = xs[tx + 32 * b][j];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const float d = qv[a] - xv[b];
                acc[a][b] = fmaf(d, d, acc[a][b]);
            }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int64_t q = q0 + tq * 4 + a;
        if (q >= nq) continue;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t x = x0 + tx + 32 * b;
            if (x < nx) D[q * ld + x] = acc[a][b];
        }
    }
}

// Row-wise top-k: 8-bit radix select of the k-th smallest key (4 passes with
// warp-aggregated shared histograms), an ordered compaction that keeps every
// key below the threshold and the first equal keys by column, then a bitonic
// sort of (key, column) pairs.
constexpr int kTopkThreads = 1024;
__global__ void __launch_bounds__(kTopkThreads)
topk_kernel(const float* __restrict__ D, int64_t rows, int64_t cols, int64_t ld, int k,
            int64_t* __restrict__ out_idx, float* __restrict__ out_val) {
    __shared__ unsigned hist[256];
    __shared__ unsigned long long sel[TOPK_MAX];
    __shared__ unsigned s_digit, s_kk;
    __shared__ unsigned wlt[32], weq[32];
    __shared__ unsigned s_nlt, s_neq;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kTopkThreads / 32;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const float* d = D + row * ld;
        unsigned prefix = 0u, mask = 0u, kk = (unsigned)k;
        for (int pass = 0; pass < 4; ++pass) {
            const int shift = 24 - 8 * pass;
            for (int i = tid; i < 256; i += kTopkThreads) hist[i] = 0u;
            __syncthreads();
            for (int64_t i0 = 0; i0 < cols; i0 += kTopkThreads) {
                const int64_t i = i0 + tid;
                const bool in = i < cols;
                const unsigned key = in ? ordered_bits(d[i]) : 0u;
                const bool take = in && ((key & mask) == prefix);
                const unsigned dig = (key >> shift) & 255u;
                const unsigned act = __ballot_sync(0xffffffffu, take);
                if (take) {
                    const unsigned peers = __match_any_sync(act, dig);
                    if (lane == __ffs(peers) - 1) atomicAdd(&hist[dig], (unsigned)__popc(peers));
                }
            }
            __syncthreads();
            if (warp == 0) {
                unsigned c[8], tot = 0;
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    c[j] = hist[lane * 8 + j];
                    tot += c[j];
                }
                unsigned incl = tot;
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                unsigned before = incl - tot;
                if (before < kk && kk <= incl) {
                    for (int j = 0; j < 8; ++j) {
                        if (before + c[j] >= kk) {
                            s_digit = (unsigned)(lane * 8 + j);
                            s_kk = kk - before;
                            break;
                        }
                        before += c[j];
                    }
                }
            }
            __syncthreads();
            prefix |= s_digit << shift;
            mask |= 255u << shift;
            kk = s_kk;
            __syncthreads();
        }
        // prefix is the k-th smallest key; take k - kk keys below it and the
        // first kk keys equal to it, in column order
        const unsigned nlt_total = (unsigned)k - kk;
        if (tid == 0) {
            s_nlt = 0u;
            s_neq = 0u;
        }
        __syncthreads();
        for (int64_t i0 = 0; i0 < cols; i0 += kTopkThreads) {
            const int64_t i = i0 + tid;
            const bool in = i < cols;
            const unsigned key = in ? ordered_bits(d[i]) : 0xFFFFFFFFu;
            const bool lt = in && key < prefix;
            const bool eq = in && key == prefix;
            const unsigned blt = __ballot_sync(0xffffffffu, lt);
            const unsigned beq = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) {
                wlt[warp] = __popc(blt);
                weq[warp] = __popc(beq);
            }
            __syncthreads();
            unsigned plt = s_nlt, peq = s_neq;
            for (int w = 0; w < warp; ++w) {
                plt += wlt[w];
                peq += weq[w];
            }
            const unsigned below = (1u << lane) - 1u;
            plt += __popc(blt & below);
            peq += __popc(beq & below);
            if (lt && plt < nlt_total) sel[plt] = ((unsigned long long)key << 32) | (unsigned)i;
            if (eq && peq < kk) sel[nlt_total + peq] = ((unsigned long long)key << 32) | (unsigned)i;
            __syncthreads();
            if (tid == 0) {
                unsigned a = 0, b = 0;
                for (int w = 0; w < nwarps; ++w) {
                    a += wlt[w];
                    b += weq[w];
                }
                s_nlt += a;
                s_neq += b;
            }
            __syncthreads();
        }
        int n2 = 1;
        while (n2 < k) n2 <<= 1;
        for (int i = k + tid; i < n2; i += kTopkThreads) sel[i] = ~0ull;
        __syncthreads();
        for (int size = 2; size <= n2; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int i = tid; i < n2; i += kTopkThreads) {
                    const int j = i ^ stride;
                    if (j > i) {
                        const bool up = (i & size) == 0;
                        const unsigned long long x = sel[i], y = sel[j];
                        if ((x > y) == up) {
                            sel[i] = y;
                            sel[j] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        for (int i = tid; i < k; i += kTopkThreads) {
            out_idx[row * k + i] = (int64_t)(sel[i] & 0xFFFFFFFFull);
            out_val[row * k + i] = from_ordered((unsigned)(sel[i] >> 32));
        }
        __syncthreads();
    }
}

__global__ void make_pairs_kernel(const int64_t* __restrict__ cand, int64_t nq, int C, int64_t q0,
                                  int64_t* __restrict__ pairs) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq * C;
         i += (int64_t)gridDim.x * blockDim.x) {
        pairs[2 * i] = q0 + i / C;
        pairs[2 * i + 1] = cand[i];
    }
}

__global__ void __launch_bounds__(256)
pair_cells_kernel(const int64_t* __restrict__ pairs, int64_t n, const int64_t* __restrict__ oa,
                  const int64_t* __restrict__ ob, unsigned long long* __restrict__ out) {
    unsigned long long acc = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = pairs[2 * i], b = pairs[2 * i + 1];
        acc += (unsigned long long)((oa[a + 1] - oa[a]) * (ob[b + 1] - ob[b]));
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void gather_cand_kernel(const int64_t* __restrict__ cand, const int64_t* __restrict__ pos,
                                   int64_t nq, int C, int k, int64_t* __restrict__ idx) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nq * k;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = i / k;
        idx[i] = cand[q * C + pos[i]];
    }
}

int grid_for(int64_t n, int threads) {
    const int64_t b = (n + threads - 1) / threads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(b, 1 << 20));
}

}  // namespace

// ======================================================================= host
size_t conv_smem_bytes(int cin) {
    return sizeof(float) * ((size_t)cin * TAPS * CH + (size_t)cin * kXsLd);
}
size_t wgrad_smem_bytes(int cin) {
    return sizeof(float) * ((size_t)TM * CH + (size_t)(TM + 4) * cin);
}

cudaError_t prepare_attributes() {
    cudaError_t e;
#define TWED_SMEM_ATTR(kern, bytes)                                                              \
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes));   \
    if (e != cudaSuccess) return e;
    TWED_SMEM_ATTR((conv_kernel<8, kEpiBiasRelu>), conv_smem_bytes(8));
    TWED_SMEM_ATTR((conv_kernel<16, kEpiBiasRelu>), conv_smem_bytes(16));
    TWED_SMEM_ATTR((conv_kernel<64, kEpiBiasRelu>), conv_smem_bytes(64));
    TWED_SMEM_ATTR((conv_kernel<64, kEpiMask>), conv_smem_bytes(64));
    TWED_SMEM_ATTR(wgrad_kernel<8>, wgrad_smem_bytes(8));
    TWED_SMEM_ATTR(wgrad_kernel<16>, wgrad_smem_bytes(16));
    TWED_SMEM_ATTR(wgrad_kernel<64>, wgrad_smem_bytes(64));
#undef TWED_SMEM_ATTR
    return cudaSuccess;
}

int conv_blocks_per_sm(int cin) {
    int occ = 0;
    cudaError_t e = cudaSuccess;
    switch (cin) {
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_kernel<8, kEpiBiasRelu>, kConvThreads, conv_smem_bytes(8)); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_kernel<16, kEpiBiasRelu>, kConvThreads, conv_smem_bytes(16)); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, conv_kernel<64, kEpiMask>, kConvThreads, conv_smem_bytes(64)); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, occ);
}

int wgrad_blocks_per_sm(int cin) {
    int occ = 0;
    cudaError_t e = cudaSuccess;
    switch (cin) {
        case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_kernel<8>, 256, wgrad_smem_bytes(8)); break;
        case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_kernel<16>, 256, wgrad_smem_bytes(16)); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, wgrad_kernel<64>, 256, wgrad_smem_bytes(64)); break;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, occ);
}

cudaError_t gather_features(const float* vals, const float* ts, const int64_t* offs,
                            const int64_t* ids, const int64_t* base, int64_t nser, int dim,
                            int p, float nu, float lambda, const float* mu, const float* sd,
                            int cin, float* X0, int32_t* rseries, cudaStream_t st) {
    if (nser < 1) return cudaSuccess;
    gather_kernel<<<(unsigned)nser, 128, 0, st>>>(vals, ts, offs, ids, base, dim, p, nu, lambda,
                                                  mu, sd, cin, X0, rseries);
    return cudaGetLastError();
}

cudaError_t feature_stats(const float* vals, const float* ts, const int64_t* offs,
                          int64_t nser, int64_t npoints, int dim, int p, float nu,
                          float lambda, double* part, float* mu, float* sd, cudaStream_t st) {
    const int nb = (int)std::min<int64_t>(kStatBlocks, nser);
    double* mean = part + (size_t)kStatBlocks * MAX_C0;
    const int c0 = dim + 2;
    stats_kernel<<<nb, kStatThreads, 0, st>>>(vals, ts, offs, nser, dim, p, nu, lambda, mean, 0, part);
    stats_finish_kernel<<<1, 32, 0, st>>>(part, nb, c0, npoints, 0, mean, mu);
    stats_kernel<<<nb, kStatThreads, 0, st>>>(vals, ts, offs, nser, dim, p, nu, lambda, mean, 1, part);
    stats_finish_kernel<<<1, 32, 0, st>>>(part, nb, c0, npoints, 1, mean, sd);
    return cudaGetLastError();
}

cudaError_t transform_weights(const float* params, const Layout& L, int cin,
                              const WeightViews& w, cudaStream_t st) {
    const int64_t total = (int64_t)cin * TAPS * CH + 4LL * CH * TAPS * CH;
    transform_kernel<<<grid_for(total, 256), 256, 0, st>>>(params, L.c0, cin, L.w1, L.w2, L.w3,
                                                           w.wt1, w.wt2, w.wt3, w.wb2, w.wb3);
    return cudaGetLastError();
}

cudaError_t conv_forward(int cin, const float* X, int64_t P, const float* wt, const float* bias,
                         const int32_t* rseries, float* Y, int grid, cudaStream_t st) {
    const size_t sm = conv_smem_bytes(cin);
    switch (cin) {
        case 8: conv_kernel<8, kEpiBiasRelu><<<grid, kConvThreads, sm, st>>>(X, P, wt, bias, nullptr, rseries, Y); break;
        case 16: conv_kernel<16, kEpiBiasRelu><<<grid, kConvThreads, sm, st>>>(X, P, wt, bias, nullptr, rseries, Y); break;
        case 64: conv_kernel<64, kEpiBiasRelu><<<grid, kConvThreads, sm, st>>>(X, P, wt, bias, nullptr, rseries, Y); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t conv_backward_data(const float* dY, int64_t P, const float* wb, const float* M,
                               float* dX, int grid, cudaStream_t st) {
    conv_kernel<64, kEpiMask><<<grid, kConvThreads, conv_smem_bytes(64), st>>>(dY, P, wb, nullptr, M,
                                                                               nullptr, dX);
    return cudaGetLastError();
}

int wgrad_parts(int cin, int grid) {
    switch (cin) {
        case 8: return grid * WgradShape<8>::RS;
        case 16: return grid * WgradShape<16>::RS;
        default: return grid * WgradShape<64>::RS;
    }
}

cudaError_t conv_wgrad(int cin, const float* X, const float* dY, int64_t P, float* part, int grid,
                       cudaStream_t st) {
    const size_t sm = wgrad_smem_bytes(cin);
    switch (cin) {
        case 8: wgrad_kernel<8><<<grid, 256, sm, st>>>(X, dY, P, part); break;
        case 16: wgrad_kernel<16><<<grid, 256, sm, st>>>(X, dY, P, part); break;
        case 64: wgrad_kernel<64><<<grid, 256, sm, st>>>(X, dY, P, part); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t wgrad_reduce(const float* part, int nparts, int cin, int c0, float* gW, float* gB,
                         cudaStream_t st) {
    const int64_t n = (int64_t)CH * c0 * TAPS + CH;
    wgrad_reduce_kernel<<<grid_for(n, 256), 256, 0, st>>>(part, nparts, cin, c0, gW, gB);
    return cudaGetLastError();
}

cudaError_t pool_forward(const float* H3, const int64_t* base, int64_t nser, float inv_mean_len,
                         const float* Wl, const float* bl, float* pooled, float* emb,
                         cudaStream_t st) {
    if (nser < 1) return cudaSuccess;
    pool_kernel<<<(unsigned)nser, 256, 0, st>>>(H3, base, inv_mean_len, Wl, bl, pooled, emb);
    return cudaGetLastError();
}

cudaError_t group_loss(const float* emb, int64_t ngroups, int gsize, const int64_t* gids,
                       const float* labels, const float* inv_sigma, float inv_npairs, float rel_floor,
                       const float* Wl, float* de, float* dpooled, float* gloss, cudaStream_t st) {
    if (gsize < 2 || gsize > kMaxGroup) return cudaErrorInvalidValue;
    group_loss_kernel<<<(unsigned)ngroups, 256, 0, st>>>(emb, gsize, gids, labels, inv_sigma,
                                                         inv_npairs, rel_floor, Wl, de, dpooled, gloss);
    return cudaGetLastError();
}

cudaError_t pool_backward(const float* H3, const int32_t* rseries, const float* dpooled,
                          float inv_mean_len, int64_t P, float* dPre, cudaStream_t st) {
    pool_backward_kernel<<<grid_for(P * (CH / 4), 256), 256, 0, st>>>(H3, rseries, dpooled,
                                                                      inv_mean_len, P, dPre);
    return cudaGetLastError();
}

cudaError_t linear_grad(const float* de, const float* pooled, int64_t nser, float* gWl, float* gbl,
                        cudaStream_t st) {
    linear_grad_kernel<<<(EMB * CH + EMB + 255) / 256, 256, 0, st>>>(de, pooled, nser, gWl, gbl);
    return cudaGetLastError();
}

cudaError_t adam(float* theta, const float* g, float* m, float* v, int64_t n, float lr,
                 float beta1, float beta2, float eps, float c1, float c2, cudaStream_t st) {
    adam_kernel<<<grid_for(n, 256), 256, 0, st>>>(theta, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t sum_scaled(const float* x, int64_t n, double scale, float* out, cudaStream_t st) {
    sum_kernel<<<1, 1024, 0, st>>>(x, n, scale, out);
    return cudaGetLastError();
}

cudaError_t search_vectors(const float* emb, int64_t n, float* zmin, float* svec, cudaStream_t st) {
    zmin_kernel<<<1, 1024, 0, st>>>(emb, n, zmin);
    svec_kernel<<<grid_for(n * EMB, 256), 256, 0, st>>>(emb, n, zmin, svec);
    return cudaGetLastError();
}

cudaError_t l2_rows(const float* qemb, int64_t nq, const float* svec, int64_t nx, float* D,
                    int64_t ld, cudaStream_t st) {
    if (nq < 1 || nx < 1) return cudaSuccess;
    if ((nq + 31) / 32 > 65535) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((nx + 127) / 128), (unsigned)((nq + 31) / 32));
    l2_kernel<<<grid, 256, 0, st>>>(qemb, nq, svec, nx, D, ld);
    return cudaGetLastError();
}

cudaError_t topk_rows(const float* D, int64_t rows, int64_t cols, int64_t ld, int k,
                      int64_t* idx, float* val, int grid, cudaStream_t st) {
    if (k < 1 || k > TOPK_MAX || cols < k || cols >= ((int64_t)1 << 31)) return cudaErrorInvalidValue;
    if (rows < 1) return cudaSuccess;
    const int g = (int)std::max<int64_t>(1, std::min<int64_t>(rows, grid));
    topk_kernel<<<g, kTopkThreads, 0, st>>>(D, rows, cols, ld, k, idx, val);
    return cudaGetLastError();
}

cudaError_t make_pairs(const int64_t* cand, int64_t nq, int C, int64_t q0, int64_t* pairs,
                       cudaStream_t st) {
    make_pairs_kernel<<<grid_for(nq * C, 256), 256, 0, st>>>(cand, nq, C, q0, pairs);
    return cudaGetLastError();
}

cudaError_t pair_cells(const int64_t* pairs, int64_t n, const int64_t* offs_a,
                       const int64_t* offs_b, unsigned long long* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (n < 1) return cudaSuccess;
    pair_cells_kernel<<<(int)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(pairs, n, offs_a,
                                                                                   offs_b, out);
    return cudaGetLastError();
}

cudaError_t gather_candidates(const int64_t* cand, const int64_t* pos, int64_t nq, int C, int k,
                              int64_t* idx, cudaStream_t st) {
    gather_cand_kernel<<<grid_for(nq * k, 256), 256, 0, st>>>(cand, pos, nq, C, k, idx);
    return cudaGetLastError();
}

}  // namespace enc
}  // namespace twed
