// Kernels of the learned k-NN candidate filter (encoder training and
// inference, embedding search, row-wise top-k).  Host code in knn.cu.
//
// Packed-row layout of a batch of S series ("gapped rows"): series s occupies
// rows base[s] .. base[s] + L_s - 1 of every activation buffer, with two zero
// rows before each series and after the last one:
//     base[0] = 2,  base[s+1] = base[s] + L_s + 2,  rows P = base[S].
// The zero rows are the convolutions' 'same' padding, so every convolution,
// its adjoint and its weight gradient run as plain dense sweeps over the
// packed rows with no per-series masking.  rseries[p] is the batch series of
// row p, or -1 for a zero row.  Activations are [P][64] row-major FP32;
// layer-1 inputs are [P][cin] with cin = 8 or 16 (zero-padded channels).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace twed {
namespace enc {

constexpr int CH = 64;    // convolution channels
constexpr int TAPS = 5;   // kernel width
constexpr int EMB = 32;   // embedding size
constexpr int PSI = 31;   // components of the shape part psi; e[31] = z
constexpr int TM = 128;   // rows per convolution tile
constexpr int MAX_C0 = 16;
constexpr int TOPK_MAX = 4096;

inline int cin_pad(int c0) { return c0 <= 8 ? 8 : 16; }

// Offsets (in floats) of the parameter blocks inside the flat array:
// W1[64][c0][5], b1[64], W2[64][64][5], b2, W3[64][64][5], b3, Wl[32][64], bl[32].
struct Layout {
    int c0 = 0;
    int64_t w1 = 0, b1 = 0, w2 = 0, b2 = 0, w3 = 0, b3 = 0, wl = 0, bl = 0, total = 0;
};
Layout layout(int dim);

// Device copies of the weights in the order the convolution kernel reads
// them: wt[ci][k][o] (forward; ci padded to cin) and, for layers 2 and 3,
// the flipped adjoint wb[o][k][ci] = W[o][ci][4-k].
struct WeightViews {
    float* wt1;  // [cin][5][64]
    float* wt2;  // [64][5][64]
    float* wt3;
    float* wb2;
    float* wb3;
};
size_t weight_views_floats(int cin);
void carve_weight_views(float* base, int cin, WeightViews* w);

// ---- inputs
cudaError_t gather_features(const float* vals, const float* ts, const int64_t* offs,
                            const int64_t* ids, const int64_t* base, int64_t nser, int dim,
                            int p, float nu, float lambda, const float* mu, const float* sd,
                            int cin, float* X0, int32_t* rseries, cudaStream_t st);
// Per-channel mean and population standard deviation over every point of a
// set (two passes, FP64 sums, fixed reduction order).  part: >= 2 * 1024 * 16 doubles.
cudaError_t feature_stats(const float* vals, const float* ts, const int64_t* offs,
                          int64_t nser, int64_t npoints, int dim, int p, float nu,
                          float lambda, double* part, float* mu, float* sd, cudaStream_t st);

// ---- layers
cudaError_t transform_weights(const float* params, const Layout& L, int cin,
                              const WeightViews& w, cudaStream_t st);
cudaError_t conv_forward(int cin, const float* X, int64_t P, const float* wt,
                         const float* bias, const int32_t* rseries, float* Y, int grid,
                         cudaStream_t st);
cudaError_t conv_backward_data(const float* dY, int64_t P, const float* wb, const float* M,
                               float* dX, int grid, cudaStream_t st);
int wgrad_parts(int cin, int grid);
cudaError_t conv_wgrad(int cin, const float* X, const float* dY, int64_t P, float* part,
                       int grid, cudaStream_t st);
cudaError_t wgrad_reduce(const float* part, int nparts, int cin, int c0, float* gW, float* gB,
                         cudaStream_t st);
cudaError_t pool_forward(const float* H3, const int64_t* base, int64_t nser, float inv_mean_len,
                         const float* Wl, const float* bl, float* pooled, float* emb,
                         cudaStream_t st);
cudaError_t group_loss(const float* emb, int64_t ngroups, int gsize, const int64_t* gids,
                       const float* labels, const float* inv_sigma, float inv_npairs, float rel_floor,
                       const float* Wl, float* de, float* dpooled, float* gloss, cudaStream_t st);
cudaError_t pool_backward(const float* H3, const int32_t* rseries, const float* dpooled,
                          float inv_mean_len, int64_t P, float* dPre, cudaStream_t st);
cudaError_t linear_grad(const float* de, const float* pooled, int64_t nser, float* gWl,
                        float* gbl, cudaStream_t st);
cudaError_t adam(float* theta, const float* g, float* m, float* v, int64_t n, float lr,
                 float beta1, float beta2, float eps, float c1, float c2, cudaStream_t st);
// out[0] = scale * sum(x[0..n)), summed in FP64 in a fixed order (one block).
cudaError_t sum_scaled(const float* x, int64_t n, double scale, float* out, cudaStream_t st);

// ---- search
// svec[x] = (psi_x, sqrt(max(z_x - z_min, 0))), z_min over all n rows.
cudaError_t search_vectors(const float* emb, int64_t n, float* zmin, float* svec,
                           cudaStream_t st);
// D[q][x] = sum_{j<31} (qemb[q][j] - svec[x][j])^2 + svec[x][31]^2, row stride ld.
cudaError_t l2_rows(const float* qemb, int64_t nq, const float* svec, int64_t nx, float* D,
                    int64_t ld, cudaStream_t st);
// k smallest of each row (ascending, ties by smaller column), k <= TOPK_MAX,
// cols < 2^31.
cudaError_t topk_rows(const float* D, int64_t rows, int64_t cols, int64_t ld, int k,
                      int64_t* idx, float* val, int grid, cudaStream_t st);
// pairs[(q*C + c)] = (q0 + q, cand[q*C + c]) for q < nq.
cudaError_t make_pairs(const int64_t* cand, int64_t nq, int C, int64_t q0, int64_t* pairs,
                       cudaStream_t st);
// out[0] = sum over pairs of len_a * len_b (interior cells), out zeroed here.
cudaError_t pair_cells(const int64_t* pairs, int64_t n, const int64_t* offs_a,
                       const int64_t* offs_b, unsigned long long* out, cudaStream_t st);
// idx[q*k + r] = cand[q*C + pos[q*k + r]].
cudaError_t gather_candidates(const int64_t* cand, const int64_t* pos, int64_t nq, int C, int k,
                              int64_t* idx, cudaStream_t st);

// Shared memory each kernel needs (for attribute setup and occupancy).
size_t conv_smem_bytes(int cin);
size_t wgrad_smem_bytes(int cin);
cudaError_t prepare_attributes();
// Resident blocks per SM of the convolution / weight-gradient kernels for
// `cin` input channels (persistent grids are this times the SM count).
int conv_blocks_per_sm(int cin);
int wgrad_blocks_per_sm(int cin);

}  // namespace enc
}  // namespace twed
