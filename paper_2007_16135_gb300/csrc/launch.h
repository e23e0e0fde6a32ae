// Host-visible argument blocks of the TWED kernels and their launchers.
// Included by the C ABI (api.cu) and by the per-precision kernel units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace twed {

// Status words shared by all warps of one launch.  `err` is cleared before
// each launch and makes every waiting warp give up once set; `sticky` keeps
// the first failure until the host reads it.
struct SyncCtl {
    unsigned* err;
    unsigned* sticky;
    unsigned long long timeout_ns;
    long long stall_strip;  // fault injection: strip that never publishes (-1 off)
    unsigned sleep_ns;      // back-off between polls of a progress word (0 = spin)
};

// Prologue: one record per point (see Rec<> in engine.cuh).
template <typename T>
struct RecordsArgs {
    const T* vals;         // [total][dim]
    const T* ts;           // [total]
    const int64_t* offs;   // [nseries + 1], device; nullptr = one series
    int64_t nseries;
    int64_t total;
    int dim, p;
    T nu, lam;
    T* rec;                // [total][rec_len]
};

// One long pair, rows split into strips that many warps run concurrently.
template <typename T>
struct CoopArgs {
    const T* rec_a;        // row series records [n]
    const T* rec_b;        // column series records [m]
    const T* vals_a;       // raw values (runtime-dimension kernels only)
    const T* vals_b;
    int n, m, dim, p;
    T nu;
    int64_t nstrips;
    void* ring;            // [nslot][ring_stride] pairs (D, c) of strip bottom rows
    int nslot;
    int64_t ring_stride;   // >= m + 1, even (a staged copy may read one pair past m)
    unsigned* flags;       // [nstrips] published columns per strip
    unsigned* strip_counter;
    T* out;                // D(n, m)
    SyncCtl sc;
};

// Many pairs, one warp per pair, strips of a pair run one after another.
enum PairMode : int { kExplicitPairs = 0, kSymmetricSorted = 1, kBlockSorted = 2 };

template <typename T>
struct PairsArgs {
    const T* rec_a;
    const T* rec_b;
    const T* vals_a;
    const T* vals_b;
    const int64_t* offs_a;
    const int64_t* offs_b;
    int mode;
    const int64_t* pairs;    // kExplicitPairs: [npairs][2]
    const int32_t* perm_a;   // sorted position -> series index (sorted modes)
    const int32_t* perm_b;
    int64_t npairs, na, nb;
    int dim, p, rmax;
    T nu;
    T* out;
    unsigned long long* counter;
    void* scratch;           // per warp: one boundary row of `scratch_cols` (D, c) pairs
    int64_t scratch_cols;    // >= longest series + 1, even
    SyncCtl sc;
    int64_t cut_cells = 0;   // > 0: pairs with more cells are skipped (run elsewhere)
    const int64_t* order = nullptr;  // kExplicitPairs: run position -> pair index (nullptr: identity)
    int dtw = 0;             // FP32 compiled layouts only: DTW instead of TWED (nu, times, delete costs unused)
    int64_t max_len = 0;     // longest series of either set; 1 .. 32 lets the short-pair kernel run (0: not known)
};

// Longest-first run order of an explicit pair list (order.cu): order[k] is
// the index of the pair to run k-th, by decreasing len_a * len_b in
// quarter-octave classes.  bins: kOrderBins device words of scratch.  A pair
// with an index outside [0, na) x [0, nb) sorts last and is not dereferenced.
constexpr int kOrderBins = 256;
cudaError_t launch_order_pairs(const int64_t* pairs, int64_t npairs, const int64_t* offs_a, int64_t na,
                               const int64_t* offs_b, int64_t nb, int64_t* order, unsigned long long* bins,
                               int sms, cudaStream_t st);

// Elements per point record for (dim, p) (16-byte multiple; see Rec<>).
template <typename T>
int rec_len(int dim, int p);

cudaError_t launch_records(const RecordsArgs<float>& a, cudaStream_t st);
cudaError_t launch_records(const RecordsArgs<double>& a, cudaStream_t st);
// Loads the FP32 records kernel that (dim, p) dispatches to (a function
// attribute query), so that its first launch does no lazy module loading.
cudaError_t records_preload_f32(int dim, int p);

// R (rows of the DP per lane) in {1, 2, 4, 8}.  kahan: compensated FP32
// running cost (float, dims with a compiled point layout only; ring entries
// are then (D_hi, D_lo, c, 0) float4).
cudaError_t launch_coop(const CoopArgs<float>& a, int R, bool kahan, int blocks, int threads,
                        cudaStream_t st);
cudaError_t launch_coop(const CoopArgs<double>& a, int R, bool kahan, int blocks, int threads,
                        cudaStream_t st);
template <typename T>
int coop_blocks_per_sm(int dim, int p, int R, bool kahan, int threads);
// One long FP32 pair by bands of `warps` strips per block (compiled point
// layouts only; strip_counter counts bands, flags[b] is band b's progress).
cudaError_t launch_band(const CoopArgs<float>& a, int R, bool kahan, int blocks, int warps,
                        cudaStream_t st);
int band_blocks_per_sm(int dim, int p, int R, bool kahan, int warps);
// true when (dim, p) has a compiled point layout (dims 1, 2, 3, 4, 8 with
// p = 1, 2): the compensated variant needs one.
bool compiled_layout(int dim, int p);

// a.rmax (largest rows per lane) is clamped to pairs_rmax_limit<T>().
cudaError_t launch_pairs(const PairsArgs<float>& a, int blocks, int threads, cudaStream_t st);
cudaError_t launch_pairs(const PairsArgs<double>& a, int blocks, int threads, cudaStream_t st);
template <typename T>
int pairs_blocks_per_sm(int dim, int p, int threads);
template <typename T>
int pairs_rmax_limit();

// Tensor-core cross-term path (xterm.cu): dim 64, p = 2, FP32.
// Records are float4 (t, delete cost, |x|^2, 0) per point.  Work items pair
// one column series with up to xterm_rows_per_item() row series taken in
// the sorted (longest-first) order; rows come from set A, columns from set
// B (set A again when symmetric).
struct XtermArgs {
    const float* vals_a;          // row set values [total_a][64], 16-byte aligned
    const float4* rec_a;          // row set records
    const float4* rec_b;          // column set records
    const int64_t* offs_a;
    const int64_t* offs_b;
    const int32_t* perm_a;        // sorted position -> series (longest first)
    const int32_t* perm_b;
    int64_t na, nb;
    int symmetric;                // 1: out[x][y] and out[y][x] for row x < column y in sorted order
    int64_t nitems;
    const int64_t* chunk_start;   // symmetric: first item of each chunk of rows [nchunks + 1]
    int64_t nchunks;
    float nu;
    float* out;
    float2* bnd;                  // per consumer warp: bnd_stride (D, c) of a strip's bottom row
    int64_t bnd_stride;           // xterm_bnd_stride(longest column series)
    unsigned long long* counter;  // work item counter, zero before the launch
    SyncCtl sc;
};
// bf16: records hold the norms of the points rounded to BF16
cudaError_t launch_xrecords(const RecordsArgs<float>& a, cudaStream_t st, bool bf16);
// The points of a column set rounded to BF16 (nvals values, a multiple of 64).
cudaError_t launch_bf16_copy(const float* src, void* dst, int64_t nvals, cudaStream_t st);
// tmap: 128-byte CUtensorMap of the column set's values (xterm_tensor_map):
// FP32, or with bf16 the set's BF16 copy
cudaError_t xterm_tensor_map(void* tmap, const void* vals, int64_t total, bool bf16);
cudaError_t launch_xterm(const void* tmap, const XtermArgs& a, int blocks, cudaStream_t st, bool bf16);
int xterm_blocks_per_sm();
int xterm_resident_blocks();
void xterm_resources(char* buf, int len);
int xterm_rows_per_item();
int xterm_warps_per_block();  // consumer warps
int xterm_threads();
int64_t xterm_bnd_stride(int64_t max_len);

// Writes 0 to out[i*n + i], i < n.
cudaError_t launch_zero_diag(void* out, bool f64, int64_t n, cudaStream_t st);

}  // namespace twed
