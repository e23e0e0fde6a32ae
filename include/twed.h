/*
 * twed.h -- C ABI of the GB300 (sm_103a) Time Warp Edit Distance library.
 *
 * What is computed (paper, section "Time Warp Edit Distance", steps 1-6, and
 * section "Improved Time Warp Edit Distance", which evaluates the same cells
 * one anti-diagonal at a time):
 *
 *   a_1..a_n, b_1..b_m points in R^dim with timestamps t_i, t'_j; a_0 = b_0 = 0,
 *   t_0 = t'_0 = 0.  d(x,y) = (sum_k |x_k - y_k|^p)^(1/p)  (|x - y| if dim == 1).
 *   c(i,j)  = d(a_i,b_j) + nu |t_i - t'_j|
 *   dA(i)   = d(a_i,a_{i-1}) + nu |t_i - t_{i-1}| + lambda   (dB likewise)
 *   D(0,0)  = 0, D(i,0) = D(0,j) = +inf
 *   D(i,j)  = min(D(i-1,j) + dA(i), D(i,j-1) + dB(j), D(i-1,j-1) + c(i,j) + c(i-1,j-1))
 *   TWED    = D(n,m)
 *
 * Conventions shared by every entry point:
 *  - A series is `len` points stored row-major as vals[len][dim] (the dim
 *    components of a point are contiguous) plus ts[len].
 *  - A packed set of series (twed_set_*_t) stores many series back to back:
 *    vals[offs[n]][dim], ts[offs[n]], offs[n+1] (int64, offs[0] = 0, non-
 *    decreasing); series s is rows offs[s] .. offs[s+1]-1.
 *  - Pointers named d_* or documented "device" must be device memory of the
 *    handle's device; others are host memory.  The caller owns every input
 *    and output buffer; the library owns its workspace (inside the handle or
 *    plan) and never frees caller memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Parameters: la, lb >= 1; dim >= 1; p >= 1 (integer lp degree; the paper's
 *    "degree"); nu >= 0 and lambda >= 0, both finite.  Anything else returns
 *    TWED_ERR_INVALID_ARG and launches nothing.
 *  - Host entry points also reject non-finite input values and timestamps.
 *    Device entry points do not read inputs on the host: non-finite device
 *    inputs give undefined (but memory-safe) results.
 *  - No exception crosses the ABI.  Every call returns a status; the text of
 *    the last failure on a handle is twed_last_error(handle).
 *  - A handle is not thread-safe: use one handle per host thread, and do not
 *    run two calls of one handle concurrently on different streams (they
 *    share its workspace).
 */
#ifndef TWED_H_
#define TWED_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TWED_OK = 0,
    TWED_ERR_INVALID_ARG = 1, /* bad pointer, size or parameter */
    TWED_ERR_CUDA = 2,        /* a CUDA runtime call failed */
    TWED_ERR_ALLOC = 3,       /* device workspace allocation failed */
    TWED_ERR_TIMEOUT = 4,     /* a bounded inter-warp wait expired; results invalid */
    TWED_ERR_UNSUPPORTED = 5  /* valid request the library does not support */
} twed_status_t;

typedef struct twed_handle_s* twed_handle_t;
typedef struct twed_plan_s* twed_plan_t;

/* Accumulation of the running cost D for single-precision entry points. */
typedef enum {
    TWED_ACCUM_AUTO = 0,  /* FP32, or compensated FP32 once n + m > 100000 */
    TWED_ACCUM_F32 = 1,   /* plain FP32 sums: within 1e-5 relative of FP64
                             only while n + m <= 100000; longer pairs drift
                             (measured 1.4e-5 at n = m = 1e5, 2.3e-5 at
                             1e6), outside the single-precision contract */
    TWED_ACCUM_KAHAN = 2  /* compensated (TwoSum) FP32 running cost */
} twed_accum_t;

/* Options (NULL = all defaults). */
typedef struct {
    int accum;          /* twed_accum_t, single precision only */
    int rows_per_lane;  /* 0 = automatic; else 1..8 rows of the DP per lane */
    int autotune;       /* plans: 1 = time candidate schedules at creation */
    double timeout_s;   /* bound on any inter-warp wait; 0 = 2 seconds */
    int64_t stall_strip;/* fault injection for tests: the given row strip never
                           publishes progress, so its successor's wait expires
                           (TWED_ERR_TIMEOUT); -1 = off */
    int xterm;          /* FP32 plans, dim 64, p = 2: TWED_XTERM_TF32 forms the
                           cross term a_i . b_j of |a_i - b_j|^2 on the tensor
                           cores (TF32 inputs, FP32 accumulation, FP32 norms);
                           TWED_XTERM_BF16 the same with the points rounded to
                           BF16 (norms of the rounded points; the plan keeps a
                           BF16 copy of the column set).  Every cost then
                           carries the inputs' rounding (TF32 about 1e-4,
                           BF16 about 1e-3 relative), so both are opt-in.
                           Values must be 16-byte aligned, else
                           TWED_ERR_UNSUPPORTED. */
} twed_opts_t;

/* twed_opts_t.xterm values. */
#define TWED_XTERM_OFF 0
#define TWED_XTERM_TF32 1
#define TWED_XTERM_BF16 2

/* A packed set of series.  vals/ts/offs are device pointers; offs_host is a
 * host copy of offs (the library reads lengths from it to plan work).
 * vals needs only the alignment of its element type.  When it is 16-byte
 * aligned, p = 2 sets at dims 16, 28 and 64 (FP32) take kernels that copy
 * points in 16-byte pieces, and sets whose series all have at most 32
 * points (dims 16 and 28, also FP64) take the short-pair kernel; the device
 * lengths must then match offs_host (a longer pair found on the device is
 * reported as TWED_ERR_INVALID_ARG with NaN as its value). */
typedef struct {
    const double* vals;
    const double* ts;
    const int64_t* offs;
    const int64_t* offs_host;
    int64_t n;
} twed_set_f64_t;

typedef struct {
    const float* vals;
    const float* ts;
    const int64_t* offs;
    const int64_t* offs_host;
    int64_t n;
} twed_set_f32_t;

/* ---- handles ----------------------------------------------------------- */

/* Create a handle on the current CUDA device.  Allocates a private stream; no
 * workspace until first use.  Returns TWED_ERR_CUDA without a usable GPU. */
twed_status_t twed_create(twed_handle_t* handle);
void twed_destroy(twed_handle_t handle);
/* Text of the last failure on `handle` (valid until the next call on it). */
const char* twed_last_error(twed_handle_t handle);
/* Library version string. */
const char* twed_version(void);
/* Waits for `stream`, then reports (and clears) the first error that a
 * device entry point enqueued on this handle raised on the GPU:
 * TWED_ERR_TIMEOUT (a bounded wait expired) or TWED_ERR_INVALID_ARG (a batch
 * pair index outside its set).  TWED_OK otherwise. */
twed_status_t twed_sync_status(twed_handle_t handle, void* stream);

/* ---- one pair ------------------------------------------------------------
 * The paper's host-managed `twed` call (section "Basic Methodology and
 * Results"): host pointers in, host scalar out, blocking.  Copies the inputs
 * to the handle's workspace, runs the wavefront, copies D(la,lb) back.
 * a[la][dim], ta[la], b[lb][dim], tb[lb]; *out receives TWED(a, b). */
twed_status_t twed_f64(twed_handle_t handle, const double* a, const double* ta, int64_t la,
                       const double* b, const double* tb, int64_t lb, int dim, double nu,
                       double lambda, int p, double* out);
twed_status_t twed_f32(twed_handle_t handle, const float* a, const float* ta, int64_t la,
                       const float* b, const float* tb, int64_t lb, int dim, float nu,
                       float lambda, int p, float* out);
/* As twed_f32 with options (accumulation mode, rows per lane, timeout). */
twed_status_t twed_f32_ex(twed_handle_t handle, const float* a, const float* ta, int64_t la,
                          const float* b, const float* tb, int64_t lb, int dim, float nu,
                          float lambda, int p, const twed_opts_t* opts, float* out);

/* The paper's device-resident `twed_dev` call: every pointer is device
 * memory, work is enqueued on `stream` and the call returns without waiting.
 * d_out[0] receives TWED.  Wait-timeouts surface through twed_sync_status. */
twed_status_t twed_dev_f64(twed_handle_t handle, const double* d_a, const double* d_ta,
                           int64_t la, const double* d_b, const double* d_tb, int64_t lb, int dim,
                           double nu, double lambda, int p, double* d_out, void* stream);
twed_status_t twed_dev_f32(twed_handle_t handle, const float* d_a, const float* d_ta, int64_t la,
                           const float* d_b, const float* d_tb, int64_t lb, int dim, float nu,
                           float lambda, int p, float* d_out, void* stream);
twed_status_t twed_dev_f64_ex(twed_handle_t handle, const double* d_a, const double* d_ta,
                              int64_t la, const double* d_b, const double* d_tb, int64_t lb,
                              int dim, double nu, double lambda, int p, const twed_opts_t* opts,
                              double* d_out, void* stream);
twed_status_t twed_dev_f32_ex(twed_handle_t handle, const float* d_a, const float* d_ta,
                              int64_t la, const float* d_b, const float* d_tb, int64_t lb,
                              int dim, float nu, float lambda, int p, const twed_opts_t* opts,
                              float* d_out, void* stream);

/* ---- explicit pairs over two packed sets ---------------------------------
 * The paper's batch mode (section "cuTWED Implementation Remarks"), here for
 * an arbitrary list of pairs: d_pairs[2k], d_pairs[2k+1] (device int64) index
 * series of A and B; d_out[k] (device) receives TWED(A[d_pairs[2k]],
 * B[d_pairs[2k+1]]).  One persistent launch, one warp per pair, pairs taken
 * in list order.  The host does not read d_pairs; the kernel checks every
 * index against its set before reading any point of it: a pair with an index
 * outside [0, A->n) x [0, B->n) gets NaN in d_out[k], and the launch reports
 * TWED_ERR_INVALID_ARG through twed_sync_status.  B may equal A. */
twed_status_t twed_batch_f64(twed_handle_t handle, const twed_set_f64_t* A,
                             const twed_set_f64_t* B, const int64_t* d_pairs, int64_t npairs,
                             int dim, double nu, double lambda, int p, double* d_out, void* stream);
twed_status_t twed_batch_f32(twed_handle_t handle, const twed_set_f32_t* A,
                             const twed_set_f32_t* B, const int64_t* d_pairs, int64_t npairs,
                             int dim, float nu, float lambda, int p, float* d_out, void* stream);

/* Run orders of an explicit pair list (the warps take pairs in run order):
 *   TWED_ORDER_LIST           the list's own order (twed_batch_*), which keeps
 *                             whatever locality the caller built into it;
 *   TWED_ORDER_LONGEST_FIRST  decreasing len_a * len_b (quarter-octave
 *                             classes), so the largest pairs do not start last.
 * Reordering is a device counting sort (workspace: 8 bytes per pair, in the
 * handle's workspace), done only when there are more pairs than resident
 * warps.  d_out[k] is always pair k's value, and values do not depend on
 * the order.  Arguments, ownership and errors as twed_batch_*; an unknown
 * `order` returns TWED_ERR_INVALID_ARG. */
#define TWED_ORDER_LIST 0
#define TWED_ORDER_LONGEST_FIRST 1
twed_status_t twed_batch_f64_ex(twed_handle_t handle, const twed_set_f64_t* A,
                                const twed_set_f64_t* B, const int64_t* d_pairs, int64_t npairs,
                                int dim, double nu, double lambda, int p, int order,
                                double* d_out, void* stream);
twed_status_t twed_batch_f32_ex(twed_handle_t handle, const twed_set_f32_t* A,
                                const twed_set_f32_t* B, const int64_t* d_pairs, int64_t npairs,
                                int dim, float nu, float lambda, int p, int order, float* d_out,
                                void* stream);

/* ---- explicit pairs without any allocation -------------------------------
 * The paper has no counterpart to this entry point.  It exists for callers
 * that must not allocate device memory: loops where a cudaMalloc/cudaFree
 * would synchronize the device and stall the work queued behind it,
 * latency-bound paths that must not wait on the allocator, and plug-ins
 * whose host framework hands them a fixed memory budget.  Everything above
 * allocates (twed_create, workspace growth, plans); this call does not.
 *
 * Same arguments and result as twed_batch_f32, minus the handle.  Its
 * working memory is one static device array of TWED_NOALLOC_SCRATCH_BYTES
 * inside the library, which every GPU that loads the library keeps until
 * the process exits.  The caller still passes (and owns) all inputs and
 * outputs.
 *
 * Set-up: the first call on each device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress), reads the SM count, and
 * loads and sizes every kernel this call can launch (attribute and occupancy
 * queries), so that later calls on that device do no lazy kernel loading.
 * Make that first call during the caller's own set-up.  The set-up belongs to the
 * device's primary context: after cudaDeviceReset of that device this entry
 * point must not be called again in the process.
 *
 * All calls share the one array and it keeps the last call's contents (the
 * call clears what must start at zero): two calls whose work overlaps on the
 * GPU -- on different streams, or from different threads -- race and give
 * undefined results.  Size limit: the per-point records (A's, plus B's
 * unless B is A; 16 to 80 bytes per point, by dim) plus four boundary rows
 * of 8 x (longest series + 2) bytes must fit in the array after 256 bytes of
 * control words; larger requests return TWED_ERR_UNSUPPORTED before
 * enqueuing anything.  No error text is kept (there is no handle); the
 * status code is the whole report, and a pair index outside its set leaves
 * NaN in that pair's output. */
#define TWED_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
twed_status_t twed_batch_f32_noalloc(const twed_set_f32_t* A, const twed_set_f32_t* B,
                                     const int64_t* d_pairs, int64_t npairs, int dim, float nu,
                                     float lambda, int p, float* d_out, void* stream);

/* ---- edit paths ----------------------------------------------------------
 * The alignment behind a TWED value, which the paper's introduction names
 * as readily obtainable from the same dynamic program (and its conclusion
 * as an extension).  A path is the list of moves after the forced first
 * match (0,0) -> (1,1): 0 = match (i+1, j+1), 1 = delete in a (i+1, j),
 * 2 = delete in b (i, j+1), ending at (la, lb).  Among optimal paths the one
 * returned is fixed by a walk back from (la, lb) that takes, at each cell,
 * the first of match, delete in a, delete in b whose candidate equals
 * D(i,j) (the forward pass records that choice per cell: 2 bits, la*lb/4
 * bytes of device memory per pair in flight, at most 8 GiB in all; a pair
 * needing more returns TWED_ERR_UNSUPPORTED).  The distance itself is the
 * same as twed_f64 / twed_f32 computes (FP64: bit for bit for p = 1, 2).
 *
 * twed_path_*: one pair, host pointers, blocking; moves (host) needs room
 * for max(la + lb - 2, 1) entries; *len receives their number and *out
 * TWED(a, b).  It runs on one warp (about la*lb / 1e8 seconds in FP64). */
twed_status_t twed_path_f64(twed_handle_t handle, const double* a, const double* ta, int64_t la,
                            const double* b, const double* tb, int64_t lb, int dim, double nu,
                            double lambda, int p, double* out, int8_t* moves, int64_t* len);
twed_status_t twed_path_f32(twed_handle_t handle, const float* a, const float* ta, int64_t la,
                            const float* b, const float* tb, int64_t lb, int dim, float nu,
                            float lambda, int p, float* out, int8_t* moves, int64_t* len);
/* Explicit pairs of two packed sets (device pointers, enqueued on `stream`):
 * pair k's distance goes to d_dist[k], its moves to d_moves[d_move_offs[k]
 * ..] (room for len_a + len_b - 2 entries, caller-allocated) and their
 * number to d_len[k].  A pair index outside its set gives NaN, d_len[k] = -1
 * and TWED_ERR_INVALID_ARG through twed_sync_status. */
twed_status_t twed_path_batch_f64(twed_handle_t handle, const twed_set_f64_t* A,
                                  const twed_set_f64_t* B, const int64_t* d_pairs, int64_t npairs,
                                  int dim, double nu, double lambda, int p, double* d_dist,
                                  int8_t* d_moves, const int64_t* d_move_offs, int64_t* d_len,
                                  void* stream);
twed_status_t twed_path_batch_f32(twed_handle_t handle, const twed_set_f32_t* A,
                                  const twed_set_f32_t* B, const int64_t* d_pairs, int64_t npairs,
                                  int dim, float nu, float lambda, int p, float* d_dist,
                                  int8_t* d_moves, const int64_t* d_move_offs, int64_t* d_len,
                                  void* stream);

/* ---- LCS and DTW on the same wavefront ------------------------------------
 * The paper's section "Generalized Dynamic Programming Extensions" carries
 * its diagonal band over to other dynamic programs, first the longest common
 * subsequence ("Direct Extension: LCS"):
 *   L(i,0) = L(0,j) = 0;  L(i,j) = L(i-1,j-1) + 1 if x_i == y_j,
 *                                 max(L(i-1,j), L(i,j-1)) otherwise,
 * and dynamic time warping, the related distance of its introduction:
 *   D(0,0) = 0, D(i,0) = D(0,j) = inf,
 *   D(i,j) = d(a_i,b_j) + min(min(D(i-1,j-1), D(i-1,j)), D(i,j-1)),
 * with the lp point distance d of TWED (no warping window).  Integer LCS
 * results are exact; FP64 DTW follows that evaluation order (bit for bit
 * against a sequential evaluation for p = 1, 2).
 *
 * A packed set of int32 symbol sequences: sym[offs[n]], offs[n+1] (device,
 * int64, offs[0] = 0), offs_host a host copy; sequences may be empty. */
typedef struct {
    const int32_t* sym;
    const int64_t* offs;
    const int64_t* offs_host;
    int64_t n;
} twed_seq_t;
/* LCS lengths of explicit pairs (device, enqueued on `stream`): d_len[k] =
 * LCS(X[d_pairs[2k]], Y[d_pairs[2k+1]]); an index outside its set gives -1
 * and TWED_ERR_INVALID_ARG through twed_sync_status. */
twed_status_t twed_lcs_batch(twed_handle_t handle, const twed_seq_t* X, const twed_seq_t* Y,
                             const int64_t* d_pairs, int64_t npairs, int32_t* d_len, void* stream);
/* One longest common subsequence of x[n], y[m] (host, blocking): xi[k],
 * yj[k] (room for min(n, m) entries) receive the matched 0-based positions
 * in increasing order, *len their number (the LCS length).  The walk back
 * takes the diagonal on equal symbols, else goes up when L(i-1,j) >=
 * L(i,j-1), else left.  Choice bits as for edit paths (n*m/4 bytes). */
twed_status_t twed_lcs_pairs(twed_handle_t handle, const int32_t* x, int64_t n, const int32_t* y,
                             int64_t m, int64_t* xi, int64_t* yj, int64_t* len);
/* DTW of explicit pairs over two packed sets (timestamps are not read and
 * may be NULL); arguments, ownership and errors as twed_batch_*. */
twed_status_t twed_dtw_batch_f64(twed_handle_t handle, const twed_set_f64_t* A,
                                 const twed_set_f64_t* B, const int64_t* d_pairs, int64_t npairs,
                                 int dim, int p, double* d_out, void* stream);
twed_status_t twed_dtw_batch_f32(twed_handle_t handle, const twed_set_f32_t* A,
                                 const twed_set_f32_t* B, const int64_t* d_pairs, int64_t npairs,
                                 int dim, int p, float* d_out, void* stream);
/* DTW of one pair from host memory (a[la][dim], b[lb][dim]), blocking. */
twed_status_t twed_dtw_f64(twed_handle_t handle, const double* a, int64_t la, const double* b,
                           int64_t lb, int dim, int p, double* out);
twed_status_t twed_dtw_f32(twed_handle_t handle, const float* a, int64_t la, const float* b,
                           int64_t lb, int dim, int p, float* out);

/* ---- all-pairs distance matrix (plan + CUDA graph) -----------------------
 * The paper's batch mode returning a distance matrix, with its suggested
 * upper-triangle saving for a symmetric matrix (section "Validation using
 * Real Datasets").  B == NULL: symmetric self-matrix of A, out[NA][NA]; only
 * i < j pairs are computed, mirrored, and the diagonal is 0 (TWED(a,a) = 0).
 * Otherwise out[NA][NB], out[i*NB + j] = TWED(A_i, B_j).
 * Creation sorts series by length (longest first) and picks a schedule; with
 * opts->autotune it times every rows-per-lane cap and resident-block count on
 * a strided sample of its own pairs (about 2e10 cells) and keeps the fastest.
 * Pairs whose cells exceed the plan's average work per warp (at most 4096 of
 * them) run after the persistent launch on the one-pair block-cooperative
 * schedule.  Execute computes the step-cost records and runs the launches
 * captured (at the first execute into a given output) in one CUDA graph.  The plan keeps pointers
 * to A and B: they must stay valid and keep their lengths; their values may
 * change between executes.  Execute enqueues one graph launch on `stream`. */
twed_status_t twed_allpairs_plan_create_f64(twed_handle_t handle, const twed_set_f64_t* A,
                                            const twed_set_f64_t* B, int dim, double nu,
                                            double lambda, int p, const twed_opts_t* opts,
                                            twed_plan_t* plan);
twed_status_t twed_allpairs_plan_create_f32(twed_handle_t handle, const twed_set_f32_t* A,
                                            const twed_set_f32_t* B, int dim, float nu,
                                            float lambda, int p, const twed_opts_t* opts,
                                            twed_plan_t* plan);
/* d_out: device float[NA*NB] (f32 plans) or double[NA*NB] (f64 plans). */
twed_status_t twed_plan_execute(twed_plan_t plan, void* d_out, void* stream);
/* Waits for `stream`, then reports (and clears) the first error the plan's
 * kernels raised on the GPU since the last call: TWED_ERR_TIMEOUT (a bounded
 * wait expired; that execute's output is invalid) or TWED_ERR_UNSUPPORTED
 * (the tensor-core kernel found its shared memory misaligned and computed
 * nothing).  TWED_OK otherwise. */
twed_status_t twed_plan_status(twed_plan_t plan, void* stream);
/* Interior cells (sum of la*lb over computed pairs) one execute evaluates. */
int64_t twed_plan_cells(twed_plan_t plan);
/* Number of pairs one execute evaluates. */
int64_t twed_plan_pairs(twed_plan_t plan);
/* Device time, in milliseconds, of the persistent pairs launch of the last
 * completed execute (CUDA events recorded inside the plan's graph around that
 * launch).  Call after the execute's stream has been synchronized. */
twed_status_t twed_plan_kernel_ms(twed_plan_t plan, float* ms);
/* Short text naming the schedule the plan chose (rows per lane, warps). */
const char* twed_plan_describe(twed_plan_t plan);
void twed_plan_destroy(twed_plan_t plan);

/* All-pairs from host memory, blocking: copies the packed set(s) in, builds
 * a plan, executes it and copies the matrix out.  B arrays NULL = symmetric.
 * a_vals[a_offs[na]][dim], a_ts[...], a_offs[na+1]; out[na*nb] (host). */
twed_status_t twed_allpairs_host_f32(twed_handle_t handle, const float* a_vals,
                                     const float* a_ts, const int64_t* a_offs, int64_t na,
                                     const float* b_vals, const float* b_ts,
                                     const int64_t* b_offs, int64_t nb, int dim, float nu,
                                     float lambda, int p, float* out);

/* ---- learned k-NN candidate filter ---------------------------------------
 * The paper has no learned component; this is a filter in front of its exact
 * batch mode.  A 1-D convolutional encoder maps a series to e in R^32,
 * e = (psi in R^31, z), trained so that the additive model
 *     |psi_a - psi_b|^2 + z_a + z_b   approximates   TWED(a, b) / sigma
 * on pairs whose TWED the library computes exactly (twed_batch_f32).  A query
 * takes the n_candidates database series with the smallest model value (an
 * L2 search: database vectors (psi, sqrt(z - z_min)) against the query vector
 * (psi, 0)), re-ranks them by exact TWED and returns the k best.
 *
 * Encoder (all FP32): per point the inputs a_i (dim values), t_i and the
 * delete cost dA(i) = d(a_i, a_{i-1}) + nu|t_i - t_{i-1}| + lambda (a_0 = 0,
 * t_0 = 0), each standardised by the database's per-channel mean and
 * standard deviation; three convolutions of 64 channels, 5 taps, zero 'same'
 * padding and ReLU; the sum over time divided by the database's mean length
 * (a mean pool weighted by length); a linear map 64 -> 32.
 * Flat parameter layout: W1[64][dim+2][5], b1[64], W2[64][64][5], b2[64],
 * W3[64][64][5], b3[64], Wl[32][64], bl[32]; conv y[t][o] = b[o] +
 * sum_k sum_c W[o][c][k] x[t+k-2][c].  dim must be <= 14.
 *
 * Training: groups of `group_size` distinct database series are drawn (seeded
 * splitmix64 shuffles); every pair inside a group is labelled with exact
 * TWED, so ~train_pairs labels come from group_size * train_pairs /
 * (group_size (group_size-1) / 2) series.  sigma = mean label.  Each Adam
 * step (beta 0.9 / 0.999, eps 1e-8, cosine-decayed learning rate) minimises
 * the mean squared error of the model over the pairs of `groups_per_step`
 * groups (with rel_floor > 0, the mean squared relative error: each
 * residual divided by label / sigma + rel_floor).  With mine_fraction f > 0, (1-f) train_pairs come from random
 * groups, used alone for the first half of the epochs; then the database is
 * embedded and f train_pairs come from mined groups -- a seeded anchor and
 * the group_size-1 series nearest to it under the current model -- labelled
 * exactly and trained on together with the random groups for the other half.
 * Then every database series is embedded. */
typedef struct twed_knn_s* twed_knn_t;
typedef struct {
    int group_size;       /* series per labelled group, 2..64 (default 32) */
    int groups_per_step;  /* groups per Adam step (default 32) */
    int epochs;           /* passes over the labelled groups (default 40) */
    int64_t train_pairs;  /* labelled pairs (default 1,000,000) */
    float lr;             /* peak learning rate (default 2e-3) */
    uint64_t seed;        /* group sampling and weight initialisation (default 1) */
    float mine_fraction;  /* share of train_pairs from mined groups, [0, 1) (default 0) */
    float rel_floor;      /* 0: squared error; > 0: squared relative error, each pair's
                             residual divided by (label / sigma + rel_floor) (default 0) */
} twed_knn_config_t;

typedef struct {
    double sigma;          /* label scale (mean training TWED) */
    double mean_len;       /* mean database series length (pool divisor) */
    double first_loss;     /* mean loss of the first epoch */
    double last_loss;      /* mean loss of the last epoch */
    int64_t label_pairs;   /* pairs labelled with exact TWED (random + mined) */
    int64_t mined_pairs;   /* of which in mined groups */
    int64_t label_cells;   /* interior cells of those pairs */
    int64_t steps;         /* Adam steps taken */
    double label_ms;       /* wall time of labelling (exact TWED) */
    double train_ms;       /* wall time of the Adam steps */
    double embed_ms;       /* wall time of embedding the database */
    int32_t rerank_rows_per_lane;  /* re-rank launch shape chosen by timing */
    int32_t rerank_blocks_per_sm;  /* (rows-per-lane cap, resident blocks per SM) */
    double tune_ms;        /* wall time of that timing */
} twed_knn_stats_t;

void twed_knn_config_default(twed_knn_config_t* cfg);
/* db: device set (offs_host required) owned by the caller; it must stay valid
 * and unchanged for the index's lifetime.  cfg NULL = defaults.  Allocates
 * the index's device memory; trains nothing yet. */
twed_status_t twed_knn_create(twed_handle_t handle, const twed_set_f32_t* db, int dim, float nu,
                              float lambda, int p, const twed_knn_config_t* cfg, twed_knn_t* knn);
/* Labels, trains and embeds the database, then times the re-rank's launch
 * shape on random database pairs (blocking; uses the handle's stream).  May
 * be called again to retrain from a fresh initialisation. */
twed_status_t twed_knn_train(twed_knn_t knn);
/* Queries (device set, offs_host required): d_idx[q*k + r] (device int64)
 * and d_dist[q*k + r] (device float, exact FP32 TWED) receive the k
 * best of the n_candidates filtered database series, ascending (ties by
 * smaller database index).  1 <= k <= n_candidates <= min(ndb, 4096).
 * Enqueued on `stream`; the call waits only for its own host-side setup. */
twed_status_t twed_knn_search(twed_knn_t knn, const twed_set_f32_t* queries, int k,
                              int n_candidates, int64_t* d_idx, float* d_dist, void* stream);
/* Exact batched k-NN (the reference the filter's recall is measured against): the full
 * queries x database TWED matrix through an all-pairs plan, then the k
 * smallest per query (ties by smaller index).  1 <= k <= min(ndb, 4096).
 * Blocking. */
twed_status_t twed_knn_exact(twed_knn_t knn, const twed_set_f32_t* queries, int k,
                             int64_t* d_idx, float* d_dist, void* stream);
/* Host-memory queries, blocking: vals[offs[nq]][dim], ts[offs[nq]],
 * offs[nq+1] (host); idx[nq*k], dist[nq*k] (host) receive the results.
 * Copies in, searches on the index's own stream, copies out. */
twed_status_t twed_knn_search_host(twed_knn_t knn, const float* vals, const float* ts,
                                   const int64_t* offs, int64_t nq, int k, int n_candidates,
                                   int64_t* idx, float* dist);
/* Device time of the phases of the last twed_knn_search (waits for it):
 * phase_ms[0] query embedding, [1] candidate search (L2 + top-C),
 * [2] exact re-rank, [3] final top-k; *rerank_cells = interior cells the
 * re-rank evaluated. */
twed_status_t twed_knn_search_profile(twed_knn_t knn, double* phase_ms, int64_t* rerank_cells);
twed_status_t twed_knn_get_stats(twed_knn_t knn, twed_knn_stats_t* out);
/* Parameters (host float[twed_encoder_param_count(dim)]). */
twed_status_t twed_knn_get_params(twed_knn_t knn, float* out, int64_t n);
/* Replace the parameters and re-embed the database (blocking).  On an index
 * whose re-rank shape was never timed, also times it (as twed_knn_train). */
twed_status_t twed_knn_set_params(twed_knn_t knn, const float* in, int64_t n);
/* Database embeddings e (device float[ndb][32]) after training. */
twed_status_t twed_knn_get_embeddings(twed_knn_t knn, float* d_out, void* stream);
void twed_knn_destroy(twed_knn_t knn);

/* ---- encoder building blocks (blocking; each allocates and frees its own
 * scratch).  They expose the kernels the index uses so each can be checked
 * on its own. */
int64_t twed_encoder_param_count(int dim);
/* d_mu[dim+2], d_sd[dim+2] (device): per-channel mean and population
 * standard deviation of the encoder inputs over every point of `set`
 * (a channel with zero spread gets 1). */
twed_status_t twed_encoder_stats_f32(twed_handle_t handle, const twed_set_f32_t* set, int dim,
                                     float nu, float lambda, int p, float* d_mu, float* d_sd);
/* d_emb[set->n][32] (device): embeddings of every series of `set`. */
twed_status_t twed_encoder_forward_f32(twed_handle_t handle, const twed_set_f32_t* set, int dim,
                                       float nu, float lambda, int p, const float* d_params,
                                       const float* d_mu, const float* d_sd, float mean_len,
                                       float* d_emb);
/* Loss and parameter gradient over groups of series of `set`:
 * groups[g*group_size + a] (host int64) index `set`; d_labels[g*npg + q]
 * (device) is the label of the q-th pair (a < b, row-major) of group g,
 * npg = group_size (group_size-1) / 2.  loss = (1/npairs) sum (model -
 * label * inv_sigma)^2; d_grad (device, param_count floats) receives its
 * gradient and d_loss[0] (device) the loss. */
twed_status_t twed_encoder_loss_grad_f32(twed_handle_t handle, const twed_set_f32_t* set,
                                         int dim, float nu, float lambda, int p,
                                         const float* d_params, const float* d_mu,
                                         const float* d_sd, float mean_len,
                                         const int64_t* groups, int64_t ngroups, int group_size,
                                         const float* d_labels, float inv_sigma, float* d_grad,
                                         float* d_loss);
/* One Adam step (step >= 1) on device arrays of n floats. */
twed_status_t twed_adam_f32(twed_handle_t handle, float* d_theta, const float* d_grad, float* d_m,
                            float* d_v, int64_t n, int64_t step, float lr, float beta1,
                            float beta2, float eps);
/* Candidate search over embeddings (device float[..][32]): for each query,
 * the k database rows with the smallest |(psi_q, 0) - (psi_x, sqrt(z_x -
 * z_min))|^2, ascending (ties by smaller index); d_idx[nq*k], d_val[nq*k]. */
twed_status_t twed_embed_search_f32(twed_handle_t handle, const float* d_db_emb, int64_t ndb,
                                    const float* d_q_emb, int64_t nq, int k, int64_t* d_idx,
                                    float* d_val);
/* Row-wise k smallest of d_D[rows][ld] over the first `cols` columns,
 * ascending, ties by smaller column; k <= 4096, cols < 2^31. */
twed_status_t twed_topk_rows_f32(twed_handle_t handle, const float* d_D, int64_t rows,
                                 int64_t cols, int64_t ld, int k, int64_t* d_idx, float* d_val,
                                 void* stream);

/* ---- pipe peaks -----------------------------------------------------------
 * Not from the paper: measures the issue rate that bounds the ALU-bound
 * kernels, for their roofline.  Independent FFMA (FP32) or DFMA (FP64)
 * chains, or (IALU32) chains of a 32-bit integer xor and max, on every SM,
 * timed with CUDA events on the legacy stream (best of three after a
 * warm-up); *ops_per_s = lane operations per second (one FMA, one xor or one
 * max = one operation).  Blocking. */
#define TWED_PEAK_FFMA32 0
#define TWED_PEAK_DFMA64 1
#define TWED_PEAK_IALU32 2
twed_status_t twed_pipe_peak(twed_handle_t handle, int kind, double* ops_per_s);

#ifdef __cplusplus
}
#endif

#endif /* TWED_H_ */
