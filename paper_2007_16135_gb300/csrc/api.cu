// C ABI of the TWED library (include/twed.h): validation, workspace,
// schedule choice, plans and CUDA-graph capture.  All arithmetic of the
// method runs in the kernels of kernels_f32.cu / kernels_f64.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <numeric>
#include <string>
#include <vector>

#include "../../include/twed.h"
#include "handle.h"
#include "launch.h"

using twed::CoopArgs;
using twed::PairsArgs;
using twed::RecordsArgs;

#define TWED_VERSION_STR "twed-gb300 0.1"

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Carves aligned sub-buffers out of one allocation.
struct Carver {
    size_t off = 0;
    size_t take(size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes);
        return o;
    }
};

}  // namespace

struct twed_handle_s {
    int device = 0;
    int sms = 0;
    unsigned sleep_ns = 32;  // poll back-off (env TWED_WAIT_SLEEP_NS)
    int band_warps = 8;      // strips per band (env TWED_BAND_WARPS: 2, 4 or 8)
    cudaStream_t stream = nullptr;
    void* ws = nullptr;  // grow-only device workspace
    size_t ws_bytes = 0;
    unsigned* ctl = nullptr;  // [0] live error word, [1] sticky error word
    std::string last_error;
};

namespace {

twed_status_t fail(twed_handle_t h, twed_status_t st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->last_error = buf;
    return st;
}

twed_status_t cuda_fail(twed_handle_t h, cudaError_t e, const char* what) {
    return fail(h, TWED_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Text of an error word a kernel left in the launch's control words.
const char* device_error_text(unsigned code) {
    switch (code) {
        case TWED_ERR_INVALID_ARG: return "a pair index lies outside its set (the pair's result is NaN)";
        case TWED_ERR_TIMEOUT: return "a bounded inter-warp wait expired";
        case TWED_ERR_UNSUPPORTED: return "the kernel's shared memory window is not 1024-byte aligned";
        default: return "a kernel reported an error";
    }
}

#define TWED_CUDA(h, call)                                          \
    do {                                                            \
        cudaError_t e_ = (call);                                    \
        if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);    \
    } while (0)

twed_status_t ensure_ws(twed_handle_t h, size_t bytes) {
    if (bytes <= h->ws_bytes) return TWED_OK;
    if (h->ws) {
        cudaError_t e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamSynchronize");
        cudaFree(h->ws);
        h->ws = nullptr;
        h->ws_bytes = 0;
    }
    size_t want = align_up(bytes + bytes / 4);
    cudaError_t e = cudaMalloc(&h->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&h->ws, bytes);
        want = bytes;
        if (e != cudaSuccess) {
            cudaGetLastError();
            h->ws = nullptr;
            return fail(h, TWED_ERR_ALLOC, "device workspace of %zu bytes: %s", bytes,
                        cudaGetErrorString(e));
        }
    }
    h->ws_bytes = want;
    return TWED_OK;
}

template <typename T>
bool finite_param(T v) {
    return std::isfinite((double)v) && v >= T(0);
}

template <typename T>
twed_status_t check_params(twed_handle_t h, int64_t la, int64_t lb, int dim, T nu, T lambda,
                           int p) {
    if (la < 1 || lb < 1) return fail(h, TWED_ERR_INVALID_ARG, "series lengths must be >= 1");
    if (la > (int64_t)1 << 30 || lb > (int64_t)1 << 30)
        return fail(h, TWED_ERR_INVALID_ARG, "series length above 2^30");
    if (dim < 1) return fail(h, TWED_ERR_INVALID_ARG, "dim must be >= 1");
    if (p < 1) return fail(h, TWED_ERR_INVALID_ARG, "p must be >= 1");
    if (!finite_param(nu)) return fail(h, TWED_ERR_INVALID_ARG, "nu must be finite and >= 0");
    if (!finite_param(lambda))
        return fail(h, TWED_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    return TWED_OK;
}

template <typename T>
bool all_finite(const T* x, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite((double)x[i])) return false;
    return true;
}

unsigned long long timeout_ns(const twed_opts_t* o) {
    double s = (o && o->timeout_s > 0) ? o->timeout_s : 2.0;
    if (s > 600.0) s = 600.0;
    return (unsigned long long)(s * 1e9);
}

twed::SyncCtl make_sync(twed_handle_t h, const twed_opts_t* o) {
    twed::SyncCtl sc;
    sc.err = h->ctl;
    sc.sticky = h->ctl + 1;
    sc.timeout_ns = timeout_ns(o);
    sc.stall_strip = o ? o->stall_strip : -1;
    sc.sleep_ns = h->sleep_ns;
    return sc;
}

// Warps the FP64 one-pair schedule keeps in flight: at most 4 per SM.
// Every FP64 operation runs on the FP64 pipe (2 DFMA per SM per clock on
// this part), so a few warps per SM already keep it busy; more strips in
// flight only lengthen the fill of the wavefront (each strip trails its
// predecessor by about kCoopLag columns).
constexpr int kCoopF64WarpsPerSm = 4;
constexpr double kCoopLag = 64.0;

// Rows per lane for one long pair.  FP64: a cost model over R in {4, 2, 1}:
// with W = min(strips, 4 x SMs) warps, the pair takes about
// (strips / W) x m + W x lag steps, each costing R x (warps per SM) FP64-pipe
// slots.  FP32 (run-time dimensions): enough strips to give every SM several
// warps, otherwise the most rows per lane (fewest shuffles per cell).
template <typename T>
int coop_rows_per_lane(twed_handle_t h, int64_t n, int64_t m, const twed_opts_t* o) {
    if (o && o->rows_per_lane > 0) {
        int r = o->rows_per_lane;
        return r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1;
    }
    if (sizeof(T) == 8) {
        int best = 1;
        double best_t = 1e300;
        for (int r : {4, 2, 1}) {
            const double strips = std::ceil((double)n / (32.0 * r));
            const double W = std::min(strips, (double)kCoopF64WarpsPerSm * h->sms);
            const double wps = std::ceil(W / h->sms);
            const double t = (strips / W * (double)m + W * kCoopLag) * r * wps;
            if (t < best_t * 0.97) {  // ties go to more rows per lane
                best_t = t;
                best = r;
            }
        }
        return best;
    }
    const int64_t want_warps = (int64_t)h->sms * 8;
    const int cand[4] = {8, 4, 2, 1};
    for (int r : cand) {
        if (sizeof(T) == 8 && r > 4) continue;
        if ((n + 32 * r - 1) / (32 * r) >= want_warps) return r;
    }
    return 1;
}

// Band schedule (FP32, compiled point layouts): strips of 32*R rows, bands of
// h->band_warps strips per block.  R is picked with a small cost model: a step
// costs the larger of one warp's dependency chain and the SM's issue slots
// shared by its active warps; consecutive strips start ~40 steps apart; bands
// beyond the resident blocks run in further rounds.

int band_rows_per_lane(twed_handle_t h, int64_t n, int64_t m, int dim, int p, bool kahan,
                       const twed_opts_t* o) {
    if (o && o->rows_per_lane > 0) {
        int r = o->rows_per_lane;
        return r >= 8 ? 8 : r >= 4 ? 4 : r >= 2 ? 2 : 1;
    }
    const double c_row = (dim > 1 ? dim : 2) + 9.0 + (kahan ? 35.0 : 0.0);  // instructions per row
    const double c_step = 24.0;                                          // per step, per warp
    const double lat_row = kahan ? 40.0 : 8.0;                           // chain cycles per row
    int best = 1;
    double best_t = 1e300;
    for (int R : {8, 4, 2, 1}) {
        const int per_sm = twed::band_blocks_per_sm(dim, p, R, kahan, h->band_warps);
        if (per_sm < 1) continue;
        const double nstrips = std::ceil((double)n / (32.0 * R));
        const double nbands = std::ceil(nstrips / h->band_warps);
        const double conc = (double)per_sm * h->sms;
        const double rounds = std::ceil(nbands / conc);
        const double active = std::min(nbands, conc);
        const double warps_sm = active * h->band_warps / h->sms;
        const double t_step = std::max(60.0 + lat_row * R, (c_row * R + c_step) * warps_sm / 4.0);
        const double t = rounds * ((double)m + active * h->band_warps * 40.0) * t_step;
        if (t < best_t) {
            best_t = t;
            best = R;
        }
    }
    return best;
}

// Workspace layout of one pair (records, boundary ring, flags) from `base`.
struct PairLayout {
    int R;
    bool kahan;
    bool band;  // block-cooperative FP32 schedule
    int64_t nstrips;
    int64_t ring_stride;
    size_t o_ra, o_rb, o_ring, o_flags, end;
};
constexpr int kRingSlots = 4;

// Compensated FP32 running cost: requested, or automatic above 1e5 points
// per pair (where plain FP32 sums along ~n+m steps start to drift).
template <typename T>
bool use_kahan(int64_t n, int64_t m, int dim, int p, const twed_opts_t* o) {
    if (sizeof(T) != 4 || !twed::compiled_layout(dim, p)) return false;
    const int acc = o ? o->accum : TWED_ACCUM_AUTO;
    if (acc == TWED_ACCUM_KAHAN) return true;
    if (acc == TWED_ACCUM_F32) return false;
    return n + m > 100000;
}

template <typename T>
PairLayout pair_layout(twed_handle_t h, int64_t n, int64_t m, int dim, int p,
                       const twed_opts_t* o, size_t base) {
    PairLayout L;
    L.kahan = use_kahan<T>(n, m, dim, p, o);
    L.band = sizeof(T) == 4 && twed::compiled_layout(dim, p);
    L.R = L.band ? band_rows_per_lane(h, n, m, dim, p, L.kahan, o) : coop_rows_per_lane<T>(h, n, m, o);
    L.nstrips = (n + 32 * L.R - 1) / (32 * L.R);
    const int rl = twed::rec_len<T>(dim, p);
    Carver cv;
    cv.off = base;
    L.o_ra = cv.take(sizeof(T) * rl * (size_t)n);
    L.o_rb = cv.take(sizeof(T) * rl * (size_t)m);
    L.ring_stride = (m + 2) & ~(int64_t)1;  // >= m + 1, even
    const size_t entry = L.kahan ? 16 : sizeof(T) * 2;
    L.o_ring = cv.take(entry * (size_t)kRingSlots * (size_t)L.ring_stride);
    L.o_flags = cv.take(sizeof(unsigned) * (size_t)(L.nstrips + 1));
    L.end = cv.off;
    return L;
}

// Launch the one-pair schedule chosen in L (band kernel for FP32 compiled
// layouts, else the cooperative strip kernel) for the pair described by ca.
template <typename T>
twed_status_t launch_pair_schedule(twed_handle_t h, const PairLayout& L, const CoopArgs<T>& ca,
                                   cudaStream_t st) {
    const int R = L.R;
    if constexpr (sizeof(T) == 4) {
        if (L.band) {
            const int bw = h->band_warps;
            const int per_sm = std::max(1, twed::band_blocks_per_sm(ca.dim, ca.p, R, L.kahan, bw));
            const int64_t nbands = (L.nstrips + bw - 1) / bw;
            const int64_t blocks = std::max<int64_t>(1, std::min<int64_t>(nbands, (int64_t)per_sm * h->sms));
            const cudaError_t e = twed::launch_band(ca, R, L.kahan, (int)blocks, bw, st);
            if (e != cudaSuccess)
                return fail(h, TWED_ERR_CUDA, "band launch (dim %d, p %d, R %d, kahan %d, blocks %lld, per_sm %d): %s",
                            ca.dim, ca.p, R, (int)L.kahan, (long long)blocks, per_sm, cudaGetErrorString(e));
            return TWED_OK;
        }
    }
    // FP64: one warp per block, so the block scheduler spreads the first
    // strips over separate SMs (a short pair's few strips each get an SM's
    // FP64 pipe) and at most kCoopF64WarpsPerSm land on one SM
    const bool f64 = sizeof(T) == 8;
    const int threads = f64 ? 32 : 128;
    const int per_sm = std::max(1, twed::coop_blocks_per_sm<T>(ca.dim, ca.p, R, L.kahan, threads));
    int64_t blocks = f64 ? std::min<int64_t>(L.nstrips, (int64_t)std::min(per_sm, kCoopF64WarpsPerSm) * h->sms)
                         : std::min<int64_t>((L.nstrips + 3) / 4, (int64_t)per_sm * h->sms);
    blocks = std::max<int64_t>(1, blocks);
    TWED_CUDA(h, twed::launch_coop(ca, R, L.kahan, (int)blocks, threads, st));
    return TWED_OK;
}

// Enqueue one pair on `st` with all inputs already on the device.
template <typename T>
twed_status_t run_pair_dev(twed_handle_t h, const T* a, const T* ta, int64_t la, const T* b,
                           const T* tb, int64_t lb, int dim, T nu, T lambda, int p,
                           const twed_opts_t* o, T* d_out, cudaStream_t st, size_t ws_base) {
    if (o && (o->accum < TWED_ACCUM_AUTO || o->accum > TWED_ACCUM_KAHAN))
        return fail(h, TWED_ERR_INVALID_ARG, "unknown accumulation mode %d", o->accum);
    if (o && o->accum == TWED_ACCUM_KAHAN && sizeof(T) == 4 && !twed::compiled_layout(dim, p))
        return fail(h, TWED_ERR_UNSUPPORTED,
                    "compensated FP32 needs dim <= 8 and p in {1,2} (dim 1: any p)");
    // rows = the longer series: more strips, more warps in flight
    if (lb > la) {
        std::swap(a, b);
        std::swap(ta, tb);
        std::swap(la, lb);
    }
    const int n = (int)la, m = (int)lb;
    const PairLayout L = pair_layout<T>(h, n, m, dim, p, o, ws_base);
    const int R = L.R;
    const int64_t nstrips = L.nstrips;
    const int nslot = kRingSlots;
    twed_status_t s = ensure_ws(h, L.end);
    if (s != TWED_OK) return s;
    char* base = (char*)h->ws;
    T* rec_a = (T*)(base + L.o_ra);
    T* rec_b = (T*)(base + L.o_rb);
    unsigned* flags = (unsigned*)(base + L.o_flags);
    const size_t o_ring = L.o_ring;

    TWED_CUDA(h, cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)(nstrips + 1), st));
    TWED_CUDA(h, cudaMemsetAsync(h->ctl, 0, sizeof(unsigned), st));

    // offs == nullptr: the records kernel treats the input as one series
    RecordsArgs<T> ra{a, ta, nullptr, 1, la, dim, p, nu, lambda, rec_a};
    TWED_CUDA(h, twed::launch_records(ra, st));
    RecordsArgs<T> rb{b, tb, nullptr, 1, lb, dim, p, nu, lambda, rec_b};
    TWED_CUDA(h, twed::launch_records(rb, st));

    CoopArgs<T> ca;
    ca.rec_a = rec_a;
    ca.rec_b = rec_b;
    ca.vals_a = a;
    ca.vals_b = b;
    ca.n = n;
    ca.m = m;
    ca.dim = dim;
    ca.p = p;
    ca.nu = nu;
    ca.nstrips = nstrips;
    ca.ring = base + o_ring;
    ca.nslot = nslot;
    ca.ring_stride = L.ring_stride;
    ca.flags = flags;
    ca.strip_counter = flags + nstrips;
    ca.out = d_out;
    ca.sc = make_sync(h, o);
    return launch_pair_schedule<T>(h, L, ca, st);
}

// Host-pointer pair: copy in, run, copy out, report wait timeouts.
template <typename T>
twed_status_t run_pair_host(twed_handle_t h, const T* a, const T* ta, int64_t la, const T* b,
                            const T* tb, int64_t lb, int dim, T nu, T lambda, int p,
                            const twed_opts_t* o, T* out) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!a || !ta || !b || !tb || !out) return fail(h, TWED_ERR_INVALID_ARG, "null pointer");
    twed_status_t s = check_params<T>(h, la, lb, dim, nu, lambda, p);
    if (s != TWED_OK) return s;
    if (!all_finite(a, la * dim) || !all_finite(ta, la) || !all_finite(b, lb * dim) ||
        !all_finite(tb, lb))
        return fail(h, TWED_ERR_INVALID_ARG, "non-finite input value or timestamp");
    Carver cv;
    const size_t o_a = cv.take(sizeof(T) * (size_t)(la * dim));
    const size_t o_ta = cv.take(sizeof(T) * (size_t)la);
    const size_t o_b = cv.take(sizeof(T) * (size_t)(lb * dim));
    const size_t o_tb = cv.take(sizeof(T) * (size_t)lb);
    const size_t o_out = cv.take(sizeof(T));
    const size_t base = cv.off;
    const PairLayout L = pair_layout<T>(h, std::max(la, lb), std::min(la, lb), dim, p, o, base);
    s = ensure_ws(h, L.end);  // sized once, so run_pair_dev never reallocates
    if (s != TWED_OK) return s;
    cudaStream_t st = h->stream;
    auto dptr = [&](size_t off) { return (T*)((char*)h->ws + off); };
    TWED_CUDA(h, cudaMemcpyAsync(dptr(o_a), a, sizeof(T) * la * dim, cudaMemcpyHostToDevice, st));
    TWED_CUDA(h, cudaMemcpyAsync(dptr(o_ta), ta, sizeof(T) * la, cudaMemcpyHostToDevice, st));
    TWED_CUDA(h, cudaMemcpyAsync(dptr(o_b), b, sizeof(T) * lb * dim, cudaMemcpyHostToDevice, st));
    TWED_CUDA(h, cudaMemcpyAsync(dptr(o_tb), tb, sizeof(T) * lb, cudaMemcpyHostToDevice, st));
    s = run_pair_dev<T>(h, dptr(o_a), dptr(o_ta), la, dptr(o_b), dptr(o_tb), lb, dim, nu, lambda,
                        p, o, dptr(o_out), st, base);
    if (s != TWED_OK) return s;
    unsigned err = 0;
    TWED_CUDA(h, cudaMemcpyAsync(out, dptr(o_out), sizeof(T), cudaMemcpyDeviceToHost, st));
    TWED_CUDA(h, cudaMemcpyAsync(&err, h->ctl, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    TWED_CUDA(h, cudaStreamSynchronize(st));
    if (err != 0) {
        unsigned zero = 0;
        cudaMemcpy(h->ctl + 1, &zero, sizeof zero, cudaMemcpyHostToDevice);
        return fail(h, (twed_status_t)err, "%s", device_error_text(err));
    }
    return TWED_OK;
}

template <typename T>
twed_status_t twed_dev_impl(twed_handle_t h, const T* a, const T* ta, int64_t la, const T* b,
                            const T* tb, int64_t lb, int dim, T nu, T lambda, int p,
                            const twed_opts_t* o, T* d_out, void* stream) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!a || !ta || !b || !tb || !d_out) return fail(h, TWED_ERR_INVALID_ARG, "null pointer");
    twed_status_t s = check_params<T>(h, la, lb, dim, nu, lambda, p);
    if (s != TWED_OK) return s;
    return run_pair_dev<T>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, o, d_out,
                           (cudaStream_t)stream, 0);
}

}  // namespace

// =========================================================== handles
extern "C" twed_status_t twed_create(twed_handle_t* out) {
    if (!out) return TWED_ERR_INVALID_ARG;
    *out = nullptr;
    twed_handle_t h = new (std::nothrow) twed_handle_s();
    if (!h) return TWED_ERR_ALLOC;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&h->ctl, 64);
    if (e == cudaSuccess) e = cudaMemset(h->ctl, 0, 64);
    if (const char* v = getenv("TWED_WAIT_SLEEP_NS")) h->sleep_ns = (unsigned)atoi(v);
    if (const char* v = getenv("TWED_BAND_WARPS")) {
        const int w = atoi(v);
        h->band_warps = (w == 2 || w == 4 || w == 8) ? w : 8;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (h->stream) cudaStreamDestroy(h->stream);
        if (h->ctl) cudaFree(h->ctl);
        delete h;
        return TWED_ERR_CUDA;
    }
    *out = h;
    return TWED_OK;
}

extern "C" void twed_destroy(twed_handle_t h) {
    if (!h) return;
    if (h->stream) cudaStreamSynchronize(h->stream);
    if (h->ws) cudaFree(h->ws);
    if (h->ctl) cudaFree(h->ctl);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

extern "C" const char* twed_last_error(twed_handle_t h) {
    return h ? h->last_error.c_str() : "null handle";
}

extern "C" const char* twed_version(void) { return TWED_VERSION_STR; }

// Internal accessors for the other translation units (handle.h).
namespace twed {
namespace detail {
twed_status_t set_error(twed_handle_t h, twed_status_t st, const char* msg) {
    if (h) h->last_error = msg;
    return st;
}
int handle_sms(twed_handle_t h) { return h ? h->sms : 0; }
void* handle_workspace(twed_handle_t h, size_t bytes, twed_status_t* st) {
    *st = ensure_ws(h, bytes);
    return *st == TWED_OK ? h->ws : nullptr;
}
void* handle_stream(twed_handle_t h) { return h ? (void*)h->stream : nullptr; }
unsigned* handle_ctl(twed_handle_t h) { return h ? h->ctl : nullptr; }
int handle_device(twed_handle_t h) { return h ? h->device : 0; }
}  // namespace detail
}  // namespace twed

extern "C" twed_status_t twed_sync_status(twed_handle_t h, void* stream) {
    if (!h) return TWED_ERR_INVALID_ARG;
    TWED_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
    TWED_CUDA(h, cudaStreamSynchronize(h->stream));
    unsigned sticky = 0, zero = 0;
    TWED_CUDA(h, cudaMemcpy(&sticky, h->ctl + 1, sizeof sticky, cudaMemcpyDeviceToHost));
    if (sticky) {
        TWED_CUDA(h, cudaMemcpy(h->ctl + 1, &zero, sizeof zero, cudaMemcpyHostToDevice));
        return fail(h, (twed_status_t)sticky, "%s", device_error_text(sticky));
    }
    return TWED_OK;
}

// =========================================================== one pair
extern "C" twed_status_t twed_f64(twed_handle_t h, const double* a, const double* ta, int64_t la,
                                  const double* b, const double* tb, int64_t lb, int dim,
                                  double nu, double lambda, int p, double* out) {
    return run_pair_host<double>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, nullptr, out);
}

extern "C" twed_status_t twed_f32(twed_handle_t h, const float* a, const float* ta, int64_t la,
                                  const float* b, const float* tb, int64_t lb, int dim, float nu,
                                  float lambda, int p, float* out) {
    return run_pair_host<float>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, nullptr, out);
}

extern "C" twed_status_t twed_f32_ex(twed_handle_t h, const float* a, const float* ta, int64_t la,
                                     const float* b, const float* tb, int64_t lb, int dim,
                                     float nu, float lambda, int p, const twed_opts_t* opts,
                                     float* out) {
    return run_pair_host<float>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, opts, out);
}

extern "C" twed_status_t twed_dev_f64(twed_handle_t h, const double* a, const double* ta,
                                      int64_t la, const double* b, const double* tb, int64_t lb,
                                      int dim, double nu, double lambda, int p, double* d_out,
                                      void* stream) {
    return twed_dev_impl<double>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, nullptr, d_out,
                                 stream);
}

extern "C" twed_status_t twed_dev_f32(twed_handle_t h, const float* a, const float* ta, int64_t la,
                                      const float* b, const float* tb, int64_t lb, int dim,
                                      float nu, float lambda, int p, float* d_out, void* stream) {
    return twed_dev_impl<float>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, nullptr, d_out,
                                stream);
}

extern "C" twed_status_t twed_dev_f64_ex(twed_handle_t h, const double* a, const double* ta,
                                         int64_t la, const double* b, const double* tb,
                                         int64_t lb, int dim, double nu, double lambda, int p,
                                         const twed_opts_t* opts, double* d_out, void* stream) {
    return twed_dev_impl<double>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, opts, d_out,
                                 stream);
}

extern "C" twed_status_t twed_dev_f32_ex(twed_handle_t h, const float* a, const float* ta,
                                         int64_t la, const float* b, const float* tb, int64_t lb,
                                         int dim, float nu, float lambda, int p,
                                         const twed_opts_t* opts, float* d_out, void* stream) {
    return twed_dev_impl<float>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, opts, d_out,
                                stream);
}

// =========================================================== many pairs
namespace {

template <typename S>
twed_status_t check_set(twed_handle_t h, const S* set, const char* name, int64_t* max_len,
                        int64_t* total, bool need_ts = true) {
    if (!set || !set->vals || (need_ts && !set->ts) || !set->offs || !set->offs_host)
        return fail(h, TWED_ERR_INVALID_ARG, "set %s: null pointer", name);
    if (set->n < 1) return fail(h, TWED_ERR_INVALID_ARG, "set %s: no series", name);
    if (set->offs_host[0] != 0) return fail(h, TWED_ERR_INVALID_ARG, "set %s: offs[0] != 0", name);
    int64_t mx = 0;
    for (int64_t s = 0; s < set->n; ++s) {
        const int64_t len = set->offs_host[s + 1] - set->offs_host[s];
        if (len < 1) return fail(h, TWED_ERR_INVALID_ARG, "set %s: series %lld is empty", name, (long long)s);
        if (len > (int64_t)1 << 30) return fail(h, TWED_ERR_INVALID_ARG, "set %s: series too long", name);
        mx = std::max(mx, len);
    }
    *max_len = mx;
    *total = set->offs_host[set->n];
    return TWED_OK;
}

}  // namespace

struct twed_plan_s {
    twed_handle_t h = nullptr;
    bool f64 = false;
    bool symmetric = false;
    int64_t na = 0, nb = 0, npairs = 0, cells = 0;
    void* mem = nullptr;
    size_t mem_bytes = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    void* bound_out = nullptr;
    int blocks = 0, threads = 128;
    // argument blocks (the out pointer is filled in at capture)
    PairsArgs<float> pf{};
    PairsArgs<double> pd{};
    RecordsArgs<float> rfa{}, rfb{};
    RecordsArgs<double> rda{}, rdb{};
    unsigned* ctl = nullptr;  // plan's own [live err, sticky err]
    unsigned long long* counter = nullptr;
    bool xterm = false;  // tensor-core cross-term kernel (dim 64, FP32)
    bool xbf16 = false;  // ... with BF16 inputs (TWED_XTERM_BF16)
    twed::XtermArgs xa{};                 // its argument block (out filled in at launch)
    alignas(64) unsigned char tmap[128];  // its TMA descriptor of the column set's values
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;  // around the pairs launch
    std::string desc;
    // pairs above the cut-over run one at a time on the one-pair schedule;
    // rows = the longer series, from set B when r_is_b
    struct LongPair {
        int64_t rfirst, cfirst;  // first point of the row / column series
        int n, m;
        bool r_is_b;
        int64_t o1, o2;  // output elements (o2 < 0: none)
    };
    std::vector<LongPair> longp;
    int dim = 0, p = 2;
    bool has_opts = false;
    twed_opts_t opts{};
    void* band_ws = nullptr;
    size_t band_ring_bytes = 0;  // ring part of one lane's slot
    size_t band_slot_bytes = 0;  // ring + flags of one lane
    // long pairs run concurrently on `nlanes` side streams (one workspace
    // slot each), forked from and joined back into the execute's stream
    static constexpr int kMaxLanes = 8;
    int nlanes = 0;
    cudaStream_t lane_st[kMaxLanes] = {};
    cudaEvent_t fork_ev = nullptr;
    cudaEvent_t join_ev[kMaxLanes] = {};
};

namespace {

template <typename T>
PairsArgs<T>& plan_pairs(twed_plan_t pl);
template <>
PairsArgs<float>& plan_pairs<float>(twed_plan_t pl) { return pl->pf; }
template <>
PairsArgs<double>& plan_pairs<double>(twed_plan_t pl) { return pl->pd; }

template <typename T>
RecordsArgs<T>& plan_rec(twed_plan_t pl, int which);
template <>
RecordsArgs<float>& plan_rec<float>(twed_plan_t pl, int w) { return w ? pl->rfb : pl->rfa; }
template <>
RecordsArgs<double>& plan_rec<double>(twed_plan_t pl, int w) { return w ? pl->rdb : pl->rda; }

// Enqueue the whole plan (prologue + persistent pairs launch) on `st`.
template <typename T>
cudaError_t launch_plan_records(twed_plan_t pl, const RecordsArgs<T>& r, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (pl->xterm) return twed::launch_xrecords(r, st, pl->xbf16);
    }
    return twed::launch_records(r, st);
}

template <typename T>
cudaError_t launch_plan_pairs(twed_plan_t pl, const PairsArgs<T>& pa, cudaStream_t st) {
    if constexpr (sizeof(T) == 4) {
        if (pl->xterm) {
            twed::XtermArgs xa = pl->xa;
            xa.out = pa.out;
            return twed::launch_xterm(pl->tmap, xa, pl->blocks, st, pl->xbf16);
        }
    }
    return twed::launch_pairs(pa, pl->blocks, pl->threads, st);
}

template <typename T>
cudaError_t plan_enqueue(twed_plan_t pl, T* out, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(pl->counter, 0, sizeof(unsigned long long), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(pl->ctl, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) e = launch_plan_records<T>(pl, plan_rec<T>(pl, 0), st);
    if (e == cudaSuccess && !pl->symmetric) e = launch_plan_records<T>(pl, plan_rec<T>(pl, 1), st);
    PairsArgs<T> pa = plan_pairs<T>(pl);
    pa.out = out;
    // inside a capture the records become graph event-record nodes
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (e == cudaSuccess) e = cudaStreamIsCapturing(st, &cs);
    const unsigned evflag = cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal : 0u;
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(pl->ev0, st, evflag);
    if (e == cudaSuccess) e = launch_plan_pairs<T>(pl, pa, st);
    if (e == cudaSuccess) e = cudaEventRecordWithFlags(pl->ev1, st, evflag);
    if (e == cudaSuccess && !pl->longp.empty()) {
        e = cudaEventRecord(pl->fork_ev, st);
        for (int k = 0; k < pl->nlanes && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(pl->lane_st[k], pl->fork_ev, 0);
    }
    for (size_t i = 0; i < pl->longp.size() && e == cudaSuccess; ++i) {
        const auto& lp = pl->longp[i];
        const int lane = (int)(i % (size_t)pl->nlanes);
        cudaStream_t ls = pl->lane_st[lane];
        char* slot = (char*)pl->band_ws + (size_t)lane * pl->band_slot_bytes;
        const twed_opts_t* o = pl->has_opts ? &pl->opts : nullptr;
        const PairLayout L = pair_layout<T>(pl->h, lp.n, lp.m, pl->dim, pl->p, o, 0);
        const int rl = twed::rec_len<T>(pl->dim, pl->p);
        unsigned* flags = (unsigned*)(slot + pl->band_ring_bytes);
        e = cudaMemsetAsync(flags, 0, sizeof(unsigned) * (size_t)(L.nstrips + 1), ls);
        if (e != cudaSuccess) break;
        CoopArgs<T> ca;
        ca.rec_a = (lp.r_is_b ? pa.rec_b : pa.rec_a) + lp.rfirst * rl;
        ca.rec_b = (lp.r_is_b ? pa.rec_a : pa.rec_b) + lp.cfirst * rl;
        ca.vals_a = (lp.r_is_b ? pa.vals_b : pa.vals_a) + lp.rfirst * pl->dim;
        ca.vals_b = (lp.r_is_b ? pa.vals_a : pa.vals_b) + lp.cfirst * pl->dim;
        ca.n = lp.n;
        ca.m = lp.m;
        ca.dim = pl->dim;
        ca.p = pl->p;
        ca.nu = pa.nu;
        ca.nstrips = L.nstrips;
        ca.ring = slot;
        ca.nslot = kRingSlots;
        ca.ring_stride = L.ring_stride;
        ca.flags = flags;
        ca.strip_counter = flags + L.nstrips;
        ca.out = out + lp.o1;
        ca.sc = pa.sc;
        if (launch_pair_schedule<T>(pl->h, L, ca, ls) != TWED_OK) {
            e = cudaErrorLaunchFailure;
            break;
        }
        if (lp.o2 >= 0) e = cudaMemcpyAsync(out + lp.o2, out + lp.o1, sizeof(T), cudaMemcpyDeviceToDevice, ls);
    }
    if (!pl->longp.empty()) {
        // join every lane back, even after a failure (a capture must end joined)
        for (int k = 0; k < pl->nlanes; ++k) {
            cudaError_t e2 = cudaEventRecord(pl->join_ev[k], pl->lane_st[k]);
            if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(st, pl->join_ev[k], 0);
            if (e == cudaSuccess) e = e2;
        }
    }
    if (e == cudaSuccess && pl->symmetric) e = twed::launch_zero_diag(out, pl->f64, pl->na, st);
    return e;
}

// Host copy of the kernels' row-major triangle enumeration {(p, q): p < q < n}.
void host_triangle_pos(int64_t w, int64_t n, int64_t& p, int64_t& q) {
    int64_t r = (int64_t)((2.0 * n - 1.0 - std::sqrt((2.0 * n - 1.0) * (2.0 * n - 1.0) - 8.0 * (double)w)) * 0.5);
    r = std::max<int64_t>(0, std::min<int64_t>(r, n - 2));
    while (r > 0 && r * (2 * n - r - 1) / 2 > w) --r;
    while (r < n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= w) ++r;
    p = r;
    q = w - r * (2 * n - r - 1) / 2 + r + 1;
}

// Autotuner: times candidate schedules of this plan on a strided sample of its
// own pairs (same length mix, about 2e10 cells) and keeps the fastest.
// Candidates: the rows-per-lane cap (many-pairs kernel) and resident blocks
// per SM (both kernels).  Timing: CUDA events on a private stream, one
// warm-up and the best of two runs per candidate.
template <typename T>
twed_status_t autotune_plan(twed_handle_t h, twed_plan_t pl, const std::vector<int32_t>& perm_a,
                            const std::vector<int32_t>& perm_b, const int64_t* offs_a,
                            const int64_t* offs_b, int max_per_sm, std::string& report) {
    PairsArgs<T>& pa = plan_pairs<T>(pl);
    if (pl->xterm) {  // the tensor-core kernel has one launch shape (2 blocks per SM)
        report = "; autotune: not applicable to the tensor-core kernel (fixed launch shape)";
        return TWED_OK;
    }
    const double target = 2e10;
    const int64_t stride = std::max<int64_t>(1, (int64_t)((double)pl->cells / target));
    std::vector<int64_t> sample;
    double scells = 0;
    for (int64_t w = 0; w < pl->npairs && (int64_t)sample.size() < 2 * (1 << 21); w += stride) {
        int64_t x, y;
        if (pl->symmetric) {
            int64_t pp, qq;
            host_triangle_pos(w, pl->na, pp, qq);
            x = perm_a[pp];
            y = perm_a[qq];
        } else {
            x = perm_a[w / pl->nb];
            y = perm_b[w % pl->nb];
        }
        sample.push_back(x);
        sample.push_back(y);
        scells += (double)(offs_a[x + 1] - offs_a[x]) * (double)(offs_b[y + 1] - offs_b[y]);
    }
    const int64_t ns = (int64_t)sample.size() / 2;
    if (ns < 1) return TWED_OK;
    void* mem = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&mem, sizeof(int64_t) * 2 * ns + sizeof(T) * ns);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(mem, sample.data(), sizeof(int64_t) * 2 * ns, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_plan_records<T>(pl, plan_rec<T>(pl, 0), st);
    if (e == cudaSuccess && !pl->symmetric) e = launch_plan_records<T>(pl, plan_rec<T>(pl, 1), st);
    struct Cand {
        int rmax, per_sm;
        float ms;
    };
    std::vector<Cand> cands;
    {
        const int lim = twed::pairs_rmax_limit<T>();
        for (int r : {2, 4, 6, 8})
            if (r <= lim)
                for (int b = 1; b <= max_per_sm; ++b) cands.push_back({r, b, 0.f});
    }
    const int64_t per_block_pairs = 4;
    const int64_t cap_blocks = std::max<int64_t>(1, std::min<int64_t>(pl->blocks, (ns + per_block_pairs - 1) / per_block_pairs));
    PairsArgs<T> q = pa;
    q.mode = twed::kExplicitPairs;
    q.pairs = (const int64_t*)mem;
    q.npairs = ns;
    q.out = (T*)((char*)mem + sizeof(int64_t) * 2 * ns);
    for (Cand& c : cands) {
        if (e != cudaSuccess) break;
        q.rmax = c.rmax;
        const int blocks = (int)std::min<int64_t>((int64_t)c.per_sm * h->sms, cap_blocks);
        float best = 1e30f;
        for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
            e = cudaMemsetAsync(pl->counter, 0, sizeof(unsigned long long), st);
            if (e == cudaSuccess) e = cudaEventRecord(e0, st);
            if (e == cudaSuccess) {
                e = twed::launch_pairs(q, blocks, pl->threads, st);
            }
            if (e == cudaSuccess) e = cudaEventRecord(e1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0) best = std::min(best, ms);
        }
        c.ms = best;
    }
    unsigned err = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&err, pl->ctl + 1, sizeof err, cudaMemcpyDeviceToHost);
    if (st) cudaStreamDestroy(st);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (mem) cudaFree(mem);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return cuda_fail(h, e, "autotune");
    }
    if (err != 0u) return fail(h, (twed_status_t)err, "autotune: a bounded wait expired");
    const Cand* best = &cands[0];
    for (const Cand& c : cands)
        if (c.ms < best->ms) best = &c;
    pa.rmax = best->rmax;
    pl->blocks = (int)std::min<int64_t>((int64_t)best->per_sm * h->sms, pl->blocks);
    char buf[160];
    snprintf(buf, sizeof buf, "; autotuned on %lld sampled pairs (%.2e cells): rows_per_lane<=%d, %d blocks/SM, %.3f ms [",
             (long long)ns, scells, best->rmax, best->per_sm, best->ms);
    report = buf;
    for (size_t i = 0; i < cands.size(); ++i) {
        snprintf(buf, sizeof buf, "%s%d/%d:%.3f", i ? " " : "", cands[i].rmax, cands[i].per_sm, cands[i].ms);
        report += buf;
    }
    report += "]";
    return TWED_OK;
}

template <typename T, typename S>
twed_status_t plan_create(twed_handle_t h, const S* A, const S* B, int dim, T nu, T lambda,
                          int p, const twed_opts_t* o, twed_plan_t* out_plan) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!out_plan) return fail(h, TWED_ERR_INVALID_ARG, "null plan pointer");
    *out_plan = nullptr;
    twed_status_t s = check_params<T>(h, 1, 1, dim, nu, lambda, p);
    if (s != TWED_OK) return s;
    int64_t maxa = 0, tota = 0, maxb = 0, totb = 0;
    s = check_set(h, A, "A", &maxa, &tota);
    if (s != TWED_OK) return s;
    const bool sym = (B == nullptr);
    if (!sym) {
        s = check_set(h, B, "B", &maxb, &totb);
        if (s != TWED_OK) return s;
    } else {
        maxb = maxa;
        totb = tota;
    }
    twed_plan_t pl = new (std::nothrow) twed_plan_s();
    if (!pl) return fail(h, TWED_ERR_ALLOC, "plan");
    pl->h = h;
    pl->f64 = sizeof(T) == 8;
    pl->symmetric = sym;
    pl->na = A->n;
    pl->nb = sym ? A->n : B->n;

    // Longest series first: the persistent warps then finish on the shortest
    // pairs, which keeps the tail of the launch short.
    auto sorted = [](const int64_t* offs, int64_t n) {
        std::vector<int32_t> perm(n);
        std::iota(perm.begin(), perm.end(), 0);
        std::stable_sort(perm.begin(), perm.end(), [&](int32_t x, int32_t y) {
            return offs[x + 1] - offs[x] > offs[y + 1] - offs[y];
        });
        return perm;
    };
    std::vector<int32_t> perm_a = sorted(A->offs_host, A->n);
    std::vector<int32_t> perm_b = sym ? std::vector<int32_t>() : sorted(B->offs_host, B->n);
    int64_t cells = 0;
    if (sym) {
        // sum_{i<j} la*lb = ((sum l)^2 - sum l^2) / 2
        long double sl = 0, sl2 = 0;
        for (int64_t i = 0; i < A->n; ++i) {
            long double l = (long double)(A->offs_host[i + 1] - A->offs_host[i]);
            sl += l;
            sl2 += l * l;
        }
        cells = (int64_t)((sl * sl - sl2) / 2);
        pl->npairs = A->n * (A->n - 1) / 2;
    } else {
        cells = tota * totb;
        pl->npairs = A->n * B->n;
    }
    pl->cells = cells;

    const bool want_x = o && (o->xterm == TWED_XTERM_TF32 || o->xterm == TWED_XTERM_BF16);
    if (o && (o->xterm < TWED_XTERM_OFF || o->xterm > TWED_XTERM_BF16)) {
        delete pl;
        return fail(h, TWED_ERR_INVALID_ARG, "unknown xterm mode %d", o->xterm);
    }
    if (want_x && (sizeof(T) != 4 || dim != 64 || p != 2)) {
        delete pl;
        return fail(h, TWED_ERR_UNSUPPORTED, "tensor-core cross term: FP32, dim 64 and p 2 only");
    }
    if (want_x && (((uintptr_t)A->vals & 15) || (!sym && ((uintptr_t)B->vals & 15)))) {
        delete pl;
        return fail(h, TWED_ERR_UNSUPPORTED, "tensor-core cross term: values must be 16-byte aligned");
    }
    pl->xterm = want_x;
    pl->xbf16 = want_x && o->xterm == TWED_XTERM_BF16;
    const int rl = pl->xterm ? 4 : twed::rec_len<T>(dim, p);
    const int threads = pl->xterm ? twed::xterm_threads() : 128;
    const int per_sm_raw = pl->xterm ? twed::xterm_blocks_per_sm()
                                     : twed::pairs_blocks_per_sm<T>(dim, p, threads);
    int per_sm = std::max(1, per_sm_raw);
    // tensor-core plans: work items = one column series x up to CH row series
    // (sorted order); symmetric plans count them per chunk of rows
    std::vector<int64_t> chunk_start;
    int64_t nitems = 0;
    if (pl->xterm) {
        // the persistent kernel claims items dynamically, so blocks beyond the
        // resident ones would only queue: size the grid from the resources
        // (shared memory, registers, tensor memory), which the occupancy
        // query does not see in full
        per_sm = std::max(per_sm, twed::xterm_resident_blocks());
        if (const char* v = getenv("TWED_XTERM_BLOCKS_PER_SM")) per_sm = std::max(1, atoi(v));
        const int64_t CH = twed::xterm_rows_per_item();
        const int64_t nch = (A->n + CH - 1) / CH;
        if (!sym) {
            nitems = nch * B->n;
        } else {
            chunk_start.resize((size_t)nch + 1);
            for (int64_t c = 0; c < nch; ++c) {
                chunk_start[(size_t)c] = nitems;
                nitems += std::min((c + 1) * CH, A->n) - 1;
            }
            chunk_start[(size_t)nch] = nitems;
        }
    }
    const int64_t want_blocks = (int64_t)per_sm * h->sms;
    const int64_t need_blocks = pl->xterm ? std::max<int64_t>(1, nitems)
                                          : std::max<int64_t>(1, (pl->npairs + 3) / 4);
    pl->blocks = (int)std::min(want_blocks, need_blocks);
    pl->threads = threads;
    const int64_t nwarps = pl->xterm ? 0 : (int64_t)pl->blocks * (threads / 32);
    const int64_t scols = (std::max(maxa, maxb) + 2) & ~(int64_t)1;  // >= longest + 1, even

    Carver cv;
    const size_t o_ra = cv.take(sizeof(T) * rl * (size_t)tota);
    const size_t o_rb = sym ? 0 : cv.take(sizeof(T) * rl * (size_t)totb);
    const size_t o_pa = cv.take(sizeof(int32_t) * perm_a.size());
    const size_t o_pb = sym ? 0 : cv.take(sizeof(int32_t) * perm_b.size());
    const size_t o_scr = cv.take(sizeof(T) * 2 * (size_t)nwarps * (size_t)scols);
    const int64_t xbnd = pl->xterm ? twed::xterm_bnd_stride(std::max(maxa, maxb)) : 0;
    const size_t o_xb = pl->xterm ? cv.take(sizeof(float) * 2 * (size_t)pl->blocks *
                                            (size_t)twed::xterm_warps_per_block() * (size_t)xbnd) : 0;
    const size_t o_cs = chunk_start.empty() ? 0 : cv.take(sizeof(int64_t) * chunk_start.size());
    const int64_t xtot = sym ? tota : totb;  // points of the column set
    const size_t o_bf = pl->xbf16 ? cv.take((size_t)2 * 64 * (size_t)xtot) : 0;  // its BF16 copy
    const size_t o_ctl = cv.take(64);
    pl->mem_bytes = cv.off;
    cudaError_t e = cudaMalloc(&pl->mem, pl->mem_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        delete pl;
        return fail(h, TWED_ERR_ALLOC, "plan memory of %zu bytes: %s", cv.off, cudaGetErrorString(e));
    }
    char* base = (char*)pl->mem;
    pl->ctl = (unsigned*)(base + o_ctl);
    pl->counter = (unsigned long long*)(base + o_ctl + 16);
    e = cudaMemcpy(base + o_pa, perm_a.data(), sizeof(int32_t) * perm_a.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !sym)
        e = cudaMemcpy(base + o_pb, perm_b.data(), sizeof(int32_t) * perm_b.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && !chunk_start.empty())
        e = cudaMemcpy(base + o_cs, chunk_start.data(), sizeof(int64_t) * chunk_start.size(),
                       cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(pl->ctl, 0, 64);
    if (e == cudaSuccess && pl->xbf16) {
        e = twed::launch_bf16_copy((const float*)(sym ? A->vals : B->vals), base + o_bf, 64 * xtot, nullptr);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess && pl->xterm)
        e = twed::xterm_tensor_map(pl->tmap, pl->xbf16 ? (const void*)(base + o_bf) : (const void*)(sym ? A->vals : B->vals),
                                   xtot, pl->xbf16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(pl->mem);
        delete pl;
        return cuda_fail(h, e, "plan set-up copies");
    }

    T* rec_a = (T*)(base + o_ra);
    T* rec_b = sym ? rec_a : (T*)(base + o_rb);
    plan_rec<T>(pl, 0) = RecordsArgs<T>{A->vals, A->ts, A->offs, A->n, tota, dim, p, nu, lambda, rec_a};
    if (!sym) plan_rec<T>(pl, 1) = RecordsArgs<T>{B->vals, B->ts, B->offs, B->n, totb, dim, p, nu, lambda, rec_b};

    PairsArgs<T>& pa = plan_pairs<T>(pl);
    pa.rec_a = rec_a;
    pa.rec_b = rec_b;
    pa.vals_a = A->vals;
    pa.vals_b = sym ? A->vals : B->vals;
    pa.offs_a = A->offs;
    pa.offs_b = sym ? A->offs : B->offs;
    pa.mode = sym ? twed::kSymmetricSorted : twed::kBlockSorted;
    pa.pairs = nullptr;
    pa.perm_a = (const int32_t*)(base + o_pa);
    pa.perm_b = sym ? pa.perm_a : (const int32_t*)(base + o_pb);
    pa.npairs = pl->npairs;
    pa.na = pl->na;
    pa.nb = pl->nb;
    pa.dim = dim;
    pa.p = p;
    pa.rmax = (o && o->rows_per_lane > 0) ? o->rows_per_lane : twed::pairs_rmax_limit<T>();
    pa.nu = nu;
    pa.out = nullptr;
    pa.counter = pl->counter;
    pa.scratch = base + o_scr;
    pa.scratch_cols = scols;
    pa.max_len = std::max(maxa, maxb);
    pa.sc.err = pl->ctl;
    pa.sc.sticky = pl->ctl + 1;
    pa.sc.timeout_ns = timeout_ns(o);
    pa.sc.stall_strip = -1;
    pa.sc.sleep_ns = h->sleep_ns;
    if constexpr (sizeof(T) == 4) {
        if (pl->xterm) {
            twed::XtermArgs& xa = pl->xa;
            xa.vals_a = A->vals;
            xa.rec_a = (const float4*)rec_a;
            xa.rec_b = (const float4*)rec_b;
            xa.offs_a = A->offs;
            xa.offs_b = sym ? A->offs : B->offs;
            xa.perm_a = pa.perm_a;
            xa.perm_b = pa.perm_b;
            xa.na = pl->na;
            xa.nb = pl->nb;
            xa.symmetric = sym ? 1 : 0;
            xa.nitems = nitems;
            xa.chunk_start = chunk_start.empty() ? nullptr : (const int64_t*)(base + o_cs);
            xa.nchunks = chunk_start.empty() ? 0 : (int64_t)chunk_start.size() - 1;
            xa.nu = nu;
            xa.out = nullptr;
            xa.bnd = (float2*)(base + o_xb);
            xa.bnd_stride = xbnd;
            xa.counter = pl->counter;
            xa.sc = pa.sc;
        }
    }

    // Schedule cut-over: a pair with more cells than the plan's average work
    // per warp would leave one warp running long after the others finish;
    // such pairs (at most kMaxLongPairs, else the load is balanced anyway)
    // run one at a time on the one-pair block-cooperative schedule.
    pl->dim = dim;
    pl->p = p;
    if (o) {
        pl->has_opts = true;
        pl->opts = *o;
    }
    if (!pl->xterm && nwarps > 0) {
        constexpr size_t kMaxLongPairs = 4096;
        const int64_t cut = std::max<int64_t>(1, cells / nwarps);
        const int64_t* oa = A->offs_host;
        const int64_t* ob = sym ? A->offs_host : B->offs_host;
        auto lena = [&](int64_t r) { const int64_t x = perm_a[r]; return oa[x + 1] - oa[x]; };
        auto lenb = [&](int64_t r) { const int64_t y = sym ? perm_a[r] : perm_b[r]; return ob[y + 1] - ob[y]; };
        bool too_many = false;
        auto add = [&](int64_t x, int64_t y, int64_t o1, int64_t o2) {
            if (pl->longp.size() >= kMaxLongPairs) {
                too_many = true;
                return;
            }
            const int64_t lx = oa[x + 1] - oa[x], ly = ob[y + 1] - ob[y];
            twed_plan_s::LongPair lp;
            lp.r_is_b = ly > lx;  // rows = the longer series
            lp.rfirst = lp.r_is_b ? ob[y] : oa[x];
            lp.cfirst = lp.r_is_b ? oa[x] : ob[y];
            lp.n = (int)std::max(lx, ly);
            lp.m = (int)std::min(lx, ly);
            lp.o1 = o1;
            lp.o2 = o2;
            pl->longp.push_back(lp);
        };
        const int64_t nb_ = sym ? A->n : B->n;
        for (int64_t pp = 0; pp < A->n && !too_many; ++pp) {
            const int64_t lp_ = lena(pp);
            const int64_t q0 = sym ? pp + 1 : 0;
            if (q0 >= nb_ || lp_ * lenb(q0) <= cut) {
                if (sym || lp_ * lenb(0) <= cut) break;
                continue;
            }
            for (int64_t qq = q0; qq < nb_ && !too_many; ++qq) {
                if (lp_ * lenb(qq) <= cut) break;
                const int64_t x = perm_a[pp], y = sym ? perm_a[qq] : perm_b[qq];
                if (sym) add(x, y, x * A->n + y, y * A->n + x);
                else add(x, y, x * nb_ + y, -1);
            }
        }
        if (too_many) pl->longp.clear();
        if (!pl->longp.empty()) {
            size_t ring = 0, flags = 0;
            for (const auto& lp : pl->longp) {
                const PairLayout L = pair_layout<T>(h, lp.n, lp.m, dim, p, o, 0);
                ring = std::max(ring, L.o_flags - L.o_ring);
                flags = std::max(flags, L.end - L.o_flags);
            }
            pl->band_ring_bytes = align_up(ring);
            pl->band_slot_bytes = align_up(pl->band_ring_bytes + flags);
            pl->nlanes = (int)std::min<size_t>(pl->longp.size(), twed_plan_s::kMaxLanes);
            e = cudaMalloc(&pl->band_ws, pl->band_slot_bytes * (size_t)pl->nlanes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->fork_ev, cudaEventDisableTiming);
            for (int k = 0; k < pl->nlanes && e == cudaSuccess; ++k) {
                e = cudaStreamCreateWithFlags(&pl->lane_st[k], cudaStreamNonBlocking);
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&pl->join_ev[k], cudaEventDisableTiming);
            }
            if (e != cudaSuccess) {
                cudaGetLastError();
                for (int k = 0; k < pl->nlanes; ++k) {
                    if (pl->lane_st[k]) cudaStreamDestroy(pl->lane_st[k]);
                    if (pl->join_ev[k]) cudaEventDestroy(pl->join_ev[k]);
                }
                if (pl->fork_ev) cudaEventDestroy(pl->fork_ev);
                if (pl->band_ws) cudaFree(pl->band_ws);
                cudaFree(pl->mem);
                delete pl;
                return fail(h, TWED_ERR_ALLOC, "plan cut-over workspace: %s", cudaGetErrorString(e));
            }
            pa.cut_cells = cut;
        }
    }

    e = cudaStreamCreateWithFlags(&pl->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&pl->ev1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(pl->mem);
        delete pl;
        return cuda_fail(h, e, "cudaStreamCreate");
    }
    std::string tuned;
    if (o && o->autotune) {
        s = autotune_plan<T>(h, pl, perm_a, perm_b, A->offs_host, sym ? A->offs_host : B->offs_host,
                             per_sm, tuned);
        if (s != TWED_OK) {
            twed_plan_destroy(pl);
            return s;
        }
    }
    char d[400];
    if (pl->xterm) {
        char r[200];
        twed::xterm_resources(r, sizeof r);
        snprintf(d, sizeof d,
                 "f32 tensor-core cross term (tf32) pairs=%lld items=%lld blocks=%d x %d threads "
                 "(%d resident per SM by shared memory, registers and TMEM; occupancy query %d; %s)",
                 (long long)pl->npairs, (long long)nitems, pl->blocks, threads, twed::xterm_resident_blocks(),
                 per_sm_raw, r);
    }
    else
        snprintf(d, sizeof d, "%s pairs=%lld warps=%lld rows_per_lane<=%d blocks=%d x %d threads",
                 sizeof(T) == 8 ? "f64" : "f32", (long long)pl->npairs, (long long)nwarps, pa.rmax,
                 pl->blocks, threads);
    pl->desc = std::string(d) + tuned;
    if (!pl->longp.empty()) {
        char c[160];
        snprintf(c, sizeof c, "; cut-over: %zu pairs above %lld cells on the one-pair schedule",
                 pl->longp.size(), (long long)pa.cut_cells);
        pl->desc += c;
    }
    *out_plan = pl;
    return TWED_OK;
}

template <typename T>
twed_status_t plan_capture(twed_plan_t pl, T* out) {
    twed_handle_t h = pl->h;
    if (pl->exec) {
        cudaGraphExecDestroy(pl->exec);
        pl->exec = nullptr;
    }
    if (pl->graph) {
        cudaGraphDestroy(pl->graph);
        pl->graph = nullptr;
    }
    TWED_CUDA(h, cudaStreamBeginCapture(pl->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = plan_enqueue<T>(pl, out, pl->cap);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(pl->cap, &g);
    if (e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, e, "capturing the plan");
    }
    if (e2 != cudaSuccess) return cuda_fail(h, e2, "cudaStreamEndCapture");
    pl->graph = g;
    TWED_CUDA(h, cudaGraphInstantiate(&pl->exec, g, 0));
    pl->bound_out = out;
    return TWED_OK;
}

}  // namespace

extern "C" twed_status_t twed_allpairs_plan_create_f64(twed_handle_t h, const twed_set_f64_t* A,
                                                       const twed_set_f64_t* B, int dim, double nu,
                                                       double lambda, int p,
                                                       const twed_opts_t* opts, twed_plan_t* plan) {
    return plan_create<double>(h, A, B, dim, nu, lambda, p, opts, plan);
}

extern "C" twed_status_t twed_allpairs_plan_create_f32(twed_handle_t h, const twed_set_f32_t* A,
                                                       const twed_set_f32_t* B, int dim, float nu,
                                                       float lambda, int p,
                                                       const twed_opts_t* opts, twed_plan_t* plan) {
    return plan_create<float>(h, A, B, dim, nu, lambda, p, opts, plan);
}

extern "C" twed_status_t twed_plan_execute(twed_plan_t pl, void* d_out, void* stream) {
    if (!pl) return TWED_ERR_INVALID_ARG;
    if (!d_out) return fail(pl->h, TWED_ERR_INVALID_ARG, "null output");
    if (d_out != pl->bound_out || !pl->exec) {
        twed_status_t s = pl->f64 ? plan_capture<double>(pl, (double*)d_out)
                                  : plan_capture<float>(pl, (float*)d_out);
        if (s != TWED_OK) return s;
    }
    TWED_CUDA(pl->h, cudaGraphLaunch(pl->exec, (cudaStream_t)stream));
    return TWED_OK;
}

extern "C" twed_status_t twed_plan_status(twed_plan_t pl, void* stream) {
    if (!pl) return TWED_ERR_INVALID_ARG;
    twed_handle_t h = pl->h;
    TWED_CUDA(h, cudaStreamSynchronize((cudaStream_t)stream));
    unsigned sticky = 0, zero = 0;
    TWED_CUDA(h, cudaMemcpy(&sticky, pl->ctl + 1, sizeof sticky, cudaMemcpyDeviceToHost));
    if (sticky) {
        TWED_CUDA(h, cudaMemcpy(pl->ctl + 1, &zero, sizeof zero, cudaMemcpyHostToDevice));
        return fail(h, (twed_status_t)sticky, "plan: %s", device_error_text(sticky));
    }
    return TWED_OK;
}

extern "C" twed_status_t twed_plan_kernel_ms(twed_plan_t pl, float* ms) {
    if (!pl || !ms) return TWED_ERR_INVALID_ARG;
    TWED_CUDA(pl->h, cudaEventElapsedTime(ms, pl->ev0, pl->ev1));
    return TWED_OK;
}

extern "C" int64_t twed_plan_cells(twed_plan_t pl) { return pl ? pl->cells : 0; }
extern "C" int64_t twed_plan_pairs(twed_plan_t pl) { return pl ? pl->npairs : 0; }
extern "C" const char* twed_plan_describe(twed_plan_t pl) { return pl ? pl->desc.c_str() : ""; }

extern "C" void twed_plan_destroy(twed_plan_t pl) {
    if (!pl) return;
    cudaStreamSynchronize(pl->cap);
    if (pl->exec) cudaGraphExecDestroy(pl->exec);
    if (pl->graph) cudaGraphDestroy(pl->graph);
    if (pl->cap) cudaStreamDestroy(pl->cap);
    if (pl->ev0) cudaEventDestroy(pl->ev0);
    if (pl->ev1) cudaEventDestroy(pl->ev1);
    cudaDeviceSynchronize();
    for (int k = 0; k < pl->nlanes; ++k) {
        if (pl->lane_st[k]) cudaStreamDestroy(pl->lane_st[k]);
        if (pl->join_ev[k]) cudaEventDestroy(pl->join_ev[k]);
    }
    if (pl->fork_ev) cudaEventDestroy(pl->fork_ev);
    if (pl->band_ws) cudaFree(pl->band_ws);
    if (pl->mem) cudaFree(pl->mem);
    delete pl;
}

// =========================================================== explicit pairs
namespace {

// rmax / per_sm: rows-per-lane cap and resident blocks per SM of the
// many-pairs kernel (0: the kernel's limit and the occupancy maximum).
template <typename T, typename S>
twed_status_t batch_impl(twed_handle_t h, const S* A, const S* B, const int64_t* d_pairs,
                         int64_t npairs, int dim, T nu, T lambda, int p, T* d_out, void* stream,
                         int order_mode = TWED_ORDER_LIST, int rmax = 0, int per_sm_req = 0,
                         bool dtw = false) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (npairs < 0) return fail(h, TWED_ERR_INVALID_ARG, "npairs < 0");
    if (order_mode != TWED_ORDER_LIST && order_mode != TWED_ORDER_LONGEST_FIRST)
        return fail(h, TWED_ERR_INVALID_ARG, "unknown pair order %d", order_mode);
    if (npairs == 0) return TWED_OK;
    if (!d_pairs || !d_out) return fail(h, TWED_ERR_INVALID_ARG, "null pointer");
    twed_status_t s = check_params<T>(h, 1, 1, dim, nu, lambda, p);
    if (s != TWED_OK) return s;
    int64_t maxa, tota, maxb, totb;
    if ((s = check_set(h, A, "A", &maxa, &tota, !dtw)) != TWED_OK) return s;
    if ((s = check_set(h, B, "B", &maxb, &totb, !dtw)) != TWED_OK) return s;
    const bool same = (A->vals == B->vals && A->offs == B->offs && A->ts == B->ts);
    const int rl = twed::rec_len<T>(dim, p);
    const int threads = 128;
    const int occ = std::max(1, twed::pairs_blocks_per_sm<T>(dim, p, threads));
    const int per_sm = per_sm_req > 0 ? std::min(per_sm_req, occ) : occ;
    const int blocks = (int)std::min<int64_t>((int64_t)per_sm * h->sms, (npairs + 3) / 4);
    const int64_t nwarps = (int64_t)blocks * (threads / 32);
    const int64_t scols = (std::max(maxa, maxb) + 2) & ~(int64_t)1;  // >= longest + 1, even
    // a run order other than the list's, when there is a queue to order
    const bool order = order_mode != TWED_ORDER_LIST && npairs > nwarps;
    Carver cv;
    const size_t o_ra = cv.take(sizeof(T) * rl * (size_t)tota);
    const size_t o_rb = same ? o_ra : cv.take(sizeof(T) * rl * (size_t)totb);
    const size_t o_scr = cv.take(sizeof(T) * 2 * (size_t)nwarps * (size_t)scols);
    const size_t o_cnt = cv.take(sizeof(unsigned long long));
    const size_t o_ord = order ? cv.take(sizeof(int64_t) * (size_t)npairs) : 0;
    const size_t o_bins = order ? cv.take(sizeof(unsigned long long) * twed::kOrderBins) : 0;
    if ((s = ensure_ws(h, cv.off)) != TWED_OK) return s;
    char* base = (char*)h->ws;
    cudaStream_t st = (cudaStream_t)stream;
    T* rec_a = (T*)(base + o_ra);
    T* rec_b = (T*)(base + o_rb);
    unsigned long long* counter = (unsigned long long*)(base + o_cnt);
    TWED_CUDA(h, cudaMemsetAsync(counter, 0, sizeof(unsigned long long), st));
    TWED_CUDA(h, cudaMemsetAsync(h->ctl, 0, sizeof(unsigned), st));
    RecordsArgs<T> ra{A->vals, A->ts, A->offs, A->n, tota, dim, p, nu, lambda, rec_a};
    TWED_CUDA(h, twed::launch_records(ra, st));
    if (!same) {
        RecordsArgs<T> rb{B->vals, B->ts, B->offs, B->n, totb, dim, p, nu, lambda, rec_b};
        TWED_CUDA(h, twed::launch_records(rb, st));
    }
    PairsArgs<T> pa{};
    pa.rec_a = rec_a;
    pa.rec_b = rec_b;
    pa.vals_a = A->vals;
    pa.vals_b = B->vals;
    pa.offs_a = A->offs;
    pa.offs_b = B->offs;
    pa.mode = twed::kExplicitPairs;
    pa.pairs = d_pairs;
    pa.npairs = npairs;
    pa.na = A->n;
    pa.nb = B->n;
    pa.dim = dim;
    pa.p = p;
    pa.rmax = rmax > 0 ? std::min(rmax, twed::pairs_rmax_limit<T>()) : twed::pairs_rmax_limit<T>();
    pa.nu = nu;
    pa.out = d_out;
    pa.counter = counter;
    pa.scratch = base + o_scr;
    pa.scratch_cols = scols;
    pa.max_len = std::max(maxa, maxb);
    pa.sc = make_sync(h, nullptr);
    pa.dtw = dtw ? 1 : 0;
    if (order) {
        int64_t* ord = (int64_t*)(base + o_ord);
        TWED_CUDA(h, twed::launch_order_pairs(d_pairs, npairs, A->offs, A->n, B->offs, B->n, ord,
                                              (unsigned long long*)(base + o_bins), h->sms, st));
        pa.order = ord;
    }
    TWED_CUDA(h, twed::launch_pairs(pa, blocks, threads, st));
    return TWED_OK;
}

}  // namespace

namespace twed {
namespace detail {
twed_status_t batch_f32_shaped(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                               const int64_t* d_pairs, int64_t npairs, int dim, float nu,
                               float lambda, int p, float* d_out, void* stream, int order,
                               int rmax, int per_sm) {
    return batch_impl<float>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_out, stream, order,
                             rmax, per_sm);
}
twed_status_t dtw_batch_f32_staged(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                                   const int64_t* d_pairs, int64_t npairs, int dim, int p, float* d_out,
                                   void* stream) {
    return batch_impl<float>(h, A, B, d_pairs, npairs, dim, 0.f, 0.f, p, d_out, stream,
                             TWED_ORDER_LONGEST_FIRST, 0, 0, true);
}
int batch_f32_max_blocks_per_sm(int dim, int p) {
    return std::max(1, twed::pairs_blocks_per_sm<float>(dim, p, 128));
}
int batch_f32_rmax_limit() { return twed::pairs_rmax_limit<float>(); }
}  // namespace detail
}  // namespace twed

extern "C" twed_status_t twed_batch_f64(twed_handle_t h, const twed_set_f64_t* A,
                                        const twed_set_f64_t* B, const int64_t* d_pairs,
                                        int64_t npairs, int dim, double nu, double lambda, int p,
                                        double* d_out, void* stream) {
    return batch_impl<double>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_out, stream);
}

extern "C" twed_status_t twed_batch_f32(twed_handle_t h, const twed_set_f32_t* A,
                                        const twed_set_f32_t* B, const int64_t* d_pairs,
                                        int64_t npairs, int dim, float nu, float lambda, int p,
                                        float* d_out, void* stream) {
    return batch_impl<float>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_out, stream);
}

extern "C" twed_status_t twed_batch_f64_ex(twed_handle_t h, const twed_set_f64_t* A,
                                           const twed_set_f64_t* B, const int64_t* d_pairs,
                                           int64_t npairs, int dim, double nu, double lambda,
                                           int p, int order, double* d_out, void* stream) {
    return batch_impl<double>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_out, stream, order);
}

extern "C" twed_status_t twed_batch_f32_ex(twed_handle_t h, const twed_set_f32_t* A,
                                           const twed_set_f32_t* B, const int64_t* d_pairs,
                                           int64_t npairs, int dim, float nu, float lambda, int p,
                                           int order, float* d_out, void* stream) {
    return batch_impl<float>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_out, stream, order);
}

// =========================================================== host all-pairs
extern "C" twed_status_t twed_allpairs_host_f32(twed_handle_t h, const float* a_vals,
                                                const float* a_ts, const int64_t* a_offs,
                                                int64_t na, const float* b_vals,
                                                const float* b_ts, const int64_t* b_offs,
                                                int64_t nb, int dim, float nu, float lambda, int p,
                                                float* out) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!a_vals || !a_ts || !a_offs || na < 1 || !out)
        return fail(h, TWED_ERR_INVALID_ARG, "null pointer or empty set");
    const bool sym = (b_vals == nullptr);
    if (!sym && (!b_ts || !b_offs || nb < 1))
        return fail(h, TWED_ERR_INVALID_ARG, "set B incomplete");
    if (dim < 1) return fail(h, TWED_ERR_INVALID_ARG, "dim must be >= 1");
    const int64_t tota = a_offs[na], totb = sym ? 0 : b_offs[nb];
    if (tota < 1 || (!sym && totb < 1)) return fail(h, TWED_ERR_INVALID_ARG, "empty set");
    if (!all_finite(a_vals, tota * dim) || !all_finite(a_ts, tota) ||
        (!sym && (!all_finite(b_vals, totb * dim) || !all_finite(b_ts, totb))))
        return fail(h, TWED_ERR_INVALID_ARG, "non-finite input value or timestamp");
    const int64_t NB = sym ? na : nb;
    Carver cv;
    const size_t o_av = cv.take(sizeof(float) * tota * dim);
    const size_t o_at = cv.take(sizeof(float) * tota);
    const size_t o_ao = cv.take(sizeof(int64_t) * (na + 1));
    const size_t o_bv = sym ? 0 : cv.take(sizeof(float) * totb * dim);
    const size_t o_bt = sym ? 0 : cv.take(sizeof(float) * totb);
    const size_t o_bo = sym ? 0 : cv.take(sizeof(int64_t) * (nb + 1));
    const size_t o_out = cv.take(sizeof(float) * na * NB);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, cv.off);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(h, TWED_ERR_ALLOC, "staging memory: %s", cudaGetErrorString(e));
    }
    char* base = (char*)mem;
    cudaStream_t st = h->stream;
    twed_status_t s = TWED_OK;
    twed_plan_t pl = nullptr;
    do {
        e = cudaMemcpyAsync(base + o_av, a_vals, sizeof(float) * tota * dim, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_at, a_ts, sizeof(float) * tota, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ao, a_offs, sizeof(int64_t) * (na + 1), cudaMemcpyHostToDevice, st);
        if (!sym) {
            if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bv, b_vals, sizeof(float) * totb * dim, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bt, b_ts, sizeof(float) * totb, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_bo, b_offs, sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, st);
        }
        if (e != cudaSuccess) { s = cuda_fail(h, e, "host to device copies"); break; }
        twed_set_f32_t A{(const float*)(base + o_av), (const float*)(base + o_at),
                         (const int64_t*)(base + o_ao), a_offs, na};
        twed_set_f32_t B{(const float*)(base + o_bv), (const float*)(base + o_bt),
                         (const int64_t*)(base + o_bo), b_offs, nb};
        s = plan_create<float>(h, &A, sym ? nullptr : &B, dim, nu, lambda, p, nullptr, &pl);
        if (s != TWED_OK) break;
        // run the plan directly (no graph): a one-shot call gains nothing from capture
        e = plan_enqueue<float>(pl, (float*)(base + o_out), st);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "all-pairs launch"); break; }
        e = cudaMemcpyAsync(out, base + o_out, sizeof(float) * na * NB, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { s = cuda_fail(h, e, "device to host copy"); break; }
        unsigned err = 0;
        cudaMemcpy(&err, pl->ctl, sizeof err, cudaMemcpyDeviceToHost);
        if (err) s = fail(h, (twed_status_t)err, "%s", device_error_text(err));
    } while (0);
    if (pl) twed_plan_destroy(pl);
    cudaStreamSynchronize(st);
    cudaFree(mem);
    return s;
}
