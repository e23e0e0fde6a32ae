// twed_batch_f32_noalloc: explicit pairs with no device allocation.
//
// For callers that must not call cudaMalloc (see include/twed.h): the
// records, boundary rows and control words of the many-pairs kernel live in
// one static device array instead of a handle's workspace.  The kernels are
// the ones twed_batch_f32 uses; only where their scratch lives differs.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>

#include "../../include/twed.h"
#include "launch.h"

namespace {

constexpr size_t kScratchBytes = TWED_NOALLOC_SCRATCH_BYTES;
constexpr size_t kAlign = 256;
constexpr int kThreads = 128;
constexpr int kWarpsPerBlock = kThreads / 32;
constexpr int kMaxDevices = 64;

// The library's only static device buffer.  In host code this name is a
// stand-in, not a device address: host code uses the address that
// cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Every (dim, p) the many-pairs dispatch can pick: dim 1 (any p); dims 2,
// 3, 4 and 8 (5-7 use the dim-8 layout) with p = 1 or 2; the wide strips of
// dims 16, 28 and 64 at p = 2; everything else on the run-time-dimension
// kernels (which also serve the wide dims when the values are not 16-byte
// aligned).  The short-pair kernel is never chosen here: this entry point
// leaves PairsArgs::max_len at 0.
constexpr int kVariants = 13;
constexpr int kRuntimeDim = 9;  // variant index of the run-time-dimension kernels
int variant_of(int dim, int p) {
    if (dim == 1) return 0;
    if (p == 2 && (dim == 16 || dim == 28 || dim == 64)) return dim == 16 ? 10 : (dim == 28 ? 11 : 12);
    const int d = dim <= 4 ? dim : (dim <= 8 ? 8 : 0);
    if (d == 0 || (p != 1 && p != 2)) return kRuntimeDim;
    const int di = d == 2 ? 0 : d == 3 ? 1 : d == 4 ? 2 : 3;
    return 1 + 2 * di + (p - 1);
}
void variant_rep(int v, int* dim, int* p) {
    static const int dims[4] = {2, 3, 4, 8};
    static const int wide[3] = {16, 28, 64};
    if (v == 0) { *dim = 1; *p = 2; }
    else if (v == kRuntimeDim) { *dim = 9; *p = 2; }
    else if (v > kRuntimeDim) { *dim = wide[v - kRuntimeDim - 1]; *p = 2; }
    else { *dim = dims[(v - 1) / 2]; *p = (v - 1) % 2 + 1; }
}

// What the first call on a device sets up, with that device current.
struct DeviceSetup {
    bool ready = false;
    unsigned char* scratch = nullptr;  // device address of g_scratch
    int sms = 0;
    int per_sm[kVariants] = {};        // resident many-pairs blocks per SM
};
std::mutex g_mu;
DeviceSetup g_dev[kMaxDevices];

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Once per device: the device address of g_scratch (cudaGetSymbolAddress),
// the SM count, and every records / many-pairs kernel variant this entry
// point can launch loaded and sized (function attribute and occupancy
// queries), so that later calls do no lazy module loading.
cudaError_t device_setup(int dev, const DeviceSetup** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceSetup& d = g_dev[dev];
    if (!d.ready) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        for (int v = 0; v < kVariants && e == cudaSuccess; ++v) {
            int vd = 0, vp = 0;
            variant_rep(v, &vd, &vp);
            e = twed::records_preload_f32(vd, vp);
            if (e == cudaSuccess) {
                d.per_sm[v] = twed::pairs_blocks_per_sm<float>(vd, vp, kThreads);
                if (d.per_sm[v] < 1) e = cudaErrorInvalidConfiguration;
            }
        }
        if (e != cudaSuccess) {
            (void)cudaGetLastError();
            return e;  // not marked ready: the next call tries again
        }
        d.scratch = static_cast<unsigned char*>(p);
        d.ready = true;
    }
    *out = &d;
    return cudaSuccess;
}

bool good_set(const twed_set_f32_t* s, int64_t* max_len, int64_t* total) {
    if (!s || !s->vals || !s->ts || !s->offs || !s->offs_host || s->n < 1) return false;
    if (s->offs_host[0] != 0) return false;
    int64_t mx = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        const int64_t len = s->offs_host[i + 1] - s->offs_host[i];
        if (len < 1 || len > ((int64_t)1 << 30)) return false;
        mx = std::max(mx, len);
    }
    *max_len = mx;
    *total = s->offs_host[s->n];
    return true;
}

}  // namespace

extern "C" twed_status_t twed_batch_f32_noalloc(const twed_set_f32_t* A, const twed_set_f32_t* B,
                                                const int64_t* d_pairs, int64_t npairs, int dim,
                                                float nu, float lambda, int p, float* d_out,
                                                void* stream) {
    if (npairs < 0) return TWED_ERR_INVALID_ARG;
    if (npairs == 0) return TWED_OK;
    if (!d_pairs || !d_out || dim < 1 || p < 1) return TWED_ERR_INVALID_ARG;
    if (!std::isfinite(nu) || nu < 0.f || !std::isfinite(lambda) || lambda < 0.f)
        return TWED_ERR_INVALID_ARG;
    int64_t maxa = 0, tota = 0, maxb = 0, totb = 0;
    if (!good_set(A, &maxa, &tota) || !good_set(B, &maxb, &totb)) return TWED_ERR_INVALID_ARG;

    // layout inside the static array: control words, records, boundary rows
    const bool same = (A->vals == B->vals && A->ts == B->ts && A->offs == B->offs);
    const size_t rl = (size_t)twed::rec_len<float>(dim, p);
    const size_t o_ctl = 0;  // [0] err, [1] sticky, [4..5] pair counter
    const size_t o_ra = align_up(o_ctl + 64);
    const size_t o_rb = same ? o_ra : align_up(o_ra + sizeof(float) * rl * (size_t)tota);
    const size_t o_rows = align_up(o_rb + sizeof(float) * rl * (size_t)totb);
    const int64_t scols = (std::max(maxa, maxb) + 2) & ~(int64_t)1;  // >= longest + 1, even
    const size_t row_bytes = sizeof(float) * 2 * (size_t)scols;
    if (o_rows > kScratchBytes) return TWED_ERR_UNSUPPORTED;
    const int64_t fit_warps = (int64_t)((kScratchBytes - o_rows) / row_bytes);
    if (fit_warps < kWarpsPerBlock) return TWED_ERR_UNSUPPORTED;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TWED_ERR_CUDA;
    const DeviceSetup* ds = nullptr;
    if (device_setup(dev, &ds) != cudaSuccess) return TWED_ERR_CUDA;
    unsigned char* base = ds->scratch;

    const int per_sm = ds->per_sm[variant_of(dim, p)];
    int64_t blocks = std::min<int64_t>((int64_t)per_sm * ds->sms, (npairs + kWarpsPerBlock - 1) / kWarpsPerBlock);
    blocks = std::min<int64_t>(blocks, fit_warps / kWarpsPerBlock);
    blocks = std::max<int64_t>(blocks, 1);

    cudaStream_t st = (cudaStream_t)stream;
    unsigned* ctl = reinterpret_cast<unsigned*>(base + o_ctl);
    // the array keeps the previous call's contents: zero the control words
    if (cudaMemsetAsync(ctl, 0, 64, st) != cudaSuccess) return TWED_ERR_CUDA;
    float* rec_a = reinterpret_cast<float*>(base + o_ra);
    float* rec_b = reinterpret_cast<float*>(base + o_rb);
    twed::RecordsArgs<float> ra{A->vals, A->ts, A->offs, A->n, tota, dim, p, nu, lambda, rec_a};
    if (twed::launch_records(ra, st) != cudaSuccess) return TWED_ERR_CUDA;
    if (!same) {
        twed::RecordsArgs<float> rb{B->vals, B->ts, B->offs, B->n, totb, dim, p, nu, lambda, rec_b};
        if (twed::launch_records(rb, st) != cudaSuccess) return TWED_ERR_CUDA;
    }
    twed::PairsArgs<float> pa{};
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
    pa.rmax = twed::pairs_rmax_limit<float>();
    pa.nu = nu;
    pa.out = d_out;
    pa.counter = reinterpret_cast<unsigned long long*>(ctl + 4);
    pa.scratch = base + o_rows;
    pa.scratch_cols = scols;
    pa.sc.err = ctl;
    pa.sc.sticky = ctl + 1;
    pa.sc.timeout_ns = 2000000000ull;
    pa.sc.stall_strip = -1;
    pa.sc.sleep_ns = 32;
    if (twed::launch_pairs(pa, (int)blocks, kThreads, st) != cudaSuccess) return TWED_ERR_CUDA;
    return TWED_OK;
}
