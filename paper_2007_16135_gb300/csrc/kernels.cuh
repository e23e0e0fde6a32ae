// TWED kernels: prologue records, one-long-pair strips, many-pairs warps.
// Included once per precision (kernels_f32.cu, kernels_f64.cu).
#pragma once

// Resident blocks per SM the many-pairs kernel is compiled for (caps its
// registers at 65536 / (128 x this)).
#ifndef TWED_PAIRS_MIN_BLOCKS
#define TWED_PAIRS_MIN_BLOCKS 1
#endif

#include <algorithm>

#include "engine.cuh"
#include "engine_f32.cuh"
#include "engine_wide.cuh"

namespace twed {

// FP32 with a compile-time dimension runs the staged engine (engine_f32.cuh);
// FP64 and run-time dimensions run run_strip (engine.cuh).
template <typename T, int DIM>
constexpr bool kStaged = (sizeof(T) == 4 && DIM > 0);

// KH = compensated running cost (staged FP32 only; other paths ignore it).
template <typename T, int DIM, bool KH = false>
__host__ __device__ constexpr int smem_per_warp() {
    if constexpr (kStaged<T, DIM>) return staged_bytes_per_warp<DIM, KH>();
    else return 0;
}

template <typename T, int DIM, int P, int R, bool KH = false, int SB = kStepBlockPairs, bool DTW = false,
          bool PATH = false>
__device__ __forceinline__ bool strip_call(const PairRef<T>& pr, int r0, int rows,
                                           const StripIO<T>& io, const SyncCtl& sc, T* o1, T* o2,
                                           unsigned char* wsmem, uint32_t* choice = nullptr, int64_t wpr = 0) {
    if constexpr (kStaged<T, DIM>) {
        float* ring = reinterpret_cast<float*>(wsmem);
        void* bring = wsmem + kRingCols * Rec<float, DIM>::kLen * 4;
        return run_strip_staged<DIM, P, R, KH, SB, DTW, PATH>(pr, r0, rows, io, sc, o1, o2, ring, bring, choice,
                                                              wpr);
    } else {
        static_assert(!DTW && !PATH, "DTW and choice bits run on the staged FP32 engine only");
        (void)choice;
        (void)wpr;
        (void)wsmem;
        return run_strip<T, DIM, P, R>(pr, r0, rows, io, sc, o1, o2);
    }
}

// ------------------------------------------------------------------ prologue
// Step 1 of the paper's algorithm: the O(n) deletion costs of every series,
// dA(i) = d(a_i, a_{i-1}) + nu |t_i - t_{i-1}| + lambda, with a_0 = 0 and
// t_0 = 0 for the first point (the paper's footnote; the DP never reads
// dA(1)).  Packed with the point itself into one record per point.
template <typename T, int DIM, int P>
__global__ void __launch_bounds__(256) records_kernel(RecordsArgs<T> a) {
    using A = Arith<T>;
    using RL = Rec<T, DIM>;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += stride) {
        bool first = (g == 0);  // offs == nullptr: one series of `total` points
        if (a.offs != nullptr) {
            int64_t lo = 0, hi = a.nseries;  // offs[lo] <= g < offs[hi]
            while (hi - lo > 1) {
                const int64_t mid = (lo + hi) >> 1;
                if (__ldg(a.offs + mid) <= g) lo = mid; else hi = mid;
            }
            first = (__ldg(a.offs + lo) == g);
        }
        // a set without timestamps (DTW reads none) gives t = 0
        const T t = a.ts ? a.ts[g] : T(0);
        const T tprev = (first || !a.ts) ? T(0) : a.ts[g - 1];
        T d;
        T* out = a.rec + g * RL::kLen;
        if constexpr (DIM > 0) {
            // a point of a.dim <= DIM components is zero-padded to DIM: the
            // padded terms are |0 - 0|^p = 0 and come after the real ones, so
            // every distance is the same, bit for bit
            T x[DIM], y[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) {
                x[k] = k < a.dim ? a.vals[g * a.dim + k] : T(0);
                y[k] = (first || k >= a.dim) ? T(0) : a.vals[(g - 1) * a.dim + k];
#pragma unroll
                for (int u = 0; u < RL::kVS; ++u) out[k * RL::kVS + u] = x[k];
            }
            d = dist<T, DIM, P>(x, y, DIM, a.p);
        } else {
            const T* x = a.vals + g * (int64_t)a.dim;
            if (!first) {
                d = dist<T, 0, P>(x, x - a.dim, a.dim, a.p);
            } else {
                // distance to the zero padding: |x_k - 0| = |x_k|
                if (a.dim == 1) {
                    d = A::absv(x[0]);
                } else if (a.p == 1) {
                    d = A::absv(x[0]);
                    for (int k = 1; k < a.dim; ++k) d = A::add(d, A::absv(x[k]));
                } else if (a.p == 2) {
                    T s = A::mul(x[0], x[0]);
                    for (int k = 1; k < a.dim; ++k) s = A::sq_acc(s, x[k]);
                    d = A::root(s);
                } else {
                    const T e = (T)a.p;
                    T s = A::powv(A::absv(x[0]), e);
                    for (int k = 1; k < a.dim; ++k) s = A::add(s, A::powv(A::absv(x[k]), e));
                    d = A::powv(s, (T)1 / e);
                }
            }
        }
        out[RL::kT] = t;
        out[RL::kDel] = A::add(A::wcost(d, a.nu, t, tprev), a.lam);
#pragma unroll
        for (int q = RL::kDel + 1; q < RL::kLen; ++q) out[q] = T(0);
    }
}

// --------------------------------------------------------- one long pair
// Rows are cut into strips of 32*R rows.  Warps take strips in increasing
// order from an atomic counter, so the strip a warp waits on was taken by a
// warp that is already running: progress never depends on a warp that has
// not started, whatever the residency.  A strip publishes its bottom row
// every 16 columns into a ring slot (release store of the column count) and
// its successor polls that count (acquire, bounded by %globaltimer).
template <typename T, int DIM, int P, int R, bool KH>
__global__ void __launch_bounds__(128) coop_kernel(CoopArgs<T> a) {
    using V2 = typename Pair2<T>::V;
    // ring entries: (D, c) pairs, or (D_hi, D_lo, c, 0) quads when KH
    using Entry = typename std::conditional<KH && kStaged<T, DIM>, float4, V2>::type;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    unsigned char* wsmem = dyn_smem + (threadIdx.x >> 5) * smem_per_warp<T, DIM, KH>();
    const int lane = threadIdx.x & 31;
    PairRef<T> pr;
    pr.rec_a = a.rec_a;
    pr.rec_b = a.rec_b;
    pr.vals_a = a.vals_a;
    pr.vals_b = a.vals_b;
    pr.a_first = 0;
    pr.b_first = 0;
    pr.n = a.n;
    pr.m = a.m;
    pr.dim = a.dim;
    pr.p = a.p;
    pr.nu = a.nu;
    Entry* ring = reinterpret_cast<Entry*>(a.ring);
    while (true) {
        unsigned k = 0;
        if (lane == 0) k = atomicAdd(a.strip_counter, 1u);
        k = __shfl_sync(kFull, k, 0);
        if ((int64_t)k >= a.nstrips) break;
        if (*(volatile unsigned*)a.sc.err != 0u) break;
        const int r0 = (int)k * 32 * R + 1;
        const int rows = min(32 * R, a.n - r0 + 1);
        const bool last = (int64_t)k == a.nstrips - 1;
        StripIO<T> io = strip_io_global<T>(
            k == 0 ? nullptr
                   : reinterpret_cast<const V2*>(ring + (int64_t)((k - 1) % a.nslot) * a.ring_stride),
            k == 0 ? nullptr : a.flags + (k - 1),
            last ? nullptr : reinterpret_cast<V2*>(ring + (int64_t)(k % a.nslot) * a.ring_stride),
            last ? nullptr : a.flags + k, (long long)k != a.sc.stall_strip);
        if (!strip_call<T, DIM, P, R, KH>(pr, r0, rows, io, a.sc, a.out, nullptr, wsmem)) break;
    }
}

// ------------------------------------------------ one long pair, by bands
// Block-cooperative variant for FP32 with a compiled point layout.  A block
// of W warps claims a band of W consecutive strips (bands in increasing order
// from an atomic counter, so every band waits only on a band that is already
// running).  Inside the band, warp w writes its bottom row straight into the
// shared-memory boundary ring of warp w+1 and publishes progress every 8
// columns with a block-scope fence; only the band's first warp reads, and its
// last warp writes, a global boundary row with gpu-scope release/acquire
// flags.  This cuts the fences on the path to one gpu-scope hand-off per W
// strips and the lag between consecutive strips to about 40 columns.
template <int DIM, int P, int R, bool KH>
__global__ void __launch_bounds__(256) band_kernel(CoopArgs<float> a) {
    using Entry = typename std::conditional<KH, float4, float2>::type;
    constexpr int SPW = smem_per_warp<float, DIM, KH>();
    constexpr int kRecBytes = kRingCols * Rec<float, DIM>::kLen * 4;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    __shared__ int prog[32], cons[32];
    __shared__ long long band_sh;
    const int W = blockDim.x >> 5;
    const int w = threadIdx.x >> 5;
    unsigned char* wsmem = dyn_smem + w * SPW;
    const long long nbands = (a.nstrips + W - 1) / W;
    Entry* ring = reinterpret_cast<Entry*>(a.ring);
    PairRef<float> pr;
    pr.rec_a = a.rec_a;
    pr.rec_b = a.rec_b;
    pr.vals_a = a.vals_a;
    pr.vals_b = a.vals_b;
    pr.a_first = 0;
    pr.b_first = 0;
    pr.n = a.n;
    pr.m = a.m;
    pr.dim = a.dim;
    pr.p = a.p;
    pr.nu = a.nu;
    while (true) {
        __syncthreads();  // every warp is done with the previous band
        if (threadIdx.x == 0) {
            const bool failed = *(volatile unsigned*)a.sc.err != 0u;
            band_sh = failed ? nbands : (long long)atomicAdd(a.strip_counter, 1u);
        }
        if (threadIdx.x < 32) {
            prog[threadIdx.x] = 0;
            cons[threadIdx.x] = 0;
        }
        __syncthreads();
        const long long b = band_sh;
        if (b >= nbands) break;
        const long long k = b * W + w;  // this warp's strip
        if (k < a.nstrips) {
            const int r0 = (int)k * 32 * R + 1;
            const int rows = min(32 * R, a.n - r0 + 1);
            const bool last_strip = (k == a.nstrips - 1);
            const bool publish = (long long)k != a.sc.stall_strip;
            StripIO<float> io = strip_io_global<float>(nullptr, nullptr, nullptr, nullptr, publish);
            if (w == 0) {
                if (b > 0) {
                    io.up = reinterpret_cast<const float2*>(ring + ((b - 1) % a.nslot) * a.ring_stride);
                    io.up_flag = a.flags + (b - 1);
                }
            } else {
                io.up_local = true;
                io.up_prog = &prog[w];
                io.my_cons = &cons[w];
            }
            if (!last_strip) {
                if (w == W - 1) {
                    io.down = reinterpret_cast<float2*>(ring + (b % a.nslot) * a.ring_stride);
                    io.down_flag = a.flags + b;
                } else {
                    io.down_local = dyn_smem + (w + 1) * SPW + kRecBytes;
                    io.down_prog = &prog[w + 1];
                    io.down_cons = &cons[w + 1];
                }
            }
            strip_call<float, DIM, P, R, KH, kStepBlockBand>(pr, r0, rows, io, a.sc, a.out, nullptr, wsmem);
        }
    }
}

// ------------------------------------------------------------- many pairs
// Explicit pair lists come from the caller: an index outside [0, na) x
// [0, nb) is rejected on the device before any record is read.
__device__ __forceinline__ bool pair_in_range(int64_t x, int64_t y, int64_t na, int64_t nb) {
    return (uint64_t)x < (uint64_t)na && (uint64_t)y < (uint64_t)nb;
}
template <typename T>
__device__ __forceinline__ void flag_bad_pair(T* out, const SyncCtl& sc) {
    *out = (T)__int_as_float(0x7fc00000);  // quiet NaN
    atomicCAS(sc.err, 0u, 1u /* TWED_ERR_INVALID_ARG */);
    atomicCAS(sc.sticky, 0u, 1u);
}

__device__ __forceinline__ void triangle_pos(int64_t w, int64_t n, int64_t& p, int64_t& q) {
    // row-major enumeration of {(p, q): 0 <= p < q < n}; row p starts at
    // p*(2n - p - 1)/2
    const double b = 2.0 * (double)n - 1.0;
    int64_t r = (int64_t)((b - sqrt(b * b - 8.0 * (double)w)) * 0.5);
    if (r < 0) r = 0;
    if (r > n - 2) r = n - 2;
    while (r > 0 && r * (2 * n - r - 1) / 2 > w) --r;
    while (r < n - 2 && (r + 1) * (2 * n - r - 2) / 2 <= w) ++r;
    p = r;
    q = w - r * (2 * n - r - 1) / 2 + r + 1;
}

}  // namespace twed
#include "engine_short.cuh"
namespace twed {

// Shared memory per warp of the many-pairs kernel (WD > 0: the wide-point
// strips of engine_wide.cuh).
template <typename T, int DIM, int WD>
__host__ __device__ constexpr int pairs_smem_per_warp() {
    if constexpr (WD > 0) return wide_bytes_per_warp<WD>();
    else return smem_per_warp<T, DIM>();
}

template <typename T, int DIM, int P, int R, int WD, bool DTW>
__device__ __forceinline__ void pairs_strip(const PairRef<T>& pr, int r0, int rows, const StripIO<T>& io,
                                            const SyncCtl& sc, T* o1, T* o2, unsigned char* wsmem) {
    if constexpr (WD > 0) {
        (void)sc;
        float* ring = reinterpret_cast<float*>(wsmem);
        float2* bring = reinterpret_cast<float2*>(wsmem + kWideRing * wide_rec_floats<WD>() * 4);
        run_strip_wide<WD, R>(pr, r0, rows, io, o1, o2, ring, bring);
    } else {
        strip_call<T, DIM, P, R, false, kStepBlockPairs, DTW>(pr, r0, rows, io, sc, o1, o2, wsmem);
    }
}

// WD > 0: FP32 points of WD components, p = 2 (DIM = 0: the records hold
// (t, delete cost) only and the points are read from the values).
template <typename T, int DIM, int P, int RMAX, int WD = 0, bool DTW = false>
__global__ void __launch_bounds__(128, TWED_PAIRS_MIN_BLOCKS) pairs_kernel(PairsArgs<T> a) {
    using V2 = typename Pair2<T>::V;
    // packed row pairs need an even number of rows per lane
    constexpr bool kEven = kStaged<T, DIM> && P == 2 && DIM >= 2;
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    unsigned char* wsmem = dyn_smem + (threadIdx.x >> 5) * pairs_smem_per_warp<T, DIM, WD>();
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    V2* row = reinterpret_cast<V2*>(a.scratch) + gw * a.scratch_cols;
    const int rmax = a.rmax < RMAX ? (a.rmax < 1 ? 1 : a.rmax) : RMAX;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(a.counter, 1ull);
        w = __shfl_sync(kFull, w, 0);
        if ((int64_t)w >= a.npairs) break;
        int64_t x, y;
        T *o1, *o2 = nullptr;
        if (a.mode == kExplicitPairs) {
            const int64_t wi = a.order ? a.order[w] : (int64_t)w;
            x = a.pairs[2 * wi];
            y = a.pairs[2 * wi + 1];
            o1 = a.out + wi;
            // a caller's index outside its set is never dereferenced: the
            // pair's result is NaN and the launch reports TWED_ERR_INVALID_ARG
            if (!pair_in_range(x, y, a.na, a.nb)) {
                if (lane == 0) flag_bad_pair(o1, a.sc);
                continue;
            }
        } else if (a.mode == kSymmetricSorted) {
            int64_t pp, qq;
            triangle_pos((int64_t)w, a.na, pp, qq);
            x = a.perm_a[pp];
            y = a.perm_a[qq];
            o1 = a.out + x * a.na + y;
            o2 = a.out + y * a.na + x;
        } else {
            const int64_t pp = (int64_t)w / a.nb, qq = (int64_t)w % a.nb;
            x = a.perm_a[pp];
            y = a.perm_b[qq];
            o1 = a.out + x * a.nb + y;
        }
        const int64_t xa = a.offs_a[x], nx = a.offs_a[x + 1] - xa;
        const int64_t yb = a.offs_b[y], ny = a.offs_b[y + 1] - yb;
        // a pair far larger than a warp's share of the work runs on the
        // block-cooperative schedule instead (the plan enqueues it)
        if (a.cut_cells > 0 && nx * ny > a.cut_cells) continue;
        // Orientation: TWED is symmetric, and the swapped evaluation performs
        // the mirrored operations, so the value is the same bit for bit.  Take
        // the one with less estimated work: over its strips, (steps) x (R + 1)
        // -- R cells per lane per step plus about one row's worth of per-step
        // overhead -- so a short series whose rows would leave lanes idle
        // goes to the columns.
        auto work = [&](int64_t rows_n, int64_t cols_m) -> int64_t {
            int64_t w_ = 0;
            for (int64_t left = rows_n; left > 0;) {
                int R = left >= 32 * rmax ? rmax : (int)((left + 31) / 32);
                if (kEven) R = min((R + 1) & ~1, rmax);
                const int64_t rows = left < 32 * (int64_t)R ? left : 32 * (int64_t)R;
                w_ += (cols_m + (rows + R - 1) / R - 1) * (R + 1);
                left -= rows;
            }
            return w_;
        };
        PairRef<T> pr;
        pr.dim = a.dim;
        pr.p = a.p;
        pr.nu = a.nu;
        if (work(nx, ny) <= work(ny, nx)) {
            pr.rec_a = a.rec_a; pr.vals_a = a.vals_a; pr.a_first = xa; pr.n = (int)nx;
            pr.rec_b = a.rec_b; pr.vals_b = a.vals_b; pr.b_first = yb; pr.m = (int)ny;
        } else {
            pr.rec_a = a.rec_b; pr.vals_a = a.vals_b; pr.a_first = yb; pr.n = (int)ny;
            pr.rec_b = a.rec_a; pr.vals_b = a.vals_a; pr.b_first = xa; pr.m = (int)nx;
        }
        int r0 = 1;
        while (r0 <= pr.n) {
            const int left = pr.n - r0 + 1;
            int R = left >= 32 * rmax ? rmax : (left + 31) / 32;
            if (kEven) R = min((R + 1) & ~1, rmax);
            const int rows = min(left, 32 * R);
            const bool last = r0 + rows > pr.n;
            StripIO<T> io = strip_io_global<T>(r0 == 1 ? nullptr : row, nullptr,
                                               last ? nullptr : row, nullptr, true);
            switch (R) {
                case 1: if constexpr (!kEven) pairs_strip<T, DIM, P, 1, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 2: if constexpr (RMAX >= 2) pairs_strip<T, DIM, P, 2, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 3: if constexpr (RMAX >= 3 && !kEven) pairs_strip<T, DIM, P, 3, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 4: if constexpr (RMAX >= 4) pairs_strip<T, DIM, P, 4, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 5: if constexpr (RMAX >= 5 && !kEven) pairs_strip<T, DIM, P, 5, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 6: if constexpr (RMAX >= 6) pairs_strip<T, DIM, P, 6, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 7: if constexpr (RMAX >= 7 && !kEven) pairs_strip<T, DIM, P, 7, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                case 8: if constexpr (RMAX >= 8) pairs_strip<T, DIM, P, 8, WD, DTW>(pr, r0, rows, io, a.sc, o1, o2, wsmem); break;
                default: break;
            }
            r0 += rows;
            __syncwarp();
        }
    }
}

template <typename T>
__global__ void zero_diag_kernel(T* out, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i * n + i] = T(0);
}

// ----------------------------------------------------------- dispatch
// (dim, p) -> compiled variant: dims 1, 2, 3, 4, 8 keep points in registers;
// any other dim uses the run-time-dimension kernels (DIM = 0).  p = 1 and
// p = 2 have closed forms; other p use pow (P = 0).
#define TWED_DISPATCH(dim, p, BODY)                                            \
    do {                                                                       \
        _Pragma("nv_diag_suppress 177")                                        \
        switch (dim) {                                                         \
            case 1: { constexpr int DIM_ = 1, P_ = 2; BODY; } break;           \
            case 2: if (p == 1) { constexpr int DIM_ = 2, P_ = 1; BODY; }      \
                    else if (p == 2) { constexpr int DIM_ = 2, P_ = 2; BODY; } \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;      \
            case 3: if (p == 1) { constexpr int DIM_ = 3, P_ = 1; BODY; }      \
                    else if (p == 2) { constexpr int DIM_ = 3, P_ = 2; BODY; } \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;      \
            case 4: if (p == 1) { constexpr int DIM_ = 4, P_ = 1; BODY; }      \
                    else if (p == 2) { constexpr int DIM_ = 4, P_ = 2; BODY; } \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;      \
            case 5: case 6: case 7: /* zero-padded to the dim-8 layout */    \
            case 8: if (p == 1) { constexpr int DIM_ = 8, P_ = 1; BODY; }      \
                    else if (p == 2) { constexpr int DIM_ = 8, P_ = 2; BODY; } \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;      \
            default: { constexpr int DIM_ = 0, P_ = 0; BODY; } break;          \
        }                                                                      \
    } while (0)

template <typename T>
cudaError_t launch_records_t(const RecordsArgs<T>& a, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    const int threads = 256;
    int64_t blocks = (a.total + threads - 1) / threads;
    if (blocks > 65535) blocks = 65535;
    TWED_DISPATCH(a.dim, a.p, (records_kernel<T, DIM_, P_><<<(int)blocks, threads, 0, st>>>(a)));
    return cudaGetLastError();
}

// Launch (or size) a kernel with `threads` threads and its per-warp dynamic
// shared memory; the opt-in above 48 KB is set on every call (cheap).
// Dynamic plus static shared memory above 48 KB needs the opt-in; kernels
// here also carry a little static shared memory, so opt in whenever the
// dynamic part is not small.
template <typename K>
cudaError_t prepare_smem(K kernel, int smem) {
    if (smem <= 32 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

// Launch errors are read with cudaGetLastError, which also returns any
// earlier unchecked failure: clear that state first so the status belongs
// to this launch.
template <typename K, typename A>
cudaError_t launch_with_smem(K kernel, int smem_warp, int blocks, int threads, cudaStream_t st,
                             const A& a) {
    const int smem = smem_warp * (threads / 32);
    cudaError_t e = prepare_smem(kernel, smem);
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    kernel<<<blocks, threads, smem, st>>>(a);
    return cudaGetLastError();
}

template <typename K>
int blocks_per_sm(K kernel, int smem_warp, int threads) {
    const int smem = smem_warp * (threads / 32);
    int nb = 0;
    if (prepare_smem(kernel, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess) {
        (void)cudaGetLastError();  // a failed query must not surface at the next launch
        return 0;
    }
    return nb;
}

// Wide FP32 points with compiled many-pairs strips: dims 16, 28 and 64 at
// p = 2 (other wide dims run the run-time-dimension kernels).
#define TWED_WIDE_DISPATCH(dim, p, BODY)                                        \
    (((p) == 2 && (dim) == 16)   ? ([&] { constexpr int WD_ = 16; BODY; }(), true) \
     : ((p) == 2 && (dim) == 28) ? ([&] { constexpr int WD_ = 28; BODY; }(), true) \
     : ((p) == 2 && (dim) == 64) ? ([&] { constexpr int WD_ = 64; BODY; }(), true) \
                                 : false)

// Short pairs (engine_short.cuh): every series of both sets at most
// kShortMax points, p = 2, dims 16 and 28 (FP32 and FP64) or 64 (FP32),
// values and records 16-byte aligned.
template <typename T>
bool short_pairs_fit(const PairsArgs<T>& a) {
    if (a.dtw || a.p != 2 || a.max_len < 1 || a.max_len > kShortMax) return false;
    if (a.cut_cells > 0 && a.cut_cells < (int64_t)kShortMax * kShortMax) return false;
    if (((uintptr_t)a.vals_a | (uintptr_t)a.vals_b | (uintptr_t)a.rec_a | (uintptr_t)a.rec_b) & 15) return false;
    return a.dim == 16 || a.dim == 28 || (sizeof(T) == 4 && a.dim == 64);
}

// The third case instantiates the FP64 kernel at dim 16 again (never taken).
#define TWED_SHORT_DISPATCH(T, dim, BODY)                                                 \
    ((dim) == 16   ? ([&] { constexpr int SD_ = 16; BODY; }(), true)                     \
     : (dim) == 28 ? ([&] { constexpr int SD_ = 28; BODY; }(), true)                     \
     : (dim) == 64 ? ([&] { constexpr int SD_ = sizeof(T) == 4 ? 64 : 16; BODY; }(), true) \
                   : false)

// Persistent grid: the resident blocks on every SM, no more than the pairs
// need (kShortGrab pairs per warp).
template <typename T, int SD>
cudaError_t launch_short_dim(const PairsArgs<T>& a, int sms, cudaStream_t st) {
    constexpr int threads = 32 * kShortWarps;
    constexpr int warp_bytes = ShortSmem<T, SD>::kWarp;
    static int nb = 0;  // resident blocks per SM (one query per process)
    if (nb == 0) nb = blocks_per_sm(short_pairs_kernel<T, SD>, warp_bytes, threads);
    const int64_t warps_needed = (a.npairs + kShortGrab - 1) / kShortGrab;
    const int64_t blocks = std::min<int64_t>((int64_t)std::max(nb, 1) * sms,
                                             (warps_needed + kShortWarps - 1) / kShortWarps);
    return launch_with_smem(short_pairs_kernel<T, SD>, warp_bytes, (int)blocks, threads, st, a);
}

template <typename T>
cudaError_t launch_short_pairs(const PairsArgs<T>& a, cudaStream_t st) {
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    TWED_SHORT_DISPATCH(T, a.dim, (e = launch_short_dim<T, SD_>(a, sms, st)));
    return e;
}

template <typename T, int RMAX_LIMIT>
cudaError_t launch_pairs_t(const PairsArgs<T>& a, int blocks, int threads, cudaStream_t st) {
    if (a.npairs <= 0) return cudaSuccess;
    if (short_pairs_fit(a)) return launch_short_pairs(a, st);
    cudaError_t e = cudaSuccess;
    if (a.dtw) {
        // DTW: FP32 compiled point layouts on the staged engine only
        if constexpr (sizeof(T) == 4) {
            e = cudaErrorInvalidValue;
            TWED_DISPATCH(a.dim, a.p, (e = DIM_ > 0 ? launch_with_smem(pairs_kernel<T, (DIM_ > 0 ? DIM_ : 1), (DIM_ > 0 ? P_ : 2), RMAX_LIMIT, 0, true>,
                                                                      smem_per_warp<T, (DIM_ > 0 ? DIM_ : 1)>(), blocks, threads, st, a)
                                                     : cudaErrorInvalidValue));
            return e;
        }
        return cudaErrorInvalidValue;
    }
    // the wide strips copy points in 16-byte pieces: unaligned values run
    // the run-time-dimension kernels
    const bool vals16 = (((uintptr_t)a.vals_a | (uintptr_t)a.vals_b) & 15) == 0;
    if constexpr (sizeof(T) == 4) {
        if (vals16 && TWED_WIDE_DISPATCH(a.dim, a.p,
                               (e = launch_with_smem(pairs_kernel<T, 0, 2, wide_rmax<WD_>(), WD_>,
                                                     wide_bytes_per_warp<WD_>(), blocks, threads, st, a))))
            return e;
    }
    TWED_DISPATCH(a.dim, a.p, (e = launch_with_smem(pairs_kernel<T, DIM_, P_, RMAX_LIMIT>,
                                                    smem_per_warp<T, DIM_>(), blocks, threads, st, a)));
    return e;
}

template <typename T, int RMAX_LIMIT>
int pairs_blocks_per_sm_t(int dim, int p, int threads) {
    int nb = 0;
    if constexpr (sizeof(T) == 4) {
        if (TWED_WIDE_DISPATCH(dim, p, (nb = blocks_per_sm(pairs_kernel<T, 0, 2, wide_rmax<WD_>(), WD_>,
                                                           wide_bytes_per_warp<WD_>(), threads))))
            return nb;
    }
    TWED_DISPATCH(dim, p, (nb = blocks_per_sm(pairs_kernel<T, DIM_, P_, RMAX_LIMIT>,
                                              smem_per_warp<T, DIM_>(), threads)));
    return nb;
}

template <bool KH>
cudaError_t launch_band_kh(const CoopArgs<float>& a, int R, int blocks, int warps, cudaStream_t st) {
    cudaError_t e = cudaErrorNotSupported;
    const int threads = 32 * warps;
#define TWED_BAND_R(RR)                                                                           \
    TWED_DISPATCH(a.dim, a.p,                                                                     \
                  (e = (DIM_ > 0 ? launch_with_smem(band_kernel<(DIM_ > 0 ? DIM_ : 1), P_, RR, KH>, \
                                                    smem_per_warp<float, (DIM_ > 0 ? DIM_ : 1), KH>(), \
                                                    blocks, threads, st, a)                         \
                                 : cudaErrorNotSupported)))
    switch (R) {
        case 1: TWED_BAND_R(1); break;
        case 2: TWED_BAND_R(2); break;
        case 4: TWED_BAND_R(4); break;
        case 8: TWED_BAND_R(8); break;
        default: return cudaErrorInvalidValue;
    }
#undef TWED_BAND_R
    return e;
}

template <bool KH>
int band_blocks_per_sm_kh(int dim, int p, int R, int warps) {
    int nb = 0;
    const int threads = 32 * warps;
#define TWED_BAND_OCC(RR)                                                                         \
    TWED_DISPATCH(dim, p, (nb = (DIM_ > 0 ? blocks_per_sm(band_kernel<(DIM_ > 0 ? DIM_ : 1), P_, RR, KH>, \
                                                          smem_per_warp<float, (DIM_ > 0 ? DIM_ : 1), KH>(), \
                                                          threads)                              \
                                          : 0)))
    switch (R) {
        case 1: TWED_BAND_OCC(1); break;
        case 2: TWED_BAND_OCC(2); break;
        case 4: TWED_BAND_OCC(4); break;
        case 8: TWED_BAND_OCC(8); break;
        default: break;
    }
#undef TWED_BAND_OCC
    return nb;
}

template <typename T, bool KH>
cudaError_t launch_coop_kh(const CoopArgs<T>& a, int R, int blocks, int threads, cudaStream_t st) {
    cudaError_t e = cudaSuccess;
    switch (R) {
        case 1: TWED_DISPATCH(a.dim, a.p, (e = launch_with_smem(coop_kernel<T, DIM_, P_, 1, KH>, smem_per_warp<T, DIM_, KH>(), blocks, threads, st, a))); break;
        case 2: TWED_DISPATCH(a.dim, a.p, (e = launch_with_smem(coop_kernel<T, DIM_, P_, 2, KH>, smem_per_warp<T, DIM_, KH>(), blocks, threads, st, a))); break;
        case 4: TWED_DISPATCH(a.dim, a.p, (e = launch_with_smem(coop_kernel<T, DIM_, P_, 4, KH>, smem_per_warp<T, DIM_, KH>(), blocks, threads, st, a))); break;
        case 8: TWED_DISPATCH(a.dim, a.p, (e = launch_with_smem(coop_kernel<T, DIM_, P_, 8, KH>, smem_per_warp<T, DIM_, KH>(), blocks, threads, st, a))); break;
        default: return cudaErrorInvalidValue;
    }
    return e;
}

template <typename T, bool KH>
int coop_blocks_per_sm_kh(int dim, int p, int R, int threads) {
    int nb = 0;
    switch (R) {
        case 1: TWED_DISPATCH(dim, p, (nb = blocks_per_sm(coop_kernel<T, DIM_, P_, 1, KH>, smem_per_warp<T, DIM_, KH>(), threads))); break;
        case 2: TWED_DISPATCH(dim, p, (nb = blocks_per_sm(coop_kernel<T, DIM_, P_, 2, KH>, smem_per_warp<T, DIM_, KH>(), threads))); break;
        case 4: TWED_DISPATCH(dim, p, (nb = blocks_per_sm(coop_kernel<T, DIM_, P_, 4, KH>, smem_per_warp<T, DIM_, KH>(), threads))); break;
        case 8: TWED_DISPATCH(dim, p, (nb = blocks_per_sm(coop_kernel<T, DIM_, P_, 8, KH>, smem_per_warp<T, DIM_, KH>(), threads))); break;
        default: break;
    }
    return nb;
}

}  // namespace twed
