// Tensor-core cross term for 64-dimensional FP32 series (p = 2).
//
// For p = 2, d(a_i, b_j)^2 = |a_i|^2 + |b_j|^2 - 2 a_i . b_j, and the dot
// products of a block of rows of series a against a tile of columns of
// series b form a dense contraction with K = 64.  It runs on the
// 5th-generation tensor cores (tcgen05.mma, TF32 inputs, FP32 accumulation in
// tensor memory); the norms stay FP32, and the cell cost c(i,j) =
// sqrt(max(d^2, 0)) + nu |t_i - t'_j| is formed in FP32 before the wavefront
// consumes it.  The recurrence itself (paper, section "Time Warp Edit
// Distance", step 5) is the same as everywhere else in this library.
//
// Work item: one column series y and up to CH row series (consecutive in the
// longest-first order).  A block holds four consumer warps; warp q owns TMEM
// lane quadrant q, and in every "sweep" each consumer runs one strip of 64
// rows (2 per lane) of its current row series against all of y's columns.
// The four strips of a sweep share every B tile (y's points): the MMA of one
// 16-column tile is 2 x (128 x 16 x 64), A = the four strips' rows in TMEM
// (row 2L + r of warp q's strip on lane 32q + L of row tile r), written there
// by the consumers themselves with tcgen05.st at the start of the sweep.
// Roles:
//   warps 0..3  consumers: per 16-step block, tcgen05.ld of their own lanes'
//               accumulators of the next tile, cost formation for it
//               (packed f32x2 over adjacent columns) interleaved with the 16
//               wavefront steps of the current tile (lane L on column
//               s - L + 1 at step s), costs through a private skewed
//               shared-memory ring whose first 16 slots are mirrored past its
//               end so that a block's reads never wrap; the bottom rows of a
//               strip go to a per-warp boundary row in global memory (two
//               columns per store), read back by the warp's next strip of the
//               same series.
//   warp 4      TMA (cp.async.bulk.tensor) of the B tiles into a 4-stage
//               ring, as far ahead as the ring allows.
//   warp 5      tcgen05.mma issue and tcgen05.commit (to the consumers'
//               accumulator barrier and to the B stage's free barrier).
// The TMA and MMA warps wait in mbarrier.try_wait with a suspend-time hint,
// so they take no issue slots from the consumers while they wait.
// Columns past m get cost +inf and column delete cost 0, which freezes every
// row at its column-m value, so all lanes can run the same number of steps.
// Every wait is bounded (%globaltimer, then the launch's error word).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <utility>

#include "kernels.cuh"
#include "tc.cuh"

namespace twed {

namespace x64 {
constexpr int D = 64;            // point dimension (MMA K)
constexpr int RT = 2;            // row tiles per block = DP rows per lane
constexpr int N = 16;            // columns per consumer tile = wavefront steps per block
constexpr int NM = 16;           // columns per MMA tile (a B tile), a multiple of N
constexpr int HALVES = NM / N;   // consumer tiles per MMA tile
constexpr int NS = 64 / NM;      // accumulator stages in TMEM (NS x RT x NM = 128 columns)
constexpr int NBS = NS;          // B tile stages in shared memory
constexpr int CW = 4;            // consumer warps (one per TMEM lane quadrant)
constexpr int TMA_WARP = CW;     // B tile loads
constexpr int MMA_WARP = CW + 1; // tcgen05.mma issue
constexpr int THREADS = 32 * (CW + 2);
constexpr int STRIP = 32 * RT;   // rows per consumer strip
constexpr int CRING = 128;       // columns in a consumer's column-record ring (staged 32 at a time)
constexpr int RING = 64;         // columns in a consumer's cost ring
constexpr int RMIR = RING + N;   // ring slots incl. a mirror of slots 0..N-1 (no wrap inside a block)
constexpr int RS = 2 * (RMIR + 2); // floats per lane: 82 float2, == 2 mod 4 (conflict-free v2 reads, v4 writes)
constexpr int CH = 64;           // row series per work item
constexpr int TMEM_COLS = 256;
constexpr int ACC_COL = RT * D;  // accumulators follow the A tiles
constexpr int BOXES = D / 4;     // TMA boxes per B tile: 4 values x NM points each
constexpr uint32_t TILE_BYTES = NM * D * 4;
static_assert(NM % N == 0 && NS * RT * NM == 128, "accumulator layout");
constexpr int BND_PAD = 32;      // boundary rows start 32 entries in (lane 31 writes from column -30)

constexpr int OFF_B = 0;
constexpr int OFF_RING = OFF_B + NBS * (int)TILE_BYTES;
constexpr int RING_WARP = 32 * RS * 4;
constexpr int OFF_CTIME = OFF_RING + CW * RING_WARP;  // per warp: CRING column times t'
constexpr int OFF_CNORM = OFF_CTIME + CW * CRING * 4; // per warp: CRING column norms |b|^2
constexpr int DMIR = CRING + N;                       // column delete costs incl. a mirror of slots 0..N-1
constexpr int OFF_DELB = OFF_CNORM + CW * CRING * 4;  // per warp: DMIR column delete costs
constexpr int OFF_BND = OFF_DELB + CW * DMIR * 4;     // per warp: 64 staged (D, c) of the row above
constexpr int OFF_BAR = OFF_BND + CW * 64 * 8;
constexpr int NBAR = NBS + NBS + NS + NS + 1;         // b_full, b_empty, acc_full, acc_empty, a_ready
constexpr int OFF_SCHED = OFF_BAR + NBAR * 8;         // per warp: its copy of the strip schedule
constexpr int SCHED_BYTES = 128;
constexpr int OFF_MISC = OFF_SCHED + (CW + 2) * SCHED_BYTES;  // tmem base, item index
constexpr int SMEM = OFF_MISC + 64;
static_assert((OFF_RING % 16) == 0 && (RING_WARP % 16) == 0, "vector access alignment");
static_assert((OFF_SCHED % 8) == 0, "schedule alignment");
}  // namespace x64

// Point records for the tensor-core path: (t, delete cost, |x|^2, 0).
// With bf16, the norm is that of the point rounded to BF16 (the values the
// BF16 contraction multiplies), so that |a|^2 + |b|^2 - 2 a.b is exact for the
// rounded points up to FP32 summation.
__global__ void __launch_bounds__(256) xrecords_kernel(RecordsArgs<float> a, bool bf16) {
    using A = Arith<float>;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < a.total; g += stride) {
        int64_t lo = 0, hi = a.nseries;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (__ldg(a.offs + mid) <= g) lo = mid; else hi = mid;
        }
        const bool first = (__ldg(a.offs + lo) == g);
        const float* x = a.vals + g * x64::D;
        float s = 0.f, nrm = 0.f;
#pragma unroll 8
        for (int k = 0; k < x64::D; ++k) {
            const float xk = x[k];
            const float d = first ? xk : xk - x[k - x64::D];
            s = fmaf(d, d, s);
            const float xr = bf16 ? __uint_as_float(tc::pack_bf16x2(xk, 0.f) << 16) : xk;
            nrm = fmaf(xr, xr, nrm);
        }
        const float t = a.ts[g];
        const float tprev = first ? 0.f : a.ts[g - 1];
        float4 r;
        r.x = t;
        r.y = A::add(A::wcost(A::root(s), a.nu, t, tprev), a.lam);
        r.z = nrm;
        r.w = 0.f;
        reinterpret_cast<float4*>(a.rec)[g] = r;
    }
}

// Points of the column set rounded to BF16 for the B tiles of the BF16 mode,
// two per 32-bit word (the lower index in the low half).
__global__ void __launch_bounds__(256) bf16_copy_kernel(const float* src, uint32_t* dst, int64_t nwords) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < nwords; g += stride) {
        const float2 v = reinterpret_cast<const float2*>(src)[g];
        dst[g] = tc::pack_bf16x2(v.x, v.y);
    }
}

namespace {

// Bounded wait on an mbarrier phase: false (and the error word set) after
// sc.timeout_ns of %globaltimer, or as soon as another role has failed.
// Bounded waits on an mbarrier phase: false (and the error word set) after
// sc.timeout_ns of %globaltimer, or as soon as another role has failed.
// They poll with the non-blocking test_wait and back off with nanosleep in
// between (try_wait would wait inside the instruction, and a warp waiting
// there keeps taking issue slots from the consumers' wavefront).  Consumers'
// waits are rare and short (16 ns back-off); the TMA and MMA warps run
// ahead and wait most of the time (longer back-off).
__device__ __forceinline__ bool xwait_fail(const SyncCtl& sc, unsigned long long t0) {
    if (*(volatile unsigned*)sc.err != 0u) return true;
    if (globaltimer() - t0 > sc.timeout_ns) {
        atomicCAS(sc.err, 0u, 4u);
        atomicCAS(sc.sticky, 0u, 4u);
        return true;
    }
    return false;
}
__device__ __forceinline__ bool xwait_sleep(uint64_t* bar, uint32_t parity, const SyncCtl& sc,
                                            unsigned ns = 128) {
    if (tc::mbar_test_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    uint32_t k = 0;
    while (!tc::mbar_test_wait(bar, parity)) {
        __nanosleep(ns);
        if ((++k & 15u) == 0 && xwait_fail(sc, t0)) return false;
    }
    return true;
}
__device__ __forceinline__ bool xwait(uint64_t* bar, uint32_t parity, const SyncCtl& sc) {
    return xwait_sleep(bar, parity, sc, 16);
}


// Waits of the TMA and MMA warps, which run ahead and wait most of the time:
// try_wait with a suspend-time hint, so a waiting warp is descheduled until
// the phase completes (or the hint expires) instead of polling.
__device__ __forceinline__ bool xwait_prod(uint64_t* bar, uint32_t parity, const SyncCtl& sc) {
    if (tc::mbar_test_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    uint32_t k = 0;
    while (!tc::mbar_try_wait_sleep(bar, parity, 50000u))
        if ((++k & 7u) == 0 && xwait_fail(sc, t0)) return false;
    return true;
}

// Predicated 8-byte global store at p + OFF bytes (no branch around it).
template <int OFF>
__device__ __forceinline__ void st_global_pred(float2* p, float a, float b, int pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %3, 0;\n\t@q st.global.v2.f32 [%0+%4], {%1, %2};\n\t}" ::"l"(p),
                 "f"(a), "f"(b), "r"(pred), "n"(OFF)
                 : "memory");
}

// Predicated 16-byte global store of two (D, c) columns at p + OFF bytes.
template <int OFF>
__device__ __forceinline__ void st_global_pred4(float2* p, float a, float b, float c, float d, int pred) {
    asm volatile("{\n\t.reg .pred q;\n\tsetp.ne.b32 q, %5, 0;\n\t@q st.global.v4.f32 [%0+%6], {%1, %2, %3, %4};\n\t}" ::"l"(p),
                 "f"(a), "f"(b), "f"(c), "f"(d), "r"(pred), "n"(OFF)
                 : "memory");
}

// f(integral_constant<int, 0>) .. f(integral_constant<int, N-1>): a loop whose
// index is a constant expression in the body.
template <typename F, int... I>
__device__ __forceinline__ void unroll_seq(F&& f, std::integer_sequence<int, I...>) {
    (f(std::integral_constant<int, I>{}), ...);
}

// One work item: column series y, row series at sorted positions [r_lo, r_hi).
struct XItem {
    int64_t y, yb;
    int m;
    int64_t r_lo, r_hi;
};

__device__ __forceinline__ XItem decode_item(const XtermArgs& a, int64_t w) {
    XItem it;
    if (!a.symmetric) {
        const int64_t c = w / a.nb, q = w % a.nb;
        it.y = a.perm_b[q];
        it.r_lo = c * x64::CH;
        it.r_hi = min(it.r_lo + (int64_t)x64::CH, a.na);
    } else {
        // chunk c holds items chunk_start[c] .. chunk_start[c+1]-1; item p of
        // chunk c is column series p against rows max(p+1, c*CH) .. hi-1
        int64_t lo = 0, hi = a.nchunks;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (a.chunk_start[mid] <= w) lo = mid; else hi = mid;
        }
        const int64_t p = w - a.chunk_start[lo];
        it.y = a.perm_b[p];
        it.r_lo = max(p + 1, lo * (int64_t)x64::CH);
        it.r_hi = min((lo + 1) * (int64_t)x64::CH, a.na);
    }
    it.yb = a.offs_b[it.y];
    it.m = (int)(a.offs_b[it.y + 1] - it.yb);
    return it;
}

// Which strip each consumer runs in a sweep: a warp whose series is done
// takes the next row series of the item.  Every warp of the block runs the
// same bookkeeping, so they agree without communicating.
struct XSched {  // 72 bytes
    int64_t next;
    int64_t pos[x64::CW];  // sorted row position of each warp's series (-1: idle)
    int rem[x64::CW];      // strips left, the current one included
    int k[x64::CW];        // current strip index
};

static_assert(sizeof(XSched) <= 80, "the next-strip record follows the schedule at byte 80");

__device__ __forceinline__ int series_len(const XtermArgs& a, int64_t pos) {
    const int64_t x = a.perm_a[pos];
    return (int)(a.offs_a[x + 1] - a.offs_a[x]);
}

__device__ __forceinline__ void sched_init(XSched& s, const XItem& it) {
    s.next = it.r_lo;
#pragma unroll
    for (int w = 0; w < x64::CW; ++w) {
        s.pos[w] = -1;
        s.rem[w] = 0;
        s.k[w] = 0;
    }
}
// Assignments of the next sweep; false when the item is finished.
__device__ __forceinline__ bool sched_begin(XSched& s, const XtermArgs& a, const XItem& it) {
    bool any = false;
#pragma unroll
    for (int w = 0; w < x64::CW; ++w) {
        if (s.rem[w] == 0) {
            if (s.next < it.r_hi) {
                s.pos[w] = s.next++;
                s.rem[w] = (series_len(a, s.pos[w]) + x64::STRIP - 1) / x64::STRIP;
                s.k[w] = 0;
            } else {
                s.pos[w] = -1;
            }
        }
        any |= s.rem[w] > 0;
    }
    return any;
}
__device__ __forceinline__ void sched_end(XSched& s) {
#pragma unroll
    for (int w = 0; w < x64::CW; ++w) {
        if (s.rem[w] > 0) {
            --s.rem[w];
            ++s.k[w];
        }
    }
}

__device__ __forceinline__ void st_shared_v4(float* p, float a, float b, float c, float d) {
    *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}

}  // namespace

// BF = false: TF32 inputs (the FP32 values as the tensor core reads them);
// BF = true: BF16 inputs (A rounded by the consumers, B from a BF16 copy).
template <bool BF>
__global__ void __launch_bounds__(x64::THREADS, 2) xterm_sweep_kernel(const __grid_constant__ CUtensorMap tmap_b,
                                                                   XtermArgs a) {
    using namespace x64;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint64_t* b_full = bar;
    uint64_t* b_empty = bar + NBS;
    uint64_t* acc_full = bar + 2 * NBS;
    uint64_t* acc_empty = bar + 2 * NBS + NS;
    uint64_t* a_ready = bar + 2 * NBS + 2 * NS;
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile long long* item_sh = reinterpret_cast<volatile long long*>(misc + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float INF = __int_as_float(0x7f800000);

    if (threadIdx.x == 0) {
        for (int i = 0; i < NBS; ++i) {
            tc::mbar_init(&b_full[i], 1);
            tc::mbar_init(&b_empty[i], 1);
        }
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&acc_full[i], 1);
            tc::mbar_init(&acc_empty[i], CW);
        }
        tc::mbar_init(a_ready, CW);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) tc::tmem_alloc(misc, TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = misc[0];
    const uint32_t idesc = BF ? tc::idesc_bf16(128, NM) : tc::idesc_tf32(128, NM);
    // B tile: BOXES_T boxes of 16 bytes x NM points (4 TF32 or 8 BF16 values
    // of K each); A: K along TMEM columns, one TF32 or two BF16 values each
    constexpr int BOXES_T = BF ? BOXES / 2 : BOXES;
    constexpr uint32_t TILE_BYTES_T = BF ? TILE_BYTES / 2 : TILE_BYTES;
    constexpr int KSTEPS = BF ? D / 16 : D / 8;  // MMAs per row tile
    constexpr int ACOLS = BF ? D / 2 : D;        // TMEM columns of one row tile of A
    // the TMA destinations need a 1024-byte aligned shared window
    const bool aligned = (tc::smem_u32(sm) & 1023u) == 0;

    // running counters, identical in every role
    uint32_t Lp = 0;               // TMA warp: B tiles loaded
    uint32_t Tp = 0, sweep_p = 0;  // MMA warp: tiles issued, sweeps
    uint32_t Tc = 0;               // consumers: accumulator tiles read
    bool ok = aligned;
    if (!aligned && threadIdx.x == 0) {
        atomicCAS(a.sc.err, 0u, 5u);
        atomicCAS(a.sc.sticky, 0u, 5u);
    }
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const bool failed = *(volatile unsigned*)a.sc.err != 0u;
            *item_sh = failed ? a.nitems : (long long)atomicAdd(a.counter, 1ull);
        }
        __syncthreads();
        const long long w = *item_sh;  // block-uniform
        if (w >= a.nitems || !ok) break;
        const XItem it = decode_item(a, w);
        const int m = it.m;
        const int ntiles = (m + N - 1) / N;     // consumer tiles (16 columns)
        const int ntilesM = (m + NM - 1) / NM;  // MMA / B tiles
        // each warp keeps its copy of the schedule in shared memory (every lane
        // computes the same values)
        XSched& sch = *reinterpret_cast<XSched*>(sm + OFF_SCHED + warp * SCHED_BYTES);
        sched_init(sch, it);
        __syncwarp();

        if (warp >= CW) {
            uint32_t total = 0;
            {
                uint32_t nsw = 0;
                while (sched_begin(sch, a, it)) {
                    ++nsw;
                    sched_end(sch);
                }
                total = nsw * (uint32_t)ntilesM;
            }
            if (warp == TMA_WARP) {
                // ======================= B tiles by TMA, up to NBS ahead of the MMA
                for (uint32_t idx = 0; idx < total; ++idx) {
                    const int st = (int)(Lp % NBS);
                    bool w2 = true;
                    if (Lp >= NBS) w2 = xwait_prod(&b_empty[st], ((Lp / NBS) - 1) & 1, a.sc);
                    if (!__all_sync(kFull, w2)) { ok = false; break; }
                    const int t = (int)(idx % (uint32_t)ntilesM);
                    unsigned char* dst = sm + OFF_B + st * TILE_BYTES;
                    if (lane == 0) tc::mbar_arrive_expect_tx(&b_full[st], TILE_BYTES_T);
                    __syncwarp();
                    if (lane < BOXES_T)
                        tc::tma_load_2d(dst + lane * (NM * 16), &tmap_b, (BF ? 8 : 4) * lane,
                                        (int)(it.yb + (int64_t)NM * t), &b_full[st]);
                    __syncwarp();
                    ++Lp;
                }
            } else {
                // ======================= MMA issue
                for (uint32_t idx = 0; idx < total; ++idx) {
                    const int st = (int)(Tp % NBS), s = (int)(Tp % NS);
                    const int t = (int)(idx % (uint32_t)ntilesM);
                    bool w2 = xwait_prod(&b_full[st], (Tp / NBS) & 1, a.sc);
                    if (w2 && t == 0) w2 = xwait_prod(a_ready, sweep_p & 1, a.sc);
                    if (w2 && Tp >= NS) w2 = xwait_prod(&acc_empty[s], ((Tp / NS) - 1) & 1, a.sc);
                    if (!__all_sync(kFull, w2)) { ok = false; break; }
                    tc::fence_after_sync();
                    // the stage's B descriptor and the accumulator base, warp-uniform;
                    // K step ks starts ks * 2 * NM * 16 bytes on (the descriptor's
                    // address field counts 16-byte units and cannot carry: shared
                    // addresses stay below 2^18)
                    const uint64_t bd0 = tc::smem_desc(tc::smem_u32(sm + OFF_B + st * TILE_BYTES), NM * 16, 128);
                    const uint32_t dt0 = tmem + (uint32_t)(ACC_COL + s * (RT * NM));
                    if (lane == 0) {
#pragma unroll
                        for (int r = 0; r < RT; ++r) {
#pragma unroll
                            for (int ks = 0; ks < KSTEPS; ++ks) {
                                // K step ks covers k-groups 2ks, 2ks+1 (boxes NM * 16 bytes apart);
                                // each further 8 points of the tile sit 128 bytes on
                                const uint64_t bd = bd0 + (uint64_t)((ks * 2 * NM * 16) >> 4);
                                const uint32_t dt = dt0 + (uint32_t)(r * NM);
                                const uint32_t at = tmem + (uint32_t)(r * ACOLS + ks * 8);
                                if constexpr (BF) tc::mma_bf16_tmem_a(dt, at, bd, idesc, ks > 0);
                                else tc::mma_tf32_tmem_a(dt, at, bd, idesc, ks > 0);
                            }
                        }
                        tc::mma_commit(&acc_full[s]);
                        tc::mma_commit(&b_empty[st]);
                    }
                    __syncwarp();
                    ++Tp;
                    if (t == ntilesM - 1) ++sweep_p;
                }
            }
        } else {
            const int q = warp;
            const uint32_t tlane = (uint32_t)(32 * q) << 16;
            float* ring = reinterpret_cast<float*>(sm + OFF_RING + q * RING_WARP);
            float* myring = ring + lane * RS;
            float* ctime = reinterpret_cast<float*>(sm + OFF_CTIME) + q * CRING;
            float* cnorm = reinterpret_cast<float*>(sm + OFF_CNORM) + q * CRING;
            float* delb_r = reinterpret_cast<float*>(sm + OFF_DELB) + q * DMIR;
            float2* bnd_r = reinterpret_cast<float2*>(sm + OFF_BND) + q * 64;
            float2* bnd_g = a.bnd + (int64_t)(blockIdx.x * CW + q) * a.bnd_stride + BND_PAD;
            const float4* rec_y = a.rec_b + it.yb;
            const float nu = a.nu;
            // the strip this warp runs in a sweep, from its copy of the schedule
            struct Strip {
                int64_t x, xa;
                int n, r0, i0, i1;
                bool idle, first, last;
            };
            auto strip_of = [&]() -> Strip {
                int64_t pos = -1;
                int kq = 0, remq = 0;
#pragma unroll
                for (int w = 0; w < CW; ++w) {
                    if (w == q) {
                        pos = sch.pos[w];
                        kq = sch.k[w];
                        remq = sch.rem[w];
                    }
                }
                Strip S;
                S.idle = pos < 0;
                S.x = a.perm_a[S.idle ? it.r_lo : pos];
                S.xa = a.offs_a[S.x];
                S.n = (int)(a.offs_a[S.x + 1] - S.xa);
                S.r0 = STRIP * kq + 1;
                S.first = S.idle || kq == 0;
                S.last = !S.idle && remq == 1;
                S.i0 = min(S.r0 + 2 * lane, S.n);
                S.i1 = min(S.r0 + 2 * lane + 1, S.n);
                return S;
            };
            // this lane's point row r (0, 1) of a strip
            auto a_src = [&](const Strip& S, int r) -> const float4* {
                return reinterpret_cast<const float4*>(a.vals_a + (S.xa + (r ? S.i1 : S.i0) - 1) * D);
            };
            auto write_a = [&](const Strip& S) {
                if (!S.idle) {
#pragma unroll
                    for (int r = 0; r < RT; ++r) {
                        const float4* src = a_src(S, r);
                        if constexpr (BF) {
                            // 64 values rounded to BF16, two per column
                            float v[32];
#pragma unroll
                            for (int u = 0; u < 16; ++u) {
                                const float4 f = __ldg(src + u);
                                v[2 * u] = __uint_as_float(tc::pack_bf16x2(f.x, f.y));
                                v[2 * u + 1] = __uint_as_float(tc::pack_bf16x2(f.z, f.w));
                            }
                            tc::tmem_st32(tmem + tlane + (uint32_t)(r * ACOLS), v);
                        } else {
#pragma unroll
                            for (int h = 0; h < 2; ++h) {
                                float v[32];
#pragma unroll
                                for (int u = 0; u < 8; ++u) {
                                    const float4 f = __ldg(src + h * 8 + u);
                                    v[4 * u] = f.x;
                                    v[4 * u + 1] = f.y;
                                    v[4 * u + 2] = f.z;
                                    v[4 * u + 3] = f.w;
                                }
                                tc::tmem_st32(tmem + tlane + (uint32_t)(r * D + 32 * h), v);
                            }
                        }
                    }
                    tc::tmem_wait_st();
                }
                tc::fence_before_sync();
                __syncwarp();
                if (lane == 0) tc::mbar_arrive(a_ready);
            };
            bool more = sched_begin(sch, a, it);
            while (ok && more) {
                const Strip cur = strip_of();  // the schedule holds this sweep's assignment
                // ---- this strip's rows into the A tiles (every MMA of the previous
                // sweep has completed: this warp read all of its accumulators)
                write_a(cur);
                const int64_t x = cur.x;
                const int n = cur.n;
                const int r0 = cur.r0;
                const bool first = cur.first, last = cur.last;
                const float4 ra0 = __ldg(a.rec_a + cur.xa + cur.i0 - 1);
                const float4 ra1 = __ldg(a.rec_a + cur.xa + cur.i1 - 1);
                // the next sweep's strip, decided now: its rows go into the A tiles
                // during this sweep's last blocks, once every MMA of this sweep has
                // completed, so that the MMA warp can start the next sweep early
                sched_end(sch);
                more = sched_begin(sch, a, it);
                if (more) {
                    const Strip nx = strip_of();
                    if (!nx.idle) {
#pragma unroll
                        for (int r = 0; r < RT; ++r) {
                            tc::prefetch_l2(a_src(nx, r));
                            tc::prefetch_l2(a_src(nx, r) + 8);
                        }
                    }
                }
                // the TMA warp keeps the B loads four tiles ahead of its own use; the
                // MMA warp, once every warp's rows are in, issues tiles 0..2

                // ---- rings.  Cost ring: columns <= 0 cost +inf (slots 32..63).  Column
                // delete costs: 0 for columns <= 0 (slots 96..127).
#pragma unroll
                for (int u = 0; u < RING / 2; u += 2) st_shared_v4(myring + 2 * (RING / 2 + u), INF, INF, INF, INF);
                delb_r[CRING - 32 + lane] = 0.f;
                // column record of column j (1-based) of y: (t', dB, |b|^2, 0); past m the
                // norm is +inf (cost +inf) and the delete cost 0, which freezes the rows
                // (loaded raw; the selects are applied when the value is stored, so
                // that no instruction waits for the load before then)
                auto colrec_ld = [&](int j) -> float4 { return __ldg(rec_y + (min(j, m) - 1)); };  // j >= 1
                auto colrec_fix = [&](float4 v, int j) -> float4 {
                    const bool in = j <= m;
                    v.x = in ? v.x : 0.f;
                    v.y = in ? v.y : 0.f;
                    v.z = in ? v.z : INF;
                    return v;
                };
                // the row above the strip at column j (1-based): (inf, 0) above a
                // series' first strip and past m
                auto rowabove_ld = [&](int j) -> float2 { return __ldcg(bnd_g + min(j, m)); };
                auto rowabove_fix = [&](float2 v, int j) -> float2 {
                    return (first || j > m) ? make_float2(INF, 0.f) : v;
                };
                // tile 0's records (lanes 16..31 write the same values again), then the
                // staged inputs of the first two blocks: records of tiles 1 and 2, the
                // row above for steps 0..31
                {
                    const float4 c0 = colrec_fix(colrec_ld((lane & (N - 1)) + 1), (lane & (N - 1)) + 1);
                    ctime[lane & (N - 1)] = c0.x;
                    cnorm[lane & (N - 1)] = c0.z;
                    delb_r[lane & (N - 1)] = c0.y;
                    delb_r[CRING + (lane & (N - 1))] = c0.y;  // mirror
                }
                float4 cr_st = colrec_ld(N + 1 + lane);
                float2 bd_st = rowabove_ld(1 + lane);
                __syncwarp();
                // ---- costs of tile 0
                const float na0 = ra0.z, na1 = ra1.z, ti0 = ra0.x, ti1 = ra1.x;
                const float rdel0 = ra0.y, rdel1 = ra1.y;
                float X0[N], X1[N];
                {
                    const int s = (int)(Tc % NS);
                    const bool w2 = xwait(&acc_full[s], (Tc / NS) & 1, a.sc);
                    if (!__all_sync(kFull, w2)) { ok = false; break; }
                    tc::fence_after_sync();
                    tc::tmem_ld16x2(tmem + tlane + (uint32_t)(ACC_COL + s * (RT * NM)),
                                    tmem + tlane + (uint32_t)(ACC_COL + s * (RT * NM) + NM), X0, X1);
                    tc::fence_before_sync();
                    __syncwarp();
                    // the stage is released after its last consumer tile has been read
                    if (HALVES == 1 || ntiles == 1) {
                        if (lane == 0) tc::mbar_arrive(&acc_empty[s]);
                        ++Tc;
                    }
                }
                // c(i, j) = sqrt(|d^2|) + nu |t_i - t'_j| with d^2 = |a_i|^2 + |b_j|^2 - 2 X.
                // d^2 < 0 only through cancellation when the true d^2 is within
                // rounding of 0; |d^2| then stays within that rounding of the
                // truth, like max(d^2, 0) would.  d^2 and t_i - t'_j are formed for
                // two adjacent columns at once (packed f32x2).
                const unsigned long long na0p = f2_pack(na0, na0), na1p = f2_pack(na1, na1);
                const unsigned long long ti0p = f2_pack(ti0, ti0), ti1p = f2_pack(ti1, ti1);
                const unsigned long long m2p = f2_pack(-2.f, -2.f);
                auto cost2 = [&](unsigned long long x2, unsigned long long nap, unsigned long long nb2,
                                 unsigned long long tip, unsigned long long tj2, float& e_lo, float& e_hi) {
                    const unsigned long long d2 = f2_fma(x2, m2p, f2_add(nap, nb2));
                    const unsigned long long dt = f2_sub(tip, tj2);
                    float s0, s1, t0, t1;
                    f2_unpack(d2, s0, s1);
                    f2_unpack(dt, t0, t1);
                    e_lo = fmaf(nu, fabsf(t0), Arith<float>::root(fabsf(s0)));
                    e_hi = fmaf(nu, fabsf(t1), Arith<float>::root(fabsf(s1)));
                };
                // the costs of 4 columns (u0 .. u0+3 of a tile) into the cost ring at
                // `dst`, and also at `dst` + the mirror offset when `mirror`
                auto cost4 = [&](int u0, const float4& tj, const float4& nb, float* dst, bool mirror) {
                    const unsigned long long nb01 = f2_pack(nb.x, nb.y), nb23 = f2_pack(nb.z, nb.w);
                    const unsigned long long tj01 = f2_pack(tj.x, tj.y), tj23 = f2_pack(tj.z, tj.w);
                    float e0, e1, e2, e3, e4, e5, e6, e7;
                    cost2(f2_pack(X0[u0], X0[u0 + 1]), na0p, nb01, ti0p, tj01, e0, e2);
                    cost2(f2_pack(X1[u0], X1[u0 + 1]), na1p, nb01, ti1p, tj01, e1, e3);
                    cost2(f2_pack(X0[u0 + 2], X0[u0 + 3]), na0p, nb23, ti0p, tj23, e4, e6);
                    cost2(f2_pack(X1[u0 + 2], X1[u0 + 3]), na1p, nb23, ti1p, tj23, e5, e7);
                    st_shared_v4(dst, e0, e1, e2, e3);
                    st_shared_v4(dst + 4, e4, e5, e6, e7);
                    if (mirror) {
                        st_shared_v4(dst + 2 * RING, e0, e1, e2, e3);
                        st_shared_v4(dst + 2 * RING + 4, e4, e5, e6, e7);
                    }
                };
#pragma unroll
                for (int u = 0; u < N; u += 4)  // tile 0 sits in slots 0..N-1: mirrored
                    cost4(u, *reinterpret_cast<const float4*>(ctime + u), *reinterpret_cast<const float4*>(cnorm + u),
                          myring + 2 * u, true);
                __syncwarp();

                // ---- the wavefront: lane L on column s - L + 1 at step s
                float Dl0 = INF, Dl1 = INF, cp0 = 0.f;
                float diagD = (r0 == 1 && lane == 0) ? 0.f : INF, diagC = 0.f;
                float botD = INF, botC = 0.f;
                const int nblk = (m + 31 + N - 1) / N;
                const int is31 = lane == 31;
                for (int b = 0; b < nblk; ++b) {
                    const int sb = N * b;
                    if (b > 0 && (sb & (RING - 1)) == 0) {
                        // this block and the next read the cost-ring slots 0..N-1 (written
                        // in the previous block) past the ring's end: mirror them there
                        const float4* from = reinterpret_cast<const float4*>(myring);
                        float4* to = reinterpret_cast<float4*>(myring + 2 * RING);
#pragma unroll
                        for (int k = 0; k < N / 2; ++k) to[k] = from[k];
                    }
                    if ((b & 1) == 0) {
                        // every 32 steps, all lanes: the staged records of tiles b+1,
                        // b+2 (columns 16b+17 ..) and the row above for steps sb ..
                        // sb+31 go to shared memory; then those of the next 32 steps
                        // are loaded (used 32 steps later)
                        const int slot = (N * (b + 1) + lane) & (CRING - 1);
                        const float4 cr = colrec_fix(cr_st, N * (b + 1) + 1 + lane);
                        ctime[slot] = cr.x;
                        cnorm[slot] = cr.z;
                        delb_r[slot] = cr.y;
                        if (slot < N) delb_r[CRING + slot] = cr.y;  // mirror
                        bnd_r[(sb + lane) & 63] = rowabove_fix(bd_st, sb + 1 + lane);
                        __syncwarp();
                        cr_st = colrec_ld(N * (b + 3) + 1 + lane);
                        bd_st = rowabove_ld(sb + 32 + 1 + lane);
                    }
                    // accumulators of tile b+1: the load is issued here and waited for
                    // three steps later, just before the costs first use them
                    // (consumer tile b+1 is part h of MMA tile (b+1) / HALVES: only its
                    // first part waits for the MMA, its last part releases the stage)
                    const bool xload = b + 1 < ntiles;
                    const int xs = (int)(Tc % NS);
                    const int xh = (b + 1) % HALVES;
                    const bool xrel = xload && (xh == HALVES - 1 || b + 2 == ntiles);
                    if (xload) {
                        if (xh == 0) {
                            const bool w2 = xwait(&acc_full[xs], (Tc / NS) & 1, a.sc);
                            if (!__all_sync(kFull, w2)) { ok = false; break; }
                        }
                        tc::fence_after_sync();
                        tc::tmem_ld16x2_async(tmem + tlane + (uint32_t)(ACC_COL + xs * (RT * NM) + xh * N),
                                              tmem + tlane + (uint32_t)(ACC_COL + xs * (RT * NM) + NM + xh * N), X0,
                                              X1);
                        if (xrel) ++Tc;
                    }
                    const int cslot = (N * (b + 1)) & (RING - 1);  // cost-ring slot of tile b+1's first column
                    const int rslot = (N * (b + 1)) & (CRING - 1);  // record-ring slot of the same column
                    float* cst = myring + 2 * cslot;
                    // lane 31's bottom row at column s - 30 (the other lanes' addresses are
                    // never stored to)
                    float2* bst = bnd_g + (sb - 30) + (lane - 31);
                    // this block's reads: slot (s - L) mod the ring for s = sb .. sb+15,
                    // which the mirrors keep contiguous from the block's first slot
                    const float2* rp = reinterpret_cast<const float2*>(myring) + ((sb - lane) & (RING - 1));
                    const float* dp = delb_r + ((sb - lane) & (CRING - 1));
                    const float2* bp = bnd_r + (sb & 63);
                    float2 cn = rp[0];
                    float dbn = dp[0];
                    float2 bn = bp[0];
                    float pD = 0.f, pC = 0.f;  // lane 31's bottom row at the previous (even) step
                    {
                      unroll_seq(
                        [&](auto UC) {
                            constexpr int u = decltype(UC)::value;
                            const float c0 = cn.x, c1 = cn.y, delb = dbn;
                            const float2 bnd = bn;
                            if constexpr (u + 1 < N) {
                                cn = rp[u + 1];
                                dbn = dp[u + 1];
                                bn = bp[u + 1];
                            }
                            float upD = __shfl_up_sync(kFull, botD, 1);
                            float upC = __shfl_up_sync(kFull, botC, 1);
                            upD = lane == 0 ? bnd.x : upD;
                            upC = lane == 0 ? bnd.y : upC;
                            const float tb0 = Dl0 + delb, tm0 = (diagD + c0) + diagC;
                            const float tb1 = Dl1 + delb, tm1 = (Dl0 + c1) + cp0;
                            const float D0 = min3f(upD + rdel0, tb0, tm0);
                            const float D1 = min3f(D0 + rdel1, tb1, tm1);
                            diagD = upD;
                            diagC = upC;
                            cp0 = c0;
                            Dl0 = D0;
                            Dl1 = D1;
                            botD = D1;
                            botC = c1;
                            // lane 31's bottom row, two columns per store: columns
                            // sb - 31 + u (even) and sb - 30 + u at odd u
                            if constexpr ((u & 1) == 0) {
                                pD = D1;
                                pC = c1;
                            } else {
                                st_global_pred4<8 * (u - 1)>(bst, pD, pC, D1, c1, is31);
                            }
                            if constexpr (u == 2) {
                                // the accumulators have landed: release the stage
                                if (xload) {
                                    tc::tmem_wait_ld_tied(X0, X1);
                                    if (xrel) {
                                        tc::fence_before_sync();
                                        __syncwarp();
                                        if (lane == 0) tc::mbar_arrive(&acc_empty[xs]);
                                    }
                                }
                            }
                            // costs of tile b+1, 4 columns every 4 steps (not read in this
                            // block; slots 0..N-1 are mirrored at the start of the next block)
                            if constexpr ((u & 3) == 3)
                                cost4(u - 3, *reinterpret_cast<const float4*>(ctime + rslot + u - 3),
                                      *reinterpret_cast<const float4*>(cnorm + rslot + u - 3), cst + 2 * (u - 3), false);
                        },
                        std::make_integer_sequence<int, N>{});
                    }

                    __syncwarp();
                }
                if (!ok) break;
                // every lane ran past column m with frozen rows: Dl = D(row, m)
                if (last) {
                    const int rr = n - r0;  // 0 .. 63
                    if (lane == (rr >> 1)) {
                        const float v = (rr & 1) ? Dl1 : Dl0;
                        if (!a.symmetric) {
                            a.out[x * a.nb + it.y] = v;
                        } else {
                            a.out[x * a.na + it.y] = v;
                            a.out[it.y * a.na + x] = v;
                        }
                    }
                }
            }
        }
        if (!ok && lane == 0) {
            atomicCAS(a.sc.err, 0u, 4u);
            atomicCAS(a.sc.sticky, 0u, 4u);
        }
    }
    // drain (bounded): B loads and MMAs in flight must land before the shared
    // memory and the TMEM are released.  Only the last NBS loads (one per
    // stage) and the last MMA group can still be pending.
    if (warp == TMA_WARP) {
        const unsigned long long t0 = globaltimer();
        for (long long l = (Lp > NBS ? Lp - NBS : 0); l < Lp; ++l)
            while (!tc::mbar_try_wait(&b_full[l % NBS], (uint32_t)((l / NBS) & 1)) &&
                   globaltimer() - t0 < a.sc.timeout_ns) {
            }
    }
    if (warp == MMA_WARP && Tp > 0) {
        const unsigned long long t0 = globaltimer();
        while (!tc::mbar_try_wait(&acc_full[(Tp - 1) % NS], (uint32_t)(((Tp - 1) / NS) & 1)) &&
               globaltimer() - t0 < a.sc.timeout_ns) {
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

cudaError_t launch_xrecords(const RecordsArgs<float>& a, cudaStream_t st, bool bf16) {
    if (a.total <= 0) return cudaSuccess;
    int64_t blocks = (a.total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    (void)cudaGetLastError();
    xrecords_kernel<<<(int)blocks, 256, 0, st>>>(a, bf16);
    return cudaGetLastError();
}

cudaError_t launch_bf16_copy(const float* src, void* dst, int64_t nvals, cudaStream_t st) {
    if (nvals <= 0) return cudaSuccess;
    const int64_t nwords = nvals / 2;  // nvals is a multiple of 64
    int64_t blocks = (nwords + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    (void)cudaGetLastError();
    bf16_copy_kernel<<<(int)blocks, 256, 0, st>>>(src, (uint32_t*)dst, nwords);
    return cudaGetLastError();
}

template <bool BF>
static cudaError_t xterm_attributes_t() {
    cudaError_t e =
        cudaFuncSetAttribute(xterm_sweep_kernel<BF>, cudaFuncAttributeMaxDynamicSharedMemorySize, x64::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xterm_sweep_kernel<BF>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}
static cudaError_t xterm_attributes() {
    cudaError_t e = xterm_attributes_t<false>();
    return e == cudaSuccess ? xterm_attributes_t<true>() : e;
}

// Tensor map of a set's 64-dimensional values for the B tiles: [total][64]
// FP32, rows 256 bytes apart; a box is 4 values (16 bytes) of NM points, so
// one tile is 16 boxes at x = 0, 4, .., 60.  With bf16, the values are the
// set's BF16 copy, rows 128 bytes apart, a box 8 values (16 bytes), 8 boxes
// per tile at x = 0, 8, .., 56.  Points past the end read 0.
cudaError_t xterm_tensor_map(void* tmap, const void* vals, int64_t total, bool bf16) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        cudaDriverEntryPointQueryResult q;
        void* fn = nullptr;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)x64::D, (cuuint64_t)total};
    const cuuint64_t strides[1] = {(cuuint64_t)x64::D * (bf16 ? 2 : 4)};
    const cuuint32_t box[2] = {bf16 ? 8u : 4u, (cuuint32_t)x64::NM};
    const cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(tmap),
                        bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                        const_cast<void*>(vals), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_xterm(const void* tmap, const XtermArgs& a, int blocks, cudaStream_t st, bool bf16) {
    if (a.nitems <= 0) return cudaSuccess;
    cudaError_t e = xterm_attributes();
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    const CUtensorMap& tm = *reinterpret_cast<const CUtensorMap*>(tmap);
    if (bf16) xterm_sweep_kernel<true><<<blocks, x64::THREADS, x64::SMEM, st>>>(tm, a);
    else xterm_sweep_kernel<false><<<blocks, x64::THREADS, x64::SMEM, st>>>(tm, a);
    return cudaGetLastError();
}

int xterm_blocks_per_sm() {
    cudaError_t e = xterm_attributes();
    int nb = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, xterm_sweep_kernel<false>, x64::THREADS, x64::SMEM);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return -(int)e;  // negative: the CUDA error code, for diagnostics
    }
    return nb;
}

// Blocks per SM allowed by shared memory (1 KB reserved per block), tensor
// memory columns and registers.
int xterm_resident_blocks() {
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0;
    if (xterm_attributes() != cudaSuccess || cudaFuncGetAttributes(&fa, xterm_sweep_kernel<false>) != cudaSuccess ||
        cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev) != cudaSuccess) {
        (void)cudaGetLastError();
        return 1;
    }
    const int by_smem = smem_sm / (x64::SMEM + (int)fa.sharedSizeBytes + 1024);
    const int regs_warp = ((fa.numRegs * 32 + 255) / 256) * 256;
    const int by_regs = regs_sm / (regs_warp * (x64::THREADS / 32));
    const int by_tmem = 512 / x64::TMEM_COLS;
    int nb = by_smem < by_regs ? by_smem : by_regs;
    nb = nb < by_tmem ? nb : by_tmem;
    return nb > 0 ? nb : 1;
}

// "regs R static S dyn D smem/SM X": what bounds the blocks per SM.
void xterm_resources(char* buf, int len) {
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, smem_blk = 0;
    (void)xterm_attributes();
    cudaFuncGetAttributes(&fa, xterm_sweep_kernel<false>);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    (void)cudaGetLastError();
    snprintf(buf, len, "regs %d static %zu dyn %d max_dyn %d smem/SM %d smem/block %d", fa.numRegs,
             fa.sharedSizeBytes, x64::SMEM, fa.maxDynamicSharedSizeBytes, smem_sm, smem_blk);
}

int xterm_rows_per_item() { return x64::CH; }
int xterm_warps_per_block() { return x64::CW; }
int xterm_threads() { return x64::THREADS; }
// even, so that every boundary row starts on a 16-byte boundary (pairs of
// columns are stored as one 16-byte vector)
int64_t xterm_bnd_stride(int64_t max_len) { return (max_len + 64 + x64::BND_PAD + 1) & ~(int64_t)1; }

}  // namespace twed
