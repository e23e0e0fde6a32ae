// Short pairs with wide points: both series at most 32 points, p = 2, dims
// 16, 28 and 64 in FP32 and 16 and 28 in FP64 (the paper's MNIST shape,
// section "Experiments": 28 rows of 28 pixels per image).
//
// The strip engines form a cell's cost when the wavefront reaches it.  A
// 28 x 28 pair then keeps its warp in the 31-step fill and drain of the
// wavefront for most of its 59 steps, and every idle lane also sits out the
// O(dim) distance, which is nearly all of a cell's work at these widths.
// Here a warp takes one pair at a time in two phases:
//
//  1. costs: lane i holds point a_{i+1} in registers and forms
//     c(i+1, j+1) = |a_{i+1} - b_{j+1}| + nu |t_{i+1} - t'_{j+1}| for every
//     column j, reading b_{j+1} from shared memory (the same address for all
//     lanes: one broadcast per 16 bytes), into a column-major cost tile;
//  2. the recurrence (Eq. 2 with the deletion and match costs of the
//     paper's definition of TWED): the anti-diagonal wavefront of the strip
//     engines, lane i on column s - i at step s with D and c handed down by
//     shuffle, now one cost load and one delete-cost load per cell.
//
// Every lane is busy in phase 1 (lanes past the pair's rows repeat its last
// row), so the fill and drain of phase 2 cost a few additions per step.
// While a pair runs, the next pair's column points and (t', delete cost)
// records are copied into the other half of a double-buffered per-warp
// stage by cp.async, and each lane loads its next row point and record into
// registers.  Warps take pairs from the launch's counter kShortGrab at a time.
//
// Cost tile layout: column j (0-based) of the pair at tile[j * 32 + i] for
// row i.  At step s lane i reads entry (s - i, i) when 0 <= s - i < m and
// otherwise takes cost +inf and delete cost 0: a lane before its first
// column then computes +inf, and a lane past its last column keeps D(i, m)
// (its own value plus a zero delete cost is the least candidate, since
// D(i, m) <= D(i-1, m) + dA(i) by the recurrence).  The lanes of one load
// read one tile row each, so the bank of a lane's address is its lane number
// and no load conflicts.
//
// Arithmetic per cell follows the strip engines (engine.cuh): FP64 sums the
// squared differences in component order with separately rounded products
// and sums, so it reproduces the sequential evaluation bit for bit; FP32 sums
// component pairs in packed f32x2 with two partial sums, within the FP32
// tolerance.
#pragma once

#include "engine_f32.cuh"

namespace twed {

constexpr int kShortMax = 32;   // longest series this kernel takes
constexpr int kShortWarps = 2;  // warps per block
constexpr int kShortGrab = 8;   // pairs a warp takes from the counter at once

// Shared memory of one warp (bytes): two stages (the column series' points
// and records), the cost tile and its delete-cost row.
template <typename T, int DIM>
struct ShortSmem {
    static constexpr int kPts = kShortMax * DIM * (int)sizeof(T);  // one series' points
    static constexpr int kRecs = kShortMax * 16;                   // its 16-byte records
    static constexpr int kStage = kPts + kRecs;
    static constexpr int kCost = kShortMax * kShortMax * (int)sizeof(T);
    static constexpr int kDelb = kShortMax * (int)sizeof(T);
    static constexpr int kWarp = 2 * kStage + kCost + kDelb;
};

__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// A lane's row point and its (t, delete cost) in registers.  FP32 keeps the
// point as component pairs (a_2k, a_2k+1), the operands of f32x2 arithmetic.
template <typename T, int DIM>
struct ShortRow;
template <int DIM>
struct ShortRow<float, DIM> {
    static_assert(DIM % 4 == 0, "points come in 16-byte pieces");
    unsigned long long v[DIM / 2];
    float t, del;
    __device__ __forceinline__ void load(const float* pt, const float* rec) {
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(pt);
#pragma unroll
        for (int q = 0; q < DIM / 4; ++q) {
            const ulonglong2 x = __ldg(p + q);
            v[2 * q] = x.x;
            v[2 * q + 1] = x.y;
        }
        const float2 r = __ldg(reinterpret_cast<const float2*>(rec));
        t = r.x;
        del = r.y;
    }
};
template <int DIM>
struct ShortRow<double, DIM> {
    static_assert(DIM % 2 == 0, "points come in 16-byte pieces");
    double v[DIM];
    double t, del;
    __device__ __forceinline__ void load(const double* pt, const double* rec) {
        const double2* p = reinterpret_cast<const double2*>(pt);
#pragma unroll
        for (int q = 0; q < DIM / 2; ++q) {
            const double2 x = __ldg(p + q);
            v[2 * q] = x.x;
            v[2 * q + 1] = x.y;
        }
        const double2 r = __ldg(reinterpret_cast<const double2*>(rec));
        t = r.x;
        del = r.y;
    }
};

// Phase 1, FP32: costs of the lane's row against the m staged columns into
// `col` (the lane's entry of tile column 0; columns 32 entries apart).
template <int DIM>
__device__ __forceinline__ void short_costs(const ShortRow<float, DIM>& a, const float* pb, const float* rb,
                                            float nu, int m, float* col) {
    constexpr int NQ = DIM / 4;
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
        const ulonglong2* bp = reinterpret_cast<const ulonglong2*>(pb + j * DIM);
        // two running sums of pairs (components 4q, 4q+1 and 4q+2, 4q+3)
        ulonglong2 v = bp[0];
        unsigned long long d0 = f2_sub(a.v[0], v.x), d1 = f2_sub(a.v[1], v.y);
        unsigned long long s0 = f2_mul(d0, d0), s1 = f2_mul(d1, d1);
#pragma unroll
        for (int q = 1; q < NQ; ++q) {
            v = bp[q];
            d0 = f2_sub(a.v[2 * q], v.x);
            d1 = f2_sub(a.v[2 * q + 1], v.y);
            s0 = f2_fma(d0, d0, s0);
            s1 = f2_fma(d1, d1, s1);
        }
        float lo, hi;
        f2_unpack(f2_add(s0, s1), lo, hi);
        col[32 * j] = Arith<float>::wcost(Arith<float>::root(lo + hi), nu, a.t, rb[4 * j]);
    }
}

// Phase 1, FP64: the oracle's order (d_k = a_k - b_k, s = d_0^2, then
// s = s + d_k^2), every operation correctly rounded.
template <int DIM>
__device__ __forceinline__ void short_costs(const ShortRow<double, DIM>& a, const double* pb, const double* rb,
                                            double nu, int m, double* col) {
    using A = Arith<double>;
#pragma unroll 2
    for (int j = 0; j < m; ++j) {
        const double2* bp = reinterpret_cast<const double2*>(pb + j * DIM);
        double2 v = bp[0];
        double d = A::sub(a.v[0], v.x);
        double s = A::mul(d, d);
        d = A::sub(a.v[1], v.y);
        s = A::sq_acc(s, d);
#pragma unroll
        for (int q = 1; q < DIM / 2; ++q) {
            v = bp[q];
            d = A::sub(a.v[2 * q], v.x);
            s = A::sq_acc(s, d);
            d = A::sub(a.v[2 * q + 1], v.y);
            s = A::sq_acc(s, d);
        }
        col[32 * j] = A::wcost(A::root(s), nu, a.t, rb[2 * j]);
    }
}

template <typename T>
__device__ __forceinline__ T short_min3(T a, T b, T c) {
    if constexpr (sizeof(T) == 4) return min3f(a, b, c);
    else return Arith<T>::minv(Arith<T>::minv(a, b), c);
}

// The many-pairs schedule for short pairs (modes and outputs as pairs_kernel;
// included by kernels.cuh after the pair helpers).  The host launches it
// only when every series of both sets has at most kShortMax points and the
// values and records are 16-byte aligned; a pair longer than that on the
// device (lengths that disagree with the host's copy) is reported like an
// out-of-range pair index.
template <typename T, int DIM>
__global__ void __launch_bounds__(32 * kShortWarps) short_pairs_kernel(PairsArgs<T> a) {
    using A = Arith<T>;
    using SM = ShortSmem<T, DIM>;
    constexpr int RL = Rec<T, 0>::kLen;  // (t, delete cost) record: 16 bytes
    static_assert(RL * (int)sizeof(T) == 16, "records are 16 bytes");
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    unsigned char* ws = dyn_smem + (threadIdx.x >> 5) * SM::kWarp;
    T* cost = reinterpret_cast<T*>(ws + 2 * SM::kStage);
    T* delb = reinterpret_cast<T*>(ws + 2 * SM::kStage + SM::kCost);
    const int lane = threadIdx.x & 31;
    const T INF = A::inf();

    struct Job {
        int64_t xa, yb;
        T* o1;
        T* o2;
        int n, m;
    };
    int64_t next_w = 0, end_w = 0;  // the warp's current grab of pair indices
    auto fetch = [&](Job& J) -> bool {
        while (true) {
            if (next_w >= end_w) {
                unsigned long long g = 0;
                if (lane == 0) g = atomicAdd(a.counter, (unsigned long long)kShortGrab);
                g = __shfl_sync(kFull, g, 0);
                if ((int64_t)g >= a.npairs) {
                    next_w = end_w = a.npairs;
                    return false;
                }
                next_w = (int64_t)g;
                end_w = min((int64_t)g + kShortGrab, a.npairs);
            }
            const int64_t w = next_w++;
            int64_t x, y;
            T* o1;
            T* o2 = nullptr;
            if (a.mode == kExplicitPairs) {
                const int64_t wi = a.order ? a.order[w] : w;
                x = a.pairs[2 * wi];
                y = a.pairs[2 * wi + 1];
                o1 = a.out + wi;
                if (!pair_in_range(x, y, a.na, a.nb)) {
                    if (lane == 0) flag_bad_pair(o1, a.sc);
                    continue;
                }
            } else if (a.mode == kSymmetricSorted) {
                int64_t pp, qq;
                triangle_pos(w, a.na, pp, qq);
                x = a.perm_a[pp];
                y = a.perm_a[qq];
                o1 = a.out + x * a.na + y;
                o2 = a.out + y * a.na + x;
            } else {
                const int64_t pp = w / a.nb, qq = w % a.nb;
                x = a.perm_a[pp];
                y = a.perm_b[qq];
                o1 = a.out + x * a.nb + y;
            }
            J.xa = a.offs_a[x];
            J.yb = a.offs_b[y];
            const int64_t n = a.offs_a[x + 1] - J.xa, m = a.offs_b[y + 1] - J.yb;
            if (n < 1 || m < 1 || n > kShortMax || m > kShortMax) {
                if (lane == 0) {
                    flag_bad_pair(o1, a.sc);
                    if (o2) *o2 = *o1;
                }
                continue;
            }
            J.n = (int)n;
            J.m = (int)m;
            J.o1 = o1;
            J.o2 = o2;
            return true;
        }
    };
    // the column series' points and records into stage `buf` (16-byte pieces)
    auto stage = [&](const Job& J, int buf) {
        unsigned char* sb = ws + buf * SM::kStage;
        constexpr int PP = DIM * (int)sizeof(T) / 16;  // pieces per point
        const unsigned char* gb = reinterpret_cast<const unsigned char*>(a.vals_b + J.yb * DIM);
        for (int c = lane; c < J.m * PP; c += 32) cp_async16(sb + 16 * c, gb + 16 * c);
        if (lane < J.m) cp_async16(sb + SM::kPts + 16 * lane, a.rec_b + (J.yb + lane) * RL);
    };
    // the lane's row (lanes past the last row repeat it; their results are never read)
    auto load_row = [&](const Job& J, ShortRow<T, DIM>& r) {
        const int64_t i = J.xa + min(lane, J.n - 1);
        r.load(a.vals_a + i * DIM, a.rec_a + i * RL);
    };
    auto compute = [&](const Job& J, int buf, const ShortRow<T, DIM>& row) {
        const unsigned char* sb = ws + buf * SM::kStage;
        const T* pb = reinterpret_cast<const T*>(sb);
        const T* rb = reinterpret_cast<const T*>(sb + SM::kPts);
        const int n = J.n, m = J.m;
        if (lane < m) delb[lane] = rb[RL * lane + 1];
        short_costs<DIM>(row, pb, rb, a.nu, m, cost + lane);
        __syncwarp();
        // the wavefront: lane i (row i+1) on column s - i at step s
        T Dl = INF, cl = T(0);                           // D and c of the lane's row at its last column
        T diagD = lane == 0 ? T(0) : INF, diagC = T(0);  // D(0, 0) = 0, c(0, 0) = 0
        const T dA = row.del;
        // step s: tile entry (s - lane, lane) is cb[32 s], its delete cost db[s]
        // (read only for 0 <= s - lane < m)
        const T* cb = cost + lane - 32 * lane;
        const T* db = delb - lane;
        // steps past n + m - 2 leave every row's value unchanged
        for (int s0 = 0; s0 < n + m - 1; s0 += 4) {
            const int r0 = s0 - lane;
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                T upD = __shfl_up_sync(kFull, Dl, 1);
                const T upC = __shfl_up_sync(kFull, cl, 1);
                upD = lane == 0 ? INF : upD;  // D(0, j) = +inf for j >= 1
                const bool in = (unsigned)(r0 + u) < (unsigned)m;
                const T c = in ? cb[32 * (s0 + u)] : INF;
                const T dbv = in ? db[s0 + u] : T(0);
                const T tb = A::add(Dl, dbv);
                const T tm = A::add(A::add(diagD, c), diagC);
                Dl = short_min3(A::add(upD, dA), tb, tm);
                cl = c;
                diagD = upD;
                diagC = upC;
            }
        }
        if (lane == n - 1) {
            *J.o1 = Dl;
            if (J.o2) *J.o2 = Dl;
        }
    };

    Job cur{}, nxt{};
    ShortRow<T, DIM> row, nrow;
    bool live = fetch(cur);
    if (live) {
        stage(cur, 0);
        load_row(cur, row);
    }
    cp_async_commit();
    int buf = 0;
    while (live) {
        const bool more = fetch(nxt);
        if (more) {
            stage(nxt, buf ^ 1);
            load_row(nxt, nrow);
        }
        cp_async_commit();
        cp_async_wait_one();  // this lane's copies of the current pair have landed
        __syncwarp();         // and every lane's
        compute(cur, buf, row);
        __syncwarp();  // the stage and the cost tile are free again
        cur = nxt;
        row = nrow;
        live = more;
        buf ^= 1;
    }
    cp_async_wait_all();
}

}  // namespace twed
