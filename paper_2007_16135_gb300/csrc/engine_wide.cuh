// FP32 wavefront strips for wide points (dims 16, 28 and 64, p = 2) on the
// many-pairs schedule.
//
// Same strip / lane / step mapping and boundary-row protocol as
// run_strip_staged (engine_f32.cuh): lane L owns R consecutive rows and at
// step s works on column j = s - L + 1, lane L-1 hands its bottom row over by
// shuffle, lane 0 reads the row above from a boundary row in global memory.
// What changes with the width of a point (the paper's section "Higher
// Dimensions": the lp distance is an O(dim) loop per cell):
//
//  * A lane keeps its rows' points in registers as pairs of adjacent
//    components, so that d^2 = sum_k (a_k - b_k)^2 runs as one packed f32x2
//    subtract and one packed multiply-add per component pair and row (two
//    running sums per row, even and odd components, added at the end).
//  * Column points are not duplicated into records: every 32 steps each lane
//    copies one column's point (dim / 4 16-byte pieces, straight from the
//    packed values) and its (t', delete cost) record into a per-warp ring of
//    96 columns, three 32-column chunks: the chunk being read, the one lane
//    31 still reads and the one in flight.  A step then reads its column in
//    16-byte pieces while it forms the next column's costs.
//
// The recurrence and its evaluation order per cell are those of the staged
// engine (canonical TWED candidate order); only the summation order of d^2
// differs (pairs of components), which the FP32 tolerance covers.
#pragma once

#include "engine_f32.cuh"

namespace twed {

constexpr int kWideRing = 96;  // staged columns per warp (three 32-column chunks)

// Ring record of a column: dim values, t', delete cost, 2 pad floats.
template <int WD>
__host__ __device__ constexpr int wide_rec_floats() {
    return WD + 4;
}
// Shared memory one warp needs: the column ring and the boundary ring.
template <int WD>
__host__ __device__ constexpr int wide_bytes_per_warp() {
    return kWideRing * (wide_rec_floats<WD>() * 4 + 8);
}
// Rows per lane the register budget allows (the rows' points take R * dim
// registers).
template <int WD>
__host__ __device__ constexpr int wide_rmax() {
    return WD <= 16 ? 8 : (WD <= 32 ? 4 : 2);
}

// One strip (rows r0 .. r0+rows-1, rows <= 32*R) of a pair whose points have
// WD components; the point values are read from pr.vals_a / pr.vals_b and the
// (t, delete cost) records (4 floats each) from pr.rec_a / pr.rec_b.
// Boundary rows hold (D, c) per column; `io.up` must have at least m+1
// readable entries.  Returns true (no wait in this schedule can fail).
template <int WD, int R>
__device__ __forceinline__ bool run_strip_wide(const PairRef<float>& pr, int r0, int rows,
                                               const StripIO<float>& io, float* result_a, float* result_b,
                                               float* ring, float2* bring) {
    static_assert(WD % 4 == 0, "wide points come in 16-byte pieces");
    constexpr int LEN = wide_rec_floats<WD>();
    constexpr int NP = WD / 2;  // component pairs per point
    constexpr int NQ = WD / 4;  // 16-byte pieces per point
    const int lane = threadIdx.x & 31;
    const float INF = __int_as_float(0x7f800000);
    const int m = pr.m;
    const bool first = io.up == nullptr;
    const int lanes_used = (rows + R - 1) / R;

    // ---- rows: points as component pairs, times, deletion costs
    unsigned long long A[R][NP];
    float rt[R], rdel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int i = r0 + lane * R + r;
        i = i < pr.n ? i : pr.n;  // rows past n repeat row n; never used
        const ulonglong2* p = reinterpret_cast<const ulonglong2*>(pr.vals_a + (pr.a_first + i - 1) * WD);
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const ulonglong2 v = __ldg(p + q);
            A[r][2 * q] = v.x;
            A[r][2 * q + 1] = v.y;
        }
        const float2 td = __ldg(reinterpret_cast<const float2*>(pr.rec_a + (pr.a_first + i - 1) * 4));
        rt[r] = td.x;
        rdel[r] = td.y;
    }
    float Dl[R], cp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        Dl[r] = INF;  // D(i, 0)
        cp[r] = 0.f;
    }
    float diagD = (r0 == 1 && lane == 0) ? 0.f : INF;
    float diagC = 0.f;
    float botD = INF, botC = 0.f;

    // ---- staging of 32-column chunks (chunk c = columns 32c+1 .. 32c+32)
    auto issue = [&](int c) {
        const int j = 32 * c + 1 + lane;
        if (j <= m) {
            const float* src = pr.vals_b + (pr.b_first + j - 1) * WD;
            float* dst = ring + ((j - 1) % kWideRing) * LEN;
#pragma unroll
            for (int q = 0; q < NQ; ++q) cp_async16(dst + 4 * q, src + 4 * q);
            cp_async16(dst + WD, pr.rec_b + (pr.b_first + j - 1) * 4);
        }
        if (!first && lane < 16) {
            const int jj = 32 * c + 1 + 2 * lane;  // columns jj, jj+1 (jj-1 even: 16-byte aligned)
            if (jj <= m) cp_async16(bring + ((jj - 1) % kWideRing), io.up + (jj - 1));
        }
        cp_async_commit();
    };
    issue(0);
    cp_async_wait_all();
    __syncwarp();
    if (33 <= m) issue(1);

    // the next column's cell costs, time and delete cost (columns clamped to
    // 1..m: a lane outside them computes values nobody reads)
    float cn[R];
    float delbn = 0.f;
    float2 bndn = make_float2(0.f, 0.f);
    auto prefetch = [&](int jn) {
        const int jc = jn < 1 ? 1 : (jn > m ? m : jn);
        const int slot = (jc - 1) % kWideRing;
        const float* rp = ring + slot * LEN;
        const float2 td = *reinterpret_cast<const float2*>(rp + WD);
        delbn = td.y;
        bndn = bring[slot];
        unsigned long long s2[R];
#pragma unroll
        for (int r = 0; r < R; ++r) s2[r] = 0ull;  // (+0, +0)
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const ulonglong2 b = *reinterpret_cast<const ulonglong2*>(rp + 4 * q);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const unsigned long long d0 = f2_sub(A[r][2 * q], b.x);
                s2[r] = f2_fma(d0, d0, s2[r]);
                const unsigned long long d1 = f2_sub(A[r][2 * q + 1], b.y);
                s2[r] = f2_fma(d1, d1, s2[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            float lo, hi;
            f2_unpack(s2[r], lo, hi);
            cn[r] = fmaf(pr.nu, fabsf(rt[r] - td.x), Arith<float>::root(lo + hi));
        }
    };
    prefetch(1 - lane);

    // One step: lane L on column j = s - L + 1.
    auto step = [&](int j) {
        float cc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) cc[r] = cn[r];
        const float delb = delbn;
        const float2 bnd = bndn;
        float upD = __shfl_up_sync(kFull, botD, 1);
        float upC = __shfl_up_sync(kFull, botC, 1);
        upD = lane == 0 ? (first ? INF : bnd.x) : upD;  // D(r0-1, j)
        upC = lane == 0 ? (first ? 0.f : bnd.y) : upC;  // c(r0-1, j)
        // a lane that has not reached column 1 sees an infinite row above: its
        // state then stays exactly at D(i, 0) = inf
        upD = j < 1 ? INF : upD;
        float tb_[R], tm_[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const float dg = r == 0 ? diagD : Dl[r - 1];
            const float cd = r == 0 ? diagC : cp[r - 1];
            tb_[r] = Dl[r] + delb;       // deletion in b
            tm_[r] = (dg + cc[r]) + cd;  // match
        }
        float d_up = upD;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            d_up = min3f(d_up + rdel[r], tb_[r], tm_[r]);  // deletion in a
            Dl[r] = d_up;
            cp[r] = cc[r];
        }
        diagD = upD;
        diagC = upC;
        botD = Dl[R - 1];
        botC = cp[R - 1];
        prefetch(j + 1);
        if (io.down != nullptr && lane == 31 && j >= 1 && j <= m) __stcg(io.down + (j - 1), make_float2(botD, botC));
        __syncwarp();
    };

    const int steps = m + lanes_used - 1;
    for (int s = 0; s < steps; ++s) {
        if (((s + 1) & 31) == 0) {
            // the prefetch of this step reads chunk (s+1)/32 (issued 32 steps
            // ago); stage the one after it over the chunk nobody reads any more
            cp_async_wait_all();
            __syncwarp();
            const int c = ((s + 1) >> 5) + 1;
            if (32 * c + 1 <= m) issue(c);
        }
        step(s - lane + 1);
    }
    // the lane holding row n ends its last step on column m
    if (lane == lanes_used - 1) {
        const int rr = pr.n - r0 - lane * R;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r == rr) {
                if (result_a) *result_a = Dl[r];
                if (result_b) *result_b = Dl[r];
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
    return true;
}

}  // namespace twed
