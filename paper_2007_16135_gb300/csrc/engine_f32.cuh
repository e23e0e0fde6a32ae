// FP32 wavefront engine with staged columns and packed row pairs.
//
// Same strip/lane/step mapping and boundary-row protocol as run_strip in
// engine.cuh (see there for the correspondence with the paper's
// anti-diagonals), with three changes that cut the instructions per cell:
//
//  * Column records are staged per warp in a shared-memory ring of 128
//    columns.  Every 32 steps each lane issues cp.async copies of one column
//    (32 columns ahead of lane 0), so a step reads its column with a few
//    shared-memory vector loads and no prefetch registers.  The boundary row
//    above the strip is staged the same way (16 lanes copy two columns each).
//  * For p = 2 two rows share one packed f32x2 subtract / multiply-add per
//    component: the record stores each component twice, so a 64-bit load is
//    the (b_k, b_k) operand.
//  * The three-way minimum is one three-input min instruction.
#pragma once

#include "engine.cuh"

namespace twed {

// ---------------------------------------------------------------- f32x2
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
    unsigned long long d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
    unsigned long long d;
    asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(lo), "f"(hi));
    return d;
}
__device__ __forceinline__ void f2_unpack(unsigned long long x, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x));
}
__device__ __forceinline__ float min3f(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Steps per straight-line block of the staged engine (a divisor of 8).
// Measured on GB300: the many-pairs kernel runs fastest with 4 (longer
// unrolled bodies of its several strip heights miss in the instruction
// cache), the one-pair band kernel with 8.
constexpr int kStepBlockPairs = 4;
constexpr int kStepBlockBand = 8;

// ---------------------------------------------------------------- cp.async
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

constexpr int kRingCols = 128;  // staged columns per warp (power of two)

// Shared memory one warp needs for DIM (bytes).  The compensated variant
// (KH) stages (D_hi, D_lo, c, 0) per boundary column instead of (D, c).
template <int DIM, bool KH = false>
__host__ __device__ constexpr int staged_bytes_per_warp() {
    return kRingCols * (Rec<float, DIM>::kLen * 4 + (KH ? 16 : 8));
}

// ---------------------------------------------------------------- TwoSum
// s + e == a + b exactly (Knuth's TwoSum, no ordering assumption).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Compensated running cost: D is carried as hi + lo.  Every candidate adds
// FP32 costs with TwoSum and folds the rounding error into lo; the minimum is
// taken on hi + lo.  An error-free border needs a finite sentinel (inf - inf
// would poison TwoSum): kBig is far above any reachable cost.
constexpr float kBig = 1.2676506e30f;  // 2^100

// One strip (rows r0 .. r0+rows-1, rows <= 32*R) of an FP32 pair with the
// dimension known at compile time.  `ring` / `bring` are this warp's staging
// areas (kRingCols records, kRingCols boundary entries).  Boundary rows hold
// (D, c) float2 per column, or (D_hi, D_lo, c, 0) float4 when KH; `io.up`
// must have at least m+1 readable entries (a staged copy may read one past m).
// DTW = true runs dynamic time warping on the same strips instead (the
// related distance of the paper's introduction): the cell cost is d(a_i,
// b_j) alone and D(i,j) = d + min(D(i-1,j), D(i,j-1), D(i-1,j-1)); times,
// delete costs and the hand-off of c are not used (many-pairs schedule, no
// compensation).
//
// PATH = true also records, per cell, which candidate gave D(i,j): the first
// of match (0), delete in a (1), delete in b (2) equal to the minimum.  A
// lane packs its rows' choices of 16 consecutive steps into one 32-bit word
// per row: step s (lane L on column j = s - L + 1) goes to word (s + 1) / 16,
// bits 2 ((s + 1) mod 16); words are stored at the block starts, row i's word
// w at choice[(i - 1) * wpr + w] (rows past n are not stored).
template <int DIM, int P, int R, bool KH = false, int kStepBlock = kStepBlockPairs, bool DTW = false,
          bool PATH = false>
__device__ __forceinline__ bool run_strip_staged(const PairRef<float>& pr, int r0, int rows,
                                                 const StripIO<float>& io, const SyncCtl& sc,
                                                 float* result_a, float* result_b, float* ring,
                                                 void* bring_v, uint32_t* choice = nullptr, int64_t wpr = 0) {
    static_assert(DIM > 0, "staged engine needs a compile-time dimension");
    static_assert(!PATH || (!KH && !DTW), "choice bits are recorded for plain TWED only");
    uint32_t wbits[PATH ? R : 1];
#pragma unroll
    for (int r = 0; r < (PATH ? R : 1); ++r) wbits[r] = 0u;
    auto flush_bits = [&](int w) {
        if constexpr (PATH) {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int i = r0 + (threadIdx.x & 31) * R + r;
                if (i <= pr.n) choice[(int64_t)(i - 1) * wpr + w] = wbits[r];
                wbits[r] = 0u;
            }
        }
    };
    using RL = Rec<float, DIM>;
    constexpr int LEN = RL::kLen;
    constexpr bool PACK = (P == 2 && DIM >= 2 && (R % 2) == 0);
    const int lane = threadIdx.x & 31;
    const float INF = KH ? kBig : __int_as_float(0x7f800000);
    const int m = pr.m;
    const bool first = (io.up == nullptr && !io.up_local);
    const bool up_global = (io.up != nullptr);
    const int lanes_used = (rows + R - 1) / R;
    const float* gcol = pr.rec_b + pr.b_first * LEN;  // column j at gcol + (j-1)*LEN
    float2* bring2 = reinterpret_cast<float2*>(bring_v);
    float4* bring4 = reinterpret_cast<float4*>(bring_v);
    const float4* up4 = reinterpret_cast<const float4*>(io.up);
    float4* down4 = reinterpret_cast<float4*>(io.down);
    float2* dloc2 = reinterpret_cast<float2*>(io.down_local);  // the next warp's ring
    float4* dloc4 = reinterpret_cast<float4*>(io.down_local);

    // ---- rows: points (packed in pairs for p = 2), times, deletion costs
    constexpr int NPR = PACK ? R / 2 : 1;
    constexpr int NSC = PACK ? 1 : R;
    unsigned long long A2[NPR][DIM];
    float ra[NSC][DIM];
    float rt[R], rdel[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int i = r0 + lane * R + r;
        i = i < pr.n ? i : pr.n;  // rows past n repeat row n; never used
        const float4* p = reinterpret_cast<const float4*>(pr.rec_a + (pr.a_first + i - 1) * LEN);
        float rec[LEN];
#pragma unroll
        for (int q = 0; q < LEN / 4; ++q) {
            const float4 v = __ldg(p + q);
            rec[4 * q] = v.x;
            rec[4 * q + 1] = v.y;
            rec[4 * q + 2] = v.z;
            rec[4 * q + 3] = v.w;
        }
        rt[r] = rec[RL::kT];
        rdel[r] = rec[RL::kDel];
        if constexpr (PACK) {
            if (r & 1) {
#pragma unroll
                for (int k = 0; k < DIM; ++k) {
                    float lo, hi;
                    f2_unpack(A2[r / 2][k], lo, hi);
                    A2[r / 2][k] = f2_pack(lo, rec[2 * k]);
                }
            } else {
#pragma unroll
                for (int k = 0; k < DIM; ++k) A2[r / 2][k] = f2_pack(rec[2 * k], 0.f);
            }
        } else {
#pragma unroll
            for (int k = 0; k < DIM; ++k) ra[r][k] = rec[2 * k];
        }
    }
    float Dl[R], Dlo[KH ? R : 1], cp[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        Dl[r] = INF;  // D(i, 0)
        if constexpr (KH) Dlo[r] = 0.f;
        cp[r] = 0.f;
    }
    float diagD = (r0 == 1 && lane == 0) ? 0.f : INF;
    float diagL = 0.f, diagC = 0.f;
    float botD = INF, botL = 0.f, botC = 0.f;

    // ---- staging of 32-column chunks (chunk c = columns 32c+1 .. 32c+32)
    auto issue = [&](int c) {
        const int j = 32 * c + 1 + lane;
        if (j <= m) {
            const float* src = gcol + (int64_t)(j - 1) * LEN;
            float* dst = ring + ((j - 1) & (kRingCols - 1)) * LEN;
#pragma unroll
            for (int q = 0; q < LEN / 4; ++q) cp_async16(dst + 4 * q, src + 4 * q);
        }
        if (up_global) {
            if constexpr (KH) {
                if (j <= m) cp_async16(bring4 + ((j - 1) & (kRingCols - 1)), up4 + (j - 1));
            } else if (lane < 16) {
                const int jj = 32 * c + 1 + 2 * lane;  // columns jj, jj+1 (jj-1 even: 16-B aligned)
                if (jj <= m) cp_async16(bring2 + ((jj - 1) & (kRingCols - 1)), io.up + (jj - 1));
            }
        }
        cp_async_commit();
    };
    if (up_global && io.up_flag != nullptr) {
        const bool w = wait_progress(io.up_flag, (unsigned)min(32, m), sc);
        if (!__all_sync(kFull, w)) return false;
    }
    issue(0);

    // The steps are software-pipelined: step s prefetches the record and the
    // boundary entry of its next column and forms all R cell costs for it
    // (none of that depends on D), so the shared-memory loads, the distance
    // arithmetic and the square roots of step s+1 overlap the min-plus chain
    // of step s.  Staging waits therefore run one step ahead of the columns.
    // Before step 0: chunk 0 resident, chunk 1 in flight, first 8 hand-off
    // columns present.
    cp_async_wait_all();
    __syncwarp();
    if (33 <= m) {
        if (up_global && io.up_flag != nullptr) {
            const bool w = wait_progress(io.up_flag, (unsigned)min(64, m), sc);
            if (__any_sync(kFull, !w)) {
                cp_async_wait_all();
                return false;
            }
        }
        issue(1);
    }
    if (io.up_local) {
        const bool w = wait_local(io.up_prog, min(8, m), sc);
        if (__any_sync(kFull, !w)) {
            cp_async_wait_all();
            return false;
        }
    }

    // next column's inputs (valid when its column is in 1..m)
    float cn[R];
    float tbn = 0.f, delbn = 0.f;
    float4 bndn = make_float4(0.f, 0.f, 0.f, 0.f);
    float recn[LEN];
    // (a) the shared-memory loads of the next column's record and boundary entry
    auto prefetch_load = [&](int jn) {
        const int jc = jn < 1 ? 1 : (jn > m ? m : jn);
        const int slot = (jc - 1) & (kRingCols - 1);
        const float4* rp = reinterpret_cast<const float4*>(ring + slot * LEN);
#pragma unroll
        for (int q = 0; q < LEN / 4; ++q) {
            const float4 v = rp[q];
            recn[4 * q] = v.x;
            recn[4 * q + 1] = v.y;
            recn[4 * q + 2] = v.z;
            recn[4 * q + 3] = v.w;
        }
        if constexpr (KH) {
            bndn = bring4[slot];
        } else {
            const float2 b2 = bring2[slot];
            bndn = make_float4(b2.x, 0.f, b2.y, 0.f);  // (D, -, c, -)
        }
    };
    // (b) the R cell costs of that column
    auto prefetch_costs = [&]() {
        tbn = recn[RL::kT];
        delbn = recn[RL::kDel];
        if constexpr (PACK) {
            unsigned long long B2[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) B2[k] = f2_pack(recn[2 * k], recn[2 * k + 1]);
#pragma unroll
            for (int q = 0; q < R / 2; ++q) {
                unsigned long long d2 = f2_sub(A2[q][0], B2[0]);
                unsigned long long s2 = f2_mul(d2, d2);
#pragma unroll
                for (int k = 1; k < DIM; ++k) {
                    d2 = f2_sub(A2[q][k], B2[k]);
                    s2 = f2_fma(d2, d2, s2);
                }
                float s0, s1;
                f2_unpack(s2, s0, s1);
                if constexpr (DTW) {
                    cn[2 * q] = Arith<float>::root(s0);
                    cn[2 * q + 1] = Arith<float>::root(s1);
                } else {
                    cn[2 * q] = fmaf(pr.nu, fabsf(rt[2 * q] - tbn), Arith<float>::root(s0));
                    cn[2 * q + 1] = fmaf(pr.nu, fabsf(rt[2 * q + 1] - tbn), Arith<float>::root(s1));
                }
            }
        } else {
            float bv[DIM];
#pragma unroll
            for (int k = 0; k < DIM; ++k) bv[k] = recn[2 * k];
#pragma unroll
            for (int r = 0; r < R; ++r)
                cn[r] = DTW ? dist<float, DIM, P>(ra[r], bv, DIM, pr.p)
                            : fmaf(pr.nu, fabsf(rt[r] - tbn), dist<float, DIM, P>(ra[r], bv, DIM, pr.p));
        }
    };
    prefetch_load(1 - lane);
    prefetch_costs();

    const int steps = m + lanes_used - 1;

    static_assert(kStepBlock == 1 || kStepBlock == 2 || kStepBlock == 4 || kStepBlock == 8,
                  "the 8-step duties need block starts at every s = 8q + 7");
    // Steps run in blocks of kStepBlock (4 or 8).  Work due every 8 steps is
    // done at steps s = 8q + 7 before that step's prefetch: publication of
    // lane 31's progress (its last finished column, s - 31) and the
    // block-local hand-off waits; every 32 steps, the staging of the next
    // 32-column chunk.  The steps of a block are straight-line code; a
    // shorter block keeps the unrolled body small enough for the
    // instruction cache when several strip heights run on one SM.
    auto boundary = [&](int s) -> bool {
        if (((s + 1) & 7) != 0) return true;
        if constexpr (PATH) {
            if (((s + 1) & 15) == 0) flush_bits(((s + 1) >> 4) - 1);  // steps s-16 .. s-1 are done
        }
        const int jp = s - 31;  // lane 31 finished columns 1..jp
        if (io.publish && jp >= 1 && jp <= m && lane == 31) {
            if (io.down_flag != nullptr && (jp & 31) == 0) st_release(io.down_flag, (unsigned)jp);
            if (io.down_local != nullptr) {
                __threadfence_block();
                *io.down_prog = jp;
            }
        }
        if (((s + 1) & 31) == 0) {
            // the prefetch of this step reads chunk (s+1)/32 (issued 32 steps ago); stage the next
            cp_async_wait_all();
            __syncwarp();
            const int c = ((s + 1) >> 5) + 1;
            if (32 * c + 1 <= m) {
                if (up_global && io.up_flag != nullptr) {
                    const bool w = wait_progress(io.up_flag, (unsigned)min(32 * c + 32, m), sc);
                    if (__any_sync(kFull, !w)) return false;
                }
                issue(c);
            }
        }
        if (io.up_local || io.down_local != nullptr) {
            // block-local hand-off, 8 columns at a time: the row above must be
            // written for lane 0's next 8 prefetches, and the warp below must
            // have consumed what lane 31's next 8 writes overwrite (ring of 128)
            bool w = true;
            if (io.up_local) {
                if (lane == 0) {
                    __threadfence_block();
                    *io.my_cons = s + 1;  // ring columns 1..s+1 are consumed
                }
                if (s + 2 <= m) w = wait_local(io.up_prog, min(s + 9, m), sc);
            }
            if (w && io.down_local != nullptr && s - 151 >= 1)
                w = wait_local(io.down_cons, s - 151, sc);
            if (__any_sync(kFull, !w)) return false;
        }
        return true;
    };

    // One step: lane L on column j = s - L + 1.  The loads and arithmetic of
    // the next column (prefetch) interleave with this column's min-plus chain.
    auto step = [&](int j) {
        // this step's inputs, prefetched by the previous step
        float cc[R];
#pragma unroll
        for (int r = 0; r < R; ++r) cc[r] = cn[r];
        const float delb = delbn;
        const float4 bnd = bndn;
        prefetch_load(j + 1);
        float upD = __shfl_up_sync(kFull, botD, 1);
        float upC = 0.f;
        if constexpr (!DTW) upC = __shfl_up_sync(kFull, botC, 1);
        float upL = 0.f;
        if constexpr (KH) upL = __shfl_up_sync(kFull, botL, 1);
        upD = lane == 0 ? (first ? INF : bnd.x) : upD;  // D(r0-1, j)
        if constexpr (!DTW) upC = lane == 0 ? (first ? 0.f : bnd.z) : upC;  // c(r0-1, j)
        if constexpr (KH) upL = lane == 0 ? (first ? 0.f : bnd.y) : upL;
        // a lane that has not reached column 1 sees an infinite row above: its
        // state then stays exactly at D(i, 0) = inf, so no branch is needed
        upD = j < 1 ? INF : upD;
        if constexpr (KH) {
            // (2) the parts of each update that do not depend on the row just
            //     above in this step: deletion in b and the match candidate
            float h2[R], l2[R], v2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dh = r == 0 ? diagD : Dl[r - 1];
                const float dl = r == 0 ? diagL : Dlo[r - 1];
                const float cd = r == 0 ? diagC : cp[r - 1];
                float sb, eb, s3, e3, s4, e4;
                two_sum(Dl[r], delb, sb, eb);
                const float lb = Dlo[r] + eb;
                const float vb = sb + lb;
                two_sum(dh, cc[r], s3, e3);
                two_sum(s3, cd, s4, e4);
                const float lm = (dl + e3) + e4;
                const float vm = s4 + lm;
                const bool mb = vm < vb;
                h2[r] = mb ? s4 : sb;
                l2[r] = mb ? lm : lb;
                v2[r] = mb ? vm : vb;
            }
            // (3) the chain down the lane's rows: deletion in a
            float uh = upD, ul = upL;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                float sa, ea;
                two_sum(uh, rdel[r], sa, ea);
                const float la = ul + ea;
                const float va = sa + la;
                const bool ma = va < v2[r];
                uh = ma ? sa : h2[r];
                ul = ma ? la : l2[r];
                Dl[r] = uh;
                Dlo[r] = ul;
                cp[r] = cc[r];
            }
        } else if constexpr (DTW) {
            // min(left, up-left) first (both from the previous column), then
            // the chain down the lane's rows: D = d + min(up, that)
            float lm_[R];
#pragma unroll
            for (int r = 0; r < R; ++r) lm_[r] = fminf(Dl[r], r == 0 ? diagD : Dl[r - 1]);
            float d_up = upD;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                d_up = cc[r] + fminf(d_up, lm_[r]);
                Dl[r] = d_up;
            }
            (void)delb;
        } else {
            float tb_[R], tm_[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float dg = r == 0 ? diagD : Dl[r - 1];
                const float cd = r == 0 ? diagC : cp[r - 1];
                tb_[r] = Dl[r] + delb;         // deletion in b
                tm_[r] = (dg + cc[r]) + cd;    // match
            }
            // (3) the chain down the lane's rows: deletion in a
            float d_up = upD;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                if constexpr (PATH) {
                    const float da = d_up + rdel[r];
                    const float v = min3f(da, tb_[r], tm_[r]);
                    const uint32_t ch = tm_[r] == v ? 0u : (da == v ? 1u : 2u);
                    wbits[r] |= ch << (2 * ((j + lane) & 15));  // j + lane = s + 1: warp-uniform
                    d_up = v;
                } else {
                    d_up = min3f(d_up + rdel[r], tb_[r], tm_[r]);
                }
                Dl[r] = d_up;
                cp[r] = cc[r];
            }
        }
        diagD = upD;
        diagC = upC;
        botD = Dl[R - 1];
        botC = cp[R - 1];
        if constexpr (KH) {
            diagL = upL;
            botL = Dlo[R - 1];
        }
        prefetch_costs();
        const bool act = (j >= 1 && j <= m);
        if (io.down != nullptr && lane == 31 && act) {
            if constexpr (KH) __stcg(down4 + (j - 1), make_float4(botD, botL, botC, 0.f));
            else __stcg(io.down + (j - 1), make_float2(botD, botC));
        }
        if (io.down_local != nullptr && lane == 31 && act) {
            const int slot_d = (j - 1) & (kRingCols - 1);
            if constexpr (KH) dloc4[slot_d] = make_float4(botD, botL, botC, 0.f);
            else dloc2[slot_d] = make_float2(botD, botC);
        }
        __syncwarp();
    };

    int s = 0;
    const int head = min(steps, kStepBlock - 1);
    for (; s < head; ++s) step(s - lane + 1);
    bool ok = true;
    while (s + kStepBlock <= steps) {
        if (!boundary(s)) {
            ok = false;
            break;
        }
#pragma unroll
        for (int u = 0; u < kStepBlock; ++u) step(s + u - lane + 1);
        s += kStepBlock;
    }
    if (ok && s < steps) {
        ok = boundary(s);
        for (; ok && s < steps; ++s) step(s - lane + 1);
    }
    if (!ok) {
        cp_async_wait_all();
        return false;
    }
    if constexpr (PATH) {
        if (ok) flush_bits(steps >> 4);  // the word of the last step, s = steps - 1
    }
    // lane 31 ends on column m when all 32 lanes hold rows: publish it
    if (io.publish && lanes_used == 32 && lane == 31) {
        if (io.down_flag != nullptr) st_release(io.down_flag, (unsigned)m);
        if (io.down_local != nullptr) {
            __threadfence_block();
            *io.down_prog = m;
        }
    }
    // the lane holding row n ends its last step on column m, so its final
    // state holds D(n, m)
    if (lane == lanes_used - 1) {
        const int rr = pr.n - r0 - lane * R;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            if (r == rr) {
                const float v = KH ? Dl[r] + Dlo[r] : Dl[r];
                if (result_a) *result_a = v;
                if (result_b) *result_b = v;
            }
        }
    }
    cp_async_wait_all();
    __syncwarp();
    return true;
}

}  // namespace twed
