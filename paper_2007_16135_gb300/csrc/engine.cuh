// Wavefront engine for the TWED dynamic program on sm_103a.
//
// The paper's method (section "Improved Time Warp Edit Distance") evaluates
// the DP one anti-diagonal d = i + j at a time, because every cell on an
// anti-diagonal depends only on the two previous anti-diagonals.  This engine
// keeps that dependence structure but maps it onto a warp:
//
//  * A "strip" is 32*R consecutive rows of the DP matrix.  Lane L of the warp
//    owns rows r0 + L*R .. r0 + L*R + R-1 and keeps their D values, their last
//    cell costs and their points in registers.
//  * At step s lane L works on column j = s - L + 1, so the warp's active
//    cells lie on a skewed anti-diagonal (the paper's ortho-diagonal, Eq. 1-2,
//    stretched by R rows per lane).  Lane L-1 hands its bottom row's D(i,j)
//    and c(i,j) to lane L with one __shfl_up per value; the up-left value and
//    c(i-1,j-1) are the same hand-off one step later.  The paper's three
//    rolling diagonals (z_d, z_{d-1}, z_{d-2}) thus live in registers.
//  * Lane 0 reads the row above the strip from a boundary row written by the
//    strip above (global memory, read 32 columns at a time by the whole warp
//    and handed to lane 0 by shuffles); lane 31 writes the strip's bottom
//    row.  Strips of one pair run one after another on one warp (batched
//    pairs) or concurrently on many warps with bounded progress flags (one
//    long pair).
//
// Arithmetic follows a fixed order (per cell):
//   c      = d(a_i,b_j) + nu*|t_i - t'_j|
//   match  = (D(i-1,j-1) + c(i,j)) + c(i-1,j-1)
//   D(i,j) = min(min(D(i-1,j) + dA(i), D(i,j-1) + dB(j)), match)
// and in FP64 every step is a correctly rounded IEEE operation without FMA
// contraction, so FP64 results reproduce a sequential evaluation of the same
// recurrence bit for bit (p = 1, 2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#include "launch.h"

namespace twed {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------- arithmetic
template <typename T>
struct Arith;

template <>
struct Arith<double> {
    using T = double;
    __device__ static __forceinline__ T add(T a, T b) { return __dadd_rn(a, b); }
    __device__ static __forceinline__ T sub(T a, T b) { return __dsub_rn(a, b); }
    __device__ static __forceinline__ T mul(T a, T b) { return __dmul_rn(a, b); }
    __device__ static __forceinline__ T sq_acc(T s, T d) { return __dadd_rn(s, __dmul_rn(d, d)); }
    __device__ static __forceinline__ T root(T x) { return __dsqrt_rn(x); }
    __device__ static __forceinline__ T absv(T x) { return fabs(x); }
    __device__ static __forceinline__ T powv(T x, T e) { return pow(x, e); }
    __device__ static __forceinline__ T inf() { return __longlong_as_double(0x7ff0000000000000LL); }
    // Every operand of a min is a sum of non-negative terms or +inf, and for
    // such doubles the IEEE bit pattern orders like a signed integer: an
    // integer min keeps the FP64 pipe (the scarce one on this part) free.
    __device__ static __forceinline__ T minv(T a, T b) {
        long long x = __double_as_longlong(a), y = __double_as_longlong(b);
        return __longlong_as_double(x < y ? x : y);
    }
    __device__ static __forceinline__ T wcost(T d, T nu, T ti, T tj) {
        return add(d, mul(nu, absv(sub(ti, tj))));
    }
};

template <>
struct Arith<float> {
    using T = float;
    __device__ static __forceinline__ T add(T a, T b) { return a + b; }
    __device__ static __forceinline__ T sub(T a, T b) { return a - b; }
    __device__ static __forceinline__ T mul(T a, T b) { return a * b; }
    __device__ static __forceinline__ T sq_acc(T s, T d) { return fmaf(d, d, s); }
    // Hardware square root with subnormal inputs flushed to zero: one MUFU
    // operation.  Without .ftz the instruction carries a rescaling path for
    // subnormal inputs that costs four more instructions per call; here a
    // subnormal argument is a squared distance below 1.2e-38, whose root
    // (below 1.1e-19) is negligible against any cost it is added to.
    __device__ static __forceinline__ T root(T x) {
        float r;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
        return r;
    }
    __device__ static __forceinline__ T absv(T x) { return fabsf(x); }
    __device__ static __forceinline__ T powv(T x, T e) { return powf(x, e); }
    __device__ static __forceinline__ T inf() { return __int_as_float(0x7f800000); }
    __device__ static __forceinline__ T minv(T a, T b) { return fminf(a, b); }
    __device__ static __forceinline__ T wcost(T d, T nu, T ti, T tj) {
        return fmaf(nu, fabsf(ti - tj), d);
    }
};

// ------------------------------------------------------------- point records
// The prologue packs every point into one 16-byte aligned record:
//   FP64:  [v_0 .. v_{DIM-1}, t, delete-cost, padding]
//   FP32:  [v_0, v_0, v_1, v_1, .., v_{DIM-1}, v_{DIM-1}, t, delete-cost, padding]
// so that a lane fetches a whole column of B with a few vector loads.  FP32
// stores every component twice: a 64-bit load then yields the (b_k, b_k)
// operand that the packed f32x2 instructions subtract from two rows at once.
// DIM == 0 means "dimension known only at run time": the record then holds
// only [t, delete-cost] and values are read from the caller's array.
template <typename T, int DIM>
struct Rec {
    static constexpr int kPer16 = 16 / (int)sizeof(T);
    static constexpr int kVS = (sizeof(T) == 4 && DIM > 0) ? 2 : 1;  // stride between components
    static constexpr int kVals = DIM > 0 ? DIM * kVS : 0;
    static constexpr int kLen = (kVals + 2 + kPer16 - 1) / kPer16 * kPer16;
    static constexpr int kQ = kLen / kPer16;
    static constexpr int kT = kVals;
    static constexpr int kDel = kVals + 1;
};

template <typename T, int DIM>
__device__ __forceinline__ void load_rec(const T* __restrict__ recs, int64_t idx,
                                         T (&r)[Rec<T, DIM>::kLen]) {
    using RL = Rec<T, DIM>;
    if constexpr (sizeof(T) == 4) {
        const float4* p = reinterpret_cast<const float4*>(recs + idx * RL::kLen);
#pragma unroll
        for (int q = 0; q < RL::kQ; ++q) {
            float4 v = __ldg(p + q);
            r[4 * q + 0] = v.x;
            r[4 * q + 1] = v.y;
            r[4 * q + 2] = v.z;
            r[4 * q + 3] = v.w;
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(recs + idx * RL::kLen);
#pragma unroll
        for (int q = 0; q < RL::kQ; ++q) {
            double2 v = __ldg(p + q);
            r[2 * q + 0] = v.x;
            r[2 * q + 1] = v.y;
        }
    }
}

// ------------------------------------------------------------- lp distance
// d(x,y) = (sum_k |x_k - y_k|^p)^(1/p), dim == 1 -> |x - y|.
// P = 1 or 2 select the closed forms; P = 0 uses pow with the runtime p.
template <typename T, int DIM, int P>
__device__ __forceinline__ T dist(const T* x, const T* y, int dim, int p) {
    using A = Arith<T>;
    if constexpr (DIM == 1) {
        return A::absv(A::sub(x[0], y[0]));
    } else if constexpr (DIM > 1) {
        if constexpr (P == 1) {
            T s = A::absv(A::sub(x[0], y[0]));
#pragma unroll
            for (int k = 1; k < DIM; ++k) s = A::add(s, A::absv(A::sub(x[k], y[k])));
            return s;
        } else if constexpr (P == 2) {
            T d = A::sub(x[0], y[0]);
            T s = A::mul(d, d);
#pragma unroll
            for (int k = 1; k < DIM; ++k) {
                d = A::sub(x[k], y[k]);
                s = A::sq_acc(s, d);
            }
            return A::root(s);
        } else {
            const T e = (T)p;
            T s = A::powv(A::absv(A::sub(x[0], y[0])), e);
#pragma unroll
            for (int k = 1; k < DIM; ++k) s = A::add(s, A::powv(A::absv(A::sub(x[k], y[k])), e));
            return A::powv(s, (T)1 / e);
        }
    } else {  // dimension known at run time; x and y point into global memory
        if (dim == 1) return A::absv(A::sub(__ldg(x), __ldg(y)));
        if (P == 1 || (P == 0 && p == 1)) {
            T s = A::absv(A::sub(__ldg(x), __ldg(y)));
            for (int k = 1; k < dim; ++k) s = A::add(s, A::absv(A::sub(__ldg(x + k), __ldg(y + k))));
            return s;
        } else if (P == 2 || (P == 0 && p == 2)) {
            T d = A::sub(__ldg(x), __ldg(y));
            T s = A::mul(d, d);
            for (int k = 1; k < dim; ++k) {
                d = A::sub(__ldg(x + k), __ldg(y + k));
                s = A::sq_acc(s, d);
            }
            return A::root(s);
        } else {
            const T e = (T)p;
            T s = A::powv(A::absv(A::sub(__ldg(x), __ldg(y))), e);
            for (int k = 1; k < dim; ++k)
                s = A::add(s, A::powv(A::absv(A::sub(__ldg(x + k), __ldg(y + k))), e));
            return A::powv(s, (T)1 / e);
        }
    }
}

// D(i,j) from its three neighbours, in the fixed order documented above.
template <typename T>
__device__ __forceinline__ T cell_update(T d_up, T d_left, T d_diag, T del_a, T del_b, T c_ij,
                                         T c_diag) {
    using A = Arith<T>;
    T da = A::add(d_up, del_a);
    T db = A::add(d_left, del_b);
    T mt = A::add(A::add(d_diag, c_ij), c_diag);
    return A::minv(A::minv(da, db), mt);
}

// ------------------------------------------------------- boundary rows / sync
template <typename T>
struct Pair2;
template <>
struct Pair2<float> {
    using V = float2;
};
template <>
struct Pair2<double> {
    using V = double2;
};

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Wait (every lane) until *flag >= target.  Returns false if the wait gave up
// (timeout, or another warp already reported an error).  Bounded: at most
// timeout_ns of %globaltimer plus one poll.
__device__ __forceinline__ bool wait_progress(const unsigned* flag, unsigned target,
                                              const SyncCtl& sc) {
    if (ld_acquire(flag) >= target) return true;
    const unsigned long long t0 = globaltimer();
    unsigned spins = 0;
    while (true) {
        if (ld_acquire(flag) >= target) return true;
        if ((++spins & 63u) == 0) {
            if (*(volatile unsigned*)sc.err != 0u) return false;
            if (globaltimer() - t0 > sc.timeout_ns) {
                atomicCAS(sc.err, 0u, 4u /* TWED_ERR_TIMEOUT */);
                atomicCAS(sc.sticky, 0u, 4u);
                return false;
            }
        }
        if (sc.sleep_ns) __nanosleep(sc.sleep_ns);
    }
}

// Where a strip reads the row above it and writes its bottom row.
template <typename T>
struct StripIO {
    using V2 = typename Pair2<T>::V;
    const V2* up;            // bottom row of the strip above (D, c) per column, global
    const unsigned* up_flag; // columns of `up` already published; nullptr = all ready
    V2* down;                // this strip's bottom row, global; nullptr = nobody needs it
    unsigned* down_flag;     // progress of `down`; nullptr = no publication
    bool publish;            // false: skip publication (fault injection)
    // Block-local hand-off (staged FP32 engine only): the warp above writes
    // the row above straight into this warp's shared-memory boundary ring.
    bool up_local;           // the row above arrives in this warp's ring
    volatile int* up_prog;   // columns the warp above has written into it
    volatile int* my_cons;   // columns of it this warp has consumed (back-pressure)
    void* down_local;        // the warp below's boundary ring; nullptr = none
    volatile int* down_prog; // its progress word
    volatile int* down_cons; // its consumption word
};

template <typename T>
__device__ __forceinline__ StripIO<T> strip_io_global(const typename Pair2<T>::V* up,
                                                      const unsigned* up_flag,
                                                      typename Pair2<T>::V* down,
                                                      unsigned* down_flag, bool publish) {
    StripIO<T> io;
    io.up = up;
    io.up_flag = up_flag;
    io.down = down;
    io.down_flag = down_flag;
    io.publish = publish;
    io.up_local = false;
    io.up_prog = nullptr;
    io.my_cons = nullptr;
    io.down_local = nullptr;
    io.down_prog = nullptr;
    io.down_cons = nullptr;
    return io;
}

// Bounded wait (whole warp) until *word >= target on a shared-memory word
// written by another warp of the block.  Gives up, like wait_progress, on
// the launch's error word or after timeout_ns.
__device__ __forceinline__ bool wait_local(volatile int* word, int target, const SyncCtl& sc) {
    if (*word >= target) {
        __threadfence_block();
        return true;
    }
    const unsigned long long t0 = globaltimer();
    unsigned spins = 0;
    while (*word < target) {
        if ((++spins & 63u) == 0) {
            if (*(volatile unsigned*)sc.err != 0u) return false;
            if (globaltimer() - t0 > sc.timeout_ns) {
                atomicCAS(sc.err, 0u, 4u /* TWED_ERR_TIMEOUT */);
                atomicCAS(sc.sticky, 0u, 4u);
                return false;
            }
        }
        if (sc.sleep_ns) __nanosleep(sc.sleep_ns);
    }
    __threadfence_block();
    return true;
}

// The series a strip works on.  Row i (1-based) of the DP is point
// a_first + i - 1 of the row set; column j is point b_first + j - 1.
template <typename T>
struct PairRef {
    const T* rec_a;
    const T* rec_b;
    const T* vals_a;  // DIM == 0 only
    const T* vals_b;
    int64_t a_first, b_first;
    int n, m;
    int dim, p;
    T nu;
};

// One strip: rows r0 .. r0 + rows - 1 (rows <= 32*R) against all m columns.
// If the strip holds row n, the lane holding it returns D(n,m) through
// *result (only that lane writes).  Returns false if a wait gave up.
template <typename T, int DIM, int P, int R>
__device__ __forceinline__ bool run_strip(const PairRef<T>& pr, int r0, int rows,
                                          const StripIO<T>& io, const SyncCtl& sc, T* result_a,
                                          T* result_b) {
    using A = Arith<T>;
    using RL = Rec<T, DIM>;
    using V2 = typename Pair2<T>::V;
    constexpr int DV = DIM > 0 ? DIM : 1;
    const int lane = threadIdx.x & 31;
    const T INF = A::inf();
    const int m = pr.m;
    const bool first = (io.up == nullptr);
    const int lanes_used = (rows + R - 1) / R;

    // ---- this lane's rows: points, times and deletion costs in registers
    T ra[R][DV];
    T rt[R], rdel[R];
    const T* rv[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        int i = r0 + lane * R + r;
        i = i < pr.n ? i : pr.n;  // rows past n repeat row n; their results are never used
        T rec[RL::kLen];
        load_rec<T, DIM>(pr.rec_a, pr.a_first + i - 1, rec);
#pragma unroll
        for (int k = 0; k < DV; ++k) ra[r][k] = DIM > 0 ? rec[k] : T(0);
        rt[r] = rec[RL::kT];
        rdel[r] = rec[RL::kDel];
        rv[r] = DIM == 0 ? pr.vals_a + (pr.a_first + i - 1) * (int64_t)pr.dim : nullptr;
    }
    T Dl[R], cp[R];  // D(i, j-1) and c(i, j-1) of each row
#pragma unroll
    for (int r = 0; r < R; ++r) {
        Dl[r] = INF;  // D(i, 0)
        cp[r] = T(0);
    }
    // D(r0-1+lane*R, j-1) and its cost: D(0,0) = 0 for the very first row, inf otherwise
    T diagD = (r0 == 1 && lane == 0) ? T(0) : INF;
    T diagC = T(0);
    T botD = INF, botC = T(0);  // this lane's bottom row at its last column

    // ---- boundary row above the strip: 16 columns per chunk, lane L (and
    // L + 16) holding column L of it; the chunk after the current one is read
    // one chunk ahead, so a strip trails the one above by about 16 + 16 + 31
    // columns (the read-ahead, the publication step of 16 and lane 31's skew)
    constexpr int CK = 16;
    const int cl = lane & (CK - 1);
    T chD = INF, chC = T(0), nxD = INF, nxC = T(0);
    bool ok = true;
    if (!first) {
        const int c0 = 1 + cl;         // chunk 0: columns 1..16
        const int c1 = 1 + CK + cl;    // chunk 1: columns 17..32
        if (io.up_flag) {
            ok = wait_progress(io.up_flag, (unsigned)min(2 * CK, m), sc);
        }
        if (ok) {
            if (c0 <= m) {
                V2 v = __ldcg(io.up + (c0 - 1));
                chD = v.x;
                chC = v.y;
            }
            if (c1 <= m) {
                V2 v = __ldcg(io.up + (c1 - 1));
                nxD = v.x;
                nxC = v.y;
            }
        }
    }
    ok = __all_sync(kFull, ok);
    if (!ok) return false;

    T cur[RL::kLen];
    int j = 1 - lane;
    {
        int jc = j < 1 ? 1 : (j > m ? m : j);
        load_rec<T, DIM>(pr.rec_b, pr.b_first + jc - 1, cur);
    }
    const int steps = m + lanes_used - 1;
    for (int s = 0; s < steps; ++s, ++j) {
        T nxt[RL::kLen];
        {
            int jn = j + 1;
            jn = jn < 1 ? 1 : (jn > m ? m : jn);
            load_rec<T, DIM>(pr.rec_b, pr.b_first + jn - 1, nxt);
        }
        T upD = __shfl_up_sync(kFull, botD, 1);
        T upC = __shfl_up_sync(kFull, botC, 1);
        if (first) {
            if (lane == 0) {
                upD = INF;  // D(0, j)
                upC = T(0);
            }
        } else {
            const int idx = s & (CK - 1);
            T bD = __shfl_sync(kFull, chD, idx);
            T bC = __shfl_sync(kFull, chC, idx);
            if (lane == 0) {
                upD = bD;
                upC = bC;
            }
            if (idx == CK - 1) {
                chD = nxD;
                chC = nxC;
                const int base = s + 2 + CK;  // first column of the chunk after next
                if (base <= m) {
                    bool w = true;
                    if (io.up_flag) w = wait_progress(io.up_flag, (unsigned)min(base + CK - 1, m), sc);
                    if (__any_sync(kFull, !w)) return false;
                    const int c = base + cl;
                    if (c <= m) {
                        V2 v = __ldcg(io.up + (c - 1));
                        nxD = v.x;
                        nxC = v.y;
                    }
                }
            }
        }
        if (j >= 1 && j <= m) {
            const T tb = cur[RL::kT];
            const T delb = cur[RL::kDel];
            const T* bv = DIM == 0 ? pr.vals_b + (pr.b_first + j - 1) * (int64_t)pr.dim : nullptr;
            T d_up = upD, d_dg = diagD, c_dg = diagC;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                T dd;
                if constexpr (DIM > 0) {
                    dd = dist<T, DIM, P>(ra[r], cur, pr.dim, pr.p);
                } else {
                    dd = dist<T, 0, P>(rv[r], bv, pr.dim, pr.p);
                }
                const T c = A::wcost(dd, pr.nu, rt[r], tb);
                const T oldD = Dl[r], oldC = cp[r];
                const T v = cell_update<T>(d_up, oldD, d_dg, rdel[r], delb, c, c_dg);
                Dl[r] = v;
                cp[r] = c;
                d_up = v;
                d_dg = oldD;
                c_dg = oldC;
            }
            diagD = upD;
            diagC = upC;
            botD = Dl[R - 1];
            botC = cp[R - 1];
            if (io.down != nullptr && lane == 31) {
                V2 o;
                o.x = botD;
                o.y = botC;
                __stcg(io.down + (j - 1), o);
                if (io.down_flag != nullptr && io.publish && (((j & (CK - 1)) == 0) || j == m)) {
                    st_release(io.down_flag, (unsigned)j);
                }
            }
        }
#pragma unroll
        for (int q = 0; q < RL::kLen; ++q) cur[q] = nxt[q];
        __syncwarp();
    }
    // the lane holding row n ends its last step on column m (and no lane
    // updates past its column m), so its final state holds D(n, m)
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
    return true;
}

}  // namespace twed
