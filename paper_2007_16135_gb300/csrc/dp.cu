// Wavefront kernels for the dynamic programs that share TWED's band: the
// longest common subsequence (LCS) and dynamic time warping (DTW) (paper,
// section "Generalized Dynamic Programming Extensions", "Direct Extension:
// LCS"), and TWED's optimal edit path (the alignment the paper's
// introduction says a TWED solver can report).
//
// One strip routine runs all three.  A warp takes a pair; its rows are cut
// into strips of 32*R rows, lane L owns R consecutive rows, and at step s
// lane L works on column j = s - L + 1 (the anti-diagonal mapping of
// engine.cuh).  Lane L-1 hands its bottom row's cell to lane L by shuffle;
// lane 0 reads the row above the strip from a boundary row in global memory
// that the strip above wrote (the same buffer, read 32 columns ahead of the
// writes).  A cell carries (value, aux); aux is TWED's cell cost c(i,j),
// which the match term needs one diagonal later, and 0 for LCS and DTW.
//
// Path recovery: the forward pass records, per cell, 2 bits of which
// candidate produced the value (16 cells per 32-bit word, row-major), and
// lane 0 walks them back from (n, m) afterwards.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

#include "../../include/twed.h"
#include "engine.cuh"
#include "handle.h"
#include "kernels.cuh"
#include "launch.h"

namespace twed {
namespace dp {

template <typename V>
struct CellV {
    V v, aux;
};

// ------------------------------------------------------------- policies
// Longest common subsequence (textbook recurrence):
//   L(i,0) = L(0,j) = 0;  L(i,j) = L(i-1,j-1) + 1 if x_i == y_j,
//   else max(L(i-1,j), L(i,j-1)).
// Choice bits: bit 0 x_i == y_j (diagonal), bit 1 L(i-1,j) >= L(i,j-1) (up).
struct Lcs {
    static constexpr bool kAux = false;  // no second value per cell to hand over
    using V = int32_t;
    using Row = int32_t;
    using Col = int32_t;
    const int32_t* x;
    const int32_t* y;
    int n, m;
    __device__ V top() const { return 0; }
    __device__ V left() const { return 0; }
    __device__ V origin() const { return 0; }
    __device__ Row row(int i) const { return __ldg(x + i - 1); }
    __device__ Col col(int j) const { return __ldg(y + j - 1); }
    __device__ V cell(V up, V, V left_, V, V diag, V, const Row& r, const Col& c, V& aux,
                      uint32_t& ch) const {
        const bool eq = r == c;
        const bool go_up = up >= left_;
        ch = (eq ? 1u : 0u) | (go_up ? 2u : 0u);
        aux = 0;
        return eq ? diag + 1 : (go_up ? up : left_);
    }
};

// Dynamic time warping (textbook recurrence, no window) with TWED's lp point
// distance:  D(0,0) = 0, D(i,0) = D(0,j) = inf,
//   D(i,j) = d(a_i,b_j) + min(min(D(i-1,j-1), D(i-1,j)), D(i,j-1)).
// Points of dim <= DIM are zero-padded to DIM (the padded terms add exact
// zeros after the real ones); DIM = 0 reads the points from global memory.
template <typename T, int DIM, int P>
struct Dtw {
    static constexpr bool kAux = false;
    using V = T;
    static constexpr int DV = DIM > 0 ? DIM : 1;
    struct Pt {
        T x[DV];
        const T* ptr;
    };
    using Row = Pt;
    using Col = Pt;
    const T* a;
    const T* b;
    int n, m, dim, p;
    __device__ V top() const { return Arith<T>::inf(); }
    __device__ V left() const { return Arith<T>::inf(); }
    __device__ V origin() const { return T(0); }
    __device__ Pt load(const T* base, int i) const {
        Pt q;
        q.ptr = base + (int64_t)(i - 1) * dim;
        if constexpr (DIM > 0) {
#pragma unroll
            for (int k = 0; k < DIM; ++k) q.x[k] = k < dim ? __ldg(q.ptr + k) : T(0);
        } else {
            q.x[0] = T(0);
        }
        return q;
    }
    __device__ Row row(int i) const { return load(a, i); }
    __device__ Col col(int j) const { return load(b, j); }
    __device__ V cell(V up, V, V left_, V, V diag, V, const Row& r, const Col& c, V& aux,
                      uint32_t& ch) const {
        using A = Arith<T>;
        T d;
        if constexpr (DIM > 0) d = dist<T, DIM, P>(r.x, c.x, DIM, p);
        else d = dist<T, 0, P>(r.ptr, c.ptr, dim, p);
        aux = T(0);
        ch = 0;
        return A::add(d, A::minv(A::minv(diag, up), left_));
    }
};

// TWED (paper, section "Time Warp Edit Distance", step 5) in the library's
// canonical order, with the choice of the first candidate (match, delete in
// a, delete in b) whose value equals the minimum: 0 match, 1 delete in a,
// 2 delete in b.
template <typename T, int DIM, int P>
struct Twed {
    static constexpr bool kAux = true;  // c(i,j), read by the diagonal successor
    using V = T;
    using RL = Rec<T, DIM>;
    static constexpr int DV = DIM > 0 ? DIM : 1;
    struct Pt {
        T x[DV];
        T t, del;
        const T* ptr;
    };
    using Row = Pt;
    using Col = Pt;
    const T* rec_a;
    const T* rec_b;
    const T* vals_a;
    const T* vals_b;
    int n, m, dim, p;
    T nu;
    __device__ V top() const { return Arith<T>::inf(); }
    __device__ V left() const { return Arith<T>::inf(); }
    __device__ V origin() const { return T(0); }
    __device__ Pt load(const T* rec, const T* vals, int i) const {
        T r[RL::kLen];
        load_rec<T, DIM>(rec, i - 1, r);
        Pt q;
#pragma unroll
        for (int k = 0; k < DV; ++k) q.x[k] = DIM > 0 ? r[k * RL::kVS] : T(0);
        q.t = r[RL::kT];
        q.del = r[RL::kDel];
        q.ptr = vals + (int64_t)(i - 1) * dim;
        return q;
    }
    __device__ Row row(int i) const { return load(rec_a, vals_a, i); }
    __device__ Col col(int j) const { return load(rec_b, vals_b, j); }
    __device__ V cell(V up, V, V left_, V, V diag, V diag_c, const Row& r, const Col& c, V& aux,
                      uint32_t& ch) const {
        using A = Arith<T>;
        T d;
        if constexpr (DIM > 0) d = dist<T, DIM, P>(r.x, c.x, DIM, p);
        else d = dist<T, 0, P>(r.ptr, c.ptr, dim, p);
        const T cc = A::wcost(d, nu, r.t, c.t);
        const T da = A::add(up, r.del);
        const T db = A::add(left_, c.del);
        const T mt = A::add(A::add(diag, cc), diag_c);
        const T v = A::minv(A::minv(da, db), mt);
        ch = (mt == v) ? 0u : (da == v ? 1u : 2u);
        aux = cc;
        return v;
    }
};

// ------------------------------------------------------------- one strip
// Rows r0 .. r0+rows-1 (rows <= 32*R) against all m columns.  `up_row`
// (nullptr for the first strip) holds the row above at [1..m]; the strip's
// bottom row goes to `down_row` (nullptr for the last strip).  The lane
// holding row n writes D(n, m) to *result.  With PATH, the choice bits of
// row i go to choice[(i-1)*wpr + (j-1)/16] (2 bits per column).
template <class Pol, int R, bool PATH>
__device__ __forceinline__ void strip(const Pol& pol, int r0, int rows, const CellV<typename Pol::V>* up_row,
                                      CellV<typename Pol::V>* down_row, uint32_t* choice, int64_t wpr,
                                      typename Pol::V* result) {
    using V = typename Pol::V;
    const int lane = threadIdx.x & 31;
    const int m = pol.m, n = pol.n;
    const bool first = up_row == nullptr;
    const int lanes_used = (rows + R - 1) / R;
    typename Pol::Row rd[R];
    V Dl[R], Cl[R];
    uint32_t bits[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int i = r0 + lane * R + r;
        rd[r] = pol.row(i < n ? i : n);
        Dl[r] = pol.left();
        Cl[r] = V(0);
        bits[r] = 0u;
    }
    // D(row above this lane's first row, 0): the origin above row 1
    V diag = (lane == 0 && r0 == 1) ? pol.origin() : pol.left();
    V diagC = V(0);
    V bot = pol.left(), botC = V(0);
    // the row above, 32 columns per chunk (one per lane), handed to lane 0
    V chD = pol.top(), chC = V(0), nxD = pol.top(), nxC = V(0);
    if (!first) {
        if (1 + lane <= m) {
            chD = up_row[1 + lane].v;
            chC = up_row[1 + lane].aux;
        }
        if (33 + lane <= m) {
            nxD = up_row[33 + lane].v;
            nxC = up_row[33 + lane].aux;
        }
    }
    const int steps = m + lanes_used - 1;
    int j = 1 - lane;
    for (int s = 0; s < steps; ++s, ++j) {
        V upD = __shfl_up_sync(kFull, bot, 1);
        V upC = V(0);
        if constexpr (Pol::kAux) upC = __shfl_up_sync(kFull, botC, 1);
        if (first) {
            if (lane == 0) {
                upD = pol.top();
                upC = V(0);
            }
        } else {
            const int idx = s & 31;
            const V bD = __shfl_sync(kFull, chD, idx);
            V bC = V(0);
            if constexpr (Pol::kAux) bC = __shfl_sync(kFull, chC, idx);
            if (lane == 0) {
                upD = bD;
                upC = bC;
            }
            if (idx == 31) {
                chD = nxD;
                chC = nxC;
                const int c = s + 34 + lane;  // the chunk after next
                if (c <= m) {
                    nxD = up_row[c].v;
                    nxC = up_row[c].aux;
                }
            }
        }
        if (j >= 1 && j <= m) {
            const typename Pol::Col col = pol.col(j);
            V d_up = upD, c_up = upC, d_dg = diag, c_dg = diagC;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                V aux;
                uint32_t ch;
                const V v = pol.cell(d_up, c_up, Dl[r], Cl[r], d_dg, c_dg, rd[r], col, aux, ch);
                d_dg = Dl[r];
                c_dg = Cl[r];
                Dl[r] = v;
                Cl[r] = aux;
                d_up = v;
                c_up = aux;
                if constexpr (PATH) {
                    bits[r] |= ch << (2 * ((j - 1) & 15));
                    const int i = r0 + lane * R + r;
                    if (((j & 15) == 0 || j == m) && i <= n) {
                        choice[(int64_t)(i - 1) * wpr + ((j - 1) >> 4)] = bits[r];
                        bits[r] = 0u;
                    }
                }
            }
            diag = upD;
            diagC = upC;
            bot = Dl[R - 1];
            botC = Cl[R - 1];
            if (down_row != nullptr && lane == 31) {
                CellV<V> o;
                o.v = bot;
                o.aux = botC;
                down_row[j] = o;
            }
        }
        __syncwarp();
    }
    if (lane == lanes_used - 1) {
        const int rr = n - r0 - lane * R;
#pragma unroll
        for (int r = 0; r < R; ++r)
            if (r == rr && result) *result = Dl[r];
    }
}

// All strips of one pair on one warp; `row` is the warp's boundary row
// (>= m + 1 cells).  Returns D(n, m) to *result.
template <class Pol, int R, bool PATH>
__device__ __forceinline__ void run_pair(const Pol& pol, CellV<typename Pol::V>* row, uint32_t* choice,
                                         int64_t wpr, typename Pol::V* result) {
    for (int r0 = 1; r0 <= pol.n; r0 += 32 * R) {
        const int rows = min(32 * R, pol.n - r0 + 1);
        const bool last = r0 + rows > pol.n;
        strip<Pol, R, PATH>(pol, r0, rows, r0 == 1 ? nullptr : row, last ? nullptr : row, choice, wpr, result);
        __syncwarp();
    }
}

__device__ __forceinline__ uint32_t choice_at(const uint32_t* choice, int64_t wpr, int i, int j) {
    return (__ldcg(choice + (int64_t)(i - 1) * wpr + ((j - 1) >> 4)) >> (2 * ((j - 1) & 15))) & 3u;
}

// ------------------------------------------------------------- kernels
struct SeqArgs {
    const int32_t* sym_x;
    const int64_t* offs_x;
    const int32_t* sym_y;
    const int64_t* offs_y;
    int64_t nx, ny;
};

// LCS lengths of explicit pairs; pairs with an empty sequence give 0.
template <int R>
__global__ void __launch_bounds__(128) lcs_pairs_kernel(SeqArgs q, const int64_t* pairs, int64_t npairs,
                                                         int32_t* out, unsigned long long* counter,
                                                         CellV<int32_t>* rows, int64_t row_stride,
                                                         SyncCtl sc) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    CellV<int32_t>* row = rows + gw * row_stride;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(counter, 1ull);
        w = __shfl_sync(kFull, w, 0);
        if ((int64_t)w >= npairs) break;
        const int64_t x = pairs[2 * w], y = pairs[2 * w + 1];
        if ((uint64_t)x >= (uint64_t)q.nx || (uint64_t)y >= (uint64_t)q.ny) {
            if (lane == 0) {
                out[w] = -1;
                atomicCAS(sc.err, 0u, 1u);
                atomicCAS(sc.sticky, 0u, 1u);
            }
            continue;
        }
        Lcs pol;
        pol.x = q.sym_x + q.offs_x[x];
        pol.y = q.sym_y + q.offs_y[y];
        pol.n = (int)(q.offs_x[x + 1] - q.offs_x[x]);
        pol.m = (int)(q.offs_y[y + 1] - q.offs_y[y]);
        if (pol.n == 0 || pol.m == 0) {
            if (lane == 0) out[w] = 0;
            continue;
        }
        run_pair<Lcs, R, false>(pol, row, nullptr, 0, out + w);
    }
}

// One LCS with its subsequence: the forward pass records choice bits, lane 0
// walks them back (the textbook rule: diagonal on equal symbols, else up when
// L(i-1,j) >= L(i,j-1), else left) and writes the matched positions.
template <int R>
__global__ void __launch_bounds__(32) lcs_path_kernel(const int32_t* x, int n, const int32_t* y, int m,
                                                       int32_t* len, CellV<int32_t>* row, uint32_t* choice,
                                                       int64_t wpr, int64_t* xi, int64_t* yj) {
    Lcs pol;
    pol.x = x;
    pol.y = y;
    pol.n = n;
    pol.m = m;
    run_pair<Lcs, R, true>(pol, row, choice, wpr, len);
    __syncwarp();
    __threadfence_block();
    if ((threadIdx.x & 31) != 0) return;
    int i = n, j = m, k = *len;
    while (i > 0 && j > 0) {
        const uint32_t ch = choice_at(choice, wpr, i, j);
        if (ch & 1u) {
            --k;
            xi[k] = i - 1;
            yj[k] = j - 1;
            --i;
            --j;
        } else if (ch & 2u) {
            --i;
        } else {
            --j;
        }
    }
}

template <typename T>
struct SetArgs {
    const T* vals_a;
    const int64_t* offs_a;
    const T* vals_b;
    const int64_t* offs_b;
    int64_t na, nb;
    int dim, p;
};

template <typename T, int DIM, int P, int R>
__global__ void __launch_bounds__(128) dtw_pairs_kernel(SetArgs<T> s, const int64_t* pairs, int64_t npairs,
                                                         T* out, unsigned long long* counter, CellV<T>* rows,
                                                         int64_t row_stride, SyncCtl sc) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    CellV<T>* row = rows + gw * row_stride;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(counter, 1ull);
        w = __shfl_sync(kFull, w, 0);
        if ((int64_t)w >= npairs) break;
        const int64_t x = pairs[2 * w], y = pairs[2 * w + 1];
        if ((uint64_t)x >= (uint64_t)s.na || (uint64_t)y >= (uint64_t)s.nb) {
            if (lane == 0) {
                out[w] = (T)__int_as_float(0x7fc00000);
                atomicCAS(sc.err, 0u, 1u);
                atomicCAS(sc.sticky, 0u, 1u);
            }
            continue;
        }
        Dtw<T, DIM, P> pol;
        pol.a = s.vals_a + s.offs_a[x] * s.dim;
        pol.b = s.vals_b + s.offs_b[y] * s.dim;
        pol.n = (int)(s.offs_a[x + 1] - s.offs_a[x]);
        pol.m = (int)(s.offs_b[y + 1] - s.offs_b[y]);
        pol.dim = s.dim;
        pol.p = s.p;
        run_pair<Dtw<T, DIM, P>, R, false>(pol, row, nullptr, 0, out + w);
    }
}

template <typename T>
struct PathArgs {
    const T* rec_a;
    const T* rec_b;
    const T* vals_a;
    const T* vals_b;
    const int64_t* offs_a;  // nullptr: one series each (pair 0 only)
    const int64_t* offs_b;
    int64_t na, nb;
    int n1, m1;             // lengths when offs_* are nullptr
    int dim, p;
    T nu;
    const int64_t* pairs;
    int64_t npairs;
    T* dist;
    int8_t* moves;
    const int64_t* move_offs;  // nullptr: pair 0's moves at moves[0..]
    int64_t* len;
    unsigned long long* counter;
    CellV<T>* rows;
    int64_t row_stride;
    uint32_t* choice;       // per warp: choice_stride words
    int64_t choice_stride;
    int64_t wpr;            // words per choice row (>= ceil(longest / 16))
    SyncCtl sc;
    const int64_t* order = nullptr;  // run position -> pair index (nullptr: list order)
};

// TWED of each pair with one optimal edit path: the forward pass records the
// first candidate equal to D(i,j) (match, delete in a, delete in b), lane 0
// walks back from (n,m) to (1,1), and the warp moves the walk's moves (0
// match, 1 delete in a, 2 delete in b, after the forced first match) to the
// front of the pair's buffer in forward order.
template <typename T, int DIM, int P, int R>
__global__ void __launch_bounds__(128) path_pairs_kernel(PathArgs<T> a) {
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    CellV<T>* row = a.rows + gw * a.row_stride;
    uint32_t* choice = a.choice + gw * a.choice_stride;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(a.counter, 1ull);
        w = __shfl_sync(kFull, w, 0);
        if ((int64_t)w >= a.npairs) break;
        if (a.order != nullptr) w = (unsigned long long)a.order[w];  // longest first
        int64_t fa = 0, fb = 0;
        int n = a.n1, m = a.m1;
        if (a.offs_a != nullptr) {
            const int64_t x = a.pairs[2 * w], y = a.pairs[2 * w + 1];
            if ((uint64_t)x >= (uint64_t)a.na || (uint64_t)y >= (uint64_t)a.nb) {
                if (lane == 0) {
                    a.dist[w] = (T)__int_as_float(0x7fc00000);
                    a.len[w] = -1;
                    atomicCAS(a.sc.err, 0u, 1u);
                    atomicCAS(a.sc.sticky, 0u, 1u);
                }
                continue;
            }
            fa = a.offs_a[x];
            fb = a.offs_b[y];
            n = (int)(a.offs_a[x + 1] - fa);
            m = (int)(a.offs_b[y + 1] - fb);
        }
        using RL = Rec<T, DIM>;
        Twed<T, DIM, P> pol;
        pol.rec_a = a.rec_a + fa * RL::kLen;
        pol.rec_b = a.rec_b + fb * RL::kLen;
        pol.vals_a = a.vals_a + fa * a.dim;
        pol.vals_b = a.vals_b + fb * a.dim;
        pol.n = n;
        pol.m = m;
        pol.dim = a.dim;
        pol.p = a.p;
        pol.nu = a.nu;
        run_pair<Twed<T, DIM, P>, R, true>(pol, row, choice, a.wpr, a.dist + w);
        __syncwarp();
        __threadfence_block();
        int8_t* mv = a.moves + (a.move_offs ? a.move_offs[w] : 0);
        const int cap = n + m - 2;
        int len = 0;
        if (lane == 0) {
            // walk back, writing the moves from the end of the buffer
            int i = n, j = m;
            while (i > 1 || j > 1) {
                const uint32_t ch = choice_at(choice, a.wpr, i, j);
                ++len;
                mv[cap - len] = (int8_t)ch;
                if (ch == 0u) {
                    --i;
                    --j;
                } else if (ch == 1u) {
                    --i;
                } else {
                    --j;
                }
            }
            a.len[w] = len;
        }
        len = __shfl_sync(kFull, len, 0);
        __syncwarp();
        __threadfence_block();
        // the moves sit at mv[cap-len .. cap-1] in forward order: move them to the front
        if (len < cap) {
            for (int k0 = 0; k0 < len; k0 += 32) {
                int8_t v = 0;
                if (k0 + lane < len) v = mv[cap - len + k0 + lane];
                __syncwarp();
                if (k0 + lane < len) mv[k0 + lane] = v;
                __syncwarp();
            }
        }
    }
}

// ------------------------------------------------------------- FP32 paths, staged engine
// Rows per lane of a strip with `left` rows to go: the rule of the
// many-pairs kernel (at most RMAX, even when rows are packed in pairs).
template <int DIM, int P, int RMAX>
__device__ __forceinline__ int path_rows_per_lane(int left) {
    constexpr bool kEven = P == 2 && DIM >= 2;
    int R = left >= 32 * RMAX ? RMAX : (left + 31) / 32;
    if (kEven) R = min((R + 1) & ~1, RMAX);
    return R;
}

// TWED with one optimal edit path, FP32 with a compiled point layout: the
// staged engine (column ring, packed rows) records the choices in words of
// 16 steps (run_strip_staged's PATH layout: row i's choice at column j sits
// at step s + 1 = j + L, L = the lane holding row i in its strip); lane 0
// walks back from (n,m) and the warp moves the moves to the front.  Pairs
// keep their orientation (the moves name a and b).
template <int DIM, int P, int RMAX>
__global__ void __launch_bounds__(128) path_staged_kernel(PathArgs<float> a) {
    extern __shared__ __align__(16) unsigned char dyn_smem[];
    unsigned char* wsmem = dyn_smem + (threadIdx.x >> 5) * smem_per_warp<float, DIM>();
    const int lane = threadIdx.x & 31;
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    float2* row = reinterpret_cast<float2*>(a.rows + gw * a.row_stride);
    uint32_t* choice = a.choice + gw * a.choice_stride;
    constexpr bool kEven = P == 2 && DIM >= 2;
    while (true) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(a.counter, 1ull);
        w = __shfl_sync(kFull, w, 0);
        if ((int64_t)w >= a.npairs) break;
        if (a.order != nullptr) w = (unsigned long long)a.order[w];  // longest first
        int64_t fa = 0, fb = 0;
        int n = a.n1, m = a.m1;
        if (a.offs_a != nullptr) {
            const int64_t x = a.pairs[2 * w], y = a.pairs[2 * w + 1];
            if ((uint64_t)x >= (uint64_t)a.na || (uint64_t)y >= (uint64_t)a.nb) {
                if (lane == 0) {
                    a.dist[w] = __int_as_float(0x7fc00000);
                    a.len[w] = -1;
                    atomicCAS(a.sc.err, 0u, 1u);
                    atomicCAS(a.sc.sticky, 0u, 1u);
                }
                continue;
            }
            fa = a.offs_a[x];
            fb = a.offs_b[y];
            n = (int)(a.offs_a[x + 1] - fa);
            m = (int)(a.offs_b[y + 1] - fb);
        }
        PairRef<float> pr;
        pr.rec_a = a.rec_a;
        pr.rec_b = a.rec_b;
        pr.vals_a = a.vals_a;
        pr.vals_b = a.vals_b;
        pr.a_first = fa;
        pr.b_first = fb;
        pr.n = n;
        pr.m = m;
        pr.dim = a.dim;
        pr.p = a.p;
        pr.nu = a.nu;
        for (int r0 = 1; r0 <= n;) {
            const int R = path_rows_per_lane<DIM, P, RMAX>(n - r0 + 1);
            const int rows = min(n - r0 + 1, 32 * R);
            const bool last = r0 + rows > n;
            const StripIO<float> io =
                strip_io_global<float>(r0 == 1 ? nullptr : row, nullptr, last ? nullptr : row, nullptr, true);
            float* o1 = a.dist + w;
            switch (R) {
#define TWED_PATH_STRIP(RR)                                                                                  \
    case RR:                                                                                                 \
        if constexpr (RR <= RMAX && (!kEven || (RR % 2) == 0))                                               \
            strip_call<float, DIM, P, RR, false, kStepBlockPairs, false, true>(pr, r0, rows, io, a.sc, o1,   \
                                                                               nullptr, wsmem, choice, a.wpr); \
        break;
                TWED_PATH_STRIP(1)
                TWED_PATH_STRIP(2)
                TWED_PATH_STRIP(3)
                TWED_PATH_STRIP(4)
                TWED_PATH_STRIP(5)
                TWED_PATH_STRIP(6)
                TWED_PATH_STRIP(7)
                TWED_PATH_STRIP(8)
#undef TWED_PATH_STRIP
                default: break;
            }
            r0 += rows;
            __syncwarp();
        }
        __syncwarp();
        __threadfence_block();
        int8_t* mv = a.moves + (a.move_offs ? a.move_offs[w] : 0);
        const int cap = n + m - 2;
        // The walk back runs on the whole warp, in windows of 32 rows (lane k
        // holds row i0 - k) by 32 columns (j0 - 31 .. j0): each lane loads
        // the choice words of its row that cover the window (at most 3) in one
        // round of loads; then every lane steps the walk in lockstep and the
        // word of the current cell comes from the lane holding its row.
        // Moves are written from the end of the buffer.
        auto lane_in_strip = [&](int ri) -> int {
            // every strip but the last holds 32 * RMAX rows (rows per lane
            // RMAX); the last holds the rest
            constexpr int kFullRows = 32 * RMAX;
            const int nfull = n / kFullRows;
            if (ri <= nfull * kFullRows) return ((ri - 1) % kFullRows) / RMAX;
            const int r0 = nfull * kFullRows + 1;
            return (ri - r0) / path_rows_per_lane<DIM, P, RMAX>(n - r0 + 1);
        };
        int i = n, j = m, len = 0;
        while (i > 1 || j > 1) {
            const int i0 = i, j0 = j;
            const int ri = i0 - lane;
            uint32_t wv0 = 0u, wv1 = 0u, wv2 = 0u;
            int myL = 0, mybase = 0;
            if (ri >= 1) {
                myL = lane_in_strip(ri);
                const uint32_t* rowp = choice + (int64_t)(ri - 1) * a.wpr;
                mybase = (max(j0 - 31, 1) + myL) >> 4;
                const int top = (j0 + myL) >> 4;
                wv0 = __ldcg(rowp + mybase);
                if (top > mybase) wv1 = __ldcg(rowp + mybase + 1);
                if (top > mybase + 1) wv2 = __ldcg(rowp + mybase + 2);
            }
            while ((i > 1 || j > 1) && i > i0 - 32 && j > j0 - 32) {
                const int t = j + myL;  // this lane's row at column j: step + 1
                const int sel = (t >> 4) - mybase;
                const uint32_t word = sel == 0 ? wv0 : (sel == 1 ? wv1 : wv2);
                const uint32_t ch = __shfl_sync(kFull, (word >> (2 * (t & 15))) & 3u, i0 - i);
                ++len;
                if (lane == 0) mv[cap - len] = (int8_t)ch;
                if (ch == 0u) {
                    --i;
                    --j;
                } else if (ch == 1u) {
                    --i;
                } else {
                    --j;
                }
            }
        }
        if (lane == 0) a.len[w] = len;
        len = __shfl_sync(kFull, len, 0);
        __syncwarp();
        __threadfence_block();
        if (len < cap) {
            for (int k0 = 0; k0 < len; k0 += 32) {
                int8_t v = 0;
                if (k0 + lane < len) v = mv[cap - len + k0 + lane];
                __syncwarp();
                if (k0 + lane < len) mv[k0 + lane] = v;
                __syncwarp();
            }
        }
    }
}

}  // namespace dp

// ------------------------------------------------------------- dispatch
#define TWED_DP_DISPATCH(dim, p, BODY)                                            \
    do {                                                                          \
        _Pragma("nv_diag_suppress 177")                                           \
        switch (dim) {                                                            \
            case 1: { constexpr int DIM_ = 1, P_ = 2; BODY; } break;              \
            case 2: if (p == 1) { constexpr int DIM_ = 2, P_ = 1; BODY; }         \
                    else if (p == 2) { constexpr int DIM_ = 2, P_ = 2; BODY; }    \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;         \
            case 3: if (p == 1) { constexpr int DIM_ = 3, P_ = 1; BODY; }         \
                    else if (p == 2) { constexpr int DIM_ = 3, P_ = 2; BODY; }    \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;         \
            case 4: if (p == 1) { constexpr int DIM_ = 4, P_ = 1; BODY; }         \
                    else if (p == 2) { constexpr int DIM_ = 4, P_ = 2; BODY; }    \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;         \
            case 5: case 6: case 7:                                               \
            case 8: if (p == 1) { constexpr int DIM_ = 8, P_ = 1; BODY; }         \
                    else if (p == 2) { constexpr int DIM_ = 8, P_ = 2; BODY; }    \
                    else { constexpr int DIM_ = 0, P_ = 0; BODY; } break;         \
            default: { constexpr int DIM_ = 0, P_ = 0; BODY; } break;             \
        }                                                                         \
    } while (0)

}  // namespace twed

// ===================================================== C ABI
namespace {

using twed::dp::CellV;

constexpr int kLcsR = 8;   // LCS rows per lane (integer cells are cheap)
constexpr int kDtwR = 4;
constexpr int kPathR = 4;
constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

twed_status_t err(twed_handle_t h, twed_status_t st, const char* msg) {
    return twed::detail::set_error(h, st, msg);
}
twed_status_t cuda_err(twed_handle_t h, cudaError_t e) {
    (void)cudaGetLastError();
    return twed::detail::set_error(h, TWED_ERR_CUDA, cudaGetErrorString(e));
}

bool good_seq(const twed_seq_t* s, int64_t* max_len) {
    if (!s || !s->sym || !s->offs || !s->offs_host || s->n < 1 || s->offs_host[0] != 0) return false;
    int64_t mx = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        const int64_t l = s->offs_host[i + 1] - s->offs_host[i];
        if (l < 0 || l > ((int64_t)1 << 30)) return false;
        mx = std::max(mx, l);
    }
    *max_len = mx;
    return true;
}

template <typename S>
bool good_set(const S* s, int64_t* max_len, int64_t* total) {
    if (!s || !s->vals || !s->offs || !s->offs_host || s->n < 1 || s->offs_host[0] != 0) return false;
    int64_t mx = 0;
    for (int64_t i = 0; i < s->n; ++i) {
        const int64_t l = s->offs_host[i + 1] - s->offs_host[i];
        if (l < 1 || l > ((int64_t)1 << 30)) return false;
        mx = std::max(mx, l);
    }
    *max_len = mx;
    *total = s->offs_host[s->n];
    return true;
}

// Persistent grid of 128-thread blocks: enough warps to fill the GPU, at
// most one per pair.
template <typename K>
int grid_for(K kernel, int64_t npairs, int sms) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 128, 0) != cudaSuccess || per_sm < 1) {
        (void)cudaGetLastError();
        per_sm = 1;
    }
    const int64_t want = (int64_t)per_sm * sms;
    return (int)std::max<int64_t>(1, std::min<int64_t>(want, (npairs + 3) / 4));
}

template <typename T, typename S>
twed_status_t dtw_batch_impl(twed_handle_t h, const S* A, const S* B, const int64_t* d_pairs, int64_t npairs,
                             int dim, int p, T* d_out, void* stream) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (npairs < 0) return err(h, TWED_ERR_INVALID_ARG, "npairs < 0");
    if (npairs == 0) return TWED_OK;
    if (!d_pairs || !d_out) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    if (dim < 1 || p < 1) return err(h, TWED_ERR_INVALID_ARG, "dim and p must be >= 1");
    int64_t maxa, tota, maxb, totb;
    if (!good_set(A, &maxa, &tota) || !good_set(B, &maxb, &totb))
        return err(h, TWED_ERR_INVALID_ARG, "bad set (null pointer, empty series or offs[0] != 0)");
    if constexpr (sizeof(T) == 4) {
        // FP32 with a compiled point layout: the staged engine's DTW mode
        // (column ring, packed rows); other cases run the generic strips here
        if (twed::compiled_layout(dim, p))
            return twed::detail::dtw_batch_f32_staged(h, A, B, d_pairs, npairs, dim, p, d_out, stream);
    }
    const int sms = twed::detail::handle_sms(h);
    int blocks = 0;
    TWED_DP_DISPATCH(dim, p, (blocks = grid_for(twed::dp::dtw_pairs_kernel<T, DIM_, P_, kDtwR>, npairs, sms)));
    const int64_t nwarps = (int64_t)blocks * 4;
    const int64_t stride = std::max(maxa, maxb) + 2;
    const size_t o_cnt = 0, o_rows = align_up(64);
    const size_t bytes = o_rows + sizeof(CellV<T>) * (size_t)nwarps * (size_t)stride;
    twed_status_t st;
    char* base = (char*)twed::detail::handle_workspace(h, bytes, &st);
    if (!base) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* ctl = twed::detail::handle_ctl(h);
    cudaError_t e = cudaMemsetAsync(base + o_cnt, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_err(h, e);
    twed::dp::SetArgs<T> sa{A->vals, A->offs, B->vals, B->offs, A->n, B->n, dim, p};
    twed::SyncCtl sc{ctl, ctl + 1, 2000000000ull, -1, 0};
    (void)cudaGetLastError();
    TWED_DP_DISPATCH(dim, p, (twed::dp::dtw_pairs_kernel<T, DIM_, P_, kDtwR><<<blocks, 128, 0, s>>>(
                                 sa, d_pairs, npairs, d_out, (unsigned long long*)(base + o_cnt),
                                 (CellV<T>*)(base + o_rows), stride, sc)));
    e = cudaGetLastError();
    return e == cudaSuccess ? TWED_OK : cuda_err(h, e);
}

template <typename T>
bool finite_all(const T* x, int64_t n) {
    for (int64_t i = 0; i < n; ++i)
        if (!std::isfinite((double)x[i])) return false;
    return true;
}

// One pair from host memory through the device batch (one pair, one warp).
template <typename T, typename S>
twed_status_t dtw_host_impl(twed_handle_t h, const T* a, int64_t la, const T* b, int64_t lb, int dim, int p,
                            T* out) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!a || !b || !out) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    if (la < 1 || lb < 1 || la > ((int64_t)1 << 30) || lb > ((int64_t)1 << 30) || dim < 1 || p < 1)
        return err(h, TWED_ERR_INVALID_ARG, "lengths, dim and p must be >= 1");
    if (!finite_all(a, la * dim) || !finite_all(b, lb * dim))
        return err(h, TWED_ERR_INVALID_ARG, "non-finite input value");
    const size_t o_a = 0, o_b = align_up(sizeof(T) * la * dim), o_o = o_b + align_up(sizeof(T) * lb * dim);
    const size_t o_p = o_o + 256, o_out = o_p + 256;
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, o_out + 256);
    if (e != cudaSuccess) return err(h, TWED_ERR_ALLOC, "device buffers");
    char* base = (char*)mem;
    cudaStream_t s = (cudaStream_t)twed::detail::handle_stream(h);
    const int64_t offs_a[2] = {0, la}, offs_b[2] = {0, lb}, pr[2] = {0, 0};
    e = cudaMemcpyAsync(base + o_a, a, sizeof(T) * la * dim, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_b, b, sizeof(T) * lb * dim, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_o, offs_a, sizeof offs_a, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_o + 16, offs_b, sizeof offs_b, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_p, pr, sizeof pr, cudaMemcpyHostToDevice, s);
    twed_status_t st = TWED_OK;
    if (e != cudaSuccess) {
        st = cuda_err(h, e);
    } else {
        S A{(const T*)(base + o_a), nullptr, (const int64_t*)(base + o_o), offs_a, 1};
        S B{(const T*)(base + o_b), nullptr, (const int64_t*)(base + o_o + 16), offs_b, 1};
        st = dtw_batch_impl<T, S>(h, &A, &B, (const int64_t*)(base + o_p), 1, dim, p, (T*)(base + o_out), s);
        if (st == TWED_OK) {
            e = cudaMemcpyAsync(out, base + o_out, sizeof(T), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = cuda_err(h, e);
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(mem);
    return st;
}

// TWED edit paths: workspace = records, boundary rows and choice bits of the
// warps in flight; the grid is cut so that the choice bits fit kPathBudget.
constexpr size_t kPathBudget = (size_t)8 << 30;
constexpr int kPathRStaged = 8;  // rows-per-lane cap of the staged path kernel

template <typename T>
twed_status_t path_launch(twed_handle_t h, twed::dp::PathArgs<T> pa, const T* vals_a, const T* ts_a,
                          const int64_t* offs_a, int64_t na, int64_t tota, const T* vals_b, const T* ts_b,
                          const int64_t* offs_b, int64_t nb, int64_t totb, int64_t maxa, int64_t maxb, int dim,
                          T nu, T lambda, int p, cudaStream_t s) {
    const int rl = twed::rec_len<T>(dim, p);
    // FP32 with a compiled point layout: the staged engine, whose choice
    // words follow its steps (up to m + 31 of them per row)
    const bool staged = sizeof(T) == 4 && twed::compiled_layout(dim, p);
    const int64_t wpr = staged ? (maxb + 31) / 16 + 2 : (maxb + 15) / 16;
    const size_t per_choice = sizeof(uint32_t) * (size_t)maxa * (size_t)wpr;
    if (per_choice > kPathBudget)
        return err(h, TWED_ERR_UNSUPPORTED, "edit path: one pair's choice bits (n x m / 4 bytes) exceed 8 GiB");
    const int sms = twed::detail::handle_sms(h);
    int blocks = 0;
    int smem_warp = 0;
    if constexpr (sizeof(T) == 4) {
        if (staged) {
            TWED_DISPATCH(dim, p, (smem_warp = twed::smem_per_warp<float, DIM_>(),
                                   blocks = DIM_ > 0 ? twed::blocks_per_sm(twed::dp::path_staged_kernel<(DIM_ > 0 ? DIM_ : 1), (DIM_ > 0 ? P_ : 2), kPathRStaged>,
                                                                           smem_warp, 128)
                                                     : 0));
            blocks = (int)std::min<int64_t>((int64_t)std::max(blocks, 1) * sms, (pa.npairs + 3) / 4);
        }
    }
    if (!staged)
        TWED_DP_DISPATCH(dim, p, (blocks = grid_for(twed::dp::path_pairs_kernel<T, DIM_, P_, kPathR>, pa.npairs, sms)));
    int64_t nwarps = (int64_t)blocks * 4;
    nwarps = std::max<int64_t>(1, std::min<int64_t>(nwarps, (int64_t)(kPathBudget / std::max<size_t>(per_choice, 1))));
    const int threads = nwarps >= 4 ? 128 : 32 * (int)nwarps;
    blocks = (int)((nwarps * 32 + threads - 1) / threads);
    nwarps = (int64_t)blocks * (threads / 32);
    const int64_t stride = (std::max(maxa, maxb) + 3) & ~(int64_t)1;  // >= longest + 2, even
    size_t off = align_up(64);
    const size_t o_ra = off;
    off = align_up(off + sizeof(T) * rl * (size_t)tota);
    const size_t o_rb = off;
    off = align_up(off + sizeof(T) * rl * (size_t)totb);
    const size_t o_rows = off;
    off = align_up(off + sizeof(CellV<T>) * (size_t)nwarps * (size_t)stride);
    const size_t o_ch = off;
    off = align_up(off + per_choice * (size_t)nwarps);
    // a pair list runs longest first, so that no large pair starts last
    const bool ordered = offs_a != nullptr && pa.pairs != nullptr && pa.npairs > 1;
    const size_t o_ord = off;
    if (ordered) off = align_up(off + sizeof(int64_t) * (size_t)pa.npairs);
    const size_t o_bins = off;
    if (ordered) off = align_up(off + sizeof(unsigned long long) * twed::kOrderBins);
    twed_status_t st;
    char* base = (char*)twed::detail::handle_workspace(h, off, &st);
    if (!base) return st;
    unsigned* ctl = twed::detail::handle_ctl(h);
    cudaError_t e = cudaMemsetAsync(base, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_err(h, e);
    twed::RecordsArgs<T> ra{vals_a, ts_a, offs_a, na, tota, dim, p, nu, lambda, (T*)(base + o_ra)};
    twed::RecordsArgs<T> rb{vals_b, ts_b, offs_b, nb, totb, dim, p, nu, lambda, (T*)(base + o_rb)};
    if ((e = twed::launch_records(ra, s)) != cudaSuccess) return cuda_err(h, e);
    if ((e = twed::launch_records(rb, s)) != cudaSuccess) return cuda_err(h, e);
    if (ordered) {
        if ((e = twed::launch_order_pairs(pa.pairs, pa.npairs, offs_a, na, offs_b, nb, (int64_t*)(base + o_ord),
                                          (unsigned long long*)(base + o_bins), sms, s)) != cudaSuccess)
            return cuda_err(h, e);
        pa.order = (const int64_t*)(base + o_ord);
    }
    pa.rec_a = (const T*)(base + o_ra);
    pa.rec_b = (const T*)(base + o_rb);
    pa.vals_a = vals_a;
    pa.vals_b = vals_b;
    pa.dim = dim;
    pa.p = p;
    pa.nu = nu;
    pa.counter = (unsigned long long*)base;
    pa.rows = (CellV<T>*)(base + o_rows);
    pa.row_stride = stride;
    pa.choice = (uint32_t*)(base + o_ch);
    pa.choice_stride = (int64_t)(per_choice / sizeof(uint32_t));
    pa.wpr = wpr;
    pa.sc = twed::SyncCtl{ctl, ctl + 1, 2000000000ull, -1, 0};
    (void)cudaGetLastError();
    if constexpr (sizeof(T) == 4) {
        if (staged) {
            TWED_DISPATCH(dim, p, (e = DIM_ > 0 ? twed::launch_with_smem(twed::dp::path_staged_kernel<(DIM_ > 0 ? DIM_ : 1), (DIM_ > 0 ? P_ : 2), kPathRStaged>,
                                                                         smem_warp, blocks, threads, s, pa)
                                                : cudaErrorInvalidValue));
            return e == cudaSuccess ? TWED_OK : cuda_err(h, e);
        }
    }
    TWED_DP_DISPATCH(dim, p, (twed::dp::path_pairs_kernel<T, DIM_, P_, kPathR><<<blocks, threads, 0, s>>>(pa)));
    e = cudaGetLastError();
    return e == cudaSuccess ? TWED_OK : cuda_err(h, e);
}

template <typename T>
twed_status_t path_host_impl(twed_handle_t h, const T* a, const T* ta, int64_t la, const T* b, const T* tb,
                             int64_t lb, int dim, T nu, T lambda, int p, T* out, int8_t* moves, int64_t* len) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!a || !ta || !b || !tb || !out || !moves || !len) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    if (la < 1 || lb < 1 || la > ((int64_t)1 << 30) || lb > ((int64_t)1 << 30) || dim < 1 || p < 1)
        return err(h, TWED_ERR_INVALID_ARG, "lengths, dim and p must be >= 1");
    if (!std::isfinite((double)nu) || nu < 0 || !std::isfinite((double)lambda) || lambda < 0)
        return err(h, TWED_ERR_INVALID_ARG, "nu and lambda must be finite and >= 0");
    if (!finite_all(a, la * dim) || !finite_all(ta, la) || !finite_all(b, lb * dim) || !finite_all(tb, lb))
        return err(h, TWED_ERR_INVALID_ARG, "non-finite input value or timestamp");
    const int64_t cap = std::max<int64_t>(la + lb - 2, 1);
    size_t off = 0;
    const size_t o_a = off;
    off = align_up(off + sizeof(T) * la * dim);
    const size_t o_ta = off;
    off = align_up(off + sizeof(T) * la);
    const size_t o_b = off;
    off = align_up(off + sizeof(T) * lb * dim);
    const size_t o_tb = off;
    off = align_up(off + sizeof(T) * lb);
    const size_t o_o = off;
    off = align_up(off + 64);
    const size_t o_d = off;
    off = align_up(off + 16);
    const size_t o_mv = off;
    off = align_up(off + (size_t)cap);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, off);
    if (e != cudaSuccess) return err(h, TWED_ERR_ALLOC, "device buffers");
    char* base = (char*)mem;
    cudaStream_t s = (cudaStream_t)twed::detail::handle_stream(h);
    const int64_t offs[4] = {0, la, 0, lb};
    e = cudaMemcpyAsync(base + o_a, a, sizeof(T) * la * dim, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_ta, ta, sizeof(T) * la, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_b, b, sizeof(T) * lb * dim, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_tb, tb, sizeof(T) * lb, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_o, offs, sizeof offs, cudaMemcpyHostToDevice, s);
    twed_status_t st = TWED_OK;
    if (e != cudaSuccess) {
        st = cuda_err(h, e);
    } else {
        twed::dp::PathArgs<T> pa{};
        pa.offs_a = nullptr;
        pa.offs_b = nullptr;
        pa.n1 = (int)la;
        pa.m1 = (int)lb;
        pa.pairs = nullptr;
        pa.npairs = 1;
        pa.dist = (T*)(base + o_d);
        pa.len = (int64_t*)(base + o_d + 8);
        pa.moves = (int8_t*)(base + o_mv);
        pa.move_offs = nullptr;
        st = path_launch<T>(h, pa, (const T*)(base + o_a), (const T*)(base + o_ta), (const int64_t*)(base + o_o), 1,
                            la, (const T*)(base + o_b), (const T*)(base + o_tb),
                            (const int64_t*)(base + o_o) + 2, 1, lb, la, lb, dim, nu, lambda, p, s);
        if (st == TWED_OK) {
            e = cudaMemcpyAsync(out, base + o_d, sizeof(T), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(len, base + o_d + 8, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e == cudaSuccess && *len > 0)
                e = cudaMemcpy(moves, base + o_mv, (size_t)*len, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) st = cuda_err(h, e);
        }
    }
    cudaStreamSynchronize(s);
    cudaFree(mem);
    return st;
}

template <typename T, typename S>
twed_status_t path_batch_impl(twed_handle_t h, const S* A, const S* B, const int64_t* d_pairs, int64_t npairs,
                              int dim, T nu, T lambda, int p, T* d_dist, int8_t* d_moves,
                              const int64_t* d_move_offs, int64_t* d_len, void* stream) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (npairs < 0) return err(h, TWED_ERR_INVALID_ARG, "npairs < 0");
    if (npairs == 0) return TWED_OK;
    if (!d_pairs || !d_dist || !d_moves || !d_move_offs || !d_len) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    if (dim < 1 || p < 1) return err(h, TWED_ERR_INVALID_ARG, "dim and p must be >= 1");
    if (!std::isfinite((double)nu) || nu < 0 || !std::isfinite((double)lambda) || lambda < 0)
        return err(h, TWED_ERR_INVALID_ARG, "nu and lambda must be finite and >= 0");
    int64_t maxa, tota, maxb, totb;
    if (!good_set(A, &maxa, &tota) || !good_set(B, &maxb, &totb) || !A->ts || !B->ts)
        return err(h, TWED_ERR_INVALID_ARG, "bad set (null pointer, empty series or offs[0] != 0)");
    twed::dp::PathArgs<T> pa{};
    pa.offs_a = A->offs;
    pa.offs_b = B->offs;
    pa.na = A->n;
    pa.nb = B->n;
    pa.pairs = d_pairs;
    pa.npairs = npairs;
    pa.dist = d_dist;
    pa.moves = d_moves;
    pa.move_offs = d_move_offs;
    pa.len = d_len;
    return path_launch<T>(h, pa, A->vals, A->ts, A->offs, A->n, tota, B->vals, B->ts, B->offs, B->n, totb, maxa,
                          maxb, dim, nu, lambda, p, (cudaStream_t)stream);
}

}  // namespace

extern "C" twed_status_t twed_lcs_batch(twed_handle_t h, const twed_seq_t* X, const twed_seq_t* Y,
                                        const int64_t* d_pairs, int64_t npairs, int32_t* d_len, void* stream) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (npairs < 0) return err(h, TWED_ERR_INVALID_ARG, "npairs < 0");
    if (npairs == 0) return TWED_OK;
    if (!d_pairs || !d_len) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    int64_t mx, my;
    if (!good_seq(X, &mx) || !good_seq(Y, &my))
        return err(h, TWED_ERR_INVALID_ARG, "bad sequence set (null pointer, negative length or offs[0] != 0)");
    const int sms = twed::detail::handle_sms(h);
    const int blocks = grid_for(twed::dp::lcs_pairs_kernel<kLcsR>, npairs, sms);
    const int64_t nwarps = (int64_t)blocks * 4;
    const int64_t stride = std::max(mx, my) + 2;
    const size_t o_rows = align_up(64);
    const size_t bytes = o_rows + sizeof(CellV<int32_t>) * (size_t)nwarps * (size_t)stride;
    twed_status_t st;
    char* base = (char*)twed::detail::handle_workspace(h, bytes, &st);
    if (!base) return st;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned* ctl = twed::detail::handle_ctl(h);
    cudaError_t e = cudaMemsetAsync(base, 0, 64, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctl, 0, sizeof(unsigned), s);
    if (e != cudaSuccess) return cuda_err(h, e);
    twed::dp::SeqArgs q{X->sym, X->offs, Y->sym, Y->offs, X->n, Y->n};
    twed::SyncCtl sc{ctl, ctl + 1, 2000000000ull, -1, 0};
    (void)cudaGetLastError();
    twed::dp::lcs_pairs_kernel<kLcsR><<<blocks, 128, 0, s>>>(q, d_pairs, npairs, d_len, (unsigned long long*)base,
                                                            (CellV<int32_t>*)(base + o_rows), stride, sc);
    e = cudaGetLastError();
    return e == cudaSuccess ? TWED_OK : cuda_err(h, e);
}

extern "C" twed_status_t twed_lcs_pairs(twed_handle_t h, const int32_t* x, int64_t n, const int32_t* y, int64_t m,
                                        int64_t* xi, int64_t* yj, int64_t* len) {
    if (!h) return TWED_ERR_INVALID_ARG;
    if (!len || (n > 0 && !x) || (m > 0 && !y)) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    if (n < 0 || m < 0 || n > ((int64_t)1 << 30) || m > ((int64_t)1 << 30))
        return err(h, TWED_ERR_INVALID_ARG, "lengths must be in [0, 2^30]");
    if (n == 0 || m == 0) {
        *len = 0;
        return TWED_OK;
    }
    if (!xi || !yj) return err(h, TWED_ERR_INVALID_ARG, "null pointer");
    const int64_t wpr = (m + 15) / 16;
    const size_t per_choice = sizeof(uint32_t) * (size_t)n * (size_t)wpr;
    if (per_choice > kPathBudget)
        return err(h, TWED_ERR_UNSUPPORTED, "LCS pairs: the choice bits (n x m / 4 bytes) exceed 8 GiB");
    const int64_t k = std::min(n, m);
    size_t off = 0;
    const size_t o_x = off;
    off = align_up(off + sizeof(int32_t) * n);
    const size_t o_y = off;
    off = align_up(off + sizeof(int32_t) * m);
    const size_t o_len = off;
    off = align_up(off + 64);
    const size_t o_xi = off;
    off = align_up(off + sizeof(int64_t) * k);
    const size_t o_yj = off;
    off = align_up(off + sizeof(int64_t) * k);
    const size_t o_row = off;
    off = align_up(off + sizeof(CellV<int32_t>) * (size_t)(std::max(n, m) + 2));
    const size_t o_ch = off;
    off = align_up(off + per_choice);
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, off);
    if (e != cudaSuccess) return err(h, TWED_ERR_ALLOC, "device buffers");
    char* base = (char*)mem;
    cudaStream_t s = (cudaStream_t)twed::detail::handle_stream(h);
    e = cudaMemcpyAsync(base + o_x, x, sizeof(int32_t) * n, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(base + o_y, y, sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
    twed_status_t st = TWED_OK;
    if (e == cudaSuccess) {
        (void)cudaGetLastError();
        twed::dp::lcs_path_kernel<kLcsR><<<1, 32, 0, s>>>((const int32_t*)(base + o_x), (int)n,
                                                           (const int32_t*)(base + o_y), (int)m,
                                                           (int32_t*)(base + o_len), (CellV<int32_t>*)(base + o_row),
                                                           (uint32_t*)(base + o_ch), wpr, (int64_t*)(base + o_xi),
                                                           (int64_t*)(base + o_yj));
        e = cudaGetLastError();
    }
    int32_t l32 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&l32, base + o_len, sizeof l32, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess && l32 > 0) {
        e = cudaMemcpy(xi, base + o_xi, sizeof(int64_t) * (size_t)l32, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(yj, base + o_yj, sizeof(int64_t) * (size_t)l32, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) st = cuda_err(h, e);
    else *len = l32;
    cudaStreamSynchronize(s);
    cudaFree(mem);
    return st;
}

extern "C" twed_status_t twed_dtw_batch_f64(twed_handle_t h, const twed_set_f64_t* A, const twed_set_f64_t* B,
                                            const int64_t* d_pairs, int64_t npairs, int dim, int p, double* d_out,
                                            void* stream) {
    return dtw_batch_impl<double>(h, A, B, d_pairs, npairs, dim, p, d_out, stream);
}
extern "C" twed_status_t twed_dtw_batch_f32(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                                            const int64_t* d_pairs, int64_t npairs, int dim, int p, float* d_out,
                                            void* stream) {
    return dtw_batch_impl<float>(h, A, B, d_pairs, npairs, dim, p, d_out, stream);
}
extern "C" twed_status_t twed_dtw_f64(twed_handle_t h, const double* a, int64_t la, const double* b, int64_t lb,
                                      int dim, int p, double* out) {
    return dtw_host_impl<double, twed_set_f64_t>(h, a, la, b, lb, dim, p, out);
}
extern "C" twed_status_t twed_dtw_f32(twed_handle_t h, const float* a, int64_t la, const float* b, int64_t lb,
                                      int dim, int p, float* out) {
    return dtw_host_impl<float, twed_set_f32_t>(h, a, la, b, lb, dim, p, out);
}
extern "C" twed_status_t twed_path_f64(twed_handle_t h, const double* a, const double* ta, int64_t la,
                                       const double* b, const double* tb, int64_t lb, int dim, double nu,
                                       double lambda, int p, double* out, int8_t* moves, int64_t* len) {
    return path_host_impl<double>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, out, moves, len);
}
extern "C" twed_status_t twed_path_f32(twed_handle_t h, const float* a, const float* ta, int64_t la,
                                       const float* b, const float* tb, int64_t lb, int dim, float nu,
                                       float lambda, int p, float* out, int8_t* moves, int64_t* len) {
    return path_host_impl<float>(h, a, ta, la, b, tb, lb, dim, nu, lambda, p, out, moves, len);
}
extern "C" twed_status_t twed_path_batch_f64(twed_handle_t h, const twed_set_f64_t* A, const twed_set_f64_t* B,
                                             const int64_t* d_pairs, int64_t npairs, int dim, double nu,
                                             double lambda, int p, double* d_dist, int8_t* d_moves,
                                             const int64_t* d_move_offs, int64_t* d_len, void* stream) {
    return path_batch_impl<double>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_dist, d_moves, d_move_offs,
                                   d_len, stream);
}
extern "C" twed_status_t twed_path_batch_f32(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                                             const int64_t* d_pairs, int64_t npairs, int dim, float nu,
                                             float lambda, int p, float* d_dist, int8_t* d_moves,
                                             const int64_t* d_move_offs, int64_t* d_len, void* stream) {
    return path_batch_impl<float>(h, A, B, d_pairs, npairs, dim, nu, lambda, p, d_dist, d_moves, d_move_offs,
                                  d_len, stream);
}
