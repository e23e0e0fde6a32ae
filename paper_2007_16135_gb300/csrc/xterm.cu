// Tensor-core cross term for 64-dimensional FP32 series (p = 2).
//
// For p = 2, d(a_i, b_j)^2 = |a_i|^2 + |b_j|^2 - 2 a_i . b_j; the dot products
// of a 128-row strip of series a against a 16-column tile of series b form a
// dense 128 x 16 x 64 contraction.  It runs on the 5th-generation tensor cores
// (tcgen05.mma, TF32 inputs, FP32 accumulation in tensor memory); the norms
// stay FP32 on CUDA cores, and the cell cost c(i,j) = sqrt(max(d^2, 0)) +
// nu |t_i - t'_j| is formed in FP32 before the wavefront consumes it.  The
// recurrence itself (paper, section "Time Warp Edit Distance", step 5) is the
// same as everywhere else in this library.
//
// One persistent block handles one pair at a time (pairs from an atomic
// counter, longest series first); four blocks share an SM (shared memory
// 54 KB and 128 TMEM columns each).  Warp roles:
//   warp 0      producer: cp.async of the column tiles (B) into a 3-deep
//               shared-memory ring in the K-major core-matrix layout, two
//               tiles ahead; tcgen05.mma issue (A from tensor memory),
//               tcgen05.commit to an mbarrier.  Also owns the TMEM.
//   warps 1..4  epilogue: at each strip, load the strip's 128 points (one
//               per thread) into tensor memory with tcgen05.st (A operand);
//               per tile, tcgen05.ld of their TMEM lane quarter, cost
//               formation, store into a 4-tile ring of cost tiles [col][row]
//               with the tile's column delete costs beside it.
//   warp 5      wavefront: 32 lanes x 4 rows = the strip's 128 rows, lane L
//               on column s - L at step s, costs read from the ring, in
//               branch-free blocks of 16 steps (one tile of lane 0).
// Every wait is bounded (%globaltimer, then the launch's error word).
#include <cuda_runtime.h>

#include <cstdio>

#include "kernels.cuh"
#include "tc.cuh"

namespace twed {

namespace x64 {
constexpr int D = 64;         // point dimension (MMA K)
constexpr int M = 128;        // rows per strip (MMA M)
constexpr int N = 16;         // columns per tile (MMA N)
constexpr int R = 4;          // wavefront rows per lane
constexpr int NB = 2;         // TMEM accumulators in flight
constexpr int NBB = 3;        // B tiles in the shared-memory ring
constexpr int PREF = 2;       // B tiles loaded ahead of the MMA
constexpr int NC = 4;         // cost tiles in the ring (wavefront span 3 + lead 1)
constexpr int MAXCOL = 1024;  // longest column series (boundary row kept in smem)
constexpr int THREADS = 192;
constexpr int TMEM_COLS = 128;  // NB*N accumulator columns + D columns of A
constexpr int ACOL = 64;        // first TMEM column of the A strip

constexpr int OFF_B = 0;                               // NBB tiles of N*D floats
constexpr int OFF_C = OFF_B + NBB * N * D * 4;         // NC tiles [N][M] costs
constexpr int OFF_DEL = OFF_C + NC * N * M * 4;        // NC tiles of N column delete costs
constexpr int OFF_ROW = OFF_DEL + NC * N * 4;          // MAXCOL + 1 float2: boundary row, spare
constexpr int OFF_BAR = OFF_ROW + (MAXCOL + 1) * 8;    // mbarriers
constexpr int NBAR = NB + NB + NC + NC + 1;            // mma_done, tmem_empty, cost_full, cost_empty, a_ready
constexpr int OFF_MISC = OFF_BAR + NBAR * 8;           // tmem base, pair index
constexpr int SMEM = OFF_MISC + 64;
}  // namespace x64

// Point records for the tensor-core path: (t, delete cost, |x|^2, 0).
__global__ void __launch_bounds__(256) xrecords_kernel(RecordsArgs<float> a) {
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
            nrm = fmaf(xk, xk, nrm);
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

namespace {

__device__ __forceinline__ void cp_async16_zfill(void* smem, const void* gmem, bool valid) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    const int n = valid ? 16 : 0;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(n) : "memory");
}

// Bounded wait on an mbarrier phase: false (and the error word set) after
// sc.timeout_ns of %globaltimer, or as soon as another role has failed.
__device__ __forceinline__ bool xwait(uint64_t* bar, uint32_t parity, const SyncCtl& sc) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    uint32_t spins = 0;
    while (!tc::mbar_try_wait(bar, parity)) {
        if ((++spins & 15u) == 0) {
            if (*(volatile unsigned*)sc.err != 0u) return false;
            if (globaltimer() - t0 > sc.timeout_ns) {
                atomicCAS(sc.err, 0u, 4u);
                atomicCAS(sc.sticky, 0u, 4u);
                return false;
            }
        }
    }
    return true;
}

}  // namespace

// cp.async.wait_group needs an immediate: wait until at most `pending`
// groups of this thread are still in flight (pending <= PREF).
__device__ __forceinline__ void cp_async_wait_pending(int pending) {
    if (pending <= 0) asm volatile("cp.async.wait_group 0;" ::: "memory");
    else if (pending == 1) asm volatile("cp.async.wait_group 1;" ::: "memory");
    else asm volatile("cp.async.wait_group 2;" ::: "memory");
}

// PairsArgs as for pairs_kernel; rec_a / rec_b hold x64 records (float4 per
// point) and vals_a / vals_b the raw 64-dimensional points (16-byte aligned).
__global__ void __launch_bounds__(x64::THREADS) xterm_pairs_kernel(PairsArgs<float> a) {
    using namespace x64;
    static_assert(PREF <= 2 && PREF < NBB, "cp_async_wait_pending covers PREF <= 2");
    extern __shared__ __align__(1024) unsigned char sm[];
    float* sC = reinterpret_cast<float*>(sm + OFF_C);
    float* sDel = reinterpret_cast<float*>(sm + OFF_DEL);
    float2* sRow = reinterpret_cast<float2*>(sm + OFF_ROW);
    uint64_t* bar = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
    uint64_t* mma_done = bar;
    uint64_t* tmem_empty = bar + NB;
    uint64_t* cost_full = bar + 2 * NB;
    uint64_t* cost_empty = bar + 2 * NB + NC;
    uint64_t* a_ready = bar + 2 * NB + 2 * NC;
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + OFF_MISC);
    volatile long long* pair_sh = reinterpret_cast<volatile long long*>(misc + 2);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float INF = __int_as_float(0x7f800000);

    if (threadIdx.x == 0) {
        for (int i = 0; i < NB; ++i) {
            tc::mbar_init(&mma_done[i], 1);
            tc::mbar_init(&tmem_empty[i], 4);
        }
        for (int i = 0; i < NC; ++i) {
            tc::mbar_init(&cost_full[i], 4);
            tc::mbar_init(&cost_empty[i], 1);
        }
        tc::mbar_init(a_ready, 4);
    }
    if (warp == 0) tc::tmem_alloc(misc, TMEM_COLS);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = misc[0];
    const uint32_t idesc = tc::idesc_tf32(M, N);

    // per-role running counters (identical sequences in every role)
    long long t_prod = 0, t_epi = 0, t_dp = 0;  // tiles
    long long s_prod = 0, s_epi = 0;            // strips
    bool ok = true;
    while (true) {
        __syncthreads();
        if (threadIdx.x == 0) {
            const bool failed = *(volatile unsigned*)a.sc.err != 0u;
            *pair_sh = failed ? a.npairs : (long long)atomicAdd(a.counter, 1ull);
        }
        __syncthreads();
        const long long w = *pair_sh;  // block-uniform: every role stops together
        if (w >= a.npairs) break;
        // ---- the pair (same mapping as pairs_kernel)
        int64_t x, y;
        float *o1, *o2 = nullptr;
        if (a.mode == kExplicitPairs) {
            x = a.pairs[2 * w];
            y = a.pairs[2 * w + 1];
            o1 = a.out + w;
            if (!pair_in_range(x, y, a.na, a.nb)) {  // block-uniform
                if (threadIdx.x == 0) flag_bad_pair(o1, a.sc);
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
        const bool swap = nx > ny;  // rows = shorter series
        const float* rvals = swap ? a.vals_b + yb * D : a.vals_a + xa * D;
        const float* cvals = swap ? a.vals_a + xa * D : a.vals_b + yb * D;
        const float4* rrec = reinterpret_cast<const float4*>(swap ? a.rec_b : a.rec_a) + (swap ? yb : xa);
        const float4* crec = reinterpret_cast<const float4*>(swap ? a.rec_a : a.rec_b) + (swap ? xa : yb);
        const int n = (int)(swap ? ny : nx), m = (int)(swap ? nx : ny);
        const int nstrips = (n + M - 1) / M, ntiles = (m + N - 1) / N;
        const int K = nstrips * ntiles;  // tiles of this pair, strip-major

        if (warp == 0) {
            // ================= producer
            const long long t_base = t_prod;
            int issued = 0;  // B tiles of this pair whose copies were issued
            // B tile k of this pair (column tile k % ntiles) into ring slot (t_base + k) % NBB;
            // the slot was last read by the MMA of tile t_base + k - NBB.  Tiles of
            // earlier pairs are all complete (every role finished them before the
            // block moved on), and waiting on their phases could alias a later
            // phase of the same barrier, so only this pair's tiles are waited for.
            auto issue_load = [&](int k) -> bool {
                const long long t = t_base + k;
                if (k >= NBB) {
                    const long long tp = t - NBB;
                    if (!xwait(&mma_done[tp % NB], (uint32_t)((tp / NB) & 1), a.sc)) return false;
                }
                unsigned char* sB = sm + OFF_B + (int)(t % NBB) * N * D * 4;
                const int c0 = (k % ntiles) * N;
                for (int c = lane; c < N * (D / 4); c += 32) {
                    const int col = c / (D / 4), kq = c % (D / 4);
                    const bool v = c0 + col < m;
                    const float* src = cvals + (int64_t)(v ? c0 + col : 0) * D + kq * 4;
                    cp_async16_zfill(sB + tc::kmajor_offset(col, kq * 4, D), src, v);
                }
                cp_async_commit();
                return true;
            };
            for (int k = 0; k < K && ok; ++k) {
                while (issued < K && issued <= k + PREF && ok) {
                    ok = __all_sync(kFull, issue_load(issued));
                    ++issued;
                }
                if (!ok) break;
                cp_async_wait_pending(issued - k - 1);  // tile k's copies are in
                tc::fence_proxy_async_smem();
                __syncwarp();
                const long long t = t_prod;
                const int b = (int)(t % NB);
                bool w2 = true;
                if (k % ntiles == 0) w2 = xwait(a_ready, (uint32_t)(s_prod & 1), a.sc);  // strip's A in TMEM
                if (w2 && t >= NB) w2 = xwait(&tmem_empty[b], (uint32_t)(((t - NB) / NB) & 1), a.sc);
                if (!__all_sync(kFull, w2)) { ok = false; break; }
                tc::fence_after_sync();
                if (lane == 0) {
                    const uint32_t bad = tc::smem_u32(sm + OFF_B + (int)(t % NBB) * N * D * 4);
#pragma unroll
                    for (int ks = 0; ks < D / 8; ++ks) {
                        const uint64_t bd = tc::smem_desc(bad + ks * 2 * tc::kmajor_lbo(), tc::kmajor_lbo(), tc::kmajor_sbo(D));
                        tc::mma_tf32_tmem_a(tmem + (uint32_t)(b * N), tmem + (uint32_t)(ACOL + ks * 8), bd, idesc, ks > 0);
                    }
                    tc::mma_commit(&mma_done[b]);
                }
                __syncwarp();
                ++t_prod;
                if (k % ntiles == ntiles - 1) ++s_prod;
            }
            cp_async_wait_all();
        } else if (warp <= 4) {
            // ================= epilogue: TMEM lane quarter q = warp % 4
            const int q = warp & 3;
            for (int st = 0; st < nstrips && ok; ++st) {
                const int row = st * M + 32 * q + lane;  // 0-based row of the pair
                const int rowc = row < n ? row : n - 1;
                const float4 ri = __ldg(rrec + rowc);
                const float na = ri.z, ti = ri.x;
                {   // this strip's A: every MMA of the previous strip has completed
                    // (this warp waited for each of them), so TMEM columns ACOL.. are free
                    const float4* src = reinterpret_cast<const float4*>(rvals + (int64_t)rowc * D);
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
                        tc::tmem_st32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ACOL + 32 * h), v);
                    }
                    tc::tmem_wait_st();
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(a_ready);
                    ++s_epi;
                }
                for (int tt = 0; tt < ntiles; ++tt, ++t_epi) {
                    const int b = (int)(t_epi % NB), cb = (int)(t_epi % NC);
                    bool w2 = xwait(&mma_done[b], (uint32_t)((t_epi / NB) & 1), a.sc);
                    if (w2 && t_epi >= NC) w2 = xwait(&cost_empty[cb], (uint32_t)(((t_epi - NC) / NC) & 1), a.sc);
                    if (!__all_sync(kFull, w2)) { ok = false; break; }
                    tc::fence_after_sync();
                    uint32_t r[16];
                    asm volatile(
                        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                          "=r"(r[14]), "=r"(r[15])
                        : "r"(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * N))
                        : "memory");
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                    tc::fence_before_sync();
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&tmem_empty[b]);
                    float* ct = sC + (size_t)cb * N * M;
                    const int c0 = tt * N;
#pragma unroll
                    for (int c = 0; c < N; ++c) {
                        const float4 ci = __ldg(crec + min(c0 + c, m - 1));  // (t', delB, |b|^2, 0)
                        const float d2 = fmaf(-2.f, __uint_as_float(r[c]), na + ci.z);
                        const float dd = Arith<float>::root(fmaxf(d2, 0.f));
                        ct[c * M + 32 * q + lane] = fmaf(a.nu, fabsf(ti - ci.x), dd);
                    }
                    // the tile's column delete costs, next to its costs: the
                    // wavefront step then reads only shared memory
                    if (q == 0 && lane < N) sDel[cb * N + lane] = __ldg(crec + min(c0 + lane, m - 1)).y;
                    __syncwarp();
                    if (lane == 0) tc::mbar_arrive(&cost_full[cb]);
                }
            }
        } else {
            // ================= wavefront (warp 5)
            // Steps run in blocks of N (= one cost tile of lane 0's columns):
            // the tile wait and release happen once per block, so the steps in
            // between are one stretch of code without branches.
            static_assert((NC * N & (NC * N - 1)) == 0, "the cost ring index wraps with a mask");
            for (int st = 0; st < nstrips && ok; ++st) {
                const int r0 = st * M + 1;  // 1-based first row of the strip
                const int rows = min(M, n - st * M);
                const int lanes_used = (rows + R - 1) / R;
                const bool first = (st == 0), last = (st == nstrips - 1);
                float rdel[R], Dl[R], cp[R];
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const int i = r0 + lane * R + r;
                    rdel[r] = __ldg(rrec + ((i <= n ? i : n) - 1)).y;
                    Dl[r] = INF;
                    cp[r] = 0.f;
                }
                float diagD = (first && lane == 0) ? 0.f : INF, diagC = 0.f;
                float botD = INF, botC = 0.f;
                const long long t0 = t_dp;
                const int cb0 = (int)(t0 % NC);  // ring slot of this strip's tile 0
                int released = 0;                // tiles of this strip handed back
                const int steps = m + lanes_used - 1;
                // column jc (1-based) of this strip sits in ring column
                // (cb0 * N + jc - 1) mod (NC * N): tiles are consecutive slots
                const int gbase = cb0 * N;
                float4 c4n = make_float4(0.f, 0.f, 0.f, 0.f);
                float delbn = 0.f;
                float2 bndn = make_float2(0.f, 0.f);
                auto prefetch = [&](int jn) {
                    const int jc = jn < 1 ? 1 : (jn > m ? m : jn);
                    const int g = (gbase + jc - 1) & (NC * N - 1);
                    c4n = *reinterpret_cast<const float4*>(sC + (size_t)g * M + lane * R);
                    delbn = sDel[g];
                    bndn = sRow[jc - 1];
                };
                // one step: lane L on column j = s - L + 1; the next column's
                // costs, delete cost and boundary entry are fetched during it
                auto step = [&](int j) {
                    const float4 c4 = c4n;
                    const float delb = delbn;
                    const float2 bnd = bndn;
                    prefetch(j + 1);
                    float upD = __shfl_up_sync(kFull, botD, 1);
                    float upC = __shfl_up_sync(kFull, botC, 1);
                    // a lane before column 1 sees an infinite row above and keeps its state
                    // lane 0 reads the row above the strip (for the pair's first
                    // strip: D(0, j) = inf, c(0, j) = 0).  A lane before column 1
                    // receives inf from the lane above, so its update keeps every
                    // value infinite: no test of j is needed.
                    upD = lane == 0 ? bnd.x : upD;
                    upC = lane == 0 ? bnd.y : upC;
                    const float cc[R] = {c4.x, c4.y, c4.z, c4.w};
                    float tb_[R], tm_[R];
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        const float dg = r == 0 ? diagD : Dl[r - 1];
                        const float cd = r == 0 ? diagC : cp[r - 1];
                        tb_[r] = Dl[r] + delb;
                        tm_[r] = (dg + cc[r]) + cd;
                    }
                    float d_up = upD;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        d_up = min3f(d_up + rdel[r], tb_[r], tm_[r]);
                        Dl[r] = d_up;
                        cp[r] = cc[r];
                    }
                    diagD = upD;
                    diagC = upC;
                    botD = Dl[R - 1];
                    botC = cp[R - 1];
                    // lane 31 hands its bottom row to the next strip; columns
                    // outside 1..m go to the spare entry (no branch)
                    if (lane == 31) sRow[(j >= 1 && j <= m) ? j - 1 : MAXCOL] = make_float2(botD, botC);
                };
                // at step s = N k - 1 lane 0's next prefetch enters tile k, and
                // lane 31 has read tile k - 3 for the last time
                auto boundary = [&](int s) -> bool {
                    const int k = (s + 1) / N;
                    if (k < ntiles) {
                        const long long tt = t0 + k;
                        const bool w2 = xwait(&cost_full[(cb0 + k) % NC], (uint32_t)((tt / NC) & 1), a.sc);
                        if (!__all_sync(kFull, w2)) return false;
                    }
                    const int kr = k - 3;
                    if (kr >= 0 && kr == released && kr < ntiles) {
                        __syncwarp();
                        if (lane == 0) tc::mbar_arrive(&cost_empty[(cb0 + kr) % NC]);
                        ++released;
                    }
                    return true;
                };
                if (first) {  // the row above the pair: D(0, j) = inf, c(0, j) = 0
                    for (int c = lane; c < m; c += 32) sRow[c] = make_float2(INF, 0.f);
                    __syncwarp();
                }
                {   // tile 0 must be in before the first prefetch
                    const bool w2 = xwait(&cost_full[cb0], (uint32_t)((t0 / NC) & 1), a.sc);
                    if (!__all_sync(kFull, w2)) ok = false;
                }
                if (ok) {
                    prefetch(1 - lane);
                    int s = 0;
                    const int head = min(steps, N - 1);
                    for (; s < head; ++s) step(s - lane + 1);
                    while (ok && s + N <= steps) {
                        if (!boundary(s)) { ok = false; break; }
#pragma unroll
                        for (int u = 0; u < N; ++u) step(s + u - lane + 1);
                        s += N;
                    }
                    if (ok && s < steps) {
                        if (!boundary(s)) ok = false;
                        for (; ok && s < steps; ++s) step(s - lane + 1);
                    }
                }
                // hand back the tiles not yet released
                __syncwarp();
                for (int k = released; k < ntiles; ++k)
                    if (lane == 0) tc::mbar_arrive(&cost_empty[(cb0 + k) % NC]);
                // the lane holding row n ends its last step on column m, so
                // its final state holds D(n, m)
                if (ok && last && lane == lanes_used - 1) {
                    const int rr = n - r0 - lane * R;
#pragma unroll
                    for (int r = 0; r < R; ++r) {
                        if (r == rr) {
                            *o1 = Dl[r];
                            if (o2) *o2 = Dl[r];
                        }
                    }
                }
                t_dp = t0 + ntiles;
            }
        }
        // a failed role stops the block at the next pair boundary
        if (!ok && lane == 0) atomicCAS(a.sc.err, 0u, 4u);
    }
    // drain: the producer's last MMAs must finish before TMEM is freed
    // (bounded by the same timeout as every other wait)
    (void)s_epi;
    if (warp == 0 && t_prod > 0) {
        const unsigned long long t0 = globaltimer();
        while (!tc::mbar_try_wait(&mma_done[(t_prod - 1) % NB], (uint32_t)(((t_prod - 1) / NB) & 1)) &&
               globaltimer() - t0 < a.sc.timeout_ns) {
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

cudaError_t launch_xrecords(const RecordsArgs<float>& a, cudaStream_t st) {
    if (a.total <= 0) return cudaSuccess;
    int64_t blocks = (a.total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    (void)cudaGetLastError();
    xrecords_kernel<<<(int)blocks, 256, 0, st>>>(a);
    return cudaGetLastError();
}

// Opt in to the shared memory the kernel needs and ask for the largest
// shared-memory carve-out, so that three blocks fit on one SM.
static cudaError_t xterm_attributes() {
    cudaError_t e = cudaFuncSetAttribute(xterm_pairs_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, x64::SMEM);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(xterm_pairs_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
    return e;
}

cudaError_t launch_xterm_pairs(const PairsArgs<float>& a, int blocks, cudaStream_t st) {
    if (a.npairs <= 0) return cudaSuccess;
    cudaError_t e = xterm_attributes();
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    xterm_pairs_kernel<<<blocks, x64::THREADS, x64::SMEM, st>>>(a);
    return cudaGetLastError();
}

int xterm_blocks_per_sm() {
    cudaError_t e = xterm_attributes();
    int nb = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, xterm_pairs_kernel, x64::THREADS, x64::SMEM);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return -(int)e;  // negative: the CUDA error code, for diagnostics
    }
    return nb;
}

int xterm_max_cols() { return x64::MAXCOL; }

// Blocks per SM allowed by shared memory (1 KB reserved per block), tensor
// memory columns and registers.
int xterm_resident_blocks() {
    cudaFuncAttributes fa{};
    int dev = 0, smem_sm = 0, regs_sm = 0;
    if (xterm_attributes() != cudaSuccess || cudaFuncGetAttributes(&fa, xterm_pairs_kernel) != cudaSuccess ||
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
    cudaFuncGetAttributes(&fa, xterm_pairs_kernel);
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&smem_blk, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    (void)cudaGetLastError();
    snprintf(buf, len, "regs %d static %zu dyn %d max_dyn %d smem/SM %d smem/block %d", fa.numRegs,
             fa.sharedSizeBytes, x64::SMEM, fa.maxDynamicSharedSizeBytes, smem_sm, smem_blk);
}

}  // namespace twed
