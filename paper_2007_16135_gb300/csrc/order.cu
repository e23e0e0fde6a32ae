// Longest-first run order of an explicit pair list.
//
// The many-pairs kernel takes pairs from an atomic counter in array order.
// This pass computes a permutation that runs them by decreasing n * m, in
// quarter-octave classes (classes are within 19% of each other in size), so
// that the largest pairs do not start last: a counting sort over 256
// classes (order inside a class is arbitrary) -- class histogram, exclusive
// scan, scatter.  Results do not depend on the order: each pair's value is
// computed by one warp from its own inputs.
#include <cuda_runtime.h>

#include <algorithm>

#include "launch.h"

namespace twed {

namespace {

struct OrderKey {
    const int64_t* pairs;
    const int64_t* oa;
    const int64_t* ob;
    int64_t na, nb;  // series in each set: indices outside are never dereferenced
};

// Class of a pair: 0 for the largest cell counts, kOrderBins - 1 for the
// smallest (4 * floor(log2 c) + the two bits after c's leading one).
__device__ __forceinline__ int cell_class(const OrderKey& k, int64_t w) {
    const int64_t x = k.pairs[2 * w], y = k.pairs[2 * w + 1];
    // a pair outside the sets runs last; the pairs kernel reports it
    if ((uint64_t)x >= (uint64_t)k.na || (uint64_t)y >= (uint64_t)k.nb) return kOrderBins - 1;
    const int64_t* oa = k.oa;
    const int64_t* ob = k.ob;
    const unsigned long long c =
        (unsigned long long)(oa[x + 1] - oa[x]) * (unsigned long long)(ob[y + 1] - ob[y]);
    if (c == 0ull) return kOrderBins - 1;
    const int e = 63 - __clzll((long long)c);
    const int f = e >= 2 ? (int)((c >> (e - 2)) & 3ull) : (int)((c << (2 - e)) & 3ull);
    return kOrderBins - 1 - (4 * e + f);
}

__global__ void __launch_bounds__(256) order_hist_kernel(OrderKey key, int64_t npairs,
                                                         unsigned long long* hist) {
    __shared__ unsigned long long h[kOrderBins];
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) h[i] = 0ull;
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < npairs; w += stride)
        atomicAdd(&h[cell_class(key, w)], 1ull);
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// hist (class counts) -> cursor (first slot of each class), in place.
__global__ void order_scan_kernel(unsigned long long* hist) {
    if (threadIdx.x != 0) return;
    unsigned long long run = 0ull;
    for (int i = 0; i < kOrderBins; ++i) {
        const unsigned long long v = hist[i];
        hist[i] = run;
        run += v;
    }
}

// Each block takes chunks of kItems * blockDim.x pairs: ranks inside the
// chunk by shared-memory counters, then one global reservation per class.
constexpr int kItems = 8;

__global__ void __launch_bounds__(256) order_scatter_kernel(OrderKey key, int64_t npairs,
                                                            unsigned long long* cursor,
                                                            int64_t* order) {
    __shared__ unsigned cnt[kOrderBins];
    __shared__ unsigned long long base[kOrderBins];
    const int64_t chunk = (int64_t)blockDim.x * kItems;
    for (int64_t c0 = (int64_t)blockIdx.x * chunk; c0 < npairs; c0 += (int64_t)gridDim.x * chunk) {
        for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) cnt[i] = 0u;
        __syncthreads();
        int cls[kItems];
        unsigned rank[kItems];
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int64_t w = c0 + (int64_t)k * blockDim.x + threadIdx.x;
            cls[k] = 0;
            rank[k] = 0u;
            if (w < npairs) {
                cls[k] = cell_class(key, w);
                rank[k] = atomicAdd(&cnt[cls[k]], 1u);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x)
            if (cnt[i]) base[i] = atomicAdd(&cursor[i], (unsigned long long)cnt[i]);
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kItems; ++k) {
            const int64_t w = c0 + (int64_t)k * blockDim.x + threadIdx.x;
            if (w < npairs) order[base[cls[k]] + rank[k]] = w;
        }
        __syncthreads();
    }
}

}  // namespace

cudaError_t launch_order_pairs(const int64_t* pairs, int64_t npairs, const int64_t* offs_a, int64_t na,
                               const int64_t* offs_b, int64_t nb, int64_t* order, unsigned long long* bins,
                               int sms, cudaStream_t st) {
    if (npairs <= 0) return cudaSuccess;
    const OrderKey key{pairs, offs_a, offs_b, na, nb};
    const int threads = 256;
    const int64_t hist_blocks = std::min<int64_t>((int64_t)sms * 4, (npairs + threads - 1) / threads);
    const int64_t chunk = (int64_t)threads * kItems;
    const int64_t scat_blocks = std::min<int64_t>((int64_t)sms * 4, (npairs + chunk - 1) / chunk);
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(unsigned long long) * kOrderBins, st);
    if (e != cudaSuccess) return e;
    (void)cudaGetLastError();
    order_hist_kernel<<<(int)hist_blocks, threads, 0, st>>>(key, npairs, bins);
    order_scan_kernel<<<1, 32, 0, st>>>(bins);
    order_scatter_kernel<<<(int)scat_blocks, threads, 0, st>>>(key, npairs, bins, order);
    return cudaGetLastError();
}

}  // namespace twed
