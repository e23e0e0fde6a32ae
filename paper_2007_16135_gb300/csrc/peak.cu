// Issue-rate microbenchmarks for the roofline denominators of the ALU-bound
// kernels: independent FP32 FFMA (or FP64 DFMA) chains on every SM, or
// chains of a 32-bit xor and max (the integer ALU pipe the LCS recurrence
// runs on).
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/twed.h"
#include "handle.h"

namespace {

constexpr int kChains = 8;
constexpr int kThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kThreads) fma_chain_kernel(int iters, T a, T b, T* out) {
    T x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (T)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = x[c] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    // never true for the arguments the host passes; keeps the chains live
    if (s == (T)-12345.0) out[blockIdx.x] = s;
}

// Two integer operations per chain and iteration: x = max(x ^ a, b).
__global__ void __launch_bounds__(kThreads) ialu_chain_kernel(int iters, int a, int b, int* out) {
    int x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (int)threadIdx.x * 7 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = max(x[c] ^ a, b);
    }
    int s = 0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s ^= x[c];
    // never true for the arguments the host passes; keeps the chains live
    if (s == -12345) out[blockIdx.x] = s;
}

struct Ialu {};

template <typename T>
struct Chain {
    static constexpr double kOpsPerIter = 1.0;
    static void* fn() { return (void*)fma_chain_kernel<T>; }
    static int iters() { return sizeof(T) == 4 ? 1 << 14 : 1 << 9; }
    static void launch(int blocks, int it, void* out) {
        fma_chain_kernel<T><<<blocks, kThreads>>>(it, (T)0.999999, (T)1e-7, (T*)out);
    }
};

template <>
struct Chain<Ialu> {
    static constexpr double kOpsPerIter = 2.0;
    static void* fn() { return (void*)ialu_chain_kernel; }
    static int iters() { return 1 << 14; }
    static void launch(int blocks, int it, void* out) {
        ialu_chain_kernel<<<blocks, kThreads>>>(it, 0x5a5a5a5a, -1000000, (int*)out);
    }
};

template <typename T>
twed_status_t run(twed_handle_t h, double* ops_per_s) {
    const int sms = twed::detail::handle_sms(h);
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, Chain<T>::fn(), kThreads, 0) != cudaSuccess)
        per_sm = 4;
    const int blocks = sms * std::max(1, per_sm);
    const int iters = Chain<T>::iters();
    void* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    twed_status_t st = TWED_OK;
    float best = 1e30f;
    if (cudaMalloc(&out, sizeof(double) * blocks) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        st = twed::detail::set_error(h, TWED_ERR_CUDA, "peak benchmark setup failed");
    }
    for (int rep = 0; rep < 4 && st == TWED_OK; ++rep) {
        cudaEventRecord(e0, nullptr);
        Chain<T>::launch(blocks, iters, out);
        cudaEventRecord(e1, nullptr);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            st = twed::detail::set_error(h, TWED_ERR_CUDA, "peak benchmark launch failed");
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);  // first run is a warm-up
    }
    if (st == TWED_OK)
        *ops_per_s = (double)blocks * kThreads * kChains * (double)iters * Chain<T>::kOpsPerIter / (best / 1e3);
    if (out) cudaFree(out);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return st;
}

}  // namespace

extern "C" twed_status_t twed_pipe_peak(twed_handle_t h, int kind, double* ops_per_s) {
    if (!h || !ops_per_s) return TWED_ERR_INVALID_ARG;
    if (kind == TWED_PEAK_FFMA32) return run<float>(h, ops_per_s);
    if (kind == TWED_PEAK_DFMA64) return run<double>(h, ops_per_s);
    if (kind == TWED_PEAK_IALU32) return run<Ialu>(h, ops_per_s);
    return twed::detail::set_error(h, TWED_ERR_INVALID_ARG, "unknown peak kind");
}
