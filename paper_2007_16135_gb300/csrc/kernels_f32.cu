// Single-precision instantiation of the TWED kernels.
#include "kernels.cuh"

namespace twed {

constexpr int kRmaxF32 = 8;

template <>
int rec_len<float>(int dim, int p) {
    int len = 0;
    TWED_DISPATCH(dim, p, (len = Rec<float, DIM_>::kLen));
    return len;
}
cudaError_t launch_records(const RecordsArgs<float>& a, cudaStream_t st) {
    return launch_records_t(a, st);
}
cudaError_t launch_coop(const CoopArgs<float>& a, int R, bool kahan, int blocks, int threads,
                        cudaStream_t st) {
    return kahan ? launch_coop_kh<float, true>(a, R, blocks, threads, st)
                 : launch_coop_kh<float, false>(a, R, blocks, threads, st);
}
template <>
int coop_blocks_per_sm<float>(int dim, int p, int R, bool kahan, int threads) {
    return kahan ? coop_blocks_per_sm_kh<float, true>(dim, p, R, threads)
                 : coop_blocks_per_sm_kh<float, false>(dim, p, R, threads);
}
cudaError_t launch_pairs(const PairsArgs<float>& a, int blocks, int threads, cudaStream_t st) {
    return launch_pairs_t<float, kRmaxF32>(a, blocks, threads, st);
}
template <>
int pairs_blocks_per_sm<float>(int dim, int p, int threads) {
    return pairs_blocks_per_sm_t<float, kRmaxF32>(dim, p, threads);
}
template <>
int pairs_rmax_limit<float>() { return kRmaxF32; }
cudaError_t launch_band(const CoopArgs<float>& a, int R, bool kahan, int blocks, int warps,
                        cudaStream_t st) {
    return kahan ? launch_band_kh<true>(a, R, blocks, warps, st)
                 : launch_band_kh<false>(a, R, blocks, warps, st);
}
int band_blocks_per_sm(int dim, int p, int R, bool kahan, int warps) {
    return kahan ? band_blocks_per_sm_kh<true>(dim, p, R, warps)
                 : band_blocks_per_sm_kh<false>(dim, p, R, warps);
}
cudaError_t records_preload_f32(int dim, int p) {
    cudaFuncAttributes fa{};
    cudaError_t e = cudaSuccess;
    TWED_DISPATCH(dim, p, (e = cudaFuncGetAttributes(&fa, records_kernel<float, DIM_, P_>)));
    return e;
}
bool compiled_layout(int dim, int p) {
    int d = 0;
    TWED_DISPATCH(dim, p, (d = DIM_));
    return d > 0;
}

}  // namespace twed

namespace twed {
cudaError_t launch_zero_diag(void* out, bool f64, int64_t n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int blocks = (int)((n + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    if (f64) zero_diag_kernel<double><<<blocks, 256, 0, st>>>((double*)out, n);
    else zero_diag_kernel<float><<<blocks, 256, 0, st>>>((float*)out, n);
    return cudaGetLastError();
}
}  // namespace twed
