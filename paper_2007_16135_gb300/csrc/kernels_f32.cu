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
cudaError_t launch_coop(const CoopArgs<float>& a, int R, int blocks, int threads, cudaStream_t st) {
    return launch_coop_t(a, R, blocks, threads, st);
}
template <>
int coop_blocks_per_sm<float>(int dim, int p, int R, int threads) {
    return coop_blocks_per_sm_t<float>(dim, p, R, threads);
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
