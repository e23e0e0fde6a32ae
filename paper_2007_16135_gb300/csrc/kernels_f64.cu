// Double-precision instantiation of the TWED kernels.
#include "kernels.cuh"

namespace twed {

constexpr int kRmaxF64 = 4;

template <>
int rec_len<double>(int dim, int p) {
    int len = 0;
    TWED_DISPATCH(dim, p, (len = Rec<double, DIM_>::kLen));
    return len;
}
cudaError_t launch_records(const RecordsArgs<double>& a, cudaStream_t st) {
    return launch_records_t(a, st);
}
cudaError_t launch_coop(const CoopArgs<double>& a, int R, bool kahan, int blocks, int threads,
                        cudaStream_t st) {
    if (kahan) return cudaErrorNotSupported;  // compensation is an FP32 option
    return launch_coop_kh<double, false>(a, R, blocks, threads, st);
}
template <>
int coop_blocks_per_sm<double>(int dim, int p, int R, bool kahan, int threads) {
    (void)kahan;
    return coop_blocks_per_sm_kh<double, false>(dim, p, R, threads);
}
cudaError_t launch_pairs(const PairsArgs<double>& a, int blocks, int threads, cudaStream_t st) {
    return launch_pairs_t<double, kRmaxF64>(a, blocks, threads, st);
}
template <>
int pairs_blocks_per_sm<double>(int dim, int p, int threads) {
    return pairs_blocks_per_sm_t<double, kRmaxF64>(dim, p, threads);
}
template <>
int pairs_rmax_limit<double>() { return kRmaxF64; }

}  // namespace twed
