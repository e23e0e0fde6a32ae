// Handle state that translation units other than api.cu may use.
#pragma once

#include "../../include/twed.h"

namespace twed {
namespace detail {
// Records `msg` as the handle's last error and returns `st`.
twed_status_t set_error(twed_handle_t h, twed_status_t st, const char* msg);
int handle_sms(twed_handle_t h);
int handle_device(twed_handle_t h);
// twed_batch_f32_ex with a chosen launch shape: rows-per-lane cap `rmax`
// and resident blocks per SM `per_sm` (0: the defaults).
twed_status_t batch_f32_shaped(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                               const int64_t* d_pairs, int64_t npairs, int dim, float nu,
                               float lambda, int p, float* d_out, void* stream, int order,
                               int rmax, int per_sm);
int batch_f32_max_blocks_per_sm(int dim, int p);
// DTW of explicit pairs on the staged FP32 engine (compiled point layouts:
// twed::compiled_layout(dim, p)); timestamps may be NULL.
twed_status_t dtw_batch_f32_staged(twed_handle_t h, const twed_set_f32_t* A, const twed_set_f32_t* B,
                                   const int64_t* d_pairs, int64_t npairs, int dim, int p, float* d_out,
                                   void* stream);
int batch_f32_rmax_limit();
// The handle's grow-only device workspace, at least `bytes` long (nullptr
// and the handle's last error set on failure; a growth synchronizes the
// handle's stream first).
void* handle_workspace(twed_handle_t h, size_t bytes, twed_status_t* st);
void* handle_stream(twed_handle_t h);
// The handle's [live error, sticky error] words (device).
unsigned* handle_ctl(twed_handle_t h);
}  // namespace detail
}  // namespace twed
