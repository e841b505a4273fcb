// Host-side internals shared by the library's translation units.
#pragma once
#include <cstdarg>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/lassogs.h"

namespace lassogs {

constexpr int64_t kMaxRows = 2048;  // rows n supported by the register-resident residual

// records the thread-local message and returns code
lasso_status set_error(lasso_status code, const char* fmt, ...);
void clear_error();

// the option checks every entry point applies (message in lasso_last_error)
lasso_status check_options(const lasso_opts& o);

// time limit of the kernels' grid-barrier waits (20 s, or LASSOGS_WAIT_LIMIT_NS)
unsigned long long wait_limit_ns();

size_t path_workspace_size(int64_t n, int64_t p, lasso_dtype xt, int64_t ldx);
lasso_status path_launch(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx, const double* y,
                         const double* ratios, int32_t T, const double* beta0, const lasso_opts& o,
                         double* beta_out, uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                         cudaStream_t stream);

// the 8 phase counters of the last single-path launch on workspace ws
lasso_status path_phase_cycles(const void* ws, uint64_t* out_host, cudaStream_t stream);

// group: CTAs per problem (opts.batch_group; <= 1 for one CTA per problem)
size_t batch_workspace_size(int64_t n, int64_t p, int64_t B, bool lockstep, int group, bool pass);
lasso_status xtr_gemm_launch(const void* Xb, int64_t n, int64_t p, int64_t ldx, const void* Rb, int64_t ldr,
                             int64_t B, float* C, int64_t ldc, int* err_dev, cudaStream_t stream, int tile_n = 0);
lasso_status batch_launch(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                          const uint8_t* row_mask, int64_t ldm, int64_t B, const double* ratios, int32_t T,
                          const double* beta0, int64_t ldb0, const lasso_opts& o, double* beta_out,
                          uint32_t* mask_out, lasso_path_stats* stats,
                          void* ws, size_t ws_bytes, cudaStream_t stream);

}  // namespace lassogs

#define CUDA_TRY(call)                                                                                   \
  do {                                                                                                   \
    cudaError_t e_ = (call);                                                                             \
    if (e_ != cudaSuccess)                                                                               \
      return ::lassogs::set_error(LASSO_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));        \
  } while (0)
