// C-ABI entry points of liblassogs: argument checking, defaults, the
// lambda grid of Sec. 3.3 and the thread-local error message.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>

#include "internal.h"

namespace lassogs {

namespace {
thread_local char g_msg[512] = "";
}

lasso_status set_error(lasso_status code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_msg, sizeof(g_msg), fmt, ap);
  va_end(ap);
  return code;
}

void clear_error() { g_msg[0] = '\0'; }

namespace {

lasso_status check_opts(const lasso_opts& o) {
  if (o.screen_period < 1) return set_error(LASSO_ERR_INVALID_ARG, "screen_period must be >= 1 (got %d)", o.screen_period);
  if (o.dual_point != 0 && o.dual_point != 1) return set_error(LASSO_ERR_INVALID_ARG, "dual_point must be 0 or 1");
  if (o.xtr_scope != 0 && o.xtr_scope != 1) return set_error(LASSO_ERR_INVALID_ARG, "xtr_scope must be 0 or 1");
  if (o.warm_start != 0 && o.warm_start != 1) return set_error(LASSO_ERR_INVALID_ARG, "warm_start must be 0 or 1");
  if (o.max_epochs < 0) return set_error(LASSO_ERR_INVALID_ARG, "max_epochs must be >= 0");
  if (!(o.gap_tol_rel >= 0.0) || !std::isfinite(o.gap_tol_rel))
    return set_error(LASSO_ERR_INVALID_ARG, "gap_tol_rel must be finite and >= 0");
  if (o.gemm_dtype != LASSO_BF16 && o.gemm_dtype != LASSO_F32)
    return set_error(LASSO_ERR_INVALID_ARG, "gemm_dtype must be LASSO_BF16 or LASSO_F32");
  if (o.batch_ctas_per_sm < 0 || o.batch_ctas_per_sm > 2)
    return set_error(LASSO_ERR_INVALID_ARG, "batch_ctas_per_sm must be 0, 1 or 2");
  if (o.gemm_tile_n != 0 && o.gemm_tile_n != 64 && o.gemm_tile_n != 128 && o.gemm_tile_n != 256)
    return set_error(LASSO_ERR_INVALID_ARG, "gemm_tile_n must be 0, 64, 128 or 256");
  if (o.batch_group < 0 || o.batch_group > 64)
    return set_error(LASSO_ERR_INVALID_ARG, "batch_group must lie in [0, 64]");
  if (o.batch_group > 1 && o.gemm_dtype != LASSO_F32)
    return set_error(LASSO_ERR_INVALID_ARG, "batch_group > 1 needs gemm_dtype = LASSO_F32");
  if (o.screen_rule != 0 && o.screen_rule != 1) return set_error(LASSO_ERR_INVALID_ARG, "screen_rule must be 0 or 1");
  if (o.refined_radius != 0 && o.refined_radius != 1)
    return set_error(LASSO_ERR_INVALID_ARG, "refined_radius must be 0 or 1");
  if (!(o.enet_alpha > 0.0 && o.enet_alpha <= 1.0)) return set_error(LASSO_ERR_INVALID_ARG, "enet_alpha must lie in (0, 1]");
  if (o.audit_bounds != 0 && o.audit_bounds != 1) return set_error(LASSO_ERR_INVALID_ARG, "audit_bounds must be 0 or 1");
  if (o.lockstep_pass != 0 && o.lockstep_pass != 1)
    return set_error(LASSO_ERR_INVALID_ARG, "lockstep_pass must be 0 or 1");
  return LASSO_OK;
}

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

lasso_status check_options(const lasso_opts& o) { return check_opts(o); }
}  // namespace lassogs

using namespace lassogs;

extern "C" {

void lasso_default_opts(lasso_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->screen_period = 10;
  o->dual_point = 0;
  o->xtr_scope = 0;
  o->warm_start = 1;
  o->max_epochs = 100000;
  o->gap_tol_rel = 1e-6;
  o->gemm_dtype = LASSO_BF16;
  o->enet_alpha = 1.0;
}

lasso_status lasso_lambda_grid(int32_t T, double delta, double* ratios_host) {
  clear_error();
  if (T < 1 || !(delta >= 0.0) || !std::isfinite(delta) || !ratios_host)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_lambda_grid: need T >= 1, finite delta >= 0, non-NULL output");
  for (int32_t t = 0; t < T; ++t)
    ratios_host[t] = (T == 1) ? 1.0 : std::pow(10.0, -delta * (double)t / (double)(T - 1));
  return LASSO_OK;
}

size_t lasso_path_workspace_size(int64_t n, int64_t p, lasso_dtype x_dtype, const lasso_opts* opts) {
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_default_opts(&o);
  if (check_opts(o) != LASSO_OK) return 0;
  // the FP32 design is used in place with its own leading dimension; the
  // size below assumes the tight one (n rounded up to 4)
  return path_workspace_size(n, p, x_dtype, (n + 3) / 4 * 4);
}

lasso_status lasso_path(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx, const double* y,
                        const double* ratios, int32_t T, const double* beta0, const lasso_opts* opts,
                        double* beta_out, uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                        void* stream) {
  clear_error();
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_default_opts(&o);
  lasso_status st = check_opts(o);
  if (st != LASSO_OK) return st;
  if (!X || !y || !ratios || !beta_out || !stats)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: X, y, lambda_ratios, beta_out and stats must be non-NULL");
  if (n < 1 || n > kMaxRows) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: need 1 <= n <= %lld (got %lld)", (long long)kMaxRows, (long long)n);
  if (p < 1 || p > (int64_t)INT32_MAX / 4) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: p out of range (got %lld)", (long long)p);
  if (T < 1) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: T must be >= 1");
  if (ldx < n) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: ldx (%lld) < n (%lld)", (long long)ldx, (long long)n);
  if (xt == LASSO_F32) {
    if (ldx % 4 != 0 || !aligned(X, 16))
      return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: an FP32 design needs ldx %% 4 == 0 and a 16-byte aligned base");
  } else if (xt == LASSO_F64) {
    if (!aligned(X, 8)) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: an FP64 design needs an 8-byte aligned base");
  } else {
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: x_dtype must be LASSO_F32 or LASSO_F64");
  }
  if (!aligned(y, 8) || !aligned(ratios, 8) || !aligned(beta_out, 8) || !aligned(stats, 8) ||
      (beta0 && !aligned(beta0, 8)) || (mask_out && !aligned(mask_out, 4)))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: misaligned vector argument");
  if (!ws || !aligned(ws, 256)) return set_error(LASSO_ERR_WORKSPACE, "lasso_path: workspace must be non-NULL and 256-byte aligned");
  const size_t need = path_workspace_size(n, p, xt, ldx);
  if (need == 0) return set_error(LASSO_ERR_INVALID_ARG, "lasso_path: unsupported sizes");
  if (ws_bytes < need)
    return set_error(LASSO_ERR_WORKSPACE, "lasso_path: workspace of %zu bytes < %zu required", ws_bytes, need);
  return path_launch(X, xt, n, p, ldx, y, ratios, T, beta0, o, beta_out, mask_out, stats, ws, ws_bytes,
                     static_cast<cudaStream_t>(stream));
}

size_t lasso_batch_workspace_size(int64_t n, int64_t p, int64_t B, const lasso_opts* opts) {
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_default_opts(&o);
  if (check_opts(o) != LASSO_OK) return 0;
  return batch_workspace_size(n, p, B, o.gemm_dtype == LASSO_BF16, o.batch_group, o.lockstep_pass == 1);
}

lasso_status lasso_batch(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                         const uint8_t* row_mask, int64_t ldm, int64_t B, const double* ratios, int32_t T,
                         const double* beta0, int64_t ldb0, const lasso_opts* opts, double* beta_out,
                         uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  lasso_opts o;
  if (opts) o = *opts;
  else lasso_default_opts(&o);
  lasso_status st = check_opts(o);
  if (st != LASSO_OK) return st;
  if (!X || !Y || !ratios || !beta_out || !stats)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: X, Y, lambda_ratios, beta_out and stats must be non-NULL");
  if (n < 1 || n > kMaxRows) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: need 1 <= n <= %lld", (long long)kMaxRows);
  if (p < 1 || p > (int64_t)INT32_MAX / 4) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: p out of range");
  if (B < 1 || B > (int64_t)INT32_MAX) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: B out of range");
  if (T < 1) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: T must be >= 1");
  if (ldx < n || ldx % 4 != 0 || !aligned(X, 16))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: X needs ldx >= n, ldx %% 4 == 0 and a 16-byte aligned base");
  if (ldy < n) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: ldy < n");
  if (row_mask && ldm < n) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: ldm < n");
  if (beta0 && ldb0 < p) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: ldb0 < p");
  if (!aligned(Y, 8) || !aligned(ratios, 8) || !aligned(beta_out, 8) || !aligned(stats, 8) ||
      (mask_out && !aligned(mask_out, 4)) || (beta0 && !aligned(beta0, 8)))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch: misaligned vector argument");
  if (!ws || !aligned(ws, 256)) return set_error(LASSO_ERR_WORKSPACE, "lasso_batch: workspace must be non-NULL and 256-byte aligned");
  return batch_launch(X, n, p, ldx, Y, ldy, row_mask, ldm, B, ratios, T, beta0, ldb0, o, beta_out, mask_out, stats, ws, ws_bytes,
                      static_cast<cudaStream_t>(stream));
}

lasso_status lasso_path_phase_cycles(const void* ws, uint64_t* cycles_host, void* stream) {
  clear_error();
  if (!ws || !aligned(ws, 256) || !cycles_host)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_path_phase_cycles: need a 256-byte aligned workspace and an output");
  return path_phase_cycles(ws, cycles_host, static_cast<cudaStream_t>(stream));
}

const char* lasso_last_error(void) { return g_msg; }

}  // extern "C"
