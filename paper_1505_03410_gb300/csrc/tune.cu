// lasso_batch_tune: picks the launch shape of the batched solver by timing.
//
// The candidates differ only in how the work is laid out on the GPU: where
// the first check of each lambda gets X^T rho (per-CTA FP32 passes or one
// split-BF16 tensor-core product per lambda), how many solver CTAs share an
// SM (two, at 128 registers per thread, or one), the N tile of the
// tensor-core product, whether a lockstep batch takes a product per lambda or
// per coordinate pass, and how many CTAs work on one problem (1, 8, 16 or
// 32; a group larger than the CTAs that rebuild its snapshots runs the
// coordinate chain in Gram form, as the single path does).
// Every candidate makes the same screening decisions (each equals the FP64
// test's), so the choice changes the time, never the result.  Each candidate
// solves the same sample of problems over the first lambdas of the grid
// twice (a warm-up, then a run timed with CUDA events on the caller's
// stream), and the fastest is returned.  A group too large for the resident
// CTAs of this GPU is skipped (its time is reported as -1).
#include <algorithm>
#include <cstring>

#include <cuda_runtime.h>

#include "internal.h"

namespace lassogs {
namespace {

struct Candidate {
  int32_t dtype, per_sm, tile_n, group, pass;
};

constexpr Candidate kCandidates[] = {
    {LASSO_F32, 2, 0, 1, 0},    {LASSO_F32, 1, 0, 1, 0},    {LASSO_BF16, 2, 128, 1, 0}, {LASSO_BF16, 1, 128, 1, 0},
    {LASSO_BF16, 2, 256, 1, 0}, {LASSO_BF16, 1, 256, 1, 0}, {LASSO_F32, 2, 0, 8, 0},    {LASSO_F32, 2, 0, 32, 0},
    {LASSO_F32, 1, 0, 16, 0},   {LASSO_BF16, 2, 128, 1, 1}, {LASSO_BF16, 1, 128, 1, 1},
};
constexpr int kNumCandidates = sizeof(kCandidates) / sizeof(kCandidates[0]);

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct TuneLayout {
  size_t solver, beta, stats, total;
};

TuneLayout tune_layout(int64_t n, int64_t p, int64_t sample, int32_t lambdas) {
  TuneLayout t{};
  // the solver's workspace: the largest any candidate shape needs
  size_t a = 0;
  for (const Candidate& c : kCandidates) {
    lasso_opts o;
    lasso_default_opts(&o);
    o.gemm_dtype = c.dtype;
    o.batch_ctas_per_sm = c.per_sm;
    o.gemm_tile_n = c.tile_n;
    o.batch_group = c.group;
    o.lockstep_pass = c.pass;
    const size_t s = lasso_batch_workspace_size(n, p, sample, &o);
    if (s == 0) return t;
    a = std::max(a, s);
  }
  t.solver = 0;
  t.beta = a256(a);
  t.stats = t.beta + a256(sizeof(double) * (size_t)sample * (size_t)lambdas * (size_t)p);
  t.total = t.stats + a256(sizeof(lasso_path_stats) * (size_t)sample * (size_t)lambdas);
  return t;
}

}  // namespace
}  // namespace lassogs

using namespace lassogs;

extern "C" {

int32_t lasso_batch_tune_candidates(void) { return kNumCandidates; }

size_t lasso_batch_tune_workspace_size(int64_t n, int64_t p, int64_t sample, int32_t lambdas) {
  if (sample < 1 || lambdas < 1) return 0;
  return tune_layout(n, p, sample, lambdas).total;
}

lasso_status lasso_batch_tune(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                              const uint8_t* row_mask, int64_t ldm, int64_t B, const double* ratios, int32_t T,
                              const double* beta0, int64_t ldb0, const lasso_opts* opts, int32_t sample,
                              int32_t lambdas, lasso_opts* tuned, float* times_ms, void* ws, size_t ws_bytes,
                              void* stream) {
  clear_error();
  if (!tuned) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch_tune: tuned must be non-NULL");
  if (sample < 1 || sample > B || lambdas < 1 || lambdas > T)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch_tune: need 1 <= sample <= B and 1 <= lambdas <= T");
  lasso_opts base;
  if (opts) base = *opts;
  else lasso_default_opts(&base);
  const TuneLayout L = tune_layout(n, p, sample, lambdas);
  if (L.total == 0) return set_error(LASSO_ERR_INVALID_ARG, "lasso_batch_tune: unsupported sizes");
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0 || ws_bytes < L.total)
    return set_error(LASSO_ERR_WORKSPACE, "lasso_batch_tune: workspace needs %zu bytes, 256-byte aligned", L.total);
  char* w = static_cast<char*>(ws);
  double* beta = reinterpret_cast<double*>(w + L.beta);
  lasso_path_stats* stats = reinterpret_cast<lasso_path_stats*>(w + L.stats);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  int best = -1;
  float best_ms = 0.f;
  lasso_status status = LASSO_OK;
  for (int c = 0; c < kNumCandidates && status == LASSO_OK; ++c) {
    lasso_opts o = base;
    o.gemm_dtype = kCandidates[c].dtype;
    o.batch_ctas_per_sm = kCandidates[c].per_sm;
    o.gemm_tile_n = kCandidates[c].tile_n;
    o.batch_group = kCandidates[c].group;
    o.lockstep_pass = kCandidates[c].pass;
    for (int rep = 0; rep < 2 && status == LASSO_OK; ++rep) {
      if (rep == 1 && cudaEventRecord(e0, st) != cudaSuccess) status = set_error(LASSO_ERR_CUDA, "event record failed");
      if (status == LASSO_OK)
        status = lasso_batch(X, n, p, ldx, Y, ldy, row_mask, ldm, sample, ratios, lambdas, beta0, ldb0, &o, beta,
                             nullptr, stats, w + L.solver, L.beta, stream);
      if (status == LASSO_OK && rep == 1 && cudaEventRecord(e1, st) != cudaSuccess)
        status = set_error(LASSO_ERR_CUDA, "event record failed");
    }
    if (status == LASSO_ERR_INVALID_ARG && kCandidates[c].group > 1) {  // the group does not fit this GPU
      status = LASSO_OK;
      if (times_ms) times_ms[c] = -1.f;
      continue;
    }
    if (status != LASSO_OK) break;
    float ms = 0.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
      status = set_error(LASSO_ERR_CUDA, "timing a candidate failed");
      break;
    }
    if (times_ms) times_ms[c] = ms;
    if (best < 0 || ms < best_ms) {
      best = c;
      best_ms = ms;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (status != LASSO_OK) return status;
  *tuned = base;
  tuned->gemm_dtype = kCandidates[best].dtype;
  tuned->batch_ctas_per_sm = kCandidates[best].per_sm;
  tuned->gemm_tile_n = kCandidates[best].tile_n;
  tuned->batch_group = kCandidates[best].group;
  tuned->lockstep_pass = kCandidates[best].pass;
  return LASSO_OK;
}

}  // extern "C"
