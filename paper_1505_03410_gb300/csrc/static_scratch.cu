// lasso_path_static: the Lasso path without a caller-supplied workspace.
//
// Some callers cannot allocate device memory at the point where they solve:
// plug-ins of a host application that owns the whole device heap through its
// own pool (a cudaMalloc of theirs would fail or fragment that pool), and
// real-time callers that are not allowed the latency or the failure modes of
// an allocation on their hot path.  For them this entry point takes its
// scratch from one fixed array in device global memory that the library
// declares itself.  The paper has no counterpart.
//
// Properties a caller must know:
//   - The array holds kStaticScratchBytes (32 MiB) on every GPU that loads the
//     library, for as long as the library stays loaded (until process exit).
//   - Problems whose workspace exceeds it are rejected with
//     LASSO_ERR_INVALID_ARG.
//   - The first call on each device looks up the array's device address with
//     cudaGetSymbolAddress while that device is current; make that first call
//     before any stream capture.  Later calls on the device reuse the address.
//   - Every call on a device uses the same array.  Calls whose work overlaps
//     on the GPU (different streams, or several host threads) race on it and
//     give wrong results; serialise them.  Each call clears the parts that
//     must start at zero (the control block and the per-CTA counters) before
//     its kernels run, so the contents left by the previous call do no harm.
//   - Nothing here calls cudaMalloc, cudaFree or any allocating routine.
#include <cstdint>
#include <mutex>

#include <cuda_runtime.h>

#include "internal.h"

namespace lassogs {
namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

// The scratch array: a device-side global, not host memory.  Host code must
// never pass its name to a kernel; it uses the address looked up below.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_static_scratch on the current device (looked up once).
lasso_status scratch_address(void** out) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return set_error(LASSO_ERR_CUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (g_scratch_addr[dev] == nullptr) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr)
      return set_error(LASSO_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s",
                       cudaGetErrorString(e));
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return LASSO_OK;
}

}  // namespace
}  // namespace lassogs

using namespace lassogs;

extern "C" lasso_status lasso_path_static(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx,
                                          const double* y, const double* ratios, int32_t T, const double* beta0,
                                          const lasso_opts* opts, double* beta_out, uint32_t* mask_out,
                                          lasso_path_stats* stats, void* stream) {
  clear_error();
  // the size lasso_path will check, with the caller's ldx; 0 means invalid
  // sizes, which lasso_path then reports with the exact reason
  const size_t need = path_workspace_size(n, p, xt, ldx);
  if (need > kStaticScratchBytes)
    return set_error(LASSO_ERR_INVALID_ARG,
                     "lasso_path_static: this problem needs %zu bytes of scratch, more than the %zu bytes of the "
                     "static array; use lasso_path with a workspace",
                     need, kStaticScratchBytes);
  void* scratch = nullptr;
  const lasso_status st = scratch_address(&scratch);
  if (st != LASSO_OK) return st;
  return lasso_path(X, xt, n, p, ldx, y, ratios, T, beta0, opts, beta_out, mask_out, stats, scratch,
                    kStaticScratchBytes, stream);
}
