// The correlation pass of a GAP SAFE check as a standalone streaming kernel:
// c = X^T r and m = ||c||_inf for an FP32 design (Eq. (7) needs every
// |x_j^T rho|, the dual rescaling of Eq. (8) needs the maximum).
//
// The pass reads each column once and does 2 flops per 4 bytes: it is bound
// by HBM bandwidth.  Columns stream through shared memory by TMA: in each CTA
// one producer thread issues 1-D bulk copies (cp.async.bulk, one per column,
// its first 4 ceil(n/4) floats) of a block of columns into a 4-stage ring
// guarded by mbarriers, and 8 consumer warps take the columns of a stage one
// per warp, with r in registers (granule g = lane + 32 k).  The copy engine
// keeps up to the whole ring (about 96 KB) in flight per CTA without using
// the SM's outstanding-load slots, which is what limited a load-based
// version.  Two CTAs per SM, grid = 2 x SMs, each striding over the blocks.
// Every wait is bounded by the global timer; after a timeout the producer
// waits (bounded) for its copies in flight before the CTA exits, and the
// maximum is reported as NaN.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "device_util.cuh"
#include "internal.h"

namespace lassogs {
namespace {

constexpr int kConsumerWarps = 8;
constexpr int kXtrThreads = (kConsumerWarps + 1) * 32;
constexpr int kXStages = 4;
constexpr int kStageTarget = 24576;  // bytes of columns per stage (a whole number of columns)

// rows >= n of the last granule are padding of the caller's buffer: zero them
__device__ __forceinline__ float4 mask_tail(float4 v, int g, int n) {
  const int r = 4 * g;
  if (r + 3 >= n) {
    if (r + 0 >= n) v.x = 0.f;
    if (r + 1 >= n) v.y = 0.f;
    if (r + 2 >= n) v.z = 0.f;
    if (r + 3 >= n) v.w = 0.f;
  }
  return v;
}

// wait on an mbarrier phase with only the time limit (used to drain copies
// in flight after an error, when the error word already says "stop")
__device__ __forceinline__ void drain_wait(uint64_t* bar, unsigned parity) {
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > kWaitLimitNs) return;
}

template <int NG>
__global__ void __launch_bounds__(kXtrThreads, 2)
    xtr_f32_kernel(const float* __restrict__ X, long long ldx, int n, int p, int cols_per_stage,
                   const float* __restrict__ r, float* __restrict__ c, unsigned* __restrict__ cmax_bits) {
  extern __shared__ __align__(128) unsigned char xsm[];
  __shared__ __align__(8) uint64_t full[kXStages], empty[kXStages];
  __shared__ int s_err;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ld4 = (n + 3) >> 2;
  const unsigned col_bytes = 16u * (unsigned)ld4;
  const long long nblocks = (p + cols_per_stage - 1) / cols_per_stage;
  if (threadIdx.x == 0) {
    for (int s = 0; s < kXStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], kConsumerWarps);
    }
    s_err = 0;
    fence_mbar_init();
  }
  __syncthreads();
  if (warp == kConsumerWarps) {
    if (lane == 0) {  // producer
      long long issued = 0;
      for (long long blk = blockIdx.x; blk < nblocks; blk += gridDim.x, ++issued) {
        const int s = (int)(issued % kXStages);
        if (issued >= kXStages && !mbar_wait(&empty[s], (unsigned)(((issued / kXStages) - 1) & 1), &s_err)) break;
        const long long j0 = blk * cols_per_stage;
        const int cols = (int)min((long long)cols_per_stage, (long long)p - j0);
        unsigned char* dst = xsm + (size_t)s * cols_per_stage * col_bytes;
        mbar_arrive_expect_tx(&full[s], (unsigned)cols * col_bytes);
        for (int cc = 0; cc < cols; ++cc)
          bulk_g2s(dst + (size_t)cc * col_bytes, X + (j0 + cc) * ldx, col_bytes, &full[s]);
      }
      if (ld_volatile(&s_err) != 0)  // copies still in flight land before the CTA exits
        for (long long k = max(0ll, issued - kXStages); k < issued; ++k)
          drain_wait(&full[k % kXStages], (unsigned)((k / kXStages) & 1));
    }
  } else {  // consumers
    float4 r4[NG];
#pragma unroll
    for (int k = 0; k < NG; ++k) {
      const int g = lane + 32 * k;
      r4[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (4 * g + 3 < n) {
        r4[k] = __ldg(reinterpret_cast<const float4*>(r) + g);
      } else if (g < ld4) {  // the ragged last granule: only the n entries of r are read
        const int i = 4 * g;
        r4[k].x = __ldg(r + i);
        if (i + 1 < n) r4[k].y = __ldg(r + i + 1);
        if (i + 2 < n) r4[k].z = __ldg(r + i + 2);
      }
    }
    float mx = 0.f;
    long long it = 0;
    for (long long blk = blockIdx.x; blk < nblocks; blk += gridDim.x, ++it) {
      const int s = (int)(it % kXStages);
      if (!mbar_wait(&full[s], (unsigned)((it / kXStages) & 1), &s_err)) break;
      const long long j0 = blk * cols_per_stage;
      const int cols = (int)min((long long)cols_per_stage, (long long)p - j0);
      const unsigned char* base = xsm + (size_t)s * cols_per_stage * col_bytes;
      for (int cc = warp; cc < cols; cc += kConsumerWarps) {
        const float4* col = reinterpret_cast<const float4*>(base + (size_t)cc * col_bytes);
        float acc = 0.f;
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const int g = lane + 32 * k;
          if (g < ld4) {
            const float4 v = mask_tail(col[g], g, n);
            acc = __fmaf_rn(v.x, r4[k].x, acc);
            acc = __fmaf_rn(v.y, r4[k].y, acc);
            acc = __fmaf_rn(v.z, r4[k].z, acc);
            acc = __fmaf_rn(v.w, r4[k].w, acc);
          }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
        if (lane == 0) c[j0 + cc] = acc;
        mx = fmaxf(mx, fabsf(acc));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
    // the maximum does not depend on the order in which warps report it
    if (lane == 0 && cmax_bits) atomicMax(cmax_bits, __float_as_uint(mx));
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_err != 0 && cmax_bits) atomicMax(cmax_bits, 0x7fc00000u);  // NaN: a wait timed out
}

template <int NG>
lasso_status launch_xtr(const float* X, int64_t n, int64_t p, int64_t ldx, const float* r, float* c, unsigned* cmax,
                        cudaStream_t st) {
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int ld4 = (int)((n + 3) / 4);
  const int col_bytes = 16 * ld4;
  const int cols = std::max(1, kStageTarget / col_bytes);
  const size_t smem = (size_t)kXStages * cols * col_bytes;
  CUDA_TRY(cudaFuncSetAttribute(xtr_f32_kernel<NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long blocks = (p + cols - 1) / cols;
  const int grid = (int)std::min<long long>(2ll * sms, blocks);
  xtr_f32_kernel<NG><<<grid, kXtrThreads, smem, st>>>(X, ldx, (int)n, (int)p, cols, r, c, cmax);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

}  // namespace
}  // namespace lassogs

using namespace lassogs;

extern "C" lasso_status lasso_correlations_f32(const float* X, int64_t n, int64_t p, int64_t ldx, const float* r,
                                               float* c, float* cmax, void* stream) {
  clear_error();
  if (!X || !r || !c) return set_error(LASSO_ERR_INVALID_ARG, "lasso_correlations_f32: NULL argument");
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_correlations_f32: need 1 <= n <= %lld and p >= 1",
                     (long long)kMaxRows);
  if (ldx < n || ldx % 4 != 0 || (reinterpret_cast<uintptr_t>(X) & 15u) || (reinterpret_cast<uintptr_t>(r) & 15u))
    return set_error(LASSO_ERR_INVALID_ARG,
                     "lasso_correlations_f32: X needs ldx >= n, ldx %% 4 == 0, X and r 16-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  unsigned* cm = reinterpret_cast<unsigned*>(cmax);
  if (cm) CUDA_TRY(cudaMemsetAsync(cm, 0, sizeof(unsigned), st));
  // NG float4 granules per lane cover n <= 128 NG rows
  if (n <= 128) return launch_xtr<1>(X, n, p, ldx, r, c, cm, st);
  if (n <= 256) return launch_xtr<2>(X, n, p, ldx, r, c, cm, st);
  if (n <= 512) return launch_xtr<4>(X, n, p, ldx, r, c, cm, st);
  if (n <= 1024) return launch_xtr<8>(X, n, p, ldx, r, c, cm, st);
  return launch_xtr<16>(X, n, p, ldx, r, c, cm, st);
}
