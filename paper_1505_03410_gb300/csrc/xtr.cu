// The correlation pass of a GAP SAFE check as a standalone streaming kernel:
// c = X^T r and m = ||c||_inf for an FP32 design (Eq. (7) needs every
// |x_j^T rho|, the dual rescaling of Eq. (8) needs the maximum).
//
// The pass reads each column once and does 2 flops per 4 bytes: it is bound
// by HBM bandwidth.  Each warp owns U adjacent columns per step and issues
// all U * NG float4 loads of them (streaming, evict-first) before it reduces,
// so every SM keeps enough bytes in flight to cover the DRAM latency; r sits
// in registers (granule g = lane + 32 k of the warp).  The grid is persistent
// (CTAs per SM from the occupancy calculator times the SM count) and strides
// over the column groups.
#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "internal.h"

namespace lassogs {
namespace {

constexpr int kXtrThreads = 256;

__device__ __forceinline__ float4 ld_stream4(const float* p) {
  return __ldcs(reinterpret_cast<const float4*>(p));
}

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

template <int NG, int U>
__global__ void __launch_bounds__(kXtrThreads) xtr_f32_kernel(const float* __restrict__ X, long long ldx, int n, int p,
                                                              const float* __restrict__ r, float* __restrict__ c,
                                                              unsigned* __restrict__ cmax_bits) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ld4 = (n + 3) >> 2;
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
  const long long gw = (long long)blockIdx.x * (kXtrThreads / 32) + warp;
  const long long nw = (long long)gridDim.x * (kXtrThreads / 32);
  float mx = 0.f;
  for (long long j0 = gw * U; j0 < p; j0 += nw * U) {
    float4 x[U][NG];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long j = j0 + u;
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const int g = lane + 32 * k;
        x[u][k] = (j < p && g < ld4) ? ld_stream4(X + j * ldx + 4 * g) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    float acc[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      float s = 0.f;
#pragma unroll
      for (int k = 0; k < NG; ++k) {
        const float4 v = mask_tail(x[u][k], lane + 32 * k, n);
        s = __fmaf_rn(v.x, r4[k].x, s);
        s = __fmaf_rn(v.y, r4[k].y, s);
        s = __fmaf_rn(v.z, r4[k].z, s);
        s = __fmaf_rn(v.w, r4[k].w, s);
      }
      acc[u] = s;
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc[u] = __fadd_rn(acc[u], __shfl_xor_sync(0xffffffffu, acc[u], o));
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const long long j = j0 + u;
      if (j < p) {
        if (lane == u) c[j] = acc[u];
        mx = fmaxf(mx, fabsf(acc[u]));
      }
    }
  }
  // the maximum does not depend on the order in which warps report it
  if (lane == 0 && cmax_bits) atomicMax(cmax_bits, __float_as_uint(mx));
}

template <int NG, int U>
lasso_status launch_xtr(const float* X, int64_t n, int64_t p, int64_t ldx, const float* r, float* c, unsigned* cmax,
                        cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, xtr_f32_kernel<NG, U>, kXtrThreads, 0));
  if (per_sm < 1) per_sm = 1;
  const long long groups = (p + U - 1) / U;
  const long long need = (groups + (kXtrThreads / 32) - 1) / (kXtrThreads / 32);
  const int grid = (int)std::min<long long>((long long)sms * per_sm, need);
  xtr_f32_kernel<NG, U><<<grid, kXtrThreads, 0, st>>>(X, ldx, (int)n, (int)p, r, c, cmax);
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
  // NG float4 granules per lane cover n <= 128 NG rows; U * NG = 16 keeps
  // 8 KB of loads in flight per warp at every n
  if (n <= 128) return launch_xtr<1, 16>(X, n, p, ldx, r, c, cm, st);
  if (n <= 256) return launch_xtr<2, 8>(X, n, p, ldx, r, c, cm, st);
  if (n <= 512) return launch_xtr<4, 4>(X, n, p, ldx, r, c, cm, st);
  if (n <= 1024) return launch_xtr<8, 2>(X, n, p, ldx, r, c, cm, st);
  return launch_xtr<16, 1>(X, n, p, ldx, r, c, cm, st);
}
