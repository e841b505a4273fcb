// Device utilities: bounded grid barrier, mbarrier and bulk-copy (TMA) PTX
// wrappers, block reductions.  Every wait has a time limit read from the
// global nanosecond timer; on expiry the wait records LASSO_ERR_TIMEOUT in
// the control block and returns false so the kernel can unwind.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lassogs {

constexpr unsigned long long kWaitLimitNs = 20ull * 1000ull * 1000ull * 1000ull;  // 20 s
constexpr int kErrTimeout = 6;
constexpr int kErrNonfinite = 2;

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void set_error(int* err, int code) { atomicCAS(err, 0, code); }

__device__ __forceinline__ int ld_volatile(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned ld_volatile_u(const unsigned* p) { return *(volatile const unsigned*)p; }

// Sense-free generation barrier across all CTAs of a cooperative launch.
// count and gen live in global memory; *err is the shared error word.  A
// waiter gives up after limit_ns nanoseconds (recording kErrTimeout).  With
// leave_on_error a waiter also leaves as soon as another CTA has recorded an
// error, instead of waiting for the generation to turn: only for callers that
// stop using the barrier after a failed wait (the single path), because the
// CTAs that leave early no longer keep the arrivals of one barrier apart from
// those of the next.
// Returns false if the wait timed out or an error is pending.
static __device__ __noinline__ bool grid_sync(unsigned* count, unsigned* gen, int* err, unsigned nblocks,
                                              unsigned long long limit_ns = kWaitLimitNs,
                                              bool leave_on_error = false) {
  __syncthreads();
  __shared__ int s_ok;
  if (nblocks == 1) {  // a one-CTA group: the block barrier is the whole barrier
    if (threadIdx.x == 0) s_ok = ld_volatile(err) == 0;
    __syncthreads();
    return s_ok != 0;
  }
  if (threadIdx.x == 0) {
    int ok = 1;
    unsigned my_gen = ld_volatile_u(gen);
    __threadfence();
    unsigned arrived = atomicAdd(count, 1u);
    if (arrived == nblocks - 1) {
      *(volatile unsigned*)count = 0u;
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned long long t0 = global_ns();
      unsigned spins = 0;
      while (ld_volatile_u(gen) == my_gen) {
        if (++spins > 64) __nanosleep(200);
        if (leave_on_error && (spins & 15u) == 0u && ld_volatile(err) != 0) {
          ok = 0;
          break;
        }
        if ((spins & 15u) == 0u && global_ns() - t0 > limit_ns) {
          set_error(err, kErrTimeout);
          ok = 0;
          break;
        }
      }
    }
    __threadfence();
    if (ld_volatile(err) != 0) ok = 0;
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// ---------------------------------------------------------------- mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait on an mbarrier phase
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (!mbar_try_wait(bar, parity)) {
    if ((++spins & 1023u) == 0u) {
      if (global_ns() - t0 > kWaitLimitNs) {
        set_error(err, kErrTimeout);
        return false;
      }
      if (ld_volatile(err) != 0) return false;
    }
  }
  return true;
}

// 1-D bulk copy global -> shared, completion counted on bar (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst_smem)),
      "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void named_bar_sync(int id, int nthreads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// ---------------------------------------------------------------- block reductions (FP64)
// Deterministic: fixed tree for a fixed blockDim.  buf: >= 32 doubles of smem.
__device__ __forceinline__ double warp_sum_d(double v) {
  for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double block_sum_d(double v, double* buf) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum_d(v);
  __syncthreads();
  if (lane == 0) buf[w] = v;
  __syncthreads();
  double r = (threadIdx.x < nw) ? buf[threadIdx.x] : 0.0;
  if (w == 0) r = warp_sum_d(r);
  if (threadIdx.x == 0) buf[0] = r;
  __syncthreads();
  r = buf[0];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_sum_i(int v, int* buf) {
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = __reduce_add_sync(0xffffffffu, v);
  __syncthreads();
  if (lane == 0) buf[w] = v;
  __syncthreads();
  int r = (threadIdx.x < nw) ? buf[threadIdx.x] : 0;
  if (w == 0) r = __reduce_add_sync(0xffffffffu, r);
  if (threadIdx.x == 0) buf[0] = r;
  __syncthreads();
  r = buf[0];
  __syncthreads();
  return r;
}

}  // namespace lassogs
