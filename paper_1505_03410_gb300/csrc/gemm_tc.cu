// Batched correlations C = X^T R on the 5th-generation tensor cores.
//
// X is the n x p design and R holds B residuals (n x B), both stored
// column-major in BF16, so both GEMM operands are K-major (K = n).  C is
// p x B FP32, column-major (problem b's correlations are contiguous).
//
// One CTA computes a 128 x BN tile of C:
//   warp 0  (one thread)  TMA producer: 2-D tiled bulk-tensor copies of a
//                         128 x 64 tile of X^T and a BN x 64 tile of R^T per
//                         stage, 128-byte swizzle, into a kStages ring
//   warp 1  (one thread)  MMA issuer: tcgen05.mma kind::f16 (BF16 x BF16 ->
//                         FP32) into a TMEM accumulator of BN columns, four
//                         K = 16 steps per stage; tcgen05.commit frees a stage
//   warps 0-3             epilogue: tcgen05.ld of the accumulator (each warp
//                         its 32 TMEM lanes = 32 rows of the tile) and
//                         coalesced stores of C
// Every wait is bounded by the global timer; a timeout sets *err and the CTA
// still releases its TMEM before returning.
#include <cstdint>
#include <cstring>
#include <mutex>

#include <cuda.h>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "internal.h"

namespace lassogs {
namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // one 128-byte swizzle row of BF16
constexpr int kStages = 4;
constexpr int kGemmThreads = 128;

struct GemmSmem {
  uint64_t full[kStages];
  uint64_t empty[kStages];
  uint64_t done;
  uint32_t tmem_base;
};

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major tile with 128-byte swizzle:
// rows of 128 bytes, 8-row atoms 1024 bytes apart (stride byte offset).
__device__ __forceinline__ uint64_t smem_desc_sw128(const void* tile) {
  const uint64_t addr = smem_u32(tile);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;          // start address
  d |= (uint64_t)1 << 16;                // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;      // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                // descriptor version (sm_100 family)
  d |= (uint64_t)2 << 61;                // layout: 128-byte swizzle
  return d;
}

// Instruction descriptor, kind::f16: BF16 A and B, FP32 accumulator,
// both operands K-major, M = 128, N = bn.
__host__ __device__ constexpr uint32_t instr_desc_bf16(int bn) {
  return (1u << 4)                       // D format: F32
         | (1u << 7)                     // A format: BF16
         | (1u << 10)                    // B format: BF16
         | ((uint32_t)(bn >> 3) << 17)   // N >> 3
         | ((uint32_t)(kBM >> 4) << 24); // M >> 4
}

template <int BN>
__global__ void __launch_bounds__(kGemmThreads, 1)
    xtr_gemm_kernel(const __grid_constant__ CUtensorMap map_x, const __grid_constant__ CUtensorMap map_r, int n,
                    int p, int B, float* __restrict__ C, long long ldc, int* err) {
  extern __shared__ __align__(1024) unsigned char gsm_raw[];
  // 1024-byte aligned stage buffers (swizzle atoms)
  unsigned char* gsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(gsm_raw) + 1023) & ~uintptr_t(1023));
  constexpr int kABytes = kBM * kBK * 2;
  constexpr int kBBytes = BN * kBK * 2;
  unsigned char* sa = gsm;
  unsigned char* sb = gsm + kStages * kABytes;
  __shared__ GemmSmem gs;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
  const int KT = (n + kBK - 1) / kBK;

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&gs.full[s], 1);
      mbar_init(&gs.empty[s], 1);
    }
    mbar_init(&gs.done, 1);
    fence_mbar_init();
  }
  if (warp == 0) {  // TMEM: BN FP32 columns x 128 lanes
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&gs.tmem_base)),
                 "r"(BN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = gs.tmem_base;

  if (warp == 0 && lane == 0) {
    // producer
    for (int kt = 0; kt < KT; ++kt) {
      const int s = kt % kStages;
      if (kt >= kStages && !mbar_wait(&gs.empty[s], ((kt / kStages) - 1) & 1, err)) break;
      mbar_arrive_expect_tx(&gs.full[s], kABytes + kBBytes);
      tma_load_2d(sa + s * kABytes, &map_x, kt * kBK, m0, &gs.full[s]);
      tma_load_2d(sb + s * kBBytes, &map_r, kt * kBK, n0, &gs.full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    constexpr uint32_t idesc = instr_desc_bf16(BN);
    bool ok = true;
    for (int kt = 0; kt < KT && ok; ++kt) {
      const int s = kt % kStages;
      if (!mbar_wait(&gs.full[s], (kt / kStages) & 1, err)) {
        ok = false;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t da = smem_desc_sw128(sa + s * kABytes);
      const uint64_t db = smem_desc_sw128(sb + s * kBBytes);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        // advance 16 BF16 = 32 bytes along K inside the swizzle row
        const uint64_t a_k = da + (uint64_t)(2 * k);
        const uint64_t b_k = db + (uint64_t)(2 * k);
        const uint32_t acc = (kt > 0 || k > 0) ? 1u : 0u;
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
            "l"(a_k), "l"(b_k), "r"(idesc), "r"(acc)
            : "memory");
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                       smem_u32(&gs.empty[s]))
                   : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(&gs.done))
                 : "memory");
  }
  __syncwarp();
  // epilogue: wait for the accumulator, TMEM -> registers -> C
  const bool ready = mbar_wait(&gs.done, 0, err);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (ready) {
    const int row = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
          "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
            "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
            "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
            "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
          : "r"(taddr));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < p) {
#pragma unroll
        for (int c = 0; c < 32; ++c) {
          const int col = n0 + c0 + c;
          if (col < B) C[(long long)row + (long long)col * ldc] = __uint_as_float(v[c]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN) : "memory");
  }
}

// ---------------------------------------------------------------- host: tensor maps
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_enc_mutex;
EncodeTiledFn g_encode = nullptr;

lasso_status get_encoder(EncodeTiledFn* out) {
  std::lock_guard<std::mutex> lock(g_enc_mutex);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    CUDA_TRY(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
    if (!fn || q != cudaDriverEntryPointSuccess)
      return set_error(LASSO_ERR_CUDA, "cuTensorMapEncodeTiled is not available from the driver");
    g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  *out = g_encode;
  return LASSO_OK;
}

// 2-D BF16 tensor: inner dimension K (contiguous), outer rows with stride ld elements
lasso_status make_map(CUtensorMap* map, const void* base, int64_t K, int64_t rows, int64_t ld, int box_rows) {
  EncodeTiledFn enc = nullptr;
  lasso_status st = get_encoder(&enc);
  if (st != LASSO_OK) return st;
  const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return set_error(LASSO_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return LASSO_OK;
}

}  // namespace

namespace {

template <int BN>
lasso_status launch_bn(const void* Xb, int64_t n, int64_t p, int64_t ldx, const void* Rb, int64_t ldr, int64_t B,
                       float* C, int64_t ldc, int* err_dev, cudaStream_t stream) {
  CUtensorMap mx, mr;
  lasso_status st = make_map(&mx, Xb, n, p, ldx, kBM);
  if (st != LASSO_OK) return st;
  st = make_map(&mr, Rb, n, B, ldr, BN);
  if (st != LASSO_OK) return st;
  const size_t smem = 1024 + (size_t)kStages * (kBM + BN) * kBK * 2;
  CUDA_TRY(cudaFuncSetAttribute(xtr_gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const dim3 grid((unsigned)((p + kBM - 1) / kBM), (unsigned)((B + BN - 1) / BN));
  xtr_gemm_kernel<BN><<<grid, kGemmThreads, smem, stream>>>(mx, mr, (int)n, (int)p, (int)B, C, ldc, err_dev);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

}  // namespace

// tile_n: the N tile (64, 128 or 256 accumulator columns of TMEM; 0 = 128)
lasso_status xtr_gemm_launch(const void* Xb, int64_t n, int64_t p, int64_t ldx, const void* Rb, int64_t ldr,
                             int64_t B, float* C, int64_t ldc, int* err_dev, cudaStream_t stream, int tile_n) {
  if (tile_n == 64) return launch_bn<64>(Xb, n, p, ldx, Rb, ldr, B, C, ldc, err_dev, stream);
  if (tile_n == 256) return launch_bn<256>(Xb, n, p, ldx, Rb, ldr, B, C, ldc, err_dev, stream);
  return launch_bn<128>(Xb, n, p, ldx, Rb, ldr, B, C, ldc, err_dev, stream);
}

}  // namespace lassogs

using namespace lassogs;

extern "C" lasso_status lasso_correlations_bf16(const void* X_bf16, int64_t n, int64_t p, int64_t ldx,
                                                const void* R_bf16, int64_t ldr, int64_t B, float* C, int64_t ldc,
                                                void* workspace, size_t workspace_bytes, void* stream) {
  clear_error();
  if (!X_bf16 || !R_bf16 || !C || !workspace)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_correlations_bf16: NULL pointer argument");
  if (n < 1 || p < 1 || B < 1 || p > (int64_t)INT32_MAX || B > (int64_t)INT32_MAX || n > (int64_t)INT32_MAX)
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_correlations_bf16: sizes out of range");
  if (ldx < n || ldr < n || ldc < p || ldx % 8 != 0 || ldr % 8 != 0)
    return set_error(LASSO_ERR_INVALID_ARG,
                     "lasso_correlations_bf16: need ldx, ldr >= n and multiples of 8, ldc >= p");
  if ((reinterpret_cast<uintptr_t>(X_bf16) % 16) || (reinterpret_cast<uintptr_t>(R_bf16) % 16) ||
      (reinterpret_cast<uintptr_t>(C) % 4))
    return set_error(LASSO_ERR_INVALID_ARG, "lasso_correlations_bf16: X and R need 16-byte aligned bases");
  if (workspace_bytes < 256 || (reinterpret_cast<uintptr_t>(workspace) % 256))
    return set_error(LASSO_ERR_WORKSPACE, "lasso_correlations_bf16: workspace of 256 aligned bytes required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* err = static_cast<int*>(workspace);
  CUDA_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  return xtr_gemm_launch(X_bf16, n, p, ldx, R_bf16, ldr, B, C, ldc, err, st);
}
