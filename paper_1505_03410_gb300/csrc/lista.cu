// Learned warm start: training and inference kernels of the unrolled ISTA
// network declared in include/lista.h.
//
// Per layer the network needs five contractions over (n, p, B):
//   forward   X beta (n x B, K = p)   and  W u (p x B, K = n)
//   backward  u gv^T (n x p, K = B),   W^T gv (n x B, K = p),   X^T gu (p x B, K = n)
// All run through one FP32 CUDA-core GEMM kernel (128 x 128 x 16 tiles, 8 x 8
// register blocking, double-buffered shared memory) instantiated for the three
// operand layouts that occur.  When the output has few tiles the K range is
// split and the partial sums are added in a fixed order by the epilogue
// kernels (which also apply the elementwise parts of each layer), so every
// result is deterministic.
#include <algorithm>
#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/lista.h"
#include "internal.h"

namespace lassogs {
namespace {

constexpr int kBM = 128, kBN = 128, kBK = 16, kGemmThreads = 256;
constexpr int kSplitTarget = 512;  // CTAs a split-K product aims for (fixed: sizes must not depend on the device)
constexpr int kEwThreads = 256;
constexpr int kLossBlocks = 256;   // fixed grid of the loss reduction (fixed summation order)
constexpr int kPowerIters = 60;
constexpr int kMaxLayers = 64;

struct Plan {
  int S;   // number of K splits
  int kc;  // K per split (a multiple of kBK)
};

Plan plan_gemm(int64_t M, int64_t N, int64_t K) {
  const int64_t tiles = ((M + kBM - 1) / kBM) * ((N + kBN - 1) / kBN);
  int64_t S = std::max<int64_t>(1, kSplitTarget / std::max<int64_t>(tiles, 1));
  S = std::min<int64_t>(S, std::max<int64_t>(1, K / 128));
  int64_t kc = (K + S - 1) / S;
  kc = std::max<int64_t>(kBK, (kc + kBK - 1) / kBK * kBK);
  S = (K + kc - 1) / kc;
  return Plan{(int)S, (int)kc};
}

size_t part_floats(int64_t M, int64_t N, int64_t K) {
  const Plan pl = plan_gemm(M, N, K);
  return (size_t)pl.S * (size_t)M * (size_t)N;
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------- GEMM
// P[z][nn][mm] = sum over the K range of split z of A(mm, k) B(k, nn), with
// A(m, k) = A[m*lda + k] (A_KC: k contiguous) or A[k*lda + m], and
// B(k, n) = B[n*ldb + k] (B_KC: k contiguous) or B[k*ldb + n].
template <bool A_KC>
__device__ __forceinline__ void tile_coord_a(int idx, int& m, int& k) {
  if (A_KC) {
    k = idx & (kBK - 1);
    m = idx >> 4;
  } else {
    m = idx & (kBM - 1);
    k = idx >> 7;
  }
}

template <bool A_KC, bool B_KC>
__global__ void __launch_bounds__(kGemmThreads) sgemm_kernel(int M, int N, int K, int kc, const float* __restrict__ A,
                                                              long long lda, const float* __restrict__ Bm,
                                                              long long ldb, float* __restrict__ P) {
  __shared__ __align__(16) float As[2][kBK][kBM + 4];
  __shared__ __align__(16) float Bs[2][kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * kBN;
  const int kb = blockIdx.z * kc, ke = min(K, kb + kc);
  float ra[8], rb[8];
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  auto load = [&](int k0) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      int m, k;
      tile_coord_a<A_KC>(tid + kGemmThreads * r, m, k);
      const int gm = m0 + m, gk = k0 + k;
      ra[r] = (gm < M && gk < ke) ? __ldg(A_KC ? A + (long long)gm * lda + gk : A + (long long)gk * lda + gm) : 0.f;
      int nn, kk;
      tile_coord_a<B_KC>(tid + kGemmThreads * r, nn, kk);
      const int gn = n0 + nn, gk2 = k0 + kk;
      rb[r] = (gn < N && gk2 < ke) ? __ldg(B_KC ? Bm + (long long)gn * ldb + gk2 : Bm + (long long)gk2 * ldb + gn)
                                   : 0.f;
    }
  };
  auto store = [&](int buf) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      int m, k;
      tile_coord_a<A_KC>(tid + kGemmThreads * r, m, k);
      As[buf][k][m] = ra[r];
      int nn, kk;
      tile_coord_a<B_KC>(tid + kGemmThreads * r, nn, kk);
      Bs[buf][kk][nn] = rb[r];
    }
  };

  load(kb);
  store(0);
  __syncthreads();
  int buf = 0;
  for (int k0 = kb; k0 < ke; k0 += kBK) {
    const bool more = k0 + kBK < ke;
    if (more) load(k0 + kBK);
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][tx * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][64 + tx * 4]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][kk][ty * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][kk][64 + ty * 4]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = __fmaf_rn(a[i], b[j], acc[i][j]);
    }
    if (more) store(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }
  float* Pz = P + (size_t)blockIdx.z * (size_t)M * (size_t)N;
  const bool vec = (M & 3) == 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int gn = n0 + (j < 4 ? ty * 4 + j : 64 + ty * 4 + j - 4);
    if (gn >= N) continue;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int gm = m0 + h * 64 + tx * 4;
      float* dst = Pz + (size_t)gn * M + gm;
      if (vec && gm + 3 < M) {
        *reinterpret_cast<float4*>(dst) = make_float4(acc[4 * h][j], acc[4 * h + 1][j], acc[4 * h + 2][j], acc[4 * h + 3][j]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (gm + c < M) dst[c] = acc[4 * h + c][j];
      }
    }
  }
}

template <bool A_KC, bool B_KC>
lasso_status gemm(int64_t M, int64_t N, int64_t K, const float* A, int64_t lda, const float* B, int64_t ldb, float* P,
                  int* S_out, cudaStream_t st) {
  const Plan pl = plan_gemm(M, N, K);
  const dim3 grid((unsigned)((M + kBM - 1) / kBM), (unsigned)((N + kBN - 1) / kBN), (unsigned)pl.S);
  if (grid.y > 65535u || grid.z > 65535u) return set_error(LASSO_ERR_INVALID_ARG, "lista: product too large");
  sgemm_kernel<A_KC, B_KC><<<grid, kGemmThreads, 0, st>>>((int)M, (int)N, (int)K, pl.kc, A, lda, B, ldb, P);
  CUDA_TRY(cudaGetLastError());
  *S_out = pl.S;
  return LASSO_OK;
}

// sum of the S partial products at linear index e (fixed order)
__device__ __forceinline__ float psum(const float* P, int S, size_t MN, size_t e) {
  float s = 0.f;
  for (int z = 0; z < S; ++z) s = __fadd_rn(s, P[(size_t)z * MN + e]);
  return s;
}

__device__ __forceinline__ float soft_threshold(float z, float t) {
  const float a = __fsub_rn(fabsf(z), t);
  return a > 0.f ? copysignf(a, z) : 0.f;
}

// ---------------------------------------------------------------- epilogues
// u[b*n + i] = ytil[b*ldyt + i] - sum_z P (S = 0: u = ytil)
__global__ void ep_residual_kernel(const float* P, int S, int n, int B, const float* ytil, long long ldyt, float* u) {
  const size_t MN = (size_t)n * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n), i = (int)(e % n);
    u[e] = __fsub_rn(ytil[(size_t)b * ldyt + i], psum(P, S, MN, e));
  }
}

// v = W u (sum of partials), z = beta + d .* v, beta_next = ST(z, tau)
__global__ void ep_layer_kernel(const float* P, int S, int p, int B, const float* beta, const float* d,
                                const float* tau_l, float* v_out, float* z_out, float* beta_next) {
  const size_t MN = (size_t)p * B;
  const float tau = *tau_l;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e % p);
    const float v = psum(P, S, MN, e);
    const float z = __fmaf_rn(d[j], v, beta ? beta[e] : 0.f);
    if (v_out) v_out[e] = v;
    if (z_out) z_out[e] = z;
    beta_next[e] = soft_threshold(z, tau);
  }
}

// out = sum_z P (+ out when accumulate)
__global__ void ep_sum_kernel(const float* P, int S, size_t MN, float* out, int accumulate) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const float s = psum(P, S, MN, e);
    out[e] = accumulate ? __fadd_rn(out[e], s) : s;
  }
}

// g = gz - sum_z P
__global__ void ep_sub_kernel(const float* P, int S, size_t MN, const float* gz, float* g) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x)
    g[e] = __fsub_rn(gz[e], psum(P, S, MN, e));
}

// ---------------------------------------------------------------- scaling
__global__ void to_f32_kernel(const double* Y, long long ldy, int n, int B, float* Yf) {
  const size_t MN = (size_t)n * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n), i = (int)(e % n);
    Yf[e] = (float)Y[(size_t)b * ldy + i];
  }
}

// one block per response: s_b = max_j |c_j b| over the partial sums of X^T y
__global__ void scale_kernel(const float* P, int S, int p, int B, float* s) {
  __shared__ float red[kEwThreads / 32];
  const int b = blockIdx.x;
  const size_t MN = (size_t)p * B;
  float m = 0.f;
  for (int j = threadIdx.x; j < p; j += blockDim.x) m = fmaxf(m, fabsf(psum(P, S, MN, (size_t)b * p + j)));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float r = 0.f;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = fmaxf(r, red[w]);
    s[b] = r;
  }
}

__global__ void ytil_kernel(const double* Y, long long ldy, const float* s, int n, int B, float* Ytil, long long ldyt) {
  const size_t MN = (size_t)n * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / n), i = (int)(e % n);
    const double sb = (double)s[b];
    Ytil[(size_t)b * ldyt + i] = sb > 0.0 ? (float)(Y[(size_t)b * ldy + i] / sb) : 0.f;
  }
}

// ---------------------------------------------------------------- backward
// g = (beta^L - t) / B; per-block partial sums of (beta^L - t)^2 in FP64
__global__ void loss_kernel(const float* betaL, const float* tgt, size_t count, int B, float* g, double* part) {
  __shared__ double red[kEwThreads / 32];
  double acc = 0.0;
  const float invB = 1.0f / (float)B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const float r = __fsub_rn(betaL[e], tgt[e]);
    g[e] = __fmul_rn(r, invB);
    acc = __fma_rn((double)r, (double)r, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = __dadd_rn(r, red[w]);
    part[blockIdx.x] = r;
  }
}

__global__ void loss_final_kernel(const double* part, int nblk, int B, double* loss_out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s = __dadd_rn(s, part[k]);
    *loss_out = 0.5 * s / (double)B;
  }
}

// Layer l of the backward pass, one thread per feature j (ascending b):
// gz = g . [|z| > tau], gv = d .* gz, gD[j] = sum_b gz v, and the block's
// partial of gtau = -sum sign(z) gz.
__global__ void bw_layer_kernel(const float* g, const float* z, const float* v, const float* d, const float* tau_l,
                                int p, int B, float* gz, float* gv, float* gD, double* tpart) {
  __shared__ double red[kEwThreads / 32];
  const float tau = *tau_l;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  double dd = 0.0, dt = 0.0;
  if (j < p) {
    const float dj = d[j];
    for (int b = 0; b < B; ++b) {
      const size_t e = (size_t)b * p + j;
      const float zz = z[e];
      const float gzv = fabsf(zz) > tau ? g[e] : 0.f;
      gz[e] = gzv;
      gv[e] = __fmul_rn(dj, gzv);
      dd = __fma_rn((double)gzv, (double)v[e], dd);
      dt = zz > 0.f ? __dsub_rn(dt, (double)gzv) : (zz < 0.f ? __dadd_rn(dt, (double)gzv) : dt);
    }
    gD[j] = (float)dd;
  }
  for (int o = 16; o > 0; o >>= 1) dt = __dadd_rn(dt, __shfl_xor_sync(0xffffffffu, dt, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = dt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = __dadd_rn(r, red[w]);
    tpart[blockIdx.x] = r;
  }
}

__global__ void tau_final_kernel(const double* tpart, int nblk, int L, float* gtau) {
  const int l = threadIdx.x;
  if (blockIdx.x == 0 && l < L) {
    double s = 0.0;
    for (int k = 0; k < nblk; ++k) s = __dadd_rn(s, tpart[(size_t)l * nblk + k]);
    gtau[l] = (float)s;
  }
}

// ---------------------------------------------------------------- optimiser, data
__global__ void adam_kernel(float* th, const float* g, float* m, float* v, size_t count, float lr, float b1, float b2,
                            float eps, float c1, float c2) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x) {
    const float ge = g[e];
    const float me = __fmaf_rn(b1, m[e], __fmul_rn(1.0f - b1, ge));
    const float ve = __fmaf_rn(b2, v[e], __fmul_rn(1.0f - b2, __fmul_rn(ge, ge)));
    m[e] = me;
    v[e] = ve;
    const float mh = __fmul_rn(me, c1), vh = __fmul_rn(ve, c2);
    th[e] = __fsub_rn(th[e], __fdiv_rn(__fmul_rn(lr, mh), __fadd_rn(sqrtf(vh), eps)));
  }
}

__global__ void gather_kernel(const float* src, long long lds, const int32_t* idx, int B, long long width, float* dst,
                              long long ldd) {
  const size_t MN = (size_t)width * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int r = (int)(e / width);
    const long long c = (long long)(e % width);
    dst[(size_t)r * ldd + c] = src[(size_t)idx[r] * lds + c];
  }
}

__global__ void targets_kernel(const double* bh, long long ldbh, const float* s, int B, int p, float* t) {
  const size_t MN = (size_t)p * B;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < MN; e += (size_t)gridDim.x * blockDim.x) {
    const int b = (int)(e / p), j = (int)(e % p);
    const double sb = (double)s[b];
    t[e] = sb > 0.0 ? (float)(bh[(size_t)b * ldbh + j] / sb) : 0.f;
  }
}

// One block per row: beta0 = s_b * beta^L, keeping only entries whose
// magnitude is among the K largest of the row (K <= 0: all).  The cut is the
// smallest t (as the bit pattern of a non-negative float, whose order is the
// order of the values) with #{|beta_j| >= t} <= K, found by bisection over
// the 31 magnitude bits; entries below t are set to 0.
__global__ void unscale_kernel(const float* betaL, const float* s, int p, long long K, double* out, long long ldo) {
  __shared__ int red[kEwThreads / 32];
  __shared__ unsigned cut;
  const int b = blockIdx.x;
  const float* row = betaL + (size_t)b * p;
  if (threadIdx.x == 0) cut = 0u;
  __syncthreads();
  if (K > 0 && K < p) {
    unsigned lo = 0u, hi = 0x7f800000u;  // #{>= hi} = 0 <= K (finite entries)
    while (lo < hi) {
      const unsigned mid = lo + ((hi - lo) >> 1);
      int cnt = 0;
      for (int j = threadIdx.x; j < p; j += blockDim.x) cnt += (__float_as_uint(fabsf(row[j])) >= mid) ? 1 : 0;
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      __syncthreads();
      if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = cnt;
      __syncthreads();
      int tot = 0;
      for (int w = 0; w < (int)(blockDim.x / 32); ++w) tot += red[w];
      if ((long long)tot <= K) hi = mid;
      else lo = mid + 1;
    }
    if (threadIdx.x == 0) cut = hi;
    __syncthreads();
  }
  const unsigned t = cut;
  const double sb = (double)s[b];
  for (int j = threadIdx.x; j < p; j += blockDim.x) {
    const float v = row[j];
    out[(size_t)b * ldo + j] = (__float_as_uint(fabsf(v)) >= t) ? sb * (double)v : 0.0;
  }
}

// ---------------------------------------------------------------- initialisation
__global__ void fill_kernel(float* x, size_t count, float v) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    x[e] = v;
}

// one block: nrm = ||sum_z P||, v = (sum_z P) / nrm
__global__ void normalize_vec_kernel(const float* P, int S, int len, float* v, double* nrm) {
  __shared__ double red[kEwThreads / 32];
  double acc = 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const double x = (double)psum(P, S, (size_t)len, i);
    acc = __fma_rn(x, x, acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  __shared__ double tot;
  if (threadIdx.x == 0) {
    double r = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) r = __dadd_rn(r, red[w]);
    tot = sqrt(r);
    *nrm = tot;
  }
  __syncthreads();
  const double inv = tot > 0.0 ? 1.0 / tot : 0.0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) v[i] = (float)((double)psum(P, S, (size_t)len, i) * inv);
}

__global__ void init_params_kernel(const float* X, long long ldx, int n, int p, int L, float ratio, const double* nrm,
                                   float* W, float* D, float* tau, float* lip_out) {
  const double lip = *nrm * 1.01;
  const float inv = lip > 0.0 ? (float)(1.0 / lip) : 0.f;
  const size_t NP = (size_t)n * p;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < NP; e += (size_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / n), i = (int)(e % n);
    W[e] = X[(size_t)j * ldx + i];
  }
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < (size_t)L * p; e += (size_t)gridDim.x * blockDim.x)
    D[e] = inv;
  if (blockIdx.x == 0 && threadIdx.x < (unsigned)L) tau[threadIdx.x] = __fmul_rn(ratio, inv);
  if (blockIdx.x == 0 && threadIdx.x == 0 && lip_out) *lip_out = (float)lip;
}

// ---------------------------------------------------------------- workspace
struct Ws {
  size_t cu, cv, cz;         // cache: L x B x n, L x B x p, L x B x p
  size_t b0, b1;             // beta ping-pong (B x p)
  size_t ub;                 // B x n scratch (u without cache, FP32 responses, gu)
  size_t g, gz, gv;          // B x p
  size_t part;               // split-K partials
  size_t red;                // FP64 partial sums
  size_t yt, s;              // normalised responses and scales (warm start)
  size_t pv, pw, pn;         // power method: v (p), w (n), norm
  size_t total;
  int nred;                  // doubles in red
};

Ws ws_layout(int64_t n, int64_t p, int64_t L, int64_t B) {
  Ws w{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += a256(bytes);
    return o;
  };
  const size_t Bn = (size_t)B * n, Bp = (size_t)B * p;
  w.cu = take(sizeof(float) * L * Bn);
  w.cv = take(sizeof(float) * L * Bp);
  w.cz = take(sizeof(float) * L * Bp);
  w.b0 = take(sizeof(float) * Bp);
  w.b1 = take(sizeof(float) * Bp);
  w.ub = take(sizeof(float) * Bn);
  w.g = take(sizeof(float) * Bp);
  w.gz = take(sizeof(float) * Bp);
  w.gv = take(sizeof(float) * Bp);
  size_t pf = 0;
  pf = std::max(pf, part_floats(n, B, p));  // X beta, W^T gv
  pf = std::max(pf, part_floats(p, B, n));  // W u, X^T gu, X^T y
  pf = std::max(pf, part_floats(n, p, B));  // u gv^T
  pf = std::max(pf, part_floats(n, 1, p));  // power method
  pf = std::max(pf, part_floats(p, 1, n));
  w.part = take(sizeof(float) * pf);
  const int64_t tblk = (p + kEwThreads - 1) / kEwThreads;
  w.nred = (int)(std::max<int64_t>(kLossBlocks, L * tblk));
  w.red = take(sizeof(double) * (size_t)w.nred);
  w.yt = take(sizeof(float) * Bn);
  w.s = take(sizeof(float) * (size_t)B);
  w.pv = take(sizeof(float) * (size_t)p);
  w.pw = take(sizeof(float) * (size_t)n);
  w.pn = take(sizeof(double));
  w.total = off;
  return w;
}

int ew_blocks(size_t count) {
  const size_t b = (count + kEwThreads - 1) / kEwThreads;
  return (int)std::max<size_t>(1, std::min<size_t>(b, 152 * 16));
}

lasso_status check_sizes(const char* who, int64_t n, int64_t p, int64_t L, int64_t B) {
  if (n < 1 || p < 1 || B < 1 || L < 1 || L > kMaxLayers || n > (int64_t)INT32_MAX / 4 || p > (int64_t)INT32_MAX / 4 ||
      B > 65535 * (int64_t)kBN)
    return set_error(LASSO_ERR_INVALID_ARG, "%s: sizes out of range (n %lld, p %lld, L %lld, B %lld)", who,
                     (long long)n, (long long)p, (long long)L, (long long)B);
  return LASSO_OK;
}

lasso_status check_ws(const char* who, const Ws& w, void* ws, size_t bytes) {
  if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) != 0)
    return set_error(LASSO_ERR_WORKSPACE, "%s: workspace must be non-NULL and 256-byte aligned", who);
  if (bytes < w.total)
    return set_error(LASSO_ERR_WORKSPACE, "%s: workspace of %zu bytes is smaller than the %zu bytes required", who,
                     bytes, w.total);
  return LASSO_OK;
}

template <typename T>
T* at(void* ws, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(ws) + off);
}

// forward pass into beta_out; the per-layer cache is kept when `keep`
lasso_status forward_impl(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                          const float* tau, int32_t L, const float* Ytil, int64_t ldyt, int64_t B, float* beta_out,
                          bool keep, const Ws& w, void* ws, cudaStream_t st) {
  float* P = at<float>(ws, w.part);
  const size_t Bn = (size_t)B * n, Bp = (size_t)B * p;
  const float* beta = nullptr;
  for (int l = 0; l < L; ++l) {
    float* u = keep ? at<float>(ws, w.cu) + (size_t)l * Bn : at<float>(ws, w.ub);
    int S = 0;
    if (l > 0) {
      lasso_status s = gemm<false, true>(n, B, p, X, ldx, beta, p, P, &S, st);  // X beta
      if (s != LASSO_OK) return s;
    }
    ep_residual_kernel<<<ew_blocks(Bn), kEwThreads, 0, st>>>(P, S, (int)n, (int)B, Ytil, ldyt, u);
    CUDA_TRY(cudaGetLastError());
    lasso_status s = gemm<true, true>(p, B, n, W, n, u, n, P, &S, st);  // W u
    if (s != LASSO_OK) return s;
    // ping-pong so that the last layer writes beta_out
    float* next = (l == L - 1) ? beta_out : at<float>(ws, ((L - 1 - l) & 1) ? w.b1 : w.b0);
    ep_layer_kernel<<<ew_blocks(Bp), kEwThreads, 0, st>>>(P, S, (int)p, (int)B, beta, D + (size_t)l * p, tau + l,
                                                           keep ? at<float>(ws, w.cv) + (size_t)l * Bp : nullptr,
                                                           keep ? at<float>(ws, w.cz) + (size_t)l * Bp : nullptr,
                                                           next);
    CUDA_TRY(cudaGetLastError());
    beta = next;
  }
  return LASSO_OK;
}

lasso_status normalize_impl(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                            int64_t B, float* Ytil, int64_t ldyt, float* s, const Ws& w, void* ws, cudaStream_t st) {
  float* Yf = at<float>(ws, w.ub);
  float* P = at<float>(ws, w.part);
  const size_t Bn = (size_t)B * n;
  to_f32_kernel<<<ew_blocks(Bn), kEwThreads, 0, st>>>(Y, ldy, (int)n, (int)B, Yf);
  CUDA_TRY(cudaGetLastError());
  int S = 0;
  lasso_status r = gemm<true, true>(p, B, n, X, ldx, Yf, n, P, &S, st);  // X^T y
  if (r != LASSO_OK) return r;
  scale_kernel<<<(unsigned)B, kEwThreads, 0, st>>>(P, S, (int)p, (int)B, s);
  CUDA_TRY(cudaGetLastError());
  ytil_kernel<<<ew_blocks(Bn), kEwThreads, 0, st>>>(Y, ldy, s, (int)n, (int)B, Ytil, ldyt);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

}  // namespace
}  // namespace lassogs

using namespace lassogs;

extern "C" {

size_t lista_workspace_size(int64_t n, int64_t p, int32_t L, int64_t B) {
  if (n < 1 || p < 1 || B < 1 || L < 1 || L > kMaxLayers) return 0;
  return ws_layout(n, p, L, B).total;
}

lasso_status lista_cache_layout(int64_t n, int64_t p, int32_t L, int64_t B, int64_t* off_u, int64_t* off_v,
                                int64_t* off_z) {
  clear_error();
  lasso_status r = check_sizes("lista_cache_layout", n, p, L, B);
  if (r != LASSO_OK) return r;
  if (!off_u || !off_v || !off_z) return set_error(LASSO_ERR_INVALID_ARG, "lista_cache_layout: NULL output");
  const Ws w = ws_layout(n, p, L, B);
  *off_u = (int64_t)w.cu;
  *off_v = (int64_t)w.cv;
  *off_z = (int64_t)w.cz;
  return LASSO_OK;
}

lasso_status lista_init(const float* X, int64_t n, int64_t p, int64_t ldx, int32_t L, float ratio, float* W, float* D,
                        float* tau, float* lip_out, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  lasso_status r = check_sizes("lista_init", n, p, L, 1);
  if (r != LASSO_OK) return r;
  if (!X || !W || !D || !tau || ldx < n) return set_error(LASSO_ERR_INVALID_ARG, "lista_init: bad arguments");
  if (!(ratio > 0.f && ratio <= 1.f)) return set_error(LASSO_ERR_INVALID_ARG, "lista_init: ratio must lie in (0, 1]");
  const Ws w = ws_layout(n, p, L, 1);
  if ((r = check_ws("lista_init", w, ws, ws_bytes)) != LASSO_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* v = at<float>(ws, w.pv);
  float* u = at<float>(ws, w.pw);
  float* P = at<float>(ws, w.part);
  double* nrm = at<double>(ws, w.pn);
  fill_kernel<<<ew_blocks(p), kEwThreads, 0, st>>>(v, (size_t)p, (float)(1.0 / std::sqrt((double)p)));
  CUDA_TRY(cudaGetLastError());
  for (int it = 0; it < kPowerIters; ++it) {
    int S = 0;
    if ((r = gemm<false, true>(n, 1, p, X, ldx, v, p, P, &S, st)) != LASSO_OK) return r;  // X v
    ep_sum_kernel<<<ew_blocks(n), kEwThreads, 0, st>>>(P, S, (size_t)n, u, 0);
    CUDA_TRY(cudaGetLastError());
    if ((r = gemm<true, true>(p, 1, n, X, ldx, u, n, P, &S, st)) != LASSO_OK) return r;  // X^T X v
    normalize_vec_kernel<<<1, kEwThreads, 0, st>>>(P, S, (int)p, v, nrm);
    CUDA_TRY(cudaGetLastError());
  }
  init_params_kernel<<<ew_blocks((size_t)n * p), kEwThreads, 0, st>>>(X, ldx, (int)n, (int)p, L, ratio, nrm, W, D,
                                                                       tau, lip_out);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

lasso_status lista_normalize(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                             int64_t B, float* Ytil, int64_t ldyt, float* s, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  lasso_status r = check_sizes("lista_normalize", n, p, 1, B);
  if (r != LASSO_OK) return r;
  if (!X || !Y || !Ytil || !s || ldx < n || ldy < n || ldyt < n)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_normalize: bad arguments");
  const Ws w = ws_layout(n, p, 1, B);
  if ((r = check_ws("lista_normalize", w, ws, ws_bytes)) != LASSO_OK) return r;
  return normalize_impl(X, n, p, ldx, Y, ldy, B, Ytil, ldyt, s, w, ws, static_cast<cudaStream_t>(stream));
}

lasso_status lista_forward(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                           const float* tau, int32_t L, const float* Ytil, int64_t ldyt, int64_t B, float* beta_out,
                           int32_t keep_cache, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  lasso_status r = check_sizes("lista_forward", n, p, L, B);
  if (r != LASSO_OK) return r;
  if (!X || !W || !D || !tau || !Ytil || !beta_out || ldx < n || ldyt < n)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_forward: bad arguments");
  const Ws w = ws_layout(n, p, L, B);
  if ((r = check_ws("lista_forward", w, ws, ws_bytes)) != LASSO_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return forward_impl(X, n, p, ldx, W, D, tau, L, Ytil, ldyt, B, beta_out, keep_cache != 0, w, ws, st);
}

lasso_status lista_backward(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                            const float* tau, int32_t L, int64_t B, const float* betaL, const float* targets,
                            float* gW, float* gD, float* gtau, double* loss_out, void* ws, size_t ws_bytes,
                            void* stream) {
  clear_error();
  lasso_status r = check_sizes("lista_backward", n, p, L, B);
  if (r != LASSO_OK) return r;
  if (!X || !W || !D || !tau || !betaL || !targets || !gW || !gD || !gtau || !loss_out || ldx < n)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_backward: bad arguments");
  const Ws w = ws_layout(n, p, L, B);
  if ((r = check_ws("lista_backward", w, ws, ws_bytes)) != LASSO_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t Bn = (size_t)B * n, Bp = (size_t)B * p;
  float* P = at<float>(ws, w.part);
  float* g = at<float>(ws, w.g);
  float* gz = at<float>(ws, w.gz);
  float* gv = at<float>(ws, w.gv);
  float* gu = at<float>(ws, w.ub);
  double* red = at<double>(ws, w.red);
  loss_kernel<<<kLossBlocks, kEwThreads, 0, st>>>(betaL, targets, Bp, (int)B, g, red);
  CUDA_TRY(cudaGetLastError());
  loss_final_kernel<<<1, 32, 0, st>>>(red, kLossBlocks, (int)B, loss_out);
  CUDA_TRY(cudaGetLastError());
  const int tblk = (int)((p + kEwThreads - 1) / kEwThreads);
  for (int l = L - 1; l >= 0; --l) {
    const float* u = at<float>(ws, w.cu) + (size_t)l * Bn;
    const float* v = at<float>(ws, w.cv) + (size_t)l * Bp;
    const float* z = at<float>(ws, w.cz) + (size_t)l * Bp;
    bw_layer_kernel<<<tblk, kEwThreads, 0, st>>>(g, z, v, D + (size_t)l * p, tau + l, (int)p, (int)B, gz, gv,
                                                  gD + (size_t)l * p, red + (size_t)l * tblk);
    CUDA_TRY(cudaGetLastError());
    int S = 0;
    if ((r = gemm<false, false>(n, p, B, u, n, gv, p, P, &S, st)) != LASSO_OK) return r;  // (gv u^T)^T
    ep_sum_kernel<<<ew_blocks((size_t)n * p), kEwThreads, 0, st>>>(P, S, (size_t)n * p, gW, l < L - 1 ? 1 : 0);
    CUDA_TRY(cudaGetLastError());
    if (l > 0) {
      if ((r = gemm<false, true>(n, B, p, W, n, gv, p, P, &S, st)) != LASSO_OK) return r;  // W^T gv
      ep_sum_kernel<<<ew_blocks(Bn), kEwThreads, 0, st>>>(P, S, Bn, gu, 0);
      CUDA_TRY(cudaGetLastError());
      if ((r = gemm<true, true>(p, B, n, X, ldx, gu, n, P, &S, st)) != LASSO_OK) return r;  // X^T gu
      ep_sub_kernel<<<ew_blocks(Bp), kEwThreads, 0, st>>>(P, S, Bp, gz, g);
      CUDA_TRY(cudaGetLastError());
    }
  }
  tau_final_kernel<<<1, 64, 0, st>>>(red, tblk, L, gtau);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

lasso_status lista_adam(float* theta, const float* grad, float* m, float* v, int64_t count, int32_t t, float lr,
                        float b1, float b2, float eps, void* stream) {
  clear_error();
  if (!theta || !grad || !m || !v || count < 1 || t < 1 || !(b1 >= 0.f && b1 < 1.f) || !(b2 >= 0.f && b2 < 1.f))
    return set_error(LASSO_ERR_INVALID_ARG, "lista_adam: bad arguments");
  const float c1 = (float)(1.0 / (1.0 - std::pow((double)b1, (double)t)));
  const float c2 = (float)(1.0 / (1.0 - std::pow((double)b2, (double)t)));
  adam_kernel<<<ew_blocks((size_t)count), kEwThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      theta, grad, m, v, (size_t)count, lr, b1, b2, eps, c1, c2);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

lasso_status lista_gather(const float* src, int64_t ld_src, const int32_t* idx, int64_t B, int64_t width, float* dst,
                          int64_t ld_dst, void* stream) {
  clear_error();
  if (!src || !idx || !dst || B < 1 || width < 1 || ld_src < width || ld_dst < width)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_gather: bad arguments");
  gather_kernel<<<ew_blocks((size_t)B * width), kEwThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      src, ld_src, idx, (int)B, width, dst, ld_dst);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

lasso_status lista_targets(const double* beta_hat, int64_t ldbh, const float* s, int64_t B, int64_t p, float* targets,
                           void* stream) {
  clear_error();
  if (!beta_hat || !s || !targets || B < 1 || p < 1 || ldbh < p)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_targets: bad arguments");
  targets_kernel<<<ew_blocks((size_t)B * p), kEwThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      beta_hat, ldbh, s, (int)B, (int)p, targets);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

lasso_status lista_warm_start(const float* X, int64_t n, int64_t p, int64_t ldx, const float* W, const float* D,
                              const float* tau, int32_t L, const double* Y, int64_t ldy, int64_t B, double* beta0,
                              int64_t ldb0, int64_t max_nonzeros, void* ws, size_t ws_bytes, void* stream) {
  clear_error();
  lasso_status r = check_sizes("lista_warm_start", n, p, L, B);
  if (r != LASSO_OK) return r;
  if (!X || !W || !D || !tau || !Y || !beta0 || ldx < n || ldy < n || ldb0 < p)
    return set_error(LASSO_ERR_INVALID_ARG, "lista_warm_start: bad arguments");
  const Ws w = ws_layout(n, p, L, B);
  if ((r = check_ws("lista_warm_start", w, ws, ws_bytes)) != LASSO_OK) return r;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  float* yt = at<float>(ws, w.yt);
  float* s = at<float>(ws, w.s);
  if ((r = normalize_impl(X, n, p, ldx, Y, ldy, B, yt, n, s, w, ws, st)) != LASSO_OK) return r;
  float* bl = at<float>(ws, w.g);
  if ((r = forward_impl(X, n, p, ldx, W, D, tau, L, yt, n, B, bl, false, w, ws, st)) != LASSO_OK) return r;
  unscale_kernel<<<(unsigned)B, kEwThreads, 0, st>>>(bl, s, (int)p, (long long)max_nonzeros, beta0, ldb0);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

}  // extern "C"
