// Host side of the path kernel: set-up kernels (precompute, residual,
// split-BF16 operands), the workspace layout and the launches of the single
// path and the batched solver.  The kernel itself is path_kernel.cuh.
#include <algorithm>
#include <vector>
#include <cstdint>
#include <cstdlib>
#include <cuda_runtime.h>

#include <cuda_bf16.h>

#include "path_kernel.cuh"

namespace lassogs {

// ---------------------------------------------------------------- setup kernels
// ||x_j||, 1/||x_j||^2, c0_j = x_j^T y -> lambda_max = ||X^T y||_inf (Sec. 1.2),
// finiteness of X, split planes of an FP64 X, beta0 in double-float.  c0 is
// kept for the dome test.
template <typename XT>
__global__ void precompute_kernel(const XT* X, long long ldx, int n, int p, const double* y, const double* beta0,
                                  float* Xh, float* Xl, long long ldh, double* nrm, float* nrmf, float4* ftab,
                                  float2* bdf, float2* b0df, double* cy, Ctrl* ctl) {
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j < p; j += nwarps) {
    const XT* col = X + (long long)j * ldx;
    double s2 = 0.0, sy = 0.0;
    bool finite = true;
    for (int i = lane; i < n; i += 32) {
      const double x = (double)col[i];
      finite = finite && isfinite(x);
      s2 = __fma_rn(x, x, s2);
      sy = __fma_rn(x, y[i], sy);
      if (Xh) {
        const float h = __double2float_rn(x);
        Xh[(long long)j * ldh + i] = h;
        Xl[(long long)j * ldh + i] = __double2float_rn(__dsub_rn(x, (double)h));
      }
    }
    if (Xh)
      for (int i = n + lane; i < ldh; i += 32) {
        Xh[(long long)j * ldh + i] = 0.f;
        Xl[(long long)j * ldh + i] = 0.f;
      }
    s2 = warp_sum_d(s2);
    sy = warp_sum_d(sy);
    finite = __all_sync(0xffffffffu, finite);
    if (lane == 0) {
      if (!finite || !isfinite(sy)) atomicExch(&ctl->nonfinite, 1);
      const double nr = __dsqrt_rn(s2);
      nrm[j] = nr;
      nrmf[j] = __double2float_ru(nr);
      cy[j] = sy;
      const df2 iv = df_from_double(s2 > 0.0 ? __drcp_rn(s2) : 0.0);
      ftab[j] = make_float4(iv.h, iv.l, 0.f, 0.f);
      if (isfinite(sy)) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(fabs(sy)));
      const df2 bd = df_from_double(beta0 ? beta0[j] : 0.0);
      bdf[j] = make_float2(bd.h, bd.l);
      b0df[j] = make_float2(bd.h, bd.l);
    }
  }
}

// rho = y - X beta0 (FP64 per row), ||y||^2, eps = tol ||y||^2
template <typename XT>
__global__ void rho_init_kernel(const XT* X, long long ldx, int n, int p, const double* y, const double* beta0,
                                float* rho_h, float* rho_l, float* rho0_h, float* rho0_l, int ldh, double tol,
                                Ctrl* ctl) {
  __shared__ double buf[32];
  for (int i = blockIdx.x; i < ldh; i += gridDim.x) {
    double acc = 0.0;
    if (beta0 && i < n)
      for (int j = threadIdx.x; j < p; j += blockDim.x) {
        const double b = beta0[j];
        if (b != 0.0) acc = __fma_rn(b, (double)X[(long long)j * ldx + i], acc);
      }
    acc = block_sum_d(acc, buf);
    if (threadIdx.x == 0) {
      const double r = (i < n) ? __dsub_rn(y[i], acc) : 0.0;
      if (!isfinite(r)) atomicExch(&ctl->nonfinite, 1);
      const df2 d = df_from_double(r);
      rho_h[i] = d.h;
      rho_l[i] = d.l;
      rho0_h[i] = d.h;
      rho0_l[i] = d.l;
    }
  }
  if (blockIdx.x == 0) {
    double yy = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) yy = __fma_rn(y[i], y[i], yy);
    yy = block_sum_d(yy, buf);
    if (threadIdx.x == 0) {
      ctl->yy = yy;
      ctl->eps = tol * yy;
    }
  }
}

// lambda_max = ||X^T y||_inf must be > 0 (otherwise every lambda_t is 0) and
// every ratio must lie in (0, 1]; violations are reported as INVALID_ARG.
// For the Elastic-Net with mixing a, beta = 0 is optimal from ||X^T y||_inf / a.
__global__ void finish_setup_kernel(Ctrl* ctl, const double* ratios, int T, double enet_alpha) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->lambda_max = __ddiv_rn(__longlong_as_double((long long)ctl->m_bits), enet_alpha);
    ctl->m_bits = 0ull;
    ctl->mlo_bits = 0u;
    bool bad = !(ctl->lambda_max > 0.0);
    for (int t = 0; t < T; ++t) bad = bad || !(ratios[t] > 0.0 && ratios[t] <= 1.0);
    if (ctl->nonfinite) ctl->err = kErrNonfinite;
    else if (bad) ctl->err = kErrInvalidArg;
  }
}

// stamp a device error into every stats record (after the path kernel)
__global__ void stats_error_kernel(Ctrl* ctl, lasso_path_stats* stats, int T) {
  const int e = ctl->err;
  if (e == 0) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
    stats[t].status = e;
    stats[t].converged = 0;
  }
}

// ---------------------------------------------------------------- split-BF16 operands
// A value v (FP32) is carried as vh = bf16(v) and vl = bf16(v - vh), so that
// |v - vh - vl| <= 2^-16 |v|.  The three products that matter,
//   x.r ~ xh.rh + xh.rl + xl.rh   (the dropped xl.rl is <= 2^-16 |x r|),
// are one GEMM over a K dimension of 3 L: the design row j is packed as
// [xh | xh | xl] and the residual of problem b as [rh | rl | rh] (L = n
// rounded up to 8, zero padded).  Every product of two BF16 values is exact
// in FP32, so the error of c~ is at most (3 2^-16 + 2^-20) |x||r| plus the
// FP32 accumulation of 3 L terms.
__device__ __forceinline__ void split_bf16(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(__fsub_rn(v, __bfloat162float(h)));
}

__global__ void pack_x_kernel(const float* __restrict__ X, long long ldx, int n, int p, int L,
                              __nv_bfloat16* __restrict__ X3) {
  const long long total = (long long)p * L;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(k / L), i = (int)(k % L);
    const float v = i < n ? X[(long long)j * ldx + i] : 0.f;
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* row = X3 + (long long)j * 3 * L;
    row[i] = h;
    row[L + i] = h;
    row[2 * L + i] = l;
  }
}

// residuals of the B problems: from the masked responses (first lambda) or
// from the FP32 high planes of the residuals kept in each problem's region
__global__ void pack_r_kernel(const double* Y, long long ldy, const uint8_t* rmask, long long ldm, const char* ws,
                              size_t region, size_t o_rho, int n, int B, int L, int from_y,
                              __nv_bfloat16* __restrict__ R3) {
  const long long total = (long long)B * L;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total; k += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(k / L), i = (int)(k % L);
    float v = 0.f;
    if (i < n) {
      if (from_y) {
        const bool in = rmask == nullptr || rmask[i + (size_t)b * ldm] != 0;
        v = in ? (float)Y[i + (size_t)b * ldy] : 0.f;
      } else {
        v = reinterpret_cast<const float*>(ws + (size_t)b * region + o_rho)[i];
      }
    }
    __nv_bfloat16 h, l;
    split_bf16(v, h, l);
    __nv_bfloat16* row = R3 + (long long)b * 3 * L;
    row[i] = h;
    row[L + i] = l;
    row[2 * L + i] = h;
  }
}

__global__ void set_int_kernel(int* p, int v) { *p = v; }

// ---------------------------------------------------------------- host side
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxGrid = 1024;
constexpr int kSCapPath = 4096;   // chain entries per round, single path
constexpr int kSCapBatch = 512;   // chain entries per round, batched (per-CTA snapshots)

// Offsets of one workspace region (the single path has one; the batched
// solver one per resident CTA).  Planes of an FP64 design follow the region.
struct Layout {
  size_t o[40];
  size_t region, planes, total;
  long long ldw;
  int s_cap, gram_cap;
};
enum {
  L_ctrl, L_cnt, L_part_l1, L_nrm, L_nrmf, L_ftab, L_bdf, L_b0df, L_rho0_h, L_rho0_l, L_ctil,
  L_mask, L_A, L_sup0, L_sup1, L_chain, L_entered, L_oldb, L_recs, L_snap, L_zl_j, L_zl_b, L_zbits, L_yb, L_sk,
  L_mref, L_msnap, L_cy, L_part_l2, L_gram, L_slot, L_feat, L_g0, L_dlt, L_anchor, L_dsnap, L_dref, L_N
};

// Slots of the Gram cache: twice the rows for the single path (a Lasso
// solution in general position has at most n nonzeros), the rows for a group
// of the batched solver (one cache per group), at least 512, at most p.
// kGramNone leaves the cache out.
enum GramKind { kGramNone = 0, kGramSingle = 1, kGramGroup = 2 };
int64_t gram_slots(int64_t n, int64_t p, int gram) {
  if (gram == kGramNone) return 0;
  const int64_t rows = gram == kGramSingle ? 2 * n : n;
  return std::min<int64_t>(p, std::max<int64_t>(512, (rows + 31) / 32 * 32));
}

// The residual rho (planes rho_h, rho_l) is snapshot 0 of the snapshot array:
// the residual a round of passes starts from.
Layout make_layout(int64_t n, int64_t p, int s_cap_max, bool planes, int gram = kGramNone) {
  Layout L{};
  const long long ldw = (n + 3) / 4 * 4;
  const int s_cap = (int)std::min<int64_t>(s_cap_max, p);
  const int64_t words = (p + 31) / 32;
  size_t off = 0;
  auto take = [&](int k, size_t bytes) {
    L.o[k] = off;
    off += align256(bytes);
  };
  take(L_ctrl, sizeof(Ctrl));
  take(L_cnt, sizeof(int) * 4 * kMaxGrid);
  take(L_part_l1, sizeof(double) * kMaxGrid);
  take(L_nrm, sizeof(double) * p);
  take(L_nrmf, sizeof(float) * p);
  take(L_ftab, sizeof(float4) * p);
  take(L_bdf, sizeof(float2) * p);
  take(L_b0df, sizeof(float2) * p);
  take(L_rho0_h, sizeof(float) * ldw);
  take(L_rho0_l, sizeof(float) * ldw);
  take(L_ctil, sizeof(float) * p);
  take(L_mask, sizeof(uint32_t) * words);
  take(L_A, sizeof(int) * p);
  take(L_sup0, sizeof(int) * p);
  take(L_sup1, sizeof(int) * p);
  take(L_chain, sizeof(int) * (s_cap + 1));
  take(L_entered, sizeof(int) * p);
  take(L_oldb, sizeof(float2) * (s_cap + 1));
  take(L_recs, sizeof(ChainRec) * (s_cap + 1));
  take(L_snap, sizeof(float) * 2 * (size_t)ldw * (size_t)(s_cap + 2));
  take(L_zl_j, sizeof(int) * p);
  take(L_zl_b, sizeof(double) * p);
  take(L_zbits, sizeof(uint32_t) * words);
  take(L_yb, sizeof(double) * ldw);
  take(L_sk, sizeof(float) * p);
  take(L_mref, sizeof(float) * p);
  take(L_msnap, sizeof(float) * (s_cap + 2));
  take(L_cy, sizeof(double) * p);
  take(L_part_l2, sizeof(double) * kMaxGrid);
  const int64_t gc = gram_slots(n, p, gram);
  take(L_gram, sizeof(float2) * (size_t)gc * (size_t)gc);
  take(L_slot, gc ? sizeof(int) * p : 0);
  take(L_feat, sizeof(int) * (size_t)gc);
  take(L_g0, gc ? sizeof(float2) * (s_cap + 1) : 0);
  take(L_dlt, gc ? sizeof(float2) * (s_cap + 1) : 0);
  take(L_anchor, sizeof(float) * ldw);
  take(L_dsnap, sizeof(float) * (s_cap + 2));
  take(L_dref, sizeof(float) * p);
  L.gram_cap = (int)gc;
  L.region = off;
  L.planes = planes ? 2 * align256(sizeof(float) * (size_t)ldw * (size_t)p) : 0;
  L.total = L.region + L.planes;
  L.ldw = ldw;
  L.s_cap = s_cap;
  return L;
}

void set_offsets(Args& a, const Layout& L) {
  a.o_ctrl = L.o[L_ctrl];
  a.o_cnt_kept = L.o[L_cnt];
  a.o_cnt_sup = L.o[L_cnt] + sizeof(int) * kMaxGrid;
  a.o_cnt_nnz = L.o[L_cnt] + 2 * sizeof(int) * kMaxGrid;
  a.o_cnt_zero = L.o[L_cnt] + 3 * sizeof(int) * kMaxGrid;
  a.o_part_l1 = L.o[L_part_l1];
  a.o_nrm = L.o[L_nrm];
  a.o_nrmf = L.o[L_nrmf];
  a.o_ftab = L.o[L_ftab];
  a.o_bdf = L.o[L_bdf];
  a.o_b0df = L.o[L_b0df];
  a.o_rho_h = L.o[L_snap];
  a.o_rho_l = L.o[L_snap] + sizeof(float) * (size_t)L.ldw;
  a.o_rho0_h = L.o[L_rho0_h];
  a.o_rho0_l = L.o[L_rho0_l];
  a.o_ctil = L.o[L_ctil];
  a.o_mask = L.o[L_mask];
  a.o_A = L.o[L_A];
  a.o_sup0 = L.o[L_sup0];
  a.o_sup1 = L.o[L_sup1];
  a.o_chain = L.o[L_chain];
  a.o_entered = L.o[L_entered];
  a.o_oldb = L.o[L_oldb];
  a.o_recs = L.o[L_recs];
  a.o_snap = L.o[L_snap];
  a.o_zl_j = L.o[L_zl_j];
  a.o_zl_b = L.o[L_zl_b];
  a.o_zbits = L.o[L_zbits];
  a.o_yb = L.o[L_yb];
  a.o_sk = L.o[L_sk];
  a.o_mref = L.o[L_mref];
  a.o_msnap = L.o[L_msnap];
  a.o_cy = L.o[L_cy];
  a.o_part_l2 = L.o[L_part_l2];
  a.o_gram = L.o[L_gram];
  a.o_slot = L.o[L_slot];
  a.o_feat = L.o[L_feat];
  a.o_g0 = L.o[L_g0];
  a.o_dlt = L.o[L_dlt];
  a.o_anchor = L.o[L_anchor];
  a.o_dsnap = L.o[L_dsnap];
  a.o_dref = L.o[L_dref];
  a.gram_cap = L.gram_cap;
  a.ldw = L.ldw;
  a.s_cap = L.s_cap;
}


// Chain shape for n rows.  A coordinate step is one warp's dependent
// instruction stream, so the chain spreads the rows until every lane holds a
// single float4 granule: one warp (no barrier, no shared-memory exchange)
// while n <= 128, four warps and 1, 2 or 4 granules per lane above.  Measured
// on the 500-row path: one warp with four granules per lane was 1.57x slower
// than four warps with one.
struct ChainShape {
  int cw, ngc;
};

ChainShape chain_shape(int64_t n, bool batch) {
  const int ld4 = (int)((n + 3) / 4);
  if (!batch && ld4 <= 32) return ChainShape{1, 1};
  return ChainShape{4, ld4 <= 128 ? 1 : (ld4 <= 256 ? 2 : 4)};
}

const void* pick_kernel(ChainShape c, bool xlo, bool batch, int per_sm = 1, bool enet = false) {
  if (batch) return enet ? path_kernel_batch_enet(c.ngc, per_sm) : path_kernel_batch(c.ngc, per_sm);
  if (enet) return xlo ? path_kernel_enet_f64(c.ngc, c.cw) : path_kernel_enet(c.ngc, c.cw);
  return xlo ? path_kernel_single_f64(c.ngc, c.cw) : path_kernel_single_f32(c.ngc, c.cw);
}

void fill_common(Args& a, int64_t n, int64_t p, int32_t T, const lasso_opts& o) {
  a.n = (int)n;
  a.p = (int)p;
  a.ld4 = (int)((n + 3) / 4);
  a.T = T;
  a.words = (int)((p + 31) / 32);
  a.f = o.screen_period;
  a.dual_point = o.dual_point;
  a.screen_rule = o.screen_rule;
  a.refined_radius = o.refined_radius;
  a.enet_alpha = o.enet_alpha;
  a.xtr_scope = o.xtr_scope;
  a.warm_start = o.warm_start;
  a.audit = o.audit_bounds;
  a.max_epochs = o.max_epochs;
  a.tol = o.gap_tol_rel;
  a.wait_ns = wait_limit_ns();
}

// dynamic shared memory of a CTA: the feature list of a round and the ring
// of kRing staged columns (each chain thread's granules, two planes for FP64)
size_t dyn_smem(int s_cap, ChainShape c, bool xlo) {
  const size_t jl_bytes = (((size_t)(s_cap + 1) * sizeof(int)) + 127) & ~(size_t)127;
  return jl_bytes + (size_t)kRing * c.ngc * 32 * c.cw * 16 * (xlo ? 2 : 1);
}

struct DevInfo {
  int sms, coop, smem_optin;
};

lasso_status dev_info(DevInfo& d) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.coop, cudaDevAttrCooperativeLaunch, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  return LASSO_OK;
}

// resident CTAs of the batched solver for a given device (fixed, so that the
// workspace size does not depend on the occupancy query)
int batch_grid(int64_t B, int sms, int per_sm = 2) {
  return (int)std::min<int64_t>(B, std::min<int64_t>((int64_t)sms * per_sm, kMaxGrid));
}

// CTAs that rebuild the snapshots of a Gram round (256 rows each); a group of
// the batched solver runs Gram rounds when it has more CTAs than these
int snapshot_ctas(long long ldw) { return (int)((ldw + kFollowRows - 1) / kFollowRows); }
bool group_gram(int64_t n, int group) { return group > 1 && group >= snapshot_ctas((n + 3) / 4 * 4) + 1; }

}  // namespace

// Time limit of the kernels' grid-barrier waits: 20 s, or the value of the
// environment variable LASSOGS_WAIT_LIMIT_NS (nanoseconds, >= 1000) when it is
// set.  The library's tests shorten it to make a wait run out on purpose and
// check that the kernel reports LASSO_ERR_TIMEOUT and returns; it is not part
// of the C ABI.
unsigned long long wait_limit_ns() {
  const char* v = std::getenv("LASSOGS_WAIT_LIMIT_NS");
  if (v != nullptr) {
    char* end = nullptr;
    const unsigned long long x = std::strtoull(v, &end, 10);
    if (end != v && x >= 1000ull) return x;
  }
  return kWaitLimitNs;
}

lasso_status path_phase_cycles(const void* ws, uint64_t* out, cudaStream_t stream) {
  static_assert(sizeof(((Ctrl*)nullptr)->prof) == 8 * sizeof(uint64_t), "eight phase counters");
  const char* base = static_cast<const char*>(ws);
  CUDA_TRY(cudaMemcpyAsync(out, base + offsetof(Ctrl, prof), 8 * sizeof(uint64_t), cudaMemcpyDeviceToHost, stream));
  CUDA_TRY(cudaStreamSynchronize(stream));
  return LASSO_OK;
}

size_t path_workspace_size(int64_t n, int64_t p, lasso_dtype xt, int64_t ldx) {
  (void)ldx;
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4) return 0;
  if (xt != LASSO_F32 && xt != LASSO_F64) return 0;
  return make_layout(n, p, kSCapPath, xt == LASSO_F64, kGramSingle).total;
}

lasso_status path_launch(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx, const double* y,
                         const double* ratios, int32_t T, const double* beta0, const lasso_opts& o,
                         double* beta_out, uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                         cudaStream_t stream) {
  const bool f64 = xt == LASSO_F64;
  const Layout L = make_layout(n, p, kSCapPath, f64, kGramSingle);
  if (ws_bytes < L.total)
    return set_error(LASSO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes required", ws_bytes,
                     L.total);
  char* base = static_cast<char*>(ws);
  Args a{};
  fill_common(a, n, p, T, o);
  set_offsets(a, L);
  a.ws = base;
  a.cta_bytes = 0;
  a.B = 1;
  a.y = y;
  a.ratios = ratios;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  float* Xh_w = reinterpret_cast<float*>(base + L.region);
  float* Xl_w = reinterpret_cast<float*>(base + L.region + L.planes / 2);
  if (f64) {
    a.Xh = Xh_w;
    a.Xl = Xl_w;
    a.ldx = L.ldw;
  } else {
    a.Xh = static_cast<const float*>(X);
    a.Xl = nullptr;
    a.ldx = ldx;
  }
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + a.o_ctrl);
  const ChainShape cs = chain_shape(n, false);
  const bool enet = o.enet_alpha < 1.0;
  const void* kfn = pick_kernel(cs, f64, false, 1, enet);
  DevInfo d{};
  lasso_status st = dev_info(d);
  if (st != LASSO_OK) return st;
  if (!d.coop) return set_error(LASSO_ERR_CUDA, "device does not support cooperative launch");
  // the direct chain's ring and the Gram round's tables share the dynamic shared memory
  const size_t dyn = std::max(dyn_smem(L.s_cap, cs, f64), kGramSmemBytes);
  if (dyn + 8192 > (size_t)d.smem_optin)
    return set_error(LASSO_ERR_INVALID_ARG, "the chain ring of %zu bytes does not fit shared memory", dyn);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, dyn));
  if (per_sm < 1) return set_error(LASSO_ERR_CUDA, "the path kernel cannot be resident (occupancy 0)");
  per_sm = std::min(per_sm, 2);
  const int grid = std::min(d.sms * per_sm, kMaxGrid);
  const int fs = (int)((p + grid - 1) / grid);
  a.fs = (fs + 31) / 32 * 32;
  // CTAs 1..nsc rebuild the snapshots of Gram rounds (256 rows each)
  a.nsc = snapshot_ctas(a.ldw);
  if (a.nsc + 1 > grid) a.gram_cap = 0;

  CUDA_TRY(cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), stream));
  CUDA_TRY(cudaMemsetAsync(base + a.o_cnt_kept, 0, sizeof(int) * 4 * kMaxGrid, stream));
  double* nrm = reinterpret_cast<double*>(base + a.o_nrm);
  float* nrmf = reinterpret_cast<float*>(base + a.o_nrmf);
  float4* ftab = reinterpret_cast<float4*>(base + a.o_ftab);
  float2* bdf = reinterpret_cast<float2*>(base + a.o_bdf);
  float2* b0df = reinterpret_cast<float2*>(base + a.o_b0df);
  double* cy = reinterpret_cast<double*>(base + a.o_cy);
  float* rho_h = reinterpret_cast<float*>(base + a.o_rho_h);
  float* rho_l = reinterpret_cast<float*>(base + a.o_rho_l);
  float* rho0_h = reinterpret_cast<float*>(base + a.o_rho0_h);
  float* rho0_l = reinterpret_cast<float*>(base + a.o_rho0_l);
  const int blocks = d.sms * 8;
  if (f64)
    precompute_kernel<double><<<blocks, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                          Xh_w, Xl_w, a.ldw, nrm, nrmf, ftab, bdf, b0df, cy, ctrl);
  else
    precompute_kernel<float><<<blocks, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                         nullptr, nullptr, a.ldw, nrm, nrmf, ftab, bdf, b0df, cy, ctrl);
  CUDA_TRY(cudaGetLastError());
  const int rb = (int)std::min<long long>(a.ldw, (long long)d.sms * 4);
  if (f64)
    rho_init_kernel<double><<<rb, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                    rho_h, rho_l, rho0_h, rho0_l, (int)a.ldw, o.gap_tol_rel, ctrl);
  else
    rho_init_kernel<float><<<rb, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                   rho_h, rho_l, rho0_h, rho0_l, (int)a.ldw, o.gap_tol_rel, ctrl);
  CUDA_TRY(cudaGetLastError());
  finish_setup_kernel<<<1, 32, 0, stream>>>(ctrl, ratios, T, o.enet_alpha);
  CUDA_TRY(cudaGetLastError());
  void* params[] = {&a};
  CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
  stats_error_kernel<<<1, 128, 0, stream>>>(ctrl, stats, T);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

// ---------------------------------------------------------------- batched
namespace {
struct BatchLayout {
  Layout L;
  int grid, regions, group;
  bool lockstep;
  long long Lk;  // K segment length of the split-BF16 operands
  size_t o_regions, o_x3, o_r3, o_c, o_gerr, o_park, o_single, single_bytes, total;
};

// group > 1: groups of CTAs per problem, one workspace region per group (at
// most 2 x SMs / group of them resident), each with its Gram cache when the
// group is large enough for Gram rounds
// tail: lockstep per pass, whose last problems may finish on the single path
// (the lambda at which each stopped, and the single path's own workspace)
BatchLayout batch_layout(int64_t n, int64_t p, int64_t B, bool lockstep, int sms, int group = 1, bool tail = false) {
  BatchLayout bl{};
  const bool groups = !lockstep && group > 1;
  bl.L = make_layout(n, p, kSCapBatch, false, groups && group_gram(n, group) ? kGramGroup : kGramNone);
  bl.grid = batch_grid(B, sms);
  bl.lockstep = lockstep;
  bl.group = groups ? group : 1;
  bl.regions = lockstep ? (int)B : groups ? (int)std::max<int64_t>(1, std::min<int64_t>(B, 2LL * sms / group)) : bl.grid;
  bl.Lk = (n + 7) / 8 * 8;
  size_t off = 256;
  bl.o_regions = off;
  off += bl.L.region * (size_t)bl.regions;
  if (lockstep) {
    bl.o_x3 = off;
    off += align256(sizeof(__nv_bfloat16) * 3 * (size_t)bl.Lk * (size_t)p);
    bl.o_r3 = off;
    off += align256(sizeof(__nv_bfloat16) * 3 * (size_t)bl.Lk * (size_t)B);
    bl.o_c = off;
    off += align256(sizeof(float) * (size_t)p * (size_t)B);
    bl.o_gerr = off;
    off += 256;
    if (tail) {
      bl.o_park = off;
      off += align256(sizeof(int) * (size_t)B);
      bl.o_single = off;
      bl.single_bytes = make_layout(n, p, kSCapPath, false, kGramSingle).total;
      off += align256(bl.single_bytes);
    }
  }
  bl.total = off;
  return bl;
}

int device_sms() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 152;
  return sms;
}
}  // namespace

size_t batch_workspace_size(int64_t n, int64_t p, int64_t B, bool lockstep, int group, bool pass) {
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4 || B < 1) return 0;
  return batch_layout(n, p, B, lockstep, device_sms(), group, lockstep && pass).total;
}

lasso_status batch_launch(const float* X, int64_t n, int64_t p, int64_t ldx, const double* Y, int64_t ldy,
                          const uint8_t* row_mask, int64_t ldm, int64_t B, const double* ratios, int32_t T,
                          const double* beta0, int64_t ldb0, const lasso_opts& o, double* beta_out,
                          uint32_t* mask_out, lasso_path_stats* stats,
                          void* ws, size_t ws_bytes, cudaStream_t stream) {
  DevInfo d{};
  lasso_status st = dev_info(d);
  if (st != LASSO_OK) return st;
  const bool lockstep = o.gemm_dtype == LASSO_BF16;
  const BatchLayout bl = batch_layout(n, p, B, lockstep, d.sms, o.batch_group, lockstep && o.lockstep_pass == 1);
  if (ws_bytes < bl.total)
    return set_error(LASSO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes required", ws_bytes,
                     bl.total);
  char* base = static_cast<char*>(ws);
  Args a{};
  fill_common(a, n, p, T, o);
  set_offsets(a, bl.L);
  a.ws = base + bl.o_regions;
  a.cta_bytes = bl.L.region;
  a.B = (int)B;
  a.y = Y;
  a.ldy = ldy;
  a.rmask = row_mask;
  a.ldm = ldm;
  a.beta0 = beta0;
  a.ldb0 = ldb0;
  a.queue = reinterpret_cast<int*>(base);
  a.ratios = ratios;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  a.Xh = X;
  a.Xl = nullptr;
  a.ldx = ldx;
  a.fs = (int)((p + 31) / 32 * 32);
  a.gsize = 1;
  const ChainShape cs = chain_shape(n, true);
  const int per_sm = o.batch_ctas_per_sm == 1 ? 1 : 2;
  const int grid = batch_grid(B, d.sms, per_sm);  // <= the regions the layout holds
  const void* kfn = pick_kernel(cs, false, true, per_sm, o.enet_alpha < 1.0);
  // groups with Gram rounds hold the round's tables in shared memory
  const size_t dyn = bl.L.gram_cap > 0 ? std::max(dyn_smem(bl.L.s_cap, cs, false), kGramSmemBytes)
                                        : dyn_smem(bl.L.s_cap, cs, false);
  if (dyn + 8192 > (size_t)d.smem_optin)
    return set_error(LASSO_ERR_INVALID_ARG, "the chain ring of %zu bytes does not fit shared memory", dyn);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  if (!lockstep && o.batch_group > 1) {
    // groups of CTAs per problem: every group's CTAs must be resident together
    // (their barrier), so the launch is cooperative and fills the resident CTAs
    const int gs = o.batch_group;
    int occ = 0;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kfn, kThreads, dyn));
    const int resident = d.sms * std::min(occ, per_sm);
    const int groups = (int)std::min<int64_t>(std::min<int64_t>(B, resident / gs), bl.regions);
    if (groups < 1)
      return set_error(LASSO_ERR_INVALID_ARG, "batch_group %d exceeds the %d resident CTAs", gs, resident);
    a.gsize = gs;
    a.nsc = snapshot_ctas(a.ldw);  // a.gram_cap (from the layout) is 0 unless gs > nsc
    const long long fsz = (p + gs - 1) / gs;
    a.fs = (int)((fsz + 31) / 32 * 32);
    // each group's control block (its barrier count) starts at zero
    CUDA_TRY(cudaMemset2DAsync(a.ws + a.o_ctrl, a.cta_bytes, 0, sizeof(Ctrl), (size_t)groups, stream));
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(groups * gs), dim3(kThreads), params, dyn, stream));
    return LASSO_OK;
  }
  if (!lockstep) {
    // each CTA solves whole paths; its first checks are CUDA-core FP32 passes
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
    return LASSO_OK;
  }
  // lockstep: per lambda, the residuals of all problems -> one tensor-core
  // product C = X^T R (split BF16) -> one launch that advances every problem
  // by one lambda, its first check reading C with the split-BF16 error factor
  const long long Lk = bl.Lk;
  __nv_bfloat16* X3 = reinterpret_cast<__nv_bfloat16*>(base + bl.o_x3);
  __nv_bfloat16* R3 = reinterpret_cast<__nv_bfloat16*>(base + bl.o_r3);
  float* C = reinterpret_cast<float*>(base + bl.o_c);
  int* gerr = reinterpret_cast<int*>(base + bl.o_gerr);
  a.lockstep = 1;
  a.cfirst = C;
  a.ldc = p;
  a.cfactor = (float)((3.0 * 0x1p-16 + 0x1p-20 + (3.0 * (double)Lk + 8.0) * 0x1p-24) * 1.05);
  CUDA_TRY(cudaMemsetAsync(gerr, 0, 256, stream));
  pack_x_kernel<<<d.sms * 8, 256, 0, stream>>>(X, ldx, (int)n, (int)p, (int)Lk, X3);
  CUDA_TRY(cudaGetLastError());
  if (o.lockstep_pass == 1) {
    // one product and one launch per coordinate pass: the product is taken
    // on the residuals every problem's next pass (or check) starts from
    // (y at the first launch of a zero start; with beta0 that first launch
    // forms rho inside and checks with its FP32 pass).  The launches stop
    // when the counter of unfinished problems (read every 4 launches) is 0;
    // each launch advances every unfinished problem, so a problem needs at
    // most T (K + 1) of them.
    int* active = gerr + 32;  // in the product's 256-byte error block, past the word it uses
    set_int_kernel<<<1, 1, 0, stream>>>(active, (int)B);
    CUDA_TRY(cudaGetLastError());
    a.pass_mode = 1;
    a.active = active;
    // the tail: once at most kParkAt problems are unfinished, each stops at its
    // next lambda boundary and the rest of its path runs on the single path,
    // whose launch uses every SM for one problem (its iterates from a lambda
    // boundary on are those of the path: the warm start carries beta, and the
    // check that starts the next lambda is the path's own).  Row subsets have
    // no single-path form, so such batches finish in lockstep.
    constexpr int kParkAt = 8;
    int* park_t = reinterpret_cast<int*>(base + bl.o_park);
    CUDA_TRY(cudaMemsetAsync(park_t, 0xff, sizeof(int) * (size_t)B, stream));
    a.park = 0;
    a.park_t = park_t;
    bool parked = false;
    const long long max_launches = (long long)T * (o.max_epochs + 1) + 1;
    for (long long step = 0; step < max_launches; ++step) {
      const bool use_gemm = !(step == 0 && beta0 != nullptr);
      if (use_gemm) {
        pack_r_kernel<<<d.sms * 4, 256, 0, stream>>>(Y, ldy, row_mask, ldm, a.ws, a.cta_bytes, a.o_rho_h, (int)n,
                                                     (int)B, (int)Lk, step == 0 ? 1 : 0, R3);
        CUDA_TRY(cudaGetLastError());
        st = xtr_gemm_launch(X3, 3 * Lk, p, 3 * Lk, R3, 3 * Lk, B, C, p, gerr, stream, o.gemm_tile_n);
        if (st != LASSO_OK) return st;
      }
      a.cfirst = use_gemm ? C : nullptr;
      a.t0 = step == 0 ? 0 : 1;
      a.t1 = T;
      CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
      void* params[] = {&a};
      CUDA_TRY(cudaLaunchKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
      if ((step & 3) == 3 || step + 1 == max_launches) {
        int left = 0;
        CUDA_TRY(cudaMemcpyAsync(&left, active, sizeof(int), cudaMemcpyDeviceToHost, stream));
        CUDA_TRY(cudaStreamSynchronize(stream));
        if (left <= 0) break;
        if (left <= kParkAt && row_mask == nullptr && !parked) {
          parked = true;
          a.park = 1;
        }
      }
    }
    if (parked) {
      std::vector<int> pt((size_t)B);
      CUDA_TRY(cudaMemcpyAsync(pt.data(), park_t, sizeof(int) * (size_t)B, cudaMemcpyDeviceToHost, stream));
      CUDA_TRY(cudaStreamSynchronize(stream));
      const int64_t words = (p + 31) / 32;
      for (int64_t b = 0; b < B; ++b) {
        const int t = pt[(size_t)b];
        if (t < 1 || t >= T) continue;
        // warm start: the solution of lambda_{t-1}; else every lambda restarts from beta0
        const double* b0 = o.warm_start ? beta_out + (size_t)p * ((size_t)(t - 1) + (size_t)T * (size_t)b)
                                        : (beta0 != nullptr ? beta0 + (size_t)b * (size_t)ldb0 : nullptr);
        const size_t off = (size_t)t + (size_t)T * (size_t)b;
        st = path_launch(X, LASSO_F32, n, p, ldx, Y + (size_t)b * (size_t)ldy, ratios + t, T - t, b0, o,
                         beta_out + (size_t)p * off, mask_out != nullptr ? mask_out + (size_t)words * off : nullptr,
                         stats + off, base + bl.o_single, bl.single_bytes, stream);
        if (st != LASSO_OK) return st;
      }
    }
    return LASSO_OK;
  }
  for (int t = 0; t < T; ++t) {
    // the product must be taken on the residual the lambda starts from: y at
    // t = 0 (zero start), rho0 = y - X beta0 when every lambda restarts, else
    // the previous lambda's final residual.  At t = 0 with beta0 the residual
    // is formed inside the launch, so that first check runs the FP32 pass.
    const bool use_gemm = !(t == 0 && beta0 != nullptr);
    if (use_gemm) {
      pack_r_kernel<<<d.sms * 4, 256, 0, stream>>>(Y, ldy, row_mask, ldm, a.ws, a.cta_bytes,
                                                   o.warm_start ? a.o_rho_h : a.o_rho0_h, (int)n, (int)B, (int)Lk,
                                                   t == 0 ? 1 : 0, R3);
      CUDA_TRY(cudaGetLastError());
      st = xtr_gemm_launch(X3, 3 * Lk, p, 3 * Lk, R3, 3 * Lk, B, C, p, gerr, stream, o.gemm_tile_n);
      if (st != LASSO_OK) return st;
    }
    a.cfirst = use_gemm ? C : nullptr;
    CUDA_TRY(cudaMemsetAsync(base, 0, 256, stream));
    a.t0 = t;
    a.t1 = t + 1;
    void* params[] = {&a};
    CUDA_TRY(cudaLaunchKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
  }
  return LASSO_OK;
}

}  // namespace lassogs
