// Lasso path by cyclic coordinate descent with GAP SAFE sphere screening
// (Fercoq, Gramfort, Salmon, ICML 2015, Algorithm 1) as one persistent
// cooperative kernel on a GB300.
//
// One lambda of the grid (Sec. 3.3 warm start, Sec. 4.1 schedule):
//   check   (all CTAs)  c~ = X^T rho in FP32 with a forward-error bound per
//                       feature; exact double-float recomputation of the
//                       features the bound leaves undecided (the maximum used
//                       by the dual point, Eq. (8), and the sphere test,
//                       Eq. (7) with the radius of Eq. (10)); FP64 objectives,
//                       gap and radius (Prop. 1); compaction of the
//                       safe-active set (Eq. (6)).
//   f passes            each pass over the safe-active list runs in rounds:
//     chain   (CTA 0)   the coordinates whose coefficient is nonzero, in
//                       ascending order, one after the other; columns are
//                       staged by bulk copies into a shared-memory ring, the
//                       residual lives in registers, and the residual after
//                       every step is kept as a snapshot.
//     verify  (all)     every other coordinate of the pass has a zero
//                       coefficient; it stays zero iff |x_j^T rho| <= lambda
//                       for the residual in force at its position (the
//                       snapshot of its segment).  All of them are tested at
//                       once; the first one that would move ends the round:
//                       the chain is rolled back to that position, the round
//                       after it starts with that coordinate.
//   A zero coefficient that stays zero leaves rho unchanged, so the iterates
//   are those of plain cyclic coordinate descent over the safe-active set.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "dfloat.cuh"
#include "internal.h"

namespace lassogs {

constexpr int kThreads = 256;   // threads per CTA
constexpr int kChainWarps = 4;  // warps of CTA 0 that run the chain
constexpr int kChainThreads = kChainWarps * 32;
constexpr int kProducerWarp = 4;
constexpr int kStatusOK = 0, kStatusNotConverged = 5;
constexpr int kNoPos = 0x7fffffff;
constexpr int kErrInvalidArg = 1;

struct Ctrl {
  unsigned bar_count, bar_gen;
  int err;
  int nonfinite;
  double lambda_max, yy, eps;
  unsigned long long m_bits;  // max |x_j^T rho| over the scope (exact), ordered bits
  unsigned mlo_bits;          // max (|c~_j| - E_j), FP32 bits
  int fstar;                  // first entering position of a round
  int nzl;                    // zero-list length (coefficients removed by screening)
  int q, s;                   // safe-active and support counts
  int pos, round_end, nc, done, sup_idx, forced, n_entered;
  float rho_bound;            // bound on ||rho|| for every snapshot of a round
  int pad0;
  // cycle counters of CTA 0 by phase (check, chain, verify, rollback/accept,
  // end of pass, setup of a round) and event counts (rounds, rollbacks)
  unsigned long long prof[8];
};

template <typename T>
__device__ __forceinline__ T vload(const T& x) {
  return *reinterpret_cast<const volatile T*>(&x);
}

struct Args {
  const float* Xh;  // n x p column-major FP32 (or the high plane of an FP64 X)
  const float* Xl;  // low plane of an FP64 X, or nullptr
  long long ldx;    // column stride of Xh / Xl (a multiple of 4)
  long long ldw;    // leading dimension of the residual planes and snapshots (4 * ld4)
  int n, p, ld4;    // ld4 = ceil(n / 4) float4 granules per column
  int T, words;
  int fs;           // features per CTA slice (multiple of 32)
  int s_cap;        // max chain entries per round
  int f;            // screen period
  int dual_point, xtr_scope, warm_start;
  long long max_epochs;
  const double* y;
  const double* ratios;
  double* beta_out;
  uint32_t* mask_out;
  lasso_path_stats* stats;
  // workspace
  Ctrl* ctrl;
  int* cnt_kept;
  int* cnt_sup;
  int* cnt_nnz;
  int* cnt_zero;
  double* part_l1;
  double* nrm;     // ||x_j|| (FP64)
  float* nrmf;     // ||x_j|| rounded up to FP32
  float4* ftab;    // {1/||x_j||^2 (h,l), lambda/||x_j||^2 (h,l)}
  float2* bdf;     // beta (double-float)
  float2* b0df;    // beta0 (double-float)
  float* rho_h;    // residual (double-float planes, length ldw)
  float* rho_l;
  float* rho0_h;   // residual of beta0
  float* rho0_l;
  float* ctil;     // c~_j of the current check
  uint32_t* mask;  // safe-active mask
  int* A;          // ascending safe-active features
  int* sup0;       // positions (into A) of nonzero coefficients, double-buffered
  int* sup1;
  int* chain;      // positions of the current round's chain
  int* entered;    // positions that entered during the current pass
  float2* oldb;    // coefficient of each chain entry before its update
  struct ChainRec* recs;  // records of the current round's chain
  float* snap;     // (s_cap + 1) snapshots, each 2 * ldw floats (h plane, l plane)
  int* zl_j;       // ascending features screened with a nonzero beta; pass scratch
  double* zl_b;    // their coefficient, indexed by feature
  uint32_t* zbits; // per mask word: features zeroed by the current check
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ float4 mask_rows(float4 x, int g, int n) {
  int r = 4 * g;
  if (r + 3 >= n) {
    if (r + 0 >= n) x.x = 0.f;
    if (r + 1 >= n) x.y = 0.f;
    if (r + 2 >= n) x.z = 0.f;
    if (r + 3 >= n) x.w = 0.f;
  }
  return x;
}
__device__ __forceinline__ float4 ld_x4(const float* col, int g, int n) {
  return mask_rows(__ldg(reinterpret_cast<const float4*>(col) + g), g, n);
}
__device__ __forceinline__ float4 ldcg4(const float* p, int g) { return __ldcg(reinterpret_cast<const float4*>(p) + g); }
__device__ __forceinline__ float2 ld_beta(const Args& a, int j) { return __ldcg(a.bdf + j); }
__device__ __forceinline__ bool nonzero2(float2 b) { return b.x != 0.f || b.y != 0.f; }

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v = __fadd_rn(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Forward-error factor of the FP32 warp dot below: each lane runs 4
// interleaved accumulators over NG granules, merges them (2 levels) and the
// warp adds 5 butterfly levels, so every product passes through at most
// NG + 7 roundings; the residual's rounding to FP32 adds one more u, a split
// FP64 column one more.  E_j = factor * ||x_j|| * ||rho|| (Cauchy-Schwarz).
template <int NG, bool XLO>
__device__ __forceinline__ float fp32_bound_factor() {
  const float u = 5.9604645e-08f;  // 2^-24
  return (float)(NG + 7 + 1 + (XLO ? 1 : 0) + 2) * u * 1.01f;
}

template <int NG>
__device__ __forceinline__ float warp_dot_f32(const float* col, const float4 (&r)[NG], int ld4, int n) {
  int lane = threadIdx.x & 31;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    int g = lane + 32 * k;
    if (g < ld4) {
      float4 x = ld_x4(col, g, n);
      a0 = __fmaf_rn(x.x, r[k].x, a0);
      a1 = __fmaf_rn(x.y, r[k].y, a1);
      a2 = __fmaf_rn(x.z, r[k].z, a2);
      a3 = __fmaf_rn(x.w, r[k].w, a3);
    }
  }
  return warp_sum_f(__fadd_rn(__fadd_rn(a0, a1), __fadd_rn(a2, a3)));
}

// Exact (double-float, order-independent) dot of column j with rho given as
// two planes in global memory; bound >= sum_i |x_ij rho_i|.  Whole warp.
template <int NG, bool XLO>
__device__ df2 warp_dot_exact(const Args& a, int j, const float* rh, const float* rl, float bound) {
  int lane = threadIdx.x & 31;
  const float* colh = a.Xh + (long long)j * a.ldx;
  const float* coll = XLO ? a.Xl + (long long)j * a.ldx : nullptr;
  float S = 0.f, C = 0.f;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    int g = lane + 32 * k;
    if (g < a.ld4) {
      float4 x = ld_x4(colh, g, a.n);
      float4 h = ldcg4(rh, g), l = ldcg4(rl, g);
      if (XLO) {
        float4 xl = ld_x4(coll, g, a.n);
        dot2_acc2(x.x, xl.x, h.x, l.x, S, C);
        dot2_acc2(x.y, xl.y, h.y, l.y, S, C);
        dot2_acc2(x.z, xl.z, h.z, l.z, S, C);
        dot2_acc2(x.w, xl.w, h.w, l.w, S, C);
      } else {
        dot2_acc(x.x, h.x, l.x, S, C);
        dot2_acc(x.y, h.y, l.y, S, C);
        dot2_acc(x.z, h.z, l.z, S, C);
        dot2_acc(x.w, h.w, l.w, S, C);
      }
    }
  }
  float sc, isc;
  limb_scale(2.0f * bound + 1e-30f, sc, isc);
  limbs3 L = limbs_add(to_limbs(S, sc), to_limbs(C, sc));
  L = warp_limbs_sum(L);
  return limbs_to_df(L, isc);
}

// Soft-threshold step of Algorithm 1 in double-float:
// b = beta + g / ||x_j||^2;  new = sign(b) (|b| - lambda/||x_j||^2)_+.
// When the coordinate is active, new - beta = q - sign(b) thr with
// q = g / ||x_j||^2; both signs are formed while b is being compared.
__device__ __forceinline__ void cd_update(df2 g, df2 beta, float4 tab, df2& nb, df2& delta) {
  const df2 inv{tab.x, tab.y}, thr{tab.z, tab.w};
  const df2 q = df_mul(g, inv);
  const df2 b = df_add(beta, q);
  const df2 dpos = df_sub(q, thr);
  const df2 dneg = df_add(q, thr);
  const bool neg = df_is_neg(b);
  const df2 ab = neg ? df_neg(b) : b;
  if (df_gt(ab, thr)) {
    delta = neg ? dneg : dpos;
    nb = df_add(beta, delta);
  } else {
    delta = df_neg(beta);
    nb = df2{0.f, 0.f};
  }
}

__device__ __forceinline__ int slice_begin(const Args& a, int c) {
  long long v = (long long)c * a.fs;
  return v < a.p ? (int)v : a.p;
}

// ---------------------------------------------------------------- the chain (CTA 0)
// One record per chain entry, built at the start of a round.
struct ChainRec {
  float4 tab;  // 1/||x_j||^2 (h,l), lambda/||x_j||^2 (h,l)
  float2 b;    // beta_j before the update
  float nf;    // ||x_j|| rounded up
  int j;       // feature
};

constexpr int kRing = 4;  // columns staged ahead by each chain thread

struct ChainSmem {
  limbs3 red[2][kChainWarps];
};

__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Stage this thread's granules of column j into ring slot s (no-op past nc).
template <int NGC, bool XLO>
__device__ __forceinline__ void stage_column(const Args& a, float4* ring, int s, int j) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + kChainThreads * k;
    if (g < a.ld4) {
      float4* dst = ring + ((size_t)(s * NGC + k) * kChainThreads + tid) * (XLO ? 2 : 1);
      cp_async16(dst, a.Xh + (long long)j * a.ldx + 4 * g);
      if (XLO) cp_async16(dst + 1, a.Xl + (long long)j * a.ldx + 4 * g);
    }
  }
}

// Coordinate updates for chain entries c = 0..nc-1 (positions into A), in
// order.  rho is held by the 128 chain threads (granules t + 128 k); each of
// them stages its own granules of the next kRing columns with cp.async, so
// no cross-thread handshake is needed for the column data.  The only
// cross-thread step per entry is the exact limb reduction of x_j^T rho.
// Writes the new coefficients to bdf, the old ones to oldb and the residual
// after entry c to snapshot c + 1.
template <int NGC, bool XLO>
__device__ void run_chain(const Args& a, ChainSmem& cs, float4* ring, int* jl, int nc, float rho_bound,
                          float4 (&rh)[NGC], float4 (&rl)[NGC]) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (nc <= 0) return;
  // records and the feature list of this round
  for (int c = tid; c < nc; c += kThreads) {
    const int j = __ldcg(a.A + __ldcg(a.chain + c));
    ChainRec r;
    r.tab = __ldcg(a.ftab + j);
    r.b = ld_beta(a, j);
    r.nf = __ldg(a.nrmf + j);
    r.j = j;
    a.recs[c] = r;
    jl[c] = j;
  }
  __syncthreads();
  if (warp < kChainWarps) {
    // prologue: stage the first kRing columns, fetch the first two records
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
      if (s < nc) stage_column<NGC, XLO>(a, ring, s, jl[s]);
      cp_async_commit();
    }
    ChainRec r0 = a.recs[0];
    ChainRec r1 = (nc > 1) ? a.recs[1] : r0;
    for (int e = 0; e < nc; ++e) {
      const int slot = e % kRing;
      cp_async_wait<kRing - 1>();  // this thread's copies for entry e have landed
      float4 xs[NGC], xls[NGC];
      float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f;
#pragma unroll
      for (int k = 0; k < NGC; ++k) {
        const int g = tid + kChainThreads * k;
        xs[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        xls[k] = xs[k];
        if (g < a.ld4) {
          const float4* src = ring + ((size_t)(slot * NGC + k) * kChainThreads + tid) * (XLO ? 2 : 1);
          xs[k] = mask_rows(src[0], g, a.n);
          if (XLO) {
            xls[k] = mask_rows(src[1], g, a.n);
            dot2_acc2(xs[k].x, xls[k].x, rh[k].x, rl[k].x, S0, C0);
            dot2_acc2(xs[k].y, xls[k].y, rh[k].y, rl[k].y, S1, C1);
            dot2_acc2(xs[k].z, xls[k].z, rh[k].z, rl[k].z, S0, C0);
            dot2_acc2(xs[k].w, xls[k].w, rh[k].w, rl[k].w, S1, C1);
          } else {
            dot2_acc(xs[k].x, rh[k].x, rl[k].x, S0, C0);
            dot2_acc(xs[k].y, rh[k].y, rl[k].y, S1, C1);
            dot2_acc(xs[k].z, rh[k].z, rl[k].z, S0, C0);
            dot2_acc(xs[k].w, rh[k].w, rl[k].w, S1, C1);
          }
        }
      }
      // refill the slot just read with entry e + kRing (always commit a group)
      if (e + kRing < nc) stage_column<NGC, XLO>(a, ring, slot, jl[e + kRing]);
      cp_async_commit();
      const ChainRec r2 = (e + 2 < nc) ? a.recs[e + 2] : r1;  // prefetch
      // |partial sums| <= ||x_j|| ||rho|| <= nf * rho_bound
      float sc, isc;
      limb_scale(2.0f * r0.nf * rho_bound + 1e-30f, sc, isc);
      limbs3 L = limbs_add(limbs_add(to_limbs(S0, sc), to_limbs(C0, sc)),
                           limbs_add(to_limbs(S1, sc), to_limbs(C1, sc)));
      L = warp_limbs_sum(L);
      if (lane == 0) cs.red[e & 1][warp] = L;
      named_bar_sync(1, kChainThreads);
      limbs3 Tl = cs.red[e & 1][0];
#pragma unroll
      for (int w = 1; w < kChainWarps; ++w) Tl = limbs_add(Tl, cs.red[e & 1][w]);
      const df2 g = limbs_to_df(Tl, isc);
      const df2 beta{r0.b.x, r0.b.y};
      df2 nb, d;
      cd_update(g, beta, r0.tab, nb, d);
      if (tid == 0) {
        a.oldb[e] = r0.b;
        a.bdf[r0.j] = make_float2(nb.h, nb.l);
      }
      if (!df_is_zero(d)) {
#pragma unroll
        for (int k = 0; k < NGC; ++k) {
          if (XLO) {
            axpy_df2(xs[k].x, xls[k].x, d.h, d.l, rh[k].x, rl[k].x);
            axpy_df2(xs[k].y, xls[k].y, d.h, d.l, rh[k].y, rl[k].y);
            axpy_df2(xs[k].z, xls[k].z, d.h, d.l, rh[k].z, rl[k].z);
            axpy_df2(xs[k].w, xls[k].w, d.h, d.l, rh[k].w, rl[k].w);
          } else {
            axpy_df(xs[k].x, d.h, d.l, rh[k].x, rl[k].x);
            axpy_df(xs[k].y, d.h, d.l, rh[k].y, rl[k].y);
            axpy_df(xs[k].z, d.h, d.l, rh[k].z, rl[k].z);
            axpy_df(xs[k].w, d.h, d.l, rh[k].w, rl[k].w);
          }
        }
      }
      float* sn = a.snap + (size_t)(e + 1) * 2 * a.ldw;
#pragma unroll
      for (int k = 0; k < NGC; ++k) {
        const int gi = tid + kChainThreads * k;
        if (gi < a.ld4) {
          __stcg(reinterpret_cast<float4*>(sn) + gi, rh[k]);
          __stcg(reinterpret_cast<float4*>(sn + a.ldw) + gi, rl[k]);
        }
      }
      r0 = r1;
      r1 = r2;
    }
    cp_async_wait<0>();
  }
  __syncthreads();
}

// rho planes (global) <-> chain registers of CTA 0 (threads >= 128 hold zeros)
template <int NGC>
__device__ __forceinline__ void load_rho_regs(const Args& a, const float* h, const float* l, float4 (&rh)[NGC],
                                              float4 (&rl)[NGC]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + kChainThreads * k;
    rh[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    rl[k] = rh[k];
    if (tid < kChainThreads && g < a.ld4) {
      rh[k] = ldcg4(h, g);
      rl[k] = ldcg4(l, g);
    }
  }
}
template <int NGC>
__device__ __forceinline__ void store_rho_regs(const Args& a, float* h, float* l, const float4 (&rh)[NGC],
                                               const float4 (&rl)[NGC]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + kChainThreads * k;
    if (tid < kChainThreads && g < a.ld4) {
      __stcg(reinterpret_cast<float4*>(h) + g, rh[k]);
      __stcg(reinterpret_cast<float4*>(l) + g, rl[k]);
    }
  }
}

// Bound on ||rho|| for every iterate of a round: CD does not increase
// P = 1/2 ||rho||^2 + lambda ||beta||_1 and only the chain coefficients move,
// so ||rho_k||^2 <= ||rho_0||^2 + 2 lambda sum_chain |beta_c|.  Rounded up.
template <int NGC>
__device__ float rho_bound_from_regs(const Args& a, const float4 (&rh)[NGC], double lam, int nc, float* fbuf) {
  const int tid = threadIdx.x;
  float ss = 0.f;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const float4 v = rh[k];
    ss = __fmaf_ru(v.x, v.x, ss);
    ss = __fmaf_ru(v.y, v.y, ss);
    ss = __fmaf_ru(v.z, v.z, ss);
    ss = __fmaf_ru(v.w, v.w, ss);
  }
  float l1 = 0.f;
  for (int c = tid; c < nc; c += kThreads) {
    const float2 b = ld_beta(a, __ldcg(a.A + __ldcg(a.chain + c)));
    l1 = __fadd_ru(l1, __fmul_ru(fabsf(b.x), 1.0001f));
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss = __fadd_ru(ss, __shfl_xor_sync(0xffffffffu, ss, o));
    l1 = __fadd_ru(l1, __shfl_xor_sync(0xffffffffu, l1, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    fbuf[tid >> 5] = ss;
    fbuf[8 + (tid >> 5)] = l1;
  }
  __syncthreads();
  float S = 0.f, L = 0.f;
  for (int w = 0; w < kThreads / 32; ++w) {
    S = __fadd_ru(S, fbuf[w]);
    L = __fadd_ru(L, fbuf[8 + w]);
  }
  __syncthreads();
  const float P2 = __fadd_ru(S, __fmul_ru(__fmul_ru(2.0f, __double2float_ru(lam)), L));
  return __fmul_ru(__fsqrt_ru(P2), 1.001f) + 1e-30f;
}

// block-wide exclusive ranks for a flag (all threads call); returns this
// thread's rank and the block total in *total.  ibuf >= 8 ints.
__device__ __forceinline__ int block_rank(bool flag, int* ibuf, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned bal = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) ibuf[warp] = __popc(bal);
  __syncthreads();
  int before = 0, tot = 0;
  for (int w = 0; w < kThreads / 32; ++w) {
    const int c = ibuf[w];
    if (w < warp) before += c;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return before + __popc(bal & ((1u << lane) - 1u));
}

__device__ __forceinline__ int lower_bound_i(const int* arr, int n, int v) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldcg(arr + mid) < v) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// ---------------------------------------------------------------- the kernel
template <int NGC, bool XLO>
__global__ void __launch_bounds__(kThreads, 1) path_kernel(Args a) {
  constexpr int NG = 4 * NGC;  // float4 granules per lane in warp-wide dots
  extern __shared__ __align__(128) unsigned char dsm[];
  __shared__ ChainSmem cs;
  __shared__ double dbuf[32];
  __shared__ int ibuf[32];
  __shared__ float fbuf[32];

  Ctrl* ctl = a.ctrl;
  const int cta = blockIdx.x, G = gridDim.x;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, nwarps = kThreads / 32;
  const int f0 = slice_begin(a, cta), f1 = slice_begin(a, cta + 1);
  // dynamic shared memory of CTA 0: feature list of a round, then the column ring
  int* jl = reinterpret_cast<int*>(dsm);
  float4* ring = reinterpret_cast<float4*>(dsm + (((size_t)(a.s_cap + 1) * sizeof(int) + 127) & ~(size_t)127));
  unsigned* bc = &ctl->bar_count;
  unsigned* bg = &ctl->bar_gen;
  int* err = &ctl->err;
  const double u64 = 1.1102230246251565e-16;  // 2^-53
  const float bf = fp32_bound_factor<NG, XLO>();
  float4 rh[NGC], rl[NGC];  // chain registers (CTA 0)
  long long tprof = clock64();
  const bool prof_thread = (cta == 0 && tid == 0);
#define PROF(k)                                   \
  do {                                            \
    if (prof_thread) {                            \
      const long long now_ = clock64();           \
      ctl->prof[k] += (unsigned long long)(now_ - tprof); \
      tprof = now_;                               \
    }                                             \
  } while (0)

#define GSYNC()                                            \
  do {                                                     \
    if (!grid_sync(bc, bg, err, (unsigned)G)) goto done;   \
  } while (0)

  if (vload(*err) != 0) goto done;  // setup found NaN/Inf

  for (int t = 0; t < a.T; ++t) {
    const double lam = __dmul_rn(vload(ctl->lambda_max), a.ratios[t]);
    // per-lambda table lambda / ||x_j||^2; full mask; optional restart
    for (int j = f0 + tid; j < f1; j += kThreads) {
      float4 tb = a.ftab[j];
      const df2 thr = df_from_double(__dmul_rn(lam, __dadd_rn((double)tb.x, (double)tb.y)));
      tb.z = thr.h;
      tb.w = thr.l;
      a.ftab[j] = tb;
      if (t > 0 && !a.warm_start) a.bdf[j] = a.b0df[j];
    }
    for (int w = f0 / 32 + tid; w < (f1 + 31) / 32; w += kThreads) {
      const int lo = w * 32, hi = min(a.p, lo + 32);
      a.mask[w] = (hi - lo == 32) ? 0xffffffffu : ((1u << (hi - lo)) - 1u);
    }
    if (cta == 0 && t > 0 && !a.warm_start)
      for (int i = tid; i < a.ldw; i += kThreads) {
        a.rho_h[i] = __ldcg(a.rho0_h + i);
        a.rho_l[i] = __ldcg(a.rho0_l + i);
      }
    long long epochs = 0, checks = 0, xcols = 0;
    int scope_n = a.p;  // X^T rho scope of the next check
    GSYNC();

    for (;;) {
      // ======================= CHECK =======================
      PROF(7);
      // (C1) ||rho||^2, y^T rho (every CTA), c~ for the slice, sum |beta| of the slice
      double rr = 0.0, yr = 0.0;
      for (int i = tid; i < a.n; i += kThreads) {
        const double r = __dadd_rn((double)__ldcg(a.rho_h + i), (double)__ldcg(a.rho_l + i));
        rr = __fma_rn(r, r, rr);
        yr = __fma_rn(a.y[i], r, yr);
      }
      rr = block_sum_d(rr, dbuf);
      yr = block_sum_d(yr, dbuf);
      const float rnormf = __fmul_ru(__fsqrt_ru(__double2float_ru(rr)), 1.0001f);
      {
        float4 r4[NG];
#pragma unroll
        for (int k = 0; k < NG; ++k) {
          const int g = lane + 32 * k;
          r4[k] = (g < a.ld4) ? ldcg4(a.rho_h, g) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        float mlo = 0.f;
        for (int j = f0 + warp; j < f1; j += nwarps) {
          const bool in = a.xtr_scope == 0 || ((__ldcg(a.mask + (j >> 5)) >> (j & 31)) & 1u);
          float c = 0.f;
          if (in) {
            c = warp_dot_f32<NG>(a.Xh + (long long)j * a.ldx, r4, a.ld4, a.n);
            const float E = __fmul_ru(__fmul_ru(bf, __ldg(a.nrmf + j)), rnormf) + 1e-37f;
            mlo = fmaxf(mlo, __fsub_rd(fabsf(c), E));
          }
          if (lane == 0) a.ctil[j] = c;
        }
        if (lane == 0) atomicMax(&ctl->mlo_bits, __float_as_uint(fmaxf(mlo, 0.f)));
        double l1p = 0.0;
        for (int j = f0 + tid; j < f1; j += kThreads) {
          const float2 b = ld_beta(a, j);
          l1p = __dadd_rn(l1p, fabs(__dadd_rn((double)b.x, (double)b.y)));
        }
        l1p = block_sum_d(l1p, dbuf);
        if (tid == 0) a.part_l1[cta] = l1p;
      }
      GSYNC();
      // (C2) exact refinement of the candidates for the maximum
      {
        const float mlo = __uint_as_float(vload(ctl->mlo_bits));
        for (int j = f0 + warp; j < f1; j += nwarps) {
          const bool in = a.xtr_scope == 0 || ((__ldcg(a.mask + (j >> 5)) >> (j & 31)) & 1u);
          if (!in) continue;
          const float c = __ldcg(a.ctil + j);
          const float nf = __ldg(a.nrmf + j);
          const float E = __fmul_ru(__fmul_ru(bf, nf), rnormf) + 1e-37f;
          if (__fadd_ru(fabsf(c), E) >= mlo) {
            const df2 ce = warp_dot_exact<NG, XLO>(a, j, a.rho_h, a.rho_l, __fmul_ru(nf, rnormf));
            const double cv = fabs(df_to_double(ce));
            if (lane == 0) atomicMax(&ctl->m_bits, (unsigned long long)__double_as_longlong(cv));
          }
        }
      }
      GSYNC();
      // (C3) objectives, gap, radius (identical in every CTA); sphere test on the slice
      double l1 = 0.0;
      for (int c = tid; c < G; c += kThreads) l1 = __dadd_rn(l1, __ldcg(a.part_l1 + c));
      l1 = block_sum_d(l1, dbuf);
      const double m = __longlong_as_double((long long)vload(ctl->m_bits));
      double alpha;
      if (a.dual_point == 0) {
        alpha = __drcp_rn(lam > m ? lam : m);
      } else if (rr == 0.0) {
        alpha = 0.0;
      } else {
        double al = __ddiv_rn(yr, __dmul_rn(lam, rr));
        if (m > 0.0) {
          const double lim = __drcp_rn(m);
          if (al < -lim) al = -lim;
          if (al > lim) al = lim;
        }
        alpha = al;
      }
      double d2 = 0.0;
      for (int i = tid; i < a.n; i += kThreads) {
        const double r = __dadd_rn((double)__ldcg(a.rho_h + i), (double)__ldcg(a.rho_l + i));
        const double dd = __dsub_rn(__dmul_rn(lam, __dmul_rn(alpha, r)), a.y[i]);
        d2 = __fma_rn(dd, dd, d2);
      }
      d2 = block_sum_d(d2, dbuf);
      const double yy = vload(ctl->yy);
      const double P = __dadd_rn(__dmul_rn(0.5, rr), __dmul_rn(lam, l1));
      const double D = __dsub_rn(__dmul_rn(0.5, yy), __dmul_rn(0.5, d2));
      const double Gap = __dsub_rn(P, D);
      const double tau = 2.0 * (double)(a.n + a.p + 8) * u64 * (rr + lam * l1 + yy + d2);
      const double Gs = (Gap > 0.0 ? Gap : 0.0) + tau;
      const double rad = __ddiv_rn(__dsqrt_rn(__dmul_rn(2.0, Gs)), lam);
      const double aa = fabs(alpha);
      ++checks;
      xcols += scope_n;
      const bool stop = Gap <= vload(ctl->eps);
      const bool cap = epochs >= a.max_epochs;
      {
        const float aaf_lo = __double2float_rd(aa), aaf_hi = __double2float_ru(aa);
        const float radf_lo = __double2float_rd(rad), radf_hi = __double2float_ru(rad);
        int kept = 0, sup = 0, nnz = 0, zero = 0;
        // each warp handles 32 consecutive features = one mask word
        for (int w0 = f0 + 32 * warp; w0 < f1; w0 += 32 * nwarps) {
          const int j = w0 + lane;
          const bool valid = j < f1;
          const uint32_t word = __ldcg(a.mask + (w0 >> 5));
          const bool was = valid && ((word >> lane) & 1u);
          bool keep = was, amb = false;
          if (was) {
            const float c = __ldcg(a.ctil + j);
            const float nf = __ldg(a.nrmf + j);
            const float E = __fmul_ru(__fmul_ru(bf, nf), rnormf) + 1e-37f;
            // rigorous FP32 brackets of mu_j = |c_j| |alpha| + r ||x_j||
            const float mu_hi = __fadd_ru(__fmul_ru(__fadd_ru(fabsf(c), E), aaf_hi), __fmul_ru(radf_hi, nf));
            const float nfl = __double2float_rd(__ldg(a.nrm + j));
            const float clo = fmaxf(__fsub_rd(fabsf(c), E), 0.f);
            const float mu_lo = __fadd_rd(__fmul_rd(clo, aaf_lo), __fmul_rd(radf_lo, nfl));
            if (mu_hi < 0.999999f) keep = false;
            else if (mu_lo >= 1.000001f) keep = true;
            else amb = true;
          }
          // exact decision for the undecided ones, as the FP64 test of Eq. (7)
          unsigned ambm = __ballot_sync(0xffffffffu, amb);
          while (ambm) {
            const int l = __ffs(ambm) - 1;
            ambm &= ambm - 1;
            const int jj = w0 + l;
            const df2 ce = warp_dot_exact<NG, XLO>(a, jj, a.rho_h, a.rho_l, __fmul_ru(__ldg(a.nrmf + jj), rnormf));
            const double mu = __dadd_rn(__dmul_rn(fabs(df_to_double(ce)), aa), __dmul_rn(rad, __ldg(a.nrm + jj)));
            if (lane == l) keep = !(mu < 1.0);
          }
          const float2 bj = valid ? ld_beta(a, j) : make_float2(0.f, 0.f);
          bool nz = nonzero2(bj);
          // a newly screened nonzero coefficient is set to zero when the
          // solver goes on (Remark 3); its residual share is added back by CTA 0
          const bool zeroed = was && !keep && nz && !stop && !cap;
          if (zeroed) {
            a.zl_b[j] = __dadd_rn((double)bj.x, (double)bj.y);
            a.bdf[j] = make_float2(0.f, 0.f);
            nz = false;
          }
          const uint32_t zw = __ballot_sync(0xffffffffu, zeroed);
          zero += __popc(zw);
          const uint32_t nwd = __ballot_sync(0xffffffffu, keep);
          if (lane == 0) {
            a.mask[w0 >> 5] = nwd;
            a.zbits[w0 >> 5] = zw;
          }
          kept += __popc(nwd);
          sup += __popc(__ballot_sync(0xffffffffu, keep && nz));
          nnz += __popc(__ballot_sync(0xffffffffu, valid && nz));
        }
        if (lane != 0) kept = sup = nnz = zero = 0;
        kept = block_sum_i(kept, ibuf);
        sup = block_sum_i(sup, ibuf);
        nnz = block_sum_i(nnz, ibuf);
        zero = block_sum_i(zero, ibuf);
        if (tid == 0) {
          a.cnt_kept[cta] = kept;
          a.cnt_sup[cta] = sup;
          a.cnt_nnz[cta] = nnz;
          a.cnt_zero[cta] = zero;
        }
      }
      GSYNC();
      // (C4) totals and this CTA's offsets; the maxima are reset for the next check
      int totk = 0, tots = 0, totn = 0, totz = 0, pk = 0, ps = 0, pz = 0;
      for (int c = tid; c < G; c += kThreads) {
        const int k = __ldcg(a.cnt_kept + c), s = __ldcg(a.cnt_sup + c), z = __ldcg(a.cnt_zero + c);
        totk += k;
        tots += s;
        totz += z;
        totn += __ldcg(a.cnt_nnz + c);
        if (c < cta) {
          pk += k;
          ps += s;
          pz += z;
        }
      }
      totk = block_sum_i(totk, ibuf);
      tots = block_sum_i(tots, ibuf);
      totn = block_sum_i(totn, ibuf);
      totz = block_sum_i(totz, ibuf);
      pk = block_sum_i(pk, ibuf);
      ps = block_sum_i(ps, ibuf);
      pz = block_sum_i(pz, ibuf);
      if (cta == 0 && tid == 0) {
        ctl->m_bits = 0ull;
        ctl->mlo_bits = 0u;
      }
      if (stop || cap) {
        // outputs of this lambda
        for (int j = f0 + tid; j < f1; j += kThreads) {
          const float2 b = ld_beta(a, j);
          a.beta_out[(long long)t * a.p + j] = __dadd_rn((double)b.x, (double)b.y);
        }
        if (a.mask_out)
          for (int w = f0 / 32 + tid; w < (f1 + 31) / 32; w += kThreads)
            a.mask_out[(long long)t * a.words + w] = __ldcg(a.mask + w);
        if (cta == 0 && tid == 0) {
          lasso_path_stats st;
          st.lambda = lam;
          st.primal = P;
          st.dual = D;
          st.gap = Gap;
          st.radius = rad;
          st.alpha = alpha;
          st.epochs = epochs;
          st.checks = checks;
          st.n_active = totk;
          st.n_nonzero = totn;
          st.x_columns = xcols;
          st.converged = stop ? 1 : 0;
          st.status = stop ? kStatusOK : kStatusNotConverged;
          a.stats[t] = st;
        }
        GSYNC();
        break;
      }
      // compaction: ascending safe-active list A, support positions sup0 and
      // the ascending list of coefficients the check set to zero
      if (warp == 0) {
        int runk = pk, runs = ps, runz = pz;
        for (int w0 = f0; w0 < f1; w0 += 32) {
          const int j = w0 + lane;
          const uint32_t word = __ldcg(a.mask + (w0 >> 5));
          const uint32_t zw = __ldcg(a.zbits + (w0 >> 5));
          const bool keep = (word >> lane) & 1u;
          const bool nz = keep && nonzero2(ld_beta(a, j));
          const unsigned lower = (1u << lane) - 1u;
          const int kpos = runk + __popc(word & lower);
          const unsigned smk = __ballot_sync(0xffffffffu, nz);
          if (keep) a.A[kpos] = j;
          if (nz) a.sup0[runs + __popc(smk & lower)] = kpos;
          if ((zw >> lane) & 1u) a.zl_j[runz + __popc(zw & lower)] = j;
          runk += __popc(word);
          runs += __popc(smk);
          runz += __popc(zw);
        }
      }
      if (cta == 0 && tid == 0) {
        ctl->q = totk;
        ctl->s = tots;
        ctl->nzl = totz;
      }
      scope_n = a.xtr_scope == 0 ? a.p : totk;
      GSYNC();
      PROF(0);
      // ======================= PASSES =======================
      {
        const int q = vload(ctl->q);
        int s = vload(ctl->s);
        int* sup = a.sup0;
        int* sup_next = a.sup1;
        if (cta == 0) {
          // residual shares of the coefficients removed by the check, ascending j
          const int nz = vload(ctl->nzl);
          if (nz > 0) {
            load_rho_regs<NGC>(a, a.rho_h, a.rho_l, rh, rl);
            for (int i = 0; i < nz; ++i) {
              const int jj = __ldcg(a.zl_j + i);
              const df2 d = df_from_double(-__ldcg(a.zl_b + jj));  // rho -= (0 - b) x_j
              const float* col = a.Xh + (long long)jj * a.ldx;
              const float* coll = XLO ? a.Xl + (long long)jj * a.ldx : nullptr;
#pragma unroll
              for (int k = 0; k < NGC; ++k) {
                const int g = tid + kChainThreads * k;
                if (tid < kChainThreads && g < a.ld4) {
                  const float4 x = ld_x4(col, g, a.n);
                  if (XLO) {
                    const float4 xl = ld_x4(coll, g, a.n);
                    axpy_df2(x.x, xl.x, d.h, d.l, rh[k].x, rl[k].x);
                    axpy_df2(x.y, xl.y, d.h, d.l, rh[k].y, rl[k].y);
                    axpy_df2(x.z, xl.z, d.h, d.l, rh[k].z, rl[k].z);
                    axpy_df2(x.w, xl.w, d.h, d.l, rh[k].w, rl[k].w);
                  } else {
                    axpy_df(x.x, d.h, d.l, rh[k].x, rl[k].x);
                    axpy_df(x.y, d.h, d.l, rh[k].y, rl[k].y);
                    axpy_df(x.z, d.h, d.l, rh[k].z, rl[k].z);
                    axpy_df(x.w, d.h, d.l, rh[k].w, rl[k].w);
                  }
                }
              }
            }
            store_rho_regs<NGC>(a, a.rho_h, a.rho_l, rh, rl);
            __syncthreads();
            if (tid == 0) ctl->nzl = 0;
          }
        }
        for (int e = 0; e < a.f && epochs < a.max_epochs; ++e) {
          // ---- one pass over the safe-active list, in rounds
          if (cta == 0) {
            load_rho_regs<NGC>(a, a.rho_h, a.rho_l, rh, rl);
            if (tid == 0) {
              ctl->pos = 0;
              ctl->sup_idx = 0;
              ctl->forced = -1;
              ctl->n_entered = 0;
            }
            __syncthreads();
          }
          for (;;) {
            PROF(7);
            // R1 (CTA 0): chain = [forced entry] + next support positions (at most s_cap)
            if (cta == 0) {
              const int si = vload(ctl->sup_idx), forced = vload(ctl->forced);
              const int take = min(s - si, a.s_cap - (forced >= 0 ? 1 : 0));
              const int nc = take + (forced >= 0 ? 1 : 0);
              const int rend = (si + take < s) ? __ldcg(sup + si + take) : q;
              for (int c = tid; c < nc; c += kThreads)
                a.chain[c] = (forced >= 0) ? (c == 0 ? forced : __ldcg(sup + si + c - 1)) : __ldcg(sup + si + c);
              __syncthreads();
              const float rb = rho_bound_from_regs<NGC>(a, rh, lam, nc, fbuf);
              if (tid == 0) {
                ctl->rho_bound = rb;
                ctl->nc = nc;
                ctl->round_end = rend;
                ctl->fstar = kNoPos;
              }
              store_rho_regs<NGC>(a, a.snap, a.snap + a.ldw, rh, rl);  // snapshot 0
              __syncthreads();
              run_chain<NGC, XLO>(a, cs, ring, jl, nc, rb, rh, rl);
              __threadfence();
              if (prof_thread) ctl->prof[5] += (unsigned long long)nc;
            }
            PROF(1);
            GSYNC();
            // R2 (all CTAs): the zero coefficients of [pos, round_end) must stay zero
            {
              const int pos = vload(ctl->pos), rend = vload(ctl->round_end), nc = vload(ctl->nc);
              const float rb = vload(ctl->rho_bound);
              const int span = rend - pos;
              const int gw = cta * nwarps + warp, nwg = G * nwarps;
              const int chunk = (span + nwg - 1) / nwg;
              const int i0 = pos + gw * chunk, i1 = min(rend, i0 + chunk);
              if (span > 0 && i0 < i1) {
                int seg = lower_bound_i(a.chain, nc, i0);
                int nextc = (seg < nc) ? __ldcg(a.chain + seg) : kNoPos;
                float4 r4[NG];
                int loaded = -1;
                const float lamf = __double2float_rn(lam);
                for (int i = i0; i < i1; ++i) {
                  if (i == nextc) {
                    ++seg;
                    nextc = (seg < nc) ? __ldcg(a.chain + seg) : kNoPos;
                    continue;
                  }
                  if (i > vload(ctl->fstar)) break;
                  const float* sh = a.snap + (size_t)seg * 2 * a.ldw;
                  if (loaded != seg) {
#pragma unroll
                    for (int k = 0; k < NG; ++k) {
                      const int g = lane + 32 * k;
                      r4[k] = (g < a.ld4) ? ldcg4(sh, g) : make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                    loaded = seg;
                  }
                  const int j = __ldcg(a.A + i);
                  const float c = warp_dot_f32<NG>(a.Xh + (long long)j * a.ldx, r4, a.ld4, a.n);
                  const float nf = __ldg(a.nrmf + j);
                  const float E = __fmul_ru(__fmul_ru(bf, nf), rb) + 1e-37f;
                  bool enters;
                  if (__fadd_ru(fabsf(c), E) < lamf * (1.0f - 1e-6f)) enters = false;
                  else if (__fsub_rd(fabsf(c), E) > lamf * (1.0f + 1e-6f)) enters = true;
                  else {
                    const df2 g = warp_dot_exact<NG, XLO>(a, j, sh, sh + a.ldw, __fmul_ru(nf, rb));
                    df2 nb, d;
                    cd_update(g, df2{0.f, 0.f}, __ldcg(a.ftab + j), nb, d);
                    enters = !df_is_zero(d);
                  }
                  if (enters) {
                    if (lane == 0) atomicMin(&ctl->fstar, i);
                    break;
                  }
                }
              }
            }
            GSYNC();
            PROF(2);
            // R3 (CTA 0): accept the round, or roll back to the first entering position
            if (cta == 0) {
              const int fst = vload(ctl->fstar), nc = vload(ctl->nc), rend = vload(ctl->round_end);
              const int forced = vload(ctl->forced), si = vload(ctl->sup_idx);
              if (fst == kNoPos) {
                if (tid == 0) {
                  if (forced >= 0 && nonzero2(ld_beta(a, __ldcg(a.A + forced))))
                    a.entered[ctl->n_entered++] = forced;
                  ctl->sup_idx = si + nc - (forced >= 0 ? 1 : 0);
                  ctl->pos = rend;
                  ctl->forced = -1;
                  ctl->done = rend >= q ? 1 : 0;
                }
              } else {
                // chain entries before the entering position stand; later ones are undone
                if (prof_thread) ctl->prof[6] += 1ull;
                const int seg = lower_bound_i(a.chain, nc, fst);
                for (int c = seg + tid; c < nc; c += kThreads) a.bdf[__ldcg(a.A + __ldcg(a.chain + c))] = a.oldb[c];
                const float* sh = a.snap + (size_t)seg * 2 * a.ldw;
                load_rho_regs<NGC>(a, sh, sh + a.ldw, rh, rl);
                __syncthreads();
                if (tid == 0) {
                  if (forced >= 0 && nonzero2(ld_beta(a, __ldcg(a.A + forced))))
                    a.entered[ctl->n_entered++] = forced;
                  ctl->sup_idx = si + seg - (forced >= 0 ? 1 : 0);
                  ctl->forced = fst;
                  ctl->pos = fst;
                  ctl->done = 0;
                }
              }
              __threadfence();
              __syncthreads();
            }
            GSYNC();
            PROF(3);
            if (vload(ctl->done)) break;
          }
          // end of pass (CTA 0): write rho; next support list = survivors of the
          // old list merged with the entered positions (both ascending)
          if (cta == 0) {
            store_rho_regs<NGC>(a, a.rho_h, a.rho_l, rh, rl);
            const int ne = vload(ctl->n_entered);
            __syncthreads();
            int nsurv = 0;
            for (int base = 0; base < s; base += kThreads) {
              const int i = base + tid;
              int posv = 0;
              bool keep = false;
              if (i < s) {
                posv = __ldcg(sup + i);
                keep = nonzero2(ld_beta(a, __ldcg(a.A + posv)));
              }
              int tot;
              const int r = block_rank(keep, ibuf, &tot);
              if (keep) a.zl_j[nsurv + r] = posv;
              nsurv += tot;
            }
            __syncthreads();
            for (int k = tid; k < nsurv; k += kThreads) {
              const int v = __ldcg(a.zl_j + k);
              sup_next[k + lower_bound_i(a.entered, ne, v)] = v;
            }
            for (int k = tid; k < ne; k += kThreads) {
              const int v = __ldcg(a.entered + k);
              sup_next[k + lower_bound_i(a.zl_j, nsurv, v)] = v;
            }
            if (tid == 0) ctl->s = nsurv + ne;
            __threadfence();
            __syncthreads();
          }
          ++epochs;
          xcols += q;
          GSYNC();
          PROF(4);
          s = vload(ctl->s);
          int* tmp = sup;
          sup = sup_next;
          sup_next = tmp;
        }
      }
      GSYNC();
    }
  }
done:
  return;
#undef GSYNC
#undef PROF
}

// ---------------------------------------------------------------- setup kernels
// ||x_j||, 1/||x_j||^2, c0_j = x_j^T y -> lambda_max = ||X^T y||_inf (Sec. 1.2),
// finiteness of X, split planes of an FP64 X, beta0 in double-float.
template <typename XT>
__global__ void precompute_kernel(const XT* X, long long ldx, int n, int p, const double* y, const double* beta0,
                                  float* Xh, float* Xl, long long ldh, double* nrm, float* nrmf, float4* ftab,
                                  float2* bdf, float2* b0df, Ctrl* ctl) {
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
__global__ void finish_setup_kernel(Ctrl* ctl, const double* ratios, int T) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    ctl->lambda_max = __longlong_as_double((long long)ctl->m_bits);
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

// ---------------------------------------------------------------- host side
namespace {

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

constexpr int kMaxGrid = 1024;

struct Layout {
  size_t ctrl, cnt, part_l1, nrm, nrmf, ftab, bdf, b0df, rho_h, rho_l, rho0_h, rho0_l, ctil, mask, A, sup0, sup1,
      chain, entered, oldb, recs, snap, zl_j, zl_b, zbits, Xh, Xl, total;
  long long ldh;
  int s_cap;
};

Layout make_layout(int64_t n, int64_t p, bool f64, int64_t ldx) {
  Layout L{};
  const long long ld_work = (n + 3) / 4 * 4;
  int s_cap = 4096;
  if ((int64_t)s_cap > p) s_cap = (int)p;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += align256(bytes);
    return o;
  };
  const int64_t words = (p + 31) / 32;
  L.ctrl = take(sizeof(Ctrl));
  L.cnt = take(sizeof(int) * 4 * kMaxGrid);
  L.part_l1 = take(sizeof(double) * kMaxGrid);
  L.nrm = take(sizeof(double) * p);
  L.nrmf = take(sizeof(float) * p);
  L.ftab = take(sizeof(float4) * p);
  L.bdf = take(sizeof(float2) * p);
  L.b0df = take(sizeof(float2) * p);
  // residual planes and snapshots use the tight leading dimension
  const long long ldh = ld_work;
  (void)ldx;
  L.rho_h = take(sizeof(float) * ldh);
  L.rho_l = take(sizeof(float) * ldh);
  L.rho0_h = take(sizeof(float) * ldh);
  L.rho0_l = take(sizeof(float) * ldh);
  L.ctil = take(sizeof(float) * p);
  L.mask = take(sizeof(uint32_t) * words);
  L.A = take(sizeof(int) * p);
  L.sup0 = take(sizeof(int) * p);
  L.sup1 = take(sizeof(int) * p);
  L.chain = take(sizeof(int) * (s_cap + 1));
  L.entered = take(sizeof(int) * p);
  L.oldb = take(sizeof(float2) * (s_cap + 1));
  L.recs = take(sizeof(ChainRec) * (s_cap + 1));
  L.snap = take(sizeof(float) * 2 * (size_t)ldh * (size_t)(s_cap + 2));
  L.zl_j = take(sizeof(int) * p);
  L.zl_b = take(sizeof(double) * p);
  L.zbits = take(sizeof(uint32_t) * words);
  if (f64) {
    L.Xh = take(sizeof(float) * (size_t)ld_work * (size_t)p);
    L.Xl = take(sizeof(float) * (size_t)ld_work * (size_t)p);
  }
  L.total = off;
  L.ldh = ldh;
  L.s_cap = s_cap;
  return L;
}

template <int NGC, bool XLO>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&path_kernel<NGC, XLO>);
}

const void* pick_kernel(int ngc, bool xlo) {
  if (xlo) return ngc == 1 ? kernel_ptr<1, true>() : ngc == 2 ? kernel_ptr<2, true>() : kernel_ptr<4, true>();
  return ngc == 1 ? kernel_ptr<1, false>() : ngc == 2 ? kernel_ptr<2, false>() : kernel_ptr<4, false>();
}

}  // namespace

size_t path_workspace_size(int64_t n, int64_t p, lasso_dtype xt, int64_t ldx) {
  if (n < 1 || n > kMaxRows || p < 1 || p > (int64_t)INT32_MAX / 4) return 0;
  if (xt != LASSO_F32 && xt != LASSO_F64) return 0;
  if (xt == LASSO_F32 && (ldx < n || ldx % 4 != 0)) ldx = (n + 3) / 4 * 4;
  return make_layout(n, p, xt == LASSO_F64, ldx).total;
}

lasso_status path_launch(const void* X, lasso_dtype xt, int64_t n, int64_t p, int64_t ldx, const double* y,
                         const double* ratios, int32_t T, const double* beta0, const lasso_opts& o,
                         double* beta_out, uint32_t* mask_out, lasso_path_stats* stats, void* ws, size_t ws_bytes,
                         cudaStream_t stream) {
  const bool f64 = xt == LASSO_F64;
  const Layout L = make_layout(n, p, f64, ldx);
  if (ws_bytes < L.total)
    return set_error(LASSO_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes required", ws_bytes,
                     L.total);
  char* base = static_cast<char*>(ws);
  Args a{};
  a.n = (int)n;
  a.p = (int)p;
  a.ldw = L.ldh;
  a.ldx = f64 ? L.ldh : ldx;
  a.ld4 = (int)((n + 3) / 4);
  a.T = T;
  a.words = (int)((p + 31) / 32);
  a.f = o.screen_period;
  a.dual_point = o.dual_point;
  a.xtr_scope = o.xtr_scope;
  a.warm_start = o.warm_start;
  a.max_epochs = o.max_epochs;
  a.y = y;
  a.ratios = ratios;
  a.beta_out = beta_out;
  a.mask_out = mask_out;
  a.stats = stats;
  a.ctrl = reinterpret_cast<Ctrl*>(base + L.ctrl);
  a.cnt_kept = reinterpret_cast<int*>(base + L.cnt);
  a.cnt_sup = a.cnt_kept + kMaxGrid;
  a.cnt_nnz = a.cnt_sup + kMaxGrid;
  a.cnt_zero = a.cnt_nnz + kMaxGrid;
  a.part_l1 = reinterpret_cast<double*>(base + L.part_l1);
  a.nrm = reinterpret_cast<double*>(base + L.nrm);
  a.nrmf = reinterpret_cast<float*>(base + L.nrmf);
  a.ftab = reinterpret_cast<float4*>(base + L.ftab);
  a.bdf = reinterpret_cast<float2*>(base + L.bdf);
  a.b0df = reinterpret_cast<float2*>(base + L.b0df);
  a.rho_h = reinterpret_cast<float*>(base + L.rho_h);
  a.rho_l = reinterpret_cast<float*>(base + L.rho_l);
  a.rho0_h = reinterpret_cast<float*>(base + L.rho0_h);
  a.rho0_l = reinterpret_cast<float*>(base + L.rho0_l);
  a.ctil = reinterpret_cast<float*>(base + L.ctil);
  a.mask = reinterpret_cast<uint32_t*>(base + L.mask);
  a.A = reinterpret_cast<int*>(base + L.A);
  a.sup0 = reinterpret_cast<int*>(base + L.sup0);
  a.sup1 = reinterpret_cast<int*>(base + L.sup1);
  a.chain = reinterpret_cast<int*>(base + L.chain);
  a.entered = reinterpret_cast<int*>(base + L.entered);
  a.oldb = reinterpret_cast<float2*>(base + L.oldb);
  a.recs = reinterpret_cast<ChainRec*>(base + L.recs);
  a.snap = reinterpret_cast<float*>(base + L.snap);
  a.zl_j = reinterpret_cast<int*>(base + L.zl_j);
  a.zl_b = reinterpret_cast<double*>(base + L.zl_b);
  a.zbits = reinterpret_cast<uint32_t*>(base + L.zbits);
  a.s_cap = L.s_cap;
  if (f64) {
    a.Xh = reinterpret_cast<const float*>(base + L.Xh);
    a.Xl = reinterpret_cast<const float*>(base + L.Xl);
  } else {
    a.Xh = static_cast<const float*>(X);
    a.Xl = nullptr;
  }

  const int ngc = (a.ld4 <= 128) ? 1 : (a.ld4 <= 256 ? 2 : 4);
  const void* kfn = pick_kernel(ngc, f64);
  int dev = 0, sms = 0, coop = 0, smem_optin = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CUDA_TRY(cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (!coop) return set_error(LASSO_ERR_CUDA, "device does not support cooperative launch");
  // CTA 0's dynamic shared memory: the feature list of a round and the ring of
  // kRing staged columns (each chain thread's granules, two planes for FP64 X)
  const size_t jl_bytes = (((size_t)(L.s_cap + 1) * sizeof(int)) + 127) & ~(size_t)127;
  const size_t dyn = jl_bytes + (size_t)kRing * ngc * kChainThreads * 16 * (f64 ? 2 : 1);
  if (dyn + 8192 > (size_t)smem_optin)
    return set_error(LASSO_ERR_INVALID_ARG, "the chain ring of %zu bytes does not fit shared memory", dyn);
  CUDA_TRY(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, kThreads, dyn));
  if (per_sm < 1) return set_error(LASSO_ERR_CUDA, "the path kernel cannot be resident (occupancy 0)");
  per_sm = std::min(per_sm, 2);
  const int grid = std::min(sms * per_sm, kMaxGrid);
  int fs = (int)((p + grid - 1) / grid);
  a.fs = (fs + 31) / 32 * 32;

  CUDA_TRY(cudaMemsetAsync(a.ctrl, 0, sizeof(Ctrl), stream));
  CUDA_TRY(cudaMemsetAsync(a.cnt_kept, 0, sizeof(int) * 4 * kMaxGrid, stream));
  const int blocks = sms * 8;
  if (f64)
    precompute_kernel<double><<<blocks, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                          const_cast<float*>(a.Xh), const_cast<float*>(a.Xl), a.ldw,
                                                          a.nrm, a.nrmf, a.ftab, a.bdf, a.b0df, a.ctrl);
  else
    precompute_kernel<float><<<blocks, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                         nullptr, nullptr, a.ldw, a.nrm, a.nrmf, a.ftab, a.bdf, a.b0df,
                                                         a.ctrl);
  CUDA_TRY(cudaGetLastError());
  const int rb = (int)std::min<long long>(a.ldw, (long long)sms * 4);
  if (f64)
    rho_init_kernel<double><<<rb, 256, 0, stream>>>(static_cast<const double*>(X), ldx, (int)n, (int)p, y, beta0,
                                                    a.rho_h, a.rho_l, a.rho0_h, a.rho0_l, (int)a.ldw, o.gap_tol_rel,
                                                    a.ctrl);
  else
    rho_init_kernel<float><<<rb, 256, 0, stream>>>(static_cast<const float*>(X), ldx, (int)n, (int)p, y, beta0,
                                                   a.rho_h, a.rho_l, a.rho0_h, a.rho0_l, (int)a.ldw, o.gap_tol_rel,
                                                   a.ctrl);
  CUDA_TRY(cudaGetLastError());
  finish_setup_kernel<<<1, 32, 0, stream>>>(a.ctrl, ratios, T);
  CUDA_TRY(cudaGetLastError());
  void* params[] = {&a};
  CUDA_TRY(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(kThreads), params, dyn, stream));
  stats_error_kernel<<<1, 128, 0, stream>>>(a.ctrl, stats, T);
  CUDA_TRY(cudaGetLastError());
  return LASSO_OK;
}

}  // namespace lassogs
