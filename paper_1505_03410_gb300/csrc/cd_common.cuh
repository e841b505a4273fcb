// Device building blocks shared by the single-path and the batched solvers:
// warp dot products (FP32 with a forward-error bound, and exact double-float
// with limb reduction), the soft-threshold step of Algorithm 1, and the
// coordinate chain (sequential updates of the nonzero coefficients with
// cp.async-staged columns).  Functions taking a context `a` need its fields
// Xh, Xl, ldx, ld4, n, ldw, A, chain, ftab, bdf, nrmf, recs, oldb, snap, msnap.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "device_util.cuh"
#include "dfloat.cuh"
#include "../../include/lassogs.h"

namespace lassogs {

constexpr int kThreads = 256;   // threads per CTA
constexpr int kChainWarps = 4;  // warps of CTA 0 that run the chain
constexpr int kChainThreads = kChainWarps * 32;
constexpr int kProducerWarp = 4;
constexpr int kStatusOK = 0, kStatusNotConverged = 5;
constexpr int kNoPos = 0x7fffffff;
constexpr int kErrInvalidArg = 1;

template <typename T>
__device__ __forceinline__ T vload(const T& x) {
  return *reinterpret_cast<const volatile T*>(&x);
}

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
// zero the rows of a granule whose bit (0..3) is clear (row subsets)
__device__ __forceinline__ float4 mask_bits(float4 x, uint32_t bits) {
  if ((bits & 15u) != 15u) {
    if (!(bits & 1u)) x.x = 0.f;
    if (!(bits & 2u)) x.y = 0.f;
    if (!(bits & 4u)) x.z = 0.f;
    if (!(bits & 8u)) x.w = 0.f;
  }
  return x;
}
__device__ __forceinline__ float4 ld_x4(const float* col, int g, int n) {
  return mask_rows(__ldg(reinterpret_cast<const float4*>(col) + g), g, n);
}
__device__ __forceinline__ float4 ldcg4(const float* p, int g) { return __ldcg(reinterpret_cast<const float4*>(p) + g); }
template <typename Ctx>
__device__ __forceinline__ float2 ld_beta(const Ctx& a, int j) { return __ldcg(a.bdf + j); }
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

// Two columns at once against the same rho: both columns' loads are issued
// before either is reduced (twice the bytes in flight per warp).  Each result
// is computed exactly as warp_dot_f32 computes it.
template <int NG>
__device__ __forceinline__ void warp_dot_f32_2(const float* ca, const float* cb, const float4 (&r)[NG], int ld4, int n,
                                               float& outa, float& outb) {
  int lane = threadIdx.x & 31;
  float4 xa[NG], xb[NG];
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    int g = lane + 32 * k;
    xa[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    xb[k] = xa[k];
    if (g < ld4) {
      xa[k] = ld_x4(ca, g, n);
      xb[k] = ld_x4(cb, g, n);
    }
  }
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f, b0 = 0.f, b1 = 0.f, b2 = 0.f, b3 = 0.f;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    int g = lane + 32 * k;
    if (g < ld4) {
      a0 = __fmaf_rn(xa[k].x, r[k].x, a0);
      a1 = __fmaf_rn(xa[k].y, r[k].y, a1);
      a2 = __fmaf_rn(xa[k].z, r[k].z, a2);
      a3 = __fmaf_rn(xa[k].w, r[k].w, a3);
      b0 = __fmaf_rn(xb[k].x, r[k].x, b0);
      b1 = __fmaf_rn(xb[k].y, r[k].y, b1);
      b2 = __fmaf_rn(xb[k].z, r[k].z, b2);
      b3 = __fmaf_rn(xb[k].w, r[k].w, b3);
    }
  }
  float sa = __fadd_rn(__fadd_rn(a0, a1), __fadd_rn(a2, a3));
  float sb = __fadd_rn(__fadd_rn(b0, b1), __fadd_rn(b2, b3));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sa = __fadd_rn(sa, __shfl_xor_sync(0xffffffffu, sa, o));
    sb = __fadd_rn(sb, __shfl_xor_sync(0xffffffffu, sb, o));
  }
  outa = sa;
  outb = sb;
}

// Exact (double-float, order-independent) dot of column j with rho given as
// two planes in global memory; bound >= sum_i |x_ij rho_i|.  Whole warp.
template <int NG, bool XLO, typename Ctx>
__device__ df2 warp_dot_exact(const Ctx& a, int j, const float* rh, const float* rl, float bound) {
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
// The chain runs on the first CW warps; granule g = tid + 32 CW k.
template <int NGC, int CW, bool XLO, typename Ctx>
__device__ __forceinline__ void stage_column(const Ctx& a, float4* ring, int s, int j) {
  constexpr int CT = 32 * CW;
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + CT * k;
    if (g < a.ld4) {
      float4* dst = ring + ((size_t)(s * NGC + k) * CT + tid) * (XLO ? 2 : 1);
      cp_async16(dst, a.Xh + (long long)j * a.ldx + 4 * g);
      if (XLO) cp_async16(dst + 1, a.Xl + (long long)j * a.ldx + 4 * g);
    }
  }
}

// Coordinate updates for chain entries c = 0..nc-1 (positions into A), in
// order.  rho is held by the 32 CW chain threads (granules t + 32 CW k); each
// of them stages its own granules of the next kRing columns with cp.async,
// so no cross-thread handshake is needed for the column data.  The only
// cross-thread step per entry is the exact limb reduction of x_j^T rho: one
// redux per limb when the chain is a single warp, plus a named barrier and a
// shared-memory exchange between warps otherwise.  Writes the new
// coefficients to bdf, the old ones to oldb and the residual after entry c to
// snapshot c + 1.
template <int NGC, int CW, bool XLO, bool EN = false, typename Ctx>
__device__ void run_chain(const Ctx& a, ChainSmem& cs, float4* ring, int* jl, int nc, float rho_bound,
                          float4 (&rh)[NGC], float4 (&rl)[NGC], uint32_t row_bits = 0xffffffffu,
                          df2 ridge = df2{0.f, 0.f}) {
  static_assert(CW >= 1 && CW <= kChainWarps, "chain warps");
  constexpr int CT = 32 * CW;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (nc <= 0) return;
  // records and the feature list of this round
  for (int c = tid; c < nc; c += kThreads) {
    const int j = __ldcg(a.A + __ldcg(a.chain + c));
    ChainRec r;
    r.tab = __ldcg(a.ftab + j);
    r.b = ld_beta(a, j);
    r.nf = __ldcg(a.nrmf + j);
    r.j = j;
    a.recs[c] = r;
    jl[c] = j;
  }
  __syncthreads();
  if (warp < CW) {
    // prologue: stage the first kRing columns, fetch the first two records
#pragma unroll
    for (int s = 0; s < kRing; ++s) {
      if (s < nc) stage_column<NGC, CW, XLO>(a, ring, s, jl[s]);
      cp_async_commit();
    }
    ChainRec r0 = a.recs[0];
    ChainRec r1 = (nc > 1) ? a.recs[1] : r0;
    // movement bound sum |delta| ||x_j|| (thread 0): snapshot e + 1 carries it
    float mv = (tid == 0) ? a.msnap[0] : 0.f;
    for (int e = 0; e < nc; ++e) {
      const int slot = e % kRing;
      cp_async_wait<kRing - 1>();  // this thread's copies for entry e have landed
      float4 xs[NGC], xls[NGC];
      // compensated accumulators: two when a lane holds one granule (fewer
      // limb conversions), four (one per float4 component) for longer dots
      constexpr bool kFour = NGC >= 2;
      float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f, S2 = 0.f, C2 = 0.f, S3 = 0.f, C3 = 0.f;
#pragma unroll
      for (int k = 0; k < NGC; ++k) {
        const int g = tid + CT * k;
        xs[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        xls[k] = xs[k];
        if (g < a.ld4) {
          const float4* src = ring + ((size_t)(slot * NGC + k) * CT + tid) * (XLO ? 2 : 1);
          xs[k] = mask_bits(mask_rows(src[0], g, a.n), row_bits >> (4 * k));
          if (XLO) {
            xls[k] = mask_bits(mask_rows(src[1], g, a.n), row_bits >> (4 * k));
            dot2_acc2(xs[k].x, xls[k].x, rh[k].x, rl[k].x, S0, C0);
            dot2_acc2(xs[k].y, xls[k].y, rh[k].y, rl[k].y, S1, C1);
            dot2_acc2(xs[k].z, xls[k].z, rh[k].z, rl[k].z, kFour ? S2 : S0, kFour ? C2 : C0);
            dot2_acc2(xs[k].w, xls[k].w, rh[k].w, rl[k].w, kFour ? S3 : S1, kFour ? C3 : C1);
          } else {
            dot2_acc(xs[k].x, rh[k].x, rl[k].x, S0, C0);
            dot2_acc(xs[k].y, rh[k].y, rl[k].y, S1, C1);
            dot2_acc(xs[k].z, rh[k].z, rl[k].z, kFour ? S2 : S0, kFour ? C2 : C0);
            dot2_acc(xs[k].w, rh[k].w, rl[k].w, kFour ? S3 : S1, kFour ? C3 : C1);
          }
        }
      }
      // refill the slot just read with entry e + kRing (always commit a group)
      if (e + kRing < nc) stage_column<NGC, CW, XLO>(a, ring, slot, jl[e + kRing]);
      cp_async_commit();
      const ChainRec r2 = (e + 2 < nc) ? a.recs[e + 2] : r1;  // prefetch
      // |partial sums| <= ||x_j|| ||rho|| <= nf * rho_bound
      float sc, isc;
      limb_scale(2.0f * r0.nf * rho_bound + 1e-30f, sc, isc);
      limbs3 L;
      if (kFour) {
        L = limbs_add(limbs_add(limbs_add(to_limbs(S0, sc), to_limbs(C0, sc)),
                                limbs_add(to_limbs(S1, sc), to_limbs(C1, sc))),
                      limbs_add(limbs_add(to_limbs(S2, sc), to_limbs(C2, sc)),
                                limbs_add(to_limbs(S3, sc), to_limbs(C3, sc))));
        // carries out of the two low limbs before the cross-thread sum: every
        // limb is then below 2^22 + 1 in magnitude, and 128 of them fit int32
        L = limbs_norm(L);
      } else {
        // one granule per lane: fold the two compensated sums first (an
        // error-free TwoSum of the leading parts, the tails added in FP32,
        // far below the double-float's 2^-48), then two limb conversions;
        // two partials per thread keep every limb sum inside int32 unnormalised
        float sh, se;
        two_sum(S0, S1, sh, se);
        const float st = __fadd_rn(__fadd_rn(C0, C1), se);
        L = limbs_add(to_limbs(sh, sc), to_limbs(st, sc));
      }
      L = warp_limbs_sum(L);
      limbs3 Tl = L;
      if (CW > 1) {
        if (lane == 0) cs.red[e & 1][warp] = L;
        named_bar_sync(1, CT);
        Tl = cs.red[e & 1][0];
#pragma unroll
        for (int w = 1; w < CW; ++w) Tl = limbs_add(Tl, cs.red[e & 1][w]);
      }
      df2 g = limbs_to_df(Tl, isc);
      const df2 beta{r0.b.x, r0.b.y};
      // Elastic-Net: the augmented column's correlation x_j^T rho - mu beta_j
      if constexpr (EN) g = df_sub(g, df_mul(ridge, beta));
      df2 nb, d;
      cd_update(g, beta, r0.tab, nb, d);
      if (tid == 0) {
        a.oldb[e] = r0.b;
        a.bdf[r0.j] = make_float2(nb.h, nb.l);
        mv = __fadd_ru(mv, __fmul_ru(__fadd_ru(fabsf(d.h), fabsf(d.l)), r0.nf));
        a.msnap[e + 1] = mv;
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
        const int gi = tid + CT * k;
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

// rho planes (global) <-> chain registers of CTA 0 (threads >= 32 CW hold zeros)
template <int NGC, int CW, typename Ctx>
__device__ __forceinline__ void load_rho_regs(const Ctx& a, const float* h, const float* l, float4 (&rh)[NGC],
                                              float4 (&rl)[NGC]) {
  constexpr int CT = 32 * CW;
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + CT * k;
    rh[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    rl[k] = rh[k];
    if (tid < CT && g < a.ld4) {
      rh[k] = ldcg4(h, g);
      rl[k] = ldcg4(l, g);
    }
  }
}
template <int NGC, int CW, typename Ctx>
__device__ __forceinline__ void store_rho_regs(const Ctx& a, float* h, float* l, const float4 (&rh)[NGC],
                                               const float4 (&rl)[NGC]) {
  constexpr int CT = 32 * CW;
  const int tid = threadIdx.x;
#pragma unroll
  for (int k = 0; k < NGC; ++k) {
    const int g = tid + CT * k;
    if (tid < CT && g < a.ld4) {
      __stcg(reinterpret_cast<float4*>(h) + g, rh[k]);
      __stcg(reinterpret_cast<float4*>(l) + g, rl[k]);
    }
  }
}

// Bound on ||rho|| for every iterate of a round: CD does not increase
// P = 1/2 ||rho||^2 + lambda ||beta||_1 and only the chain coefficients move,
// so ||rho_k||^2 <= ||rho_0||^2 + 2 lambda sum_chain |beta_c|.  With the
// Elastic-Net's ridge term (mu/2) ||beta||^2 in P the bound gains
// mu sum_chain beta_c^2.  Rounded up.
template <int NGC, bool EN = false, typename Ctx>
__device__ float rho_bound_from_regs(const Ctx& a, const float4 (&rh)[NGC], double lam, int nc, float* fbuf,
                                     double ridge = 0.0) {
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
  float l1 = 0.f, l2 = 0.f;
  for (int c = tid; c < nc; c += kThreads) {
    const float2 b = ld_beta(a, __ldcg(a.A + __ldcg(a.chain + c)));
    const float ab = __fmul_ru(fabsf(b.x), 1.0001f);
    l1 = __fadd_ru(l1, ab);
    if constexpr (EN) l2 = __fmaf_ru(ab, ab, l2);
  }
  for (int o = 16; o > 0; o >>= 1) {
    ss = __fadd_ru(ss, __shfl_xor_sync(0xffffffffu, ss, o));
    l1 = __fadd_ru(l1, __shfl_xor_sync(0xffffffffu, l1, o));
    if constexpr (EN) l2 = __fadd_ru(l2, __shfl_xor_sync(0xffffffffu, l2, o));
  }
  __syncthreads();
  if ((tid & 31) == 0) {
    fbuf[tid >> 5] = ss;
    fbuf[8 + (tid >> 5)] = l1;
    if constexpr (EN) fbuf[16 + (tid >> 5)] = l2;
  }
  __syncthreads();
  float S = 0.f, L = 0.f, L2 = 0.f;
  for (int w = 0; w < kThreads / 32; ++w) {
    S = __fadd_ru(S, fbuf[w]);
    L = __fadd_ru(L, fbuf[8 + w]);
    if constexpr (EN) L2 = __fadd_ru(L2, fbuf[16 + w]);
  }
  __syncthreads();
  float P2 = __fadd_ru(S, __fmul_ru(__fmul_ru(2.0f, __double2float_ru(lam)), L));
  if constexpr (EN) P2 = __fadd_ru(P2, __fmul_ru(__double2float_ru(ridge), L2));
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

}  // namespace lassogs
