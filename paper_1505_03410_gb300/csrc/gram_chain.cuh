// Building blocks of the Gram (covariance) form of the coordinate chain.
//
// Cyclic coordinate descent over the nonzero coefficients S of a round needs,
// at step c, g_c = x_c^T rho_c with rho_c the residual after the c earlier
// steps of the round.  rho_c = rho_0 - sum_{c' < c} delta_c' x_c', so
//   g_c = x_c^T rho_0 - sum_{c' < c} delta_c' G[c][c'],   G = X_S^T X_S
// (Friedman, Hastie, Tibshirani, "Regularization paths for generalized linear
// models via coordinate descent", J. Stat. Softw. 2010, Sec. 2.2: covariance
// updates).  With G cached and x_c^T rho_0 computed before the round, a step
// no longer reads x_c nor reduces an n-long dot product: the coordinates of
// a block of 32 live in the lanes of one warp, and a step is the
// soft-threshold of one lane, a broadcast, and one multiply-add per later
// lane.  The iterates are those of the sequential method up to rounding:
// every term is a double-float (about 48 bits), as the residual updates of
// the direct form are.
//
// This file holds the exact dot products that fill g and G (double-float
// results of exact, order-independent limb sums, with the limb scale taken
// from the data) and the double-float multiply-adds of the updates.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cd_common.cuh"

namespace lassogs {

constexpr int kGramMaxNc = 2048;  // chain entries of a Gram round (held in shared memory)
constexpr int kGramHelpers = 6;   // helper warps of CTA 0: warps 1, 2, 3, 5, 6, 7

// Exact sum over the 32 lanes of S + C (double-float result).  The limb scale
// comes from the largest |S| + |C| of the warp, so no outside bound is needed:
// 64 terms of magnitude <= m sum to <= 64 m, below 2^(E-1) for the scale.
__device__ __forceinline__ df2 warp_exact_sum(float S, float C) {
  const float m = __fadd_ru(fabsf(S), fabsf(C));
  const unsigned mb = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  float sc, isc;
  limb_scale(__fmul_ru(__uint_as_float(mb), 64.0f), sc, isc);
  limbs3 L = limbs_add(to_limbs(S, sc), to_limbs(C, sc));
  L = warp_limbs_sum(L);
  return limbs_to_df(L, isc);
}

// (S, C) += x * y for binary32 x, y: TwoProduct into a compensated sum
__device__ __forceinline__ void dot1_acc(float x, float y, float& S, float& C) {
  const float p = __fmul_rn(x, y);
  const float e = __fmaf_rn(x, y, -p);
  float s, t;
  two_sum(S, p, s, t);
  S = s;
  C = __fadd_rn(C, __fadd_rn(t, e));
}

// merge two compensated partial sums into one (leading part exact, tails in FP32)
__device__ __forceinline__ void merge_partials(float S0, float C0, float S1, float C1, float& S, float& C) {
  float sh, se;
  two_sum(S0, S1, sh, se);
  S = sh;
  C = __fadd_rn(__fadd_rn(C0, C1), se);
}

// Exact x^T rho of a column (x = xh + xl when XLO) with a residual given as two
// planes in global memory.  Whole warp; rows >= n of the column are masked.
template <int NG, bool XLO>
__device__ df2 warp_dot_col_rho(const float* colh, const float* coll, const float* rh, const float* rl, int ld4, int n) {
  const int lane = threadIdx.x & 31;
  float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    const int g = lane + 32 * k;
    if (g < ld4) {
      const float4 x = ld_x4(colh, g, n);
      const float4 h = ldcg4(rh, g), l = ldcg4(rl, g);
      if (XLO) {
        const float4 xl = ld_x4(coll, g, n);
        dot2_acc2(x.x, xl.x, h.x, l.x, S0, C0);
        dot2_acc2(x.y, xl.y, h.y, l.y, S1, C1);
        dot2_acc2(x.z, xl.z, h.z, l.z, S0, C0);
        dot2_acc2(x.w, xl.w, h.w, l.w, S1, C1);
      } else {
        dot2_acc(x.x, h.x, l.x, S0, C0);
        dot2_acc(x.y, h.y, l.y, S1, C1);
        dot2_acc(x.z, h.z, l.z, S0, C0);
        dot2_acc(x.w, h.w, l.w, S1, C1);
      }
    }
  }
  float S, C;
  merge_partials(S0, C0, S1, C1, S, C);
  return warp_exact_sum(S, C);
}

// Exact x_a^T x_b of two columns (each xh + xl when XLO; the product of the
// two low parts, below 2^-48 of the total, is left out).  Whole warp.  rm
// (nullptr: every row) restricts the sum to the rows i with rm[i] != 0 (the
// row subset of a batched problem).
template <int NG, bool XLO>
__device__ df2 warp_dot_cols(const float* ah, const float* al, const float* bh, const float* bl, int ld4, int n,
                             const uint8_t* rm = nullptr) {
  const int lane = threadIdx.x & 31;
  float S0 = 0.f, C0 = 0.f, S1 = 0.f, C1 = 0.f;
#pragma unroll
  for (int k = 0; k < NG; ++k) {
    const int g = lane + 32 * k;
    if (g < ld4) {
      float4 x = ld_x4(ah, g, n);
      const float4 y = ld_x4(bh, g, n);
      if (rm != nullptr) {
        const int r = 4 * g;
        if (!rm[r]) x.x = 0.f;
        if (r + 1 < n && !rm[r + 1]) x.y = 0.f;
        if (r + 2 < n && !rm[r + 2]) x.z = 0.f;
        if (r + 3 < n && !rm[r + 3]) x.w = 0.f;
      }
      if (XLO) {
        float4 xl = ld_x4(al, g, n);
        const float4 yl = ld_x4(bl, g, n);
        if (x.x == 0.f) xl.x = 0.f;
        if (x.y == 0.f) xl.y = 0.f;
        if (x.z == 0.f) xl.z = 0.f;
        if (x.w == 0.f) xl.w = 0.f;
        dot2_acc2(x.x, xl.x, y.x, yl.x, S0, C0);
        dot2_acc2(x.y, xl.y, y.y, yl.y, S1, C1);
        dot2_acc2(x.z, xl.z, y.z, yl.z, S0, C0);
        dot2_acc2(x.w, xl.w, y.w, yl.w, S1, C1);
      } else {
        dot1_acc(x.x, y.x, S0, C0);
        dot1_acc(x.y, y.y, S1, C1);
        dot1_acc(x.z, y.z, S0, C0);
        dot1_acc(x.w, y.w, S1, C1);
      }
    }
  }
  float S, C;
  merge_partials(S0, C0, S1, C1, S, C);
  return warp_exact_sum(S, C);
}

// g - d * G for double-floats: the product's error terms and the tail are
// combined as in axpy_df, then renormalised.
__device__ __forceinline__ df2 df_sub_mul(df2 g, df2 d, df2 G) {
  const float p = __fmul_rn(d.h, G.h);
  float e = __fmaf_rn(d.h, G.h, -p);
  e = __fmaf_rn(d.h, G.l, e);
  e = __fmaf_rn(d.l, G.h, e);
  float s, t;
  two_sum(g.h, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(g.l, e));
  df2 r;
  two_sum(s, t, r.h, r.l);
  return r;
}

// sign(u) (|u| - thr)_+ in double-float (the soft-threshold of Algorithm 1's
// coordinate update), with both candidates u - thr and u + thr formed at once.
// The sign of a double-float difference is exact, so the decision is the one
// of |u| > thr on the double-float values.
__device__ __forceinline__ df2 soft_threshold_df(df2 u, df2 thr) {
  const df2 cp = df_sub(u, thr), cn = df_add(u, thr);
  const bool pos = cp.h > 0.f || (cp.h == 0.f && cp.l > 0.f);
  const bool neg = cn.h < 0.f || (cn.h == 0.f && cn.l < 0.f);
  return pos ? cp : (neg ? cn : df2{0.f, 0.f});
}

// (h, l) -= d * x for two rows at once (axpy_df per component, with the two
// dependency chains written out side by side so that they interleave)
__device__ __forceinline__ void axpy2_df(float2 x, float dh, float dl, float2& h, float2& l) {
  const float p0 = __fmul_rn(dh, x.x), p1 = __fmul_rn(dh, x.y);
  float e0 = __fmaf_rn(dh, x.x, -p0), e1 = __fmaf_rn(dh, x.y, -p1);
  e0 = __fmaf_rn(dl, x.x, e0);
  e1 = __fmaf_rn(dl, x.y, e1);
  const float s0 = __fadd_rn(h.x, -p0), s1 = __fadd_rn(h.y, -p1);
  const float v0 = __fsub_rn(s0, h.x), v1 = __fsub_rn(s1, h.y);
  float t0 = __fadd_rn(__fsub_rn(h.x, __fsub_rn(s0, v0)), __fsub_rn(-p0, v0));
  float t1 = __fadd_rn(__fsub_rn(h.y, __fsub_rn(s1, v1)), __fsub_rn(-p1, v1));
  t0 = __fadd_rn(t0, __fsub_rn(l.x, e0));
  t1 = __fadd_rn(t1, __fsub_rn(l.y, e1));
  const float h0 = __fadd_rn(s0, t0), h1 = __fadd_rn(s1, t1);
  const float w0 = __fsub_rn(h0, s0), w1 = __fsub_rn(h1, s1);
  l.x = __fadd_rn(__fsub_rn(s0, __fsub_rn(h0, w0)), __fsub_rn(t0, w0));
  l.y = __fadd_rn(__fsub_rn(s1, __fsub_rn(h1, w1)), __fsub_rn(t1, w1));
  h = make_float2(h0, h1);
}

// the same with x = xh + xl (a binary64 column held as two binary32 planes), as axpy_df2
__device__ __forceinline__ void axpy2_df2(float2 xh, float2 xl, float dh, float dl, float2& h, float2& l) {
  const float p0 = __fmul_rn(dh, xh.x), p1 = __fmul_rn(dh, xh.y);
  float e0 = __fmaf_rn(dh, xh.x, -p0), e1 = __fmaf_rn(dh, xh.y, -p1);
  e0 = __fmaf_rn(dl, xh.x, e0);
  e1 = __fmaf_rn(dl, xh.y, e1);
  e0 = __fmaf_rn(dh, xl.x, e0);
  e1 = __fmaf_rn(dh, xl.y, e1);
  const float s0 = __fadd_rn(h.x, -p0), s1 = __fadd_rn(h.y, -p1);
  const float v0 = __fsub_rn(s0, h.x), v1 = __fsub_rn(s1, h.y);
  float t0 = __fadd_rn(__fsub_rn(h.x, __fsub_rn(s0, v0)), __fsub_rn(-p0, v0));
  float t1 = __fadd_rn(__fsub_rn(h.y, __fsub_rn(s1, v1)), __fsub_rn(-p1, v1));
  t0 = __fadd_rn(t0, __fsub_rn(l.x, e0));
  t1 = __fadd_rn(t1, __fsub_rn(l.y, e1));
  const float h0 = __fadd_rn(s0, t0), h1 = __fadd_rn(s1, t1);
  const float w0 = __fsub_rn(h0, s0), w1 = __fsub_rn(h1, s1);
  l.x = __fadd_rn(__fsub_rn(s0, __fsub_rn(h0, w0)), __fsub_rn(t0, w0));
  l.y = __fadd_rn(__fsub_rn(s1, __fsub_rn(h1, w1)), __fsub_rn(t1, w1));
  h = make_float2(h0, h1);
}

__device__ __forceinline__ void cp_async8(void* dst_smem, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst_smem)), "l"(src) : "memory");
}

// Row index i > k of the strictly lower triangle element number t
// (t = i (i - 1) / 2 + k), for the rebuild of the Gram cache.
__device__ __forceinline__ void tri_index(long long t, int& i, int& k) {
  int r = (int)((1.0 + sqrt(1.0 + 8.0 * (double)t)) * 0.5);
  while ((long long)r * (r - 1) / 2 > t) --r;
  while ((long long)(r + 1) * r / 2 <= t) ++r;
  i = r;
  k = (int)(t - (long long)r * (r - 1) / 2);
}

// Bounded spin of one warp on a shared-memory counter: true once *p >= target,
// false when *abort is set or limit_ns has passed (then *abort is set too).
__device__ __forceinline__ bool smem_wait_ge(volatile int* p, int target, volatile int* abort,
                                             unsigned long long limit_ns, bool sleep) {
  if (*p >= target) return true;
  const unsigned long long t0 = global_ns();
  unsigned spins = 0;
  while (*p < target) {
    if (*abort) return false;
    if (sleep) __nanosleep(32);
    if ((++spins & 255u) == 0u && global_ns() - t0 > limit_ns) {
      *abort = 1;
      return false;
    }
  }
  return true;
}

}  // namespace lassogs
