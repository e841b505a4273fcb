// Double-float arithmetic (unevaluated sums h + l of two binary32 values,
// about 48 significand bits) and exact fixed-point reductions.
//
// GB300 issues FP64 at about 1/64 of the FP32 rate with a 64-cycle latency,
// so the coordinate-descent inner loop keeps beta and the residual in
// double-float and never touches the FP64 pipe.  The building blocks are the
// error-free transformations of Knuth (TwoSum), Dekker (FastTwoSum) and the
// FMA-based TwoProduct, combined as in the compensated dot product of Ogita,
// Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 2005).
// Every operation uses the explicit _rn intrinsics so that the compiler can
// neither contract nor reassociate them.
//
// Cross-thread sums are exact: each thread's double-float partial is cut into
// three 23-bit integer limbs on a common power-of-two scale, the limbs are
// summed with integer adds (warp: redux.sync), and the carry-normalised total
// is turned back into a double-float.  Integer addition is associative, so the
// result does not depend on the reduction order.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace lassogs {

struct df2 {
  float h, l;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}

// requires |a| >= |b| or a == 0
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}

__device__ __forceinline__ df2 df_make(float h) { return df2{h, 0.0f}; }

__device__ __forceinline__ df2 df_add(df2 a, df2 b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  e = __fadd_rn(e, __fadd_rn(a.l, b.l));
  df2 r;
  two_sum(s, e, r.h, r.l);
  return r;
}

__device__ __forceinline__ df2 df_neg(df2 a) { return df2{-a.h, -a.l}; }
__device__ __forceinline__ df2 df_sub(df2 a, df2 b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df2 df_mul(df2 a, df2 b) {
  float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  df2 r;
  two_sum(p, e, r.h, r.l);
  return r;
}

// a > b for normalised pairs
__device__ __forceinline__ bool df_gt(df2 a, df2 b) { return a.h > b.h || (a.h == b.h && a.l > b.l); }
__device__ __forceinline__ bool df_is_neg(df2 a) { return a.h < 0.0f || (a.h == 0.0f && a.l < 0.0f); }
__device__ __forceinline__ bool df_is_zero(df2 a) { return a.h == 0.0f && a.l == 0.0f; }
__device__ __forceinline__ df2 df_abs(df2 a) { return df_is_neg(a) ? df_neg(a) : a; }

// FP64 <-> double-float (these run on the FP64 pipe: keep out of inner loops)
__device__ __forceinline__ df2 df_from_double(double x) {
  float h = __double2float_rn(x);
  float l = __double2float_rn(__dsub_rn(x, (double)h));
  return df2{h, l};
}
__device__ __forceinline__ double df_to_double(df2 a) { return __dadd_rn((double)a.h, (double)a.l); }

// ---------------------------------------------------------------- dot / axpy
// (S, C) += x * (h + l): TwoProduct of x*h, the small product x*l folded
// into the error term, TwoSum into the running sum.
__device__ __forceinline__ void dot2_acc(float x, float h, float l, float& S, float& C) {
  float p = __fmul_rn(x, h);
  float e = __fmaf_rn(x, h, -p);
  e = __fmaf_rn(x, l, e);
  float s, t;
  two_sum(S, p, s, t);
  S = s;
  C = __fadd_rn(C, __fadd_rn(t, e));
}
// the same with x = xh + xl (a binary64 column split into two binary32 planes)
__device__ __forceinline__ void dot2_acc2(float xh, float xl, float h, float l, float& S, float& C) {
  float p = __fmul_rn(xh, h);
  float e = __fmaf_rn(xh, h, -p);
  e = __fmaf_rn(xh, l, e);
  e = __fmaf_rn(xl, h, e);
  float s, t;
  two_sum(S, p, s, t);
  S = s;
  C = __fadd_rn(C, __fadd_rn(t, e));
}

// (h, l) -= d * x   with d = (dh, dl)
__device__ __forceinline__ void axpy_df(float x, float dh, float dl, float& h, float& l) {
  float p = __fmul_rn(dh, x);
  float e = __fmaf_rn(dh, x, -p);
  e = __fmaf_rn(dl, x, e);
  float s, t;
  two_sum(h, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(l, e));
  two_sum(s, t, h, l);
}
// (h, l) -= d * (xh + xl)
__device__ __forceinline__ void axpy_df2(float xh, float xl, float dh, float dl, float& h, float& l) {
  float p = __fmul_rn(dh, xh);
  float e = __fmaf_rn(dh, xh, -p);
  e = __fmaf_rn(dl, xh, e);
  e = __fmaf_rn(dh, xl, e);
  float s, t;
  two_sum(h, -p, s, t);
  t = __fadd_rn(t, __fsub_rn(l, e));
  two_sum(s, t, h, l);
}

// ---------------------------------------------------------------- exact limb sums
// Integer nearest to w (|w| <= 2^22) via the 1.5*2^23 shift; rem = w - it.
__device__ __forceinline__ int rint_shift(float w, float& rem) {
  const float M = 12582912.0f;  // 1.5 * 2^23
  float t = __fadd_rn(w, M);
  float r = __fsub_rn(t, M);
  rem = __fsub_rn(w, r);
  return __float_as_int(t) - 0x4B400000;
}

struct limbs3 {
  int a, b, c;
};

// v * scale = a + b 2^-23 + c 2^-46 + O(2^-47); requires |v * scale| <= 2^22
__device__ __forceinline__ limbs3 to_limbs(float v, float scale) {
  limbs3 L;
  float r;
  float w = __fmul_rn(v, scale);
  L.a = rint_shift(w, r);
  w = __fmul_rn(r, 8388608.0f);
  L.b = rint_shift(w, r);
  w = __fmul_rn(r, 8388608.0f);
  L.c = rint_shift(w, r);
  return L;
}

__device__ __forceinline__ limbs3 limbs_add(limbs3 x, limbs3 y) { return limbs3{x.a + y.a, x.b + y.b, x.c + y.c}; }

// the same value with carries moved up: |b|, |c| <= 2^22 afterwards
__device__ __forceinline__ limbs3 limbs_norm(limbs3 L) {
  const int cc = (L.c + (1 << 22)) >> 23;
  L.c -= cc << 23;
  L.b += cc;
  const int cb = (L.b + (1 << 22)) >> 23;
  L.b -= cb << 23;
  L.a += cb;
  return L;
}

__device__ __forceinline__ limbs3 warp_limbs_sum(limbs3 L) {
  return limbs3{__reduce_add_sync(0xffffffffu, L.a), __reduce_add_sync(0xffffffffu, L.b),
                __reduce_add_sync(0xffffffffu, L.c)};
}

// (a + b 2^-23 + c 2^-46) / scale as a double-float.  |a| < 2^24 after the
// carries, which holds when the sum of |partials| is <= 2^22 / scale.
__device__ __forceinline__ df2 limbs_to_df(limbs3 L, float inv_scale) {
  int A = L.a, B = L.b, C = L.c;
  int cc = (C + (1 << 22)) >> 23;
  C -= cc << 23;
  B += cc;
  int cb = (B + (1 << 22)) >> 23;
  B -= cb << 23;
  A += cb;
  float a = (float)A;
  float b = __fmul_rn((float)B, 1.1920928955078125e-07f);  // 2^-23
  float c = __fmul_rn((float)C, 1.4210854715202004e-14f);  // 2^-46
  float s, e;
  fast_two_sum(a, b, s, e);  // a integer, |b| <= 1/2
  e = __fadd_rn(e, c);
  df2 r;
  two_sum(s, e, r.h, r.l);
  r.h = __fmul_rn(r.h, inv_scale);
  r.l = __fmul_rn(r.l, inv_scale);
  return r;
}

// Power-of-two scale for limbs: 2^(22 - E) with 2^(E-1) > bound, from the
// exponent bits of bound (bound >= 0; zero, subnormal or huge bounds clamp E).
__device__ __forceinline__ void limb_scale(float bound, float& scale, float& inv_scale) {
  int e = (int)((__float_as_uint(bound) >> 23) & 0xffu);  // biased exponent
  int E = (e == 0) ? -90 : e - 126 + 1;                  // bound < 2^(e-126)
  E = max(-90, min(100, E));
  scale = __uint_as_float((unsigned)(127 + 22 - E) << 23);
  inv_scale = __uint_as_float((unsigned)(127 - 22 + E) << 23);
}

}  // namespace lassogs
