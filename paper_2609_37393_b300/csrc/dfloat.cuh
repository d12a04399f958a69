// Double-float ("two-float") arithmetic on the FP32 pipe.
//
// On B300 an FP64 FMA issues at 2 per clock per SM against about 124 FP32 FMAs,
// so the precision-critical sums of the likelihood are carried as unevaluated
// pairs hi + lo of floats (about 48 significant bits) built from the published
// error-free transformations:
//   TwoSum      Knuth, TAOCP vol. 2 (1969): a + b = s + e exactly, 6 flops
//   FastTwoSum  Dekker (1971): same when |a| >= |b|, 3 flops
//   TwoProduct  with a fused multiply-add: a * b = p + e exactly, 2 flops
// and the pair operations of Dekker (1971) built on them.  The compensated
// dot product accumulates exact products with TwoSum in the style of
// Ogita, Rump and Oishi, "Accurate sum and dot product", SISC 26 (2005).
// All functions are written for -fmad=true builds: every product that must be
// exact uses fmaf explicitly, every sum that must not be contracted is an
// explicit __fadd_rn / __fsub_rn.
#pragma once
#include <cuda_runtime.h>

namespace rift {

struct df {
  float hi, lo;
};

__device__ __forceinline__ df df_make(float hi, float lo = 0.f) { return df{hi, lo}; }

__device__ __forceinline__ df two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return df{s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  float e = fmaf(a, b, -p);
  return df{p, e};
}

// (a.hi + a.lo) + (b.hi + b.lo): the high parts summed exactly (TwoSum), the
// low parts added once.  The absolute error stays within about
// u^2 (|a| + |b|) (u = 2^-24) however much the terms cancel, which is the
// accuracy every caller needs: the terms carry the scale the result is judged
// against (an angle, a time, a template).  (Dekker's sum with a second TwoSum
// on the low parts, relatively accurate under cancellation, costs 20
// operations instead of 11 and buys nothing here.)
__device__ __forceinline__ df df_add(df a, df b) {
  df s = two_sum(a.hi, b.hi);
  s.lo = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
  return fast_two_sum(s.hi, s.lo);
}

// a - b for a range reduction, where the high parts subtract exactly: b.hi = 0,
// or a.hi and b.hi of one sign within a factor of two (Sterbenz's lemma), as for
// a - k c with k = rint(a / c) != 0.  4 operations.
__device__ __forceinline__ df df_sub_reduce(df a, df b) {
  return fast_two_sum(__fsub_rn(a.hi, b.hi), __fsub_rn(a.lo, b.lo));
}

__device__ __forceinline__ df df_add_f(df a, float b) {
  df s = two_sum(a.hi, b);
  s.lo = __fadd_rn(s.lo, a.lo);
  return fast_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ df df_mul(df a, df b) {
  df p = two_prod(a.hi, b.hi);
  p.lo = fmaf(a.hi, b.lo, p.lo);
  p.lo = fmaf(a.lo, b.hi, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
  df p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return fast_two_sum(p.hi, p.lo);
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

__device__ __forceinline__ df df_from_double(double x) {
  float hi = __double2float_rn(x);
  float lo = __double2float_rn(x - (double)hi);
  return df{hi, lo};
}

// Compensated accumulator: a running sum kept as (s, c) where s collects the
// rounded sum of exact high parts through TwoSum and c collects every
// rounding error and low part.  Used for the dot products whose result must
// be accurate to ~1e-10 relative although the terms are ~1e6.
struct dacc {
  float s, c;
};

__device__ __forceinline__ dacc dacc_zero() { return dacc{0.f, 0.f}; }

// acc += a * (b.hi + b.lo) with the a*b.hi product exact.
__device__ __forceinline__ void dacc_fma(dacc& acc, float a, df b) {
  df p = two_prod(a, b.hi);
  df t = two_sum(acc.s, p.hi);
  acc.s = t.hi;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, p.lo));
  acc.c = fmaf(a, b.lo, acc.c);
}

// acc += a * b (both floats) exactly rounded into the pair.
__device__ __forceinline__ void dacc_fma_ff(dacc& acc, float a, float b) {
  df p = two_prod(a, b);
  df t = two_sum(acc.s, p.hi);
  acc.s = t.hi;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, p.lo));
}

__device__ __forceinline__ void dacc_add(dacc& acc, df x) {
  df t = two_sum(acc.s, x.hi);
  acc.s = t.hi;
  acc.c = __fadd_rn(acc.c, __fadd_rn(t.lo, x.lo));
}

__device__ __forceinline__ df dacc_result(dacc acc) { return fast_two_sum(acc.s, acc.c); }

// ---- two pairs at once: the packed FP32 instructions of sm_100 and later
// (FADD2 / FMUL2 / FFMA2, each two operations in one issue slot).  Every
// component goes through exactly the operations of the scalar functions
// above, so the results are the same bit for bit.
struct df2 {
  float2 hi, lo;  // component 0 is (hi.x, lo.x), component 1 (hi.y, lo.y)
};

__device__ __forceinline__ df2 df2_make(df a, df b) {
  return df2{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)};
}
__device__ __forceinline__ df df2_x(const df2& a) { return df{a.hi.x, a.lo.x}; }
__device__ __forceinline__ df df2_y(const df2& a) { return df{a.hi.y, a.lo.y}; }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
// a - b rounded once, as a single packed instruction (b (-1) + a)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

__device__ __forceinline__ df2 two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  const float2 bb = sub2(s, a);
  const float2 e = __fadd2_rn(sub2(a, sub2(s, bb)), sub2(b, bb));
  return df2{s, e};
}

__device__ __forceinline__ df2 fast_two_sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return df2{s, sub2(b, sub2(s, a))};
}

__device__ __forceinline__ df2 two_prod2(float2 a, float2 b) {
  const float2 p = __fmul2_rn(a, b);
  return df2{p, __ffma2_rn(a, b, neg2(p))};
}

__device__ __forceinline__ df2 df2_neg(const df2& a) { return df2{neg2(a.hi), neg2(a.lo)}; }

__device__ __forceinline__ df2 df_add2(const df2& a, const df2& b) {
  df2 s = two_sum2(a.hi, b.hi);
  s.lo = __fadd2_rn(s.lo, __fadd2_rn(a.lo, b.lo));
  return fast_two_sum2(s.hi, s.lo);
}

__device__ __forceinline__ df2 df_mul2(const df2& a, const df2& b) {
  df2 p = two_prod2(a.hi, b.hi);
  p.lo = __ffma2_rn(a.hi, b.lo, p.lo);
  p.lo = __ffma2_rn(a.lo, b.hi, p.lo);
  return fast_two_sum2(p.hi, p.lo);
}

__device__ __forceinline__ df2 df_add_f2(const df2& a, float2 b) {
  df2 s = two_sum2(a.hi, b);
  s.lo = __fadd2_rn(s.lo, a.lo);
  return fast_two_sum2(s.hi, s.lo);
}

}  // namespace rift
