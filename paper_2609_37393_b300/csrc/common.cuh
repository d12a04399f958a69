// Device helpers shared by the FP64 and FP32-mixed likelihood kernels.
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include "dfloat.cuh"
#include "rift_ile_internal.h"

namespace rift {

// Copies one PointParams record into shared memory (whole block).
__device__ __forceinline__ void stage_point(PointParams& dst, const PointParams* __restrict__ src) {
  const int words = (int)(sizeof(PointParams) / sizeof(int));
  int* d = reinterpret_cast<int*>(&dst);
  const int* s = reinterpret_cast<const int*>(src);
  for (int i = threadIdx.x; i < words; i += blockDim.x) d[i] = __ldg(s + i);
}

// The draws are read once: streaming loads (evict-first in L1 and L2), so that
// they do not displace the point's tables from L1.
__device__ __forceinline__ double load_param_d(const DrawsParams& dp, int which, long long i) {
  return dp.f64 ? __ldcs((const double*)dp.p[which] + i) : (double)__ldcs((const float*)dp.p[which] + i);
}

__device__ __forceinline__ float load_param_f(const DrawsParams& dp, int which, long long i) {
  return dp.f64 ? (float)__ldcs((const double*)dp.p[which] + i) : __ldcs((const float*)dp.p[which] + i);
}

__device__ __forceinline__ double load_logw_d(const DrawsParams& dp, long long i) {
  if (!dp.logw) return 0.0;
  return dp.f64 ? __ldcs((const double*)dp.logw + i) : (double)__ldcs((const float*)dp.logw + i);
}

// The t parameter of an FP32 draw set is exact in a float; an FP64 draw set
// keeps its double value as a (hi, lo) pair.
__device__ __forceinline__ df load_param_df(const DrawsParams& dp, int which, long long i) {
  if (dp.f64) return df_from_double(__ldcs((const double*)dp.p[which] + i));
  return df{__ldcs((const float*)dp.p[which] + i), 0.f};
}

// -2Y_lm(iota, phi) of mode i from the polynomial coefficients of the point:
// e^{i m phi} sum_r a_r c^(k0+2r) s^(2l-k0-2r), c = cos(iota/2), s = sin(iota/2);
// eiphi = e^{i phi}.  T is float or double.
template <typename T>
__device__ __forceinline__ void sylm_eval(const PointParams& P, int i, T c, T s, T eiphi_re,
                                          T eiphi_im, const T* coef, T& yre, T& yim) {
  const int l = P.ell[i], m = P.em[i], nt = P.ynt[i], k0 = P.yk0[i];
  // prefactor c^k0 s^(2l - k0 - 2(nt-1)), then homogeneous Horner in (c^2, s^2)
  T pre = T(1);
  for (int q = 0; q < k0; ++q) pre *= c;
  const int es = 2 * l - k0 - 2 * (nt - 1);
  for (int q = 0; q < es; ++q) pre *= s;
  const T X = c * c, Ys = s * s;
  T poly = coef[nt - 1];
  T yp = T(1);
  for (int r = nt - 2; r >= 0; --r) {
    yp *= Ys;
    poly = poly * X + coef[r] * yp;
  }
  T amp = pre * poly;
  // e^{i m phi} by repeated multiplication (|m| <= 8)
  T er = T(1), ei = T(0);
  const int am = m < 0 ? -m : m;
  for (int q = 0; q < am; ++q) {
    T nr = er * eiphi_re - ei * eiphi_im;
    T ni = er * eiphi_im + ei * eiphi_re;
    er = nr;
    ei = ni;
  }
  if (m < 0) ei = -ei;
  yre = amp * er;
  yim = amp * ei;
}

// d/d iota of the real amplitude of -2Y_lm (mode i): the Goldberg sum
// sum_r a_r c^p s^q, p = k0 + 2r, q = 2l - p, c = cos(iota/2), s = sin(iota/2),
// differentiated term by term (dc/d iota = -s/2, ds/d iota = c/2).
__device__ __forceinline__ double sylm_damp_dincl(const PointParams& P, int i, double c, double s) {
  const int l = P.ell[i], nt = P.ynt[i], k0 = P.yk0[i];
  double damp = 0.0;
  for (int r = 0; r < nt; ++r) {
    const int pp = k0 + 2 * r, qq = 2 * l - pp;
    double cpm = 1.0, sqm = 1.0;
    for (int u = 0; u < pp - 1; ++u) cpm *= c;
    for (int u = 0; u < qq - 1; ++u) sqm *= s;
    double t = 0.0;
    if (pp > 0) t -= pp * cpm * (qq > 0 ? sqm * s : 1.0) * s;
    if (qq > 0) t += qq * (pp > 0 ? cpm * c : 1.0) * c * sqm;
    damp += 0.5 * P.ycoef[i][r] * t;
  }
  return damp;
}

// a^T D b with D stored as xx, xy, xz, yy, yz, zz.
template <typename T>
__device__ __forceinline__ T quad3(const T* D, const T a[3], const T b[3]) {
  T d0 = D[0] * b[0] + D[1] * b[1] + D[2] * b[2];
  T d1 = D[1] * b[0] + D[3] * b[1] + D[4] * b[2];
  T d2 = D[2] * b[0] + D[4] * b[1] + D[5] * b[2];
  return a[0] * d0 + a[1] * d1 + a[2] * d2;
}

// Lagrange cubic on nodes -1, 0, 1, 2 at offset f, and the f-derivative.
__device__ __forceinline__ void lagrange4_d(double f, double w[4], double dw[4]) {
  double a = f + 1.0, b = f, c = f - 1.0, d = f - 2.0;
  w[0] = -(b * c * d) * (1.0 / 6.0);
  w[1] = (a * c * d) * 0.5;
  w[2] = -(a * b * d) * 0.5;
  w[3] = (a * b * c) * (1.0 / 6.0);
  dw[0] = -(c * d + b * d + b * c) * (1.0 / 6.0);
  dw[1] = (c * d + a * d + a * c) * 0.5;
  dw[2] = -(b * d + a * d + a * b) * 0.5;
  dw[3] = (b * c + a * c + a * b) * (1.0 / 6.0);
}

// ------------------------------------------------- distance marginalisation

// Node of the table nearest x (x_j decreasing in j), by bisection.
__device__ __forceinline__ int dist_nearest(const DistParams& dp, double x) {
  int lo = 0, hi = dp.n - 1;
  if (!(x < dp.x[0])) return 0;
  if (!(x > dp.x[hi])) return hi;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (dp.x[mid] > x) lo = mid;
    else hi = mid;
  }
  return (dp.x[lo] - x < x - dp.x[hi]) ? lo : hi;
}

// e^d for d <= 0 in FP64, for the LSE merges (FP64 issues at 2 per clock per
// SM on this part, so the merge exponential is kept short): Cody-Waite
// reduction d = k ln2 + r with ln2 split into a 31-bit head (k * head exact
// for |k| < 2^21) and the rest, |r| <= ln2/2, then the Taylor polynomial of
// e^r to degree 13 (remainder below 2^-57 relative) and the exact scaling by
// 2^k.  Zero below the double range.
__device__ __forceinline__ double lse_exp(double d) {
  if (!(d > -745.0)) return 0.0;
  const double k = rint(d * 1.4426950408889634);
  double r = fma(-k, 0.6931471803691238, d);
  r = fma(-k, 1.9082149292705877e-10, r);
  double p = 1.6059043836821613e-10;  // 1/13!
  p = fma(p, r, 2.08767569878681e-09);
  p = fma(p, r, 2.505210838544172e-08);
  p = fma(p, r, 2.755731922398589e-07);
  p = fma(p, r, 2.7557319223985893e-06);
  p = fma(p, r, 2.48015873015873e-05);
  p = fma(p, r, 0.0001984126984126984);
  p = fma(p, r, 0.001388888888888889);
  p = fma(p, r, 0.008333333333333333);
  p = fma(p, r, 0.041666666666666664);
  p = fma(p, r, 0.16666666666666666);
  p = fma(p, r, 0.5);
  p = fma(p, r, 1.0);
  p = fma(p, r, 1.0);
  return scalbn(p, (int)k);
}

// ln sum_j exp(K x_j - R x_j^2 / 2 + ln w_j) (eq. ap:dexp on the node table),
// written as K^2/(2R) + ln sum_j exp(ln w_j - R (x_j - x*)^2 / 2), x* = K/R,
// visiting only nodes whose term can exceed the running maximum minus 40:
// from the node nearest x* outwards, stopping in each direction once
// max_j ln w_j - R (x_j - x*)^2 / 2 is below that level (the quadratic only
// grows away from x*), in IEEE double.  peak = K^2/(2R) is returned
// separately; the return value is the node sum.  R <= 0
// (no template power) sums every node of K x_j + ln w_j instead, relative to
// peak = max_j K x_j.
//
// With ex (may be NULL) the node posterior moments E[x] and E[x^2] are
// returned in ex[0], ex[1] (the distance-marginal gradient is
// E[x] dK - E[x^2] dR / 2).
__device__ __forceinline__ double dist_lse(const DistParams& dp, double K, double R, double xs,
                                           double* peak, double* ex = nullptr) {
  if (!(R > 0.0)) {
    double m = -CUDART_INF;
    for (int j = 0; j < dp.n; ++j) m = fmax(m, K * dp.x[j] - 0.5 * R * dp.x[j] * dp.x[j] + dp.lnw[j]);
    double s = 0.0, s1 = 0.0, s2 = 0.0;
    for (int j = 0; j < dp.n; ++j) {
      const double e = lse_exp(K * dp.x[j] - 0.5 * R * dp.x[j] * dp.x[j] + dp.lnw[j] - m);
      s += e;
      s1 += e * dp.x[j];
      s2 += e * dp.x[j] * dp.x[j];
    }
    *peak = 0.0;
    if (ex) {
      ex[0] = s1 / s;
      ex[1] = s2 / s;
    }
    return m + log(s);
  }
  const int j0 = dist_nearest(dp, xs);
  double m = -CUDART_INF, s = 0.0, s1 = 0.0, s2 = 0.0;
  for (int dir = -1; dir <= 1; dir += 2) {
    for (int j = (dir < 0 ? j0 : j0 + 1); j >= 0 && j < dp.n; j += dir) {
      const double xj = dp.x[j];
      const double d = xj - xs;
      const double q = 0.5 * R * d * d;
      if (dp.lnw_max - q < m - 40.0) break;
      const double t = dp.lnw[j] - q;
      if (t > m) {
        const double r = lse_exp(m - t);
        s = s * r + 1.0;
        s1 = s1 * r + xj;
        s2 = s2 * r + xj * xj;
        m = t;
      } else {
        const double e = lse_exp(t - m);
        s += e;
        s1 += e * xj;
        s2 += e * xj * xj;
      }
    }
  }
  *peak = 0.5 * K * xs;
  if (ex) {
    ex[0] = s1 / s;
    ex[1] = s2 / s;
  }
  return m + log(s);
}

// ---------------------------------------------------------------- LSE state

// Per-thread online log-sum-exp of v_i = lnL_i + ln w_i, with the running
// maximum m kept as a double-float pair so that v - m is exact for the
// draws that carry weight even when lnL ~ 1e6.
struct ThreadLse {
  df m;
  float s, s2;
  int nan_seen;
};

__device__ __forceinline__ ThreadLse tlse_init() {
  ThreadLse t;
  t.m = df{-CUDART_INF_F, 0.f};
  t.s = 0.f;
  t.s2 = 0.f;
  t.nan_seen = 0;
  return t;
}

__device__ __forceinline__ void tlse_push(ThreadLse& t, df v) {
  if (isnan(v.hi)) {
    t.nan_seen = 1;
    return;
  }
  if (!(v.hi > -CUDART_INF_F)) return;  // zero weight
  const bool bigger = (v.hi > t.m.hi) || (v.hi == t.m.hi && v.lo > t.m.lo);
  float d = __fadd_rn(__fsub_rn(v.hi, t.m.hi), __fsub_rn(v.lo, t.m.lo));
  if (bigger) {
    float e = (t.m.hi == -CUDART_INF_F) ? 0.f : __expf(-d);
    t.s = fmaf(t.s, e, 1.f);
    t.s2 = fmaf(t.s2, e * e, 1.f);
    t.m = v;
  } else {
    float e = __expf(d);
    t.s += e;
    t.s2 = fmaf(e, e, t.s2);
  }
}

// Pushes lnL + ln w with a float ln w that may be infinite: a zero weight
// (ln w = -inf) is skipped unless lnL is NaN, +inf dominates; the pair sum
// of a finite lnL and an infinite ln w would otherwise be NaN.  Written with
// selects instead of branches (the same arithmetic as tlse_push), so that
// the update does not split the draw loop into divergent blocks.
__device__ __forceinline__ void tlse_push_lw(ThreadLse& t, df lnl, float lw) {
  const bool nan_in = isnan(lw) || isnan(lnl.hi);
  const bool lw_inf = isinf(lw);
  df v = df_add_f(lnl, lw_inf ? 0.f : lw);
  if (lw_inf) v = df{lw, 0.f};
  const bool skip = nan_in || !(v.hi > -CUDART_INF_F);
  const bool bigger = (v.hi > t.m.hi) || (v.hi == t.m.hi && v.lo > t.m.lo);
  const float d = __fadd_rn(__fsub_rn(v.hi, t.m.hi), __fsub_rn(v.lo, t.m.lo));
  const float e = __expf(bigger ? -d : d);  // 0 when t is empty (d = +inf)
  const float s_new = bigger ? fmaf(t.s, e, 1.f) : t.s + e;
  const float s2_new = bigger ? fmaf(t.s2, e * e, 1.f) : fmaf(e, e, t.s2);
  t.nan_seen |= nan_in ? 1 : 0;
  t.s = skip ? t.s : s_new;
  t.s2 = skip ? t.s2 : s2_new;
  const bool take = !skip && bigger;
  t.m.hi = take ? v.hi : t.m.hi;
  t.m.lo = take ? v.lo : t.m.lo;
}

// Exact merge of two states: the smaller maximum is rescaled to the larger
// one (one exponential).
__device__ __forceinline__ LseState lse_merge(LseState a, LseState b) {
  if (isnan(a.m) || isnan(b.m)) return LseState{CUDART_NAN, CUDART_NAN, CUDART_NAN, a.n + b.n};
  if (a.m == -CUDART_INF) return LseState{b.m, b.s, b.s2, a.n + b.n};
  if (b.m == -CUDART_INF) return LseState{a.m, a.s, a.s2, a.n + b.n};
  if (a.m >= b.m) {
    const double e = lse_exp(b.m - a.m);
    return LseState{a.m, fma(b.s, e, a.s), fma(b.s2, e * e, a.s2), a.n + b.n};
  }
  const double e = lse_exp(a.m - b.m);
  return LseState{b.m, fma(a.s, e, b.s), fma(a.s2, e * e, b.s2), a.n + b.n};
}

__device__ __forceinline__ LseState lse_shfl_down(LseState v, int off) {
  LseState o;
  o.m = __shfl_down_sync(0xffffffffu, v.m, off);
  o.s = __shfl_down_sync(0xffffffffu, v.s, off);
  o.s2 = __shfl_down_sync(0xffffffffu, v.s2, off);
  o.n = __shfl_down_sync(0xffffffffu, v.n, off);
  return o;
}

// Merge of the 32 lanes' states into lane 0 by a fixed shuffle tree (the
// same pairing every call, so the result is reproducible bit for bit).
__device__ __forceinline__ LseState warp_lse_reduce(LseState v) {
  for (int off = 16; off > 0; off >>= 1) v = lse_merge(v, lse_shfl_down(v, off));
  return v;
}

// Merge of one state per thread into thread 0 (blockDim a multiple of 32,
// at most 1024): shuffle trees within and then across warps.
__device__ __forceinline__ LseState block_lse_reduce(LseState v) {
  __shared__ LseState warp_part[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_lse_reduce(v);
  if (lane == 0) warp_part[wid] = v;
  __syncthreads();
  if (wid == 0) {
    v = lane < nw ? warp_part[lane] : LseState{-CUDART_INF, 0.0, 0.0, 0.0};
    v = warp_lse_reduce(v);
  }
  return v;
}

// Block-level reduction of the per-thread states; thread 0 writes the block
// partial (with n = 0; draw counts are added by the caller).  FP32 merges inside a warp (the state's m is a pair), then FP64
// across warps through shared memory, always in the same order.
__device__ __forceinline__ void block_lse_write(ThreadLse t, LseState* out) {
  // warp merge in float with the pair-valued maximum
  for (int off = 16; off > 0; off >>= 1) {
    float mh = __shfl_down_sync(0xffffffffu, t.m.hi, off);
    float ml = __shfl_down_sync(0xffffffffu, t.m.lo, off);
    float os = __shfl_down_sync(0xffffffffu, t.s, off);
    float os2 = __shfl_down_sync(0xffffffffu, t.s2, off);
    int on = __shfl_down_sync(0xffffffffu, t.nan_seen, off);
    t.nan_seen |= on;
    if (mh == -CUDART_INF_F) continue;
    if (t.m.hi == -CUDART_INF_F) {
      t.m = df{mh, ml};
      t.s = os;
      t.s2 = os2;
      continue;
    }
    const bool other_bigger = (mh > t.m.hi) || (mh == t.m.hi && ml > t.m.lo);
    float d = __fadd_rn(__fsub_rn(mh, t.m.hi), __fsub_rn(ml, t.m.lo));
    if (other_bigger) {
      float e = __expf(-d);
      t.s = fmaf(t.s, e, os);
      t.s2 = fmaf(t.s2, e * e, os2);
      t.m = df{mh, ml};
    } else {
      float e = __expf(d);
      t.s = fmaf(os, e, t.s);
      t.s2 = fmaf(os2, e * e, t.s2);
    }
  }
  __shared__ LseState warp_state[32];
  __shared__ int warp_nan[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    warp_state[wid] = LseState{(double)t.m.hi + (double)t.m.lo, (double)t.s, (double)t.s2, 0.0};
    warp_nan[wid] = t.nan_seen;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    LseState acc{-CUDART_INF, 0.0, 0.0, 0.0};
    int nan_any = 0;
    const int nw = (blockDim.x + 31) >> 5;
    for (int w = 0; w < nw; ++w) {
      acc = lse_merge(acc, warp_state[w]);
      nan_any |= warp_nan[w];
    }
    acc.n = 0.0;  // the caller knows the draw count
    if (nan_any) acc.m = acc.s = acc.s2 = CUDART_NAN;
    *out = acc;
  }
}

// The same reduction in IEEE double throughout (FP64 path).
struct ThreadLse64 {
  LseState st;
  int nan_seen;
};

__device__ __forceinline__ ThreadLse64 tlse64_init() {
  ThreadLse64 t;
  t.st = LseState{-CUDART_INF, 0.0, 0.0, 0.0};
  t.nan_seen = 0;
  return t;
}

__device__ __forceinline__ void tlse64_push(ThreadLse64& t, double v) {
  if (isnan(v)) {
    t.nan_seen = 1;
    return;
  }
  if (!(v > -CUDART_INF)) return;
  if (v > t.st.m) {
    double e = (t.st.m == -CUDART_INF) ? 0.0 : lse_exp(t.st.m - v);
    t.st.s = fma(t.st.s, e, 1.0);
    t.st.s2 = fma(t.st.s2, e * e, 1.0);
    t.st.m = v;
  } else {
    double e = lse_exp(v - t.st.m);
    t.st.s += e;
    t.st.s2 = fma(e, e, t.st.s2);
  }
}

__device__ __forceinline__ void block_lse64_write(ThreadLse64 t, LseState* out) {
  const int nan_any = __syncthreads_or(t.nan_seen);
  LseState acc = block_lse_reduce(t.st);
  if (threadIdx.x == 0) {
    acc.n = 0.0;
    if (nan_any) acc.m = acc.s = acc.s2 = CUDART_NAN;
    *out = acc;
  }
}

}  // namespace rift
