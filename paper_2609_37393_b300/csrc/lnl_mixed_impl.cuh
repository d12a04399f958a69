// FP32-mixed likelihood kernels (included once per mode-count translation
// unit lnl_mixed_m*.cu, which instantiates them for one MM; the host
// dispatch and the anchor tables' contents live in lnl_mixed.cu).
//
// The same lnL as the FP64 path (eq. def:lnL:Decomposed), arranged for a GPU
// whose FP64 pipe is ~60x narrower than its FP32 pipe.  Per detector, in the
// whitened coordinates built by point.cu,
//     lnL_k = 1/2 |e(t_k)|^2 - 1/2 |e(t_k) - w_k|^2,
//     w_k = x (Re F_k a1 + Im F_k a2),  a1 = A y,  a2 = A J y,  y = (Re Y, Im Y),
// where a1 and a2 are shared by the detectors of one class.
//
// Precision: a rounding of the template w by a relative eps moves lnL by
// <delta h | d - h> ~ eps rho |d - h|, i.e. ~1e-3 nat at rho = 1000 for
// FP32's eps = 6e-8 at 50 nat from the peak.  So the template is carried to
// ~1e-10: the sky angles, psi, iota/2, m phi go through an anchored
// double-float sine/cosine, x through an anchored double-float exponential,
// Y_lm, F_k and w in double-float, and a1, a2 through an error-free split
// product (the head/tail split in lnl_mixed_draw).  The arrival time is also double-float (1 ns
// is ~1e-3 nat).  1/2|e|^2 comes from the tabulated interval polynomial by
// double-float Horner; only the residual e - w, which is small where the
// likelihood matters, is formed in FP32 (its error enters as
// (e - w) . delta, ~1e-5 nat).
#pragma once
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>
#include <utility>
#include <vector>

#include "common.cuh"
#include "kernels.h"

// Tuning knobs (compile-time): the minimum resident blocks per SM given to
// __launch_bounds__, and whether the large double-float helpers are real
// calls (smaller code, fewer instruction-cache misses) or inlined.
#ifndef RIFT_MIXED_MIN_BLOCKS
#define RIFT_MIXED_MIN_BLOCKS 4
#endif
#ifndef RIFT_MIXED_MIN_BLOCKS_GRAD  // kernels that carry the adjoint
#define RIFT_MIXED_MIN_BLOCKS_GRAD 3
#endif
// RIFT_MIXED_A_SMEM: keep a1, a2 of the current class in a per-thread slice
// of shared memory instead of registers (for widths RR <= 12).
#ifndef RIFT_MIXED_A_SMEM
#define RIFT_MIXED_A_SMEM 1
#endif
#ifndef RIFT_MIXED_NOINLINE
#define RIFT_MIXED_NOINLINE 0
#endif
#if RIFT_MIXED_NOINLINE
#define RIFT_HELPER __device__ __noinline__
#else
#define RIFT_HELPER __device__ __forceinline__
#endif

namespace rift {

// The anchor tables: every translation unit that includes this file has its
// own copy (filled by upload_anchor_tables_mm below).
static __device__ float4 g_anchor[2 * kAnchorHalf + 1];  // (sin hi, sin lo, cos hi, cos lo) of j 2^-7
static __device__ float2 g_exp_anchor[2 * kExpHalf + 1];  // e^(j/128) as (hi, lo)

namespace {

constexpr int kMixedThreads = 128;  // block size of every FP32-mixed kernel

template <int RR>
struct A12Smem {
  static constexpr bool on = RIFT_MIXED_A_SMEM && RR <= 12;
};

// Float4 count of the split whitening of every class (two per direction pair
// and mode), and bytes of it plus gm1 at the start of the shared memory of the
// FP32-mixed kernels.
__host__ __device__ inline size_t split_a_f4(int ncls, int R, int M) {
  return (size_t)ncls * R * M;
}
__host__ __device__ inline size_t split_a_bytes(int ncls, int R, int M) {
  return split_a_f4(ncls, R, M) * 16 + (((size_t)ncls * R * 4 + 15) & ~(size_t)15);
}

// Bytes of dynamic shared memory of a FP32-mixed kernel: the split whitening
// of every class, gm1, (A12Smem) the per-thread a1, a2 slices, and the
// per-thread x F_k of the K detectors.
template <int RR>
__host__ __device__ inline size_t mixed_smem_bytes(int ncls, int R, int M, int K) {
  size_t b = split_a_bytes(ncls, R, M);
  if (A12Smem<RR>::on) b += (size_t)RR * kMixedThreads * 16;
  return b + (size_t)K * kMixedThreads * 16;
}

template <int RR>
__device__ __forceinline__ float4* a12_slice(float4* smem4, int ncls, int R, int M) {
  if (!A12Smem<RR>::on) return nullptr;
  const size_t off = split_a_bytes(ncls, R, M);
  return reinterpret_cast<float4*>(reinterpret_cast<char*>(smem4) + off) + threadIdx.x;
}

// This thread's slots of x F_k (as head/tail pairs), slot k at [k * kMixedThreads].
template <int RR>
__device__ __forceinline__ float4* xf_slice(float4* smem4, int ncls, int R, int M) {
  size_t off = split_a_bytes(ncls, R, M);
  if (A12Smem<RR>::on) off += (size_t)RR * kMixedThreads * 16;
  return reinterpret_cast<float4*>(reinterpret_cast<char*>(smem4) + off) + threadIdx.x;
}

// sin and cos of a double-float angle to ~1e-15 absolute: reduce by 2 pi (pair
// constant), take the nearest anchor a_j = j 2^-7, and add the residual
// d (|d| <= 2^-8) through sin d = d - d^3/6 + d^5/120, cos d = 1 - d^2/2 + d^4/24.
// Unroll factors of the mode loop and of the detector loop (0: the
// compiler's choice).
#ifndef RIFT_MIXED_MODE_UNROLL
#define RIFT_MIXED_MODE_UNROLL 0
#endif
#ifndef RIFT_MIXED_DET_UNROLL
#define RIFT_MIXED_DET_UNROLL 0
#endif
constexpr int kModeUnroll = RIFT_MIXED_MODE_UNROLL;
constexpr int kDetUnroll = RIFT_MIXED_DET_UNROLL;
#ifndef RIFT_MIXED_SINCOS_CALL  // 1: the anchored sine/cosine is a real call (less code)
#define RIFT_MIXED_SINCOS_CALL 0
#endif
#if RIFT_MIXED_SINCOS_CALL
__device__ __noinline__
#else
RIFT_HELPER
#endif
void sincos_df(df a, df& s_out, df& c_out) {
  const float kTwoPiHi = 6.28318548202514648f;
  const float kTwoPiLo = -1.7484555314695172e-07f;
  float k = rintf(a.hi * 0.159154943091895336f);
  df kp = two_prod(k, kTwoPiHi);
  kp.lo = fmaf(k, kTwoPiLo, kp.lo);
  df r = df_sub_reduce(a, kp);
  int j = __float2int_rn(r.hi * kAnchorInvStep);
  j = max(-kAnchorHalf, min(kAnchorHalf, j));
  const float dh = __fsub_rn(r.hi, (float)j * kAnchorStep);  // exact
  const float dl = r.lo;
  const float d2 = dh * dh;
  const float sb = fmaf(dh * d2, fmaf(d2, 1.f / 120.f, -1.f / 6.f), dl);  // sin d - dh
  const float cb = fmaf(d2, fmaf(d2, 1.f / 24.f, -0.5f), -dh * dl);       // cos d - 1
  const float4 an = g_anchor[j + kAnchorHalf];
  // sin(a_j + d) = S (1 + cb) + C (dh + sb);  cos(a_j + d) = C (1 + cb) - S (dh + sb)
  df p = two_prod(an.z, dh);
  p.lo = fmaf(an.w, dh, p.lo);
  p.lo = fmaf(an.z, sb, p.lo);
  p.lo = fmaf(an.x, cb, p.lo);
  s_out = df_add(df{an.x, an.y}, p);
  df q = two_prod(an.x, dh);
  q.lo = fmaf(an.y, dh, q.lo);
  q.lo = fmaf(an.x, sb, q.lo);
  q.lo = fmaf(-an.z, cb, q.lo);
  c_out = df_add(df{an.z, an.w}, df_neg(q));
}

// e^a for a double-float a: a = k ln2 + j/128 + d, |d| <= 2^-8, e^d by its
// Taylor series to d^4, anchors e^(j/128) from the table.
RIFT_HELPER df exp_df(df a) {
  const float kLn2Hi = 0.693147182464599609f;
  const float kLn2Lo = -1.904654323148236e-09f;
  float k = rintf(a.hi * 1.44269504088896341f);
  df kp = two_prod(k, kLn2Hi);
  kp.lo = fmaf(k, kLn2Lo, kp.lo);
  df r = df_sub_reduce(a, kp);
  int j = __float2int_rn(r.hi * 128.f);
  j = max(-kExpHalf, min(kExpHalf, j));
  const float dh = __fsub_rn(r.hi, (float)j * (1.f / 128.f));
  const float d = dh + r.lo;
  // e^d - 1 - dh = r.lo + d^2/2 + d^3/6 + d^4/24
  const float tail = fmaf(d * d, fmaf(d, fmaf(d, 1.f / 24.f, 1.f / 6.f), 0.5f), r.lo);
  df ed = fast_two_sum(1.f, dh);
  ed.lo = __fadd_rn(ed.lo, tail);
  const float2 an = g_exp_anchor[j + kExpHalf];
  df v = df_mul(df{an.x, an.y}, ed);
  const int ki = (int)k;
  return df{ldexpf(v.hi, ki), ldexpf(v.lo, ki)};
}

__device__ __forceinline__ df df_pow(df b, int n) {
  df r = df{1.f, 0.f};
  for (int q = 0; q < n; ++q) r = df_mul(r, b);
  return r;
}

// Per-detector and per-mode values the draw loop reads, copied from the
// point parameters into shared memory once per block (and once per point in
// the batch kernel): whole 16-byte vectors indexed by the loop variables
// instead of scalar constant-bank loads with register-indexed addresses.
struct MixedTables {
  float4 ah[kMaxDet][3];  // acoef_h[0..9] (head of the antenna coefficients)
  float4 at[kMaxDet][3];  // acoef_t[0..9] (their tails)
  float4 pos_hi[kMaxDet];  // (pos_hi[0..2], t0_hi)
  float4 pos_lo[kMaxDet];  // (pos_lo[0..2], t0_lo)
  int4 mode[kMaxModes];    // visiting order j: (mode index, m, l, ypar)
  float2 yz[kMaxModes][kMaxEll + 1];  // visiting order j: (hi, lo) of yz
};

__device__ __forceinline__ void stage_tables(const PointParams& P, MixedTables& T) {
  for (int t = threadIdx.x; t < P.K; t += blockDim.x) {
    float h[12] = {}, tl[12] = {};
    for (int c = 0; c < 10; ++c) {
      h[c] = P.acoef_h[t][c];
      tl[c] = P.acoef_t[t][c];
    }
    for (int v = 0; v < 3; ++v) {
      T.ah[t][v] = make_float4(h[4 * v], h[4 * v + 1], h[4 * v + 2], h[4 * v + 3]);
      T.at[t][v] = make_float4(tl[4 * v], tl[4 * v + 1], tl[4 * v + 2], tl[4 * v + 3]);
    }
    T.pos_hi[t] = make_float4(P.pos_hi[t][0], P.pos_hi[t][1], P.pos_hi[t][2], P.t0_hi[t]);
    T.pos_lo[t] = make_float4(P.pos_lo[t][0], P.pos_lo[t][1], P.pos_lo[t][2], P.t0_lo[t]);
  }
  for (int j = threadIdx.x; j < P.M; j += blockDim.x) {
    const int a = P.morder[j];
    T.mode[j] = make_int4(a, P.em[a], P.ell[a], P.ypar[a]);
    for (int q = 0; q <= P.ell[a]; ++q) T.yz[j][q] = make_float2(P.yz_hi[a][q], P.yz_lo[a][q]);
  }
}

// One double-float Horner step acc x + c: the product and the sum of the high
// parts exact, the low parts added in FP32, the result left unnormalised (after
// cancellation its low part can exceed half an ulp of the high part; the next
// step takes acc.lo through an FMA, so the absolute error stays at
// u^2 |terms| and only the final value needs normalising, if at all).
__device__ __forceinline__ df horner_step(df acc, df x, float ch, float cl) {
  df pr = two_prod(acc.hi, x.hi);
  pr.lo = fmaf(acc.hi, x.lo, fmaf(acc.lo, x.hi, pr.lo));
  const df sm = two_sum(pr.hi, ch);
  return df{sm.hi, __fadd_rn(__fadd_rn(pr.lo, sm.lo), cl)};
}

// The same with x a float (no low part).
__device__ __forceinline__ df horner_step_f(df acc, float x, float ch, float cl) {
  df pr = two_prod(acc.hi, x);
  pr.lo = fmaf(acc.lo, x, pr.lo);
  const df sm = two_sum(pr.hi, ch);
  return df{sm.hi, __fadd_rn(__fadd_rn(pr.lo, sm.lo), cl)};
}

// The real amplitude of -2Y_lm(iota, 0) of the mode visited j-th (degree l,
// parity par) in double-float from z = cos(iota) and sz = sin(iota):
// sz^par sum_q yz[q] z^q by Horner (horner_step), normalised at the end.
RIFT_HELPER df sylm_amp_df(const MixedTables& T, int j, int l, int par, df z, df sz) {
  float2 c = T.yz[j][l];
  df acc = df{c.x, c.y};
  for (int q = l - 1; q >= 0; --q) {
    c = T.yz[j][q];
    acc = horner_step(acc, z, c.x, c.y);
  }
  return par ? df_mul(acc, sz) : fast_two_sum(acc.hi, acc.lo);
}

// pos . s for a position (hi, lo vectors) and a direction of pairs: the three
// high products exact and summed by TwoSum, every low term once in FP32
// (absolute error ~u^2 |pos|).
__device__ __forceinline__ df dot3_df(float4 ph, float4 pl, df s0, df s1, df s2) {
  const df p0 = two_prod(ph.x, s0.hi), p1 = two_prod(ph.y, s1.hi), p2 = two_prod(ph.z, s2.hi);
  const df a = two_sum(p0.hi, p1.hi), b = two_sum(a.hi, p2.hi);
  float lo = __fadd_rn(__fadd_rn(p0.lo, p1.lo), __fadd_rn(p2.lo, __fadd_rn(a.lo, b.lo)));
  lo = fmaf(ph.x, s0.lo, fmaf(pl.x, s0.hi, lo));
  lo = fmaf(ph.y, s1.lo, fmaf(pl.y, s1.hi, lo));
  lo = fmaf(ph.z, s2.lo, fmaf(pl.z, s2.hi, lo));
  return fast_two_sum(b.hi, lo);
}

// Complex product of pairs.
__device__ __forceinline__ void cmul_df(df ar, df ai, df br, df bi, df& cr, df& ci) {
  cr = df_add(df_mul(ar, br), df_neg(df_mul(ai, bi)));
  ci = df_add(df_mul(ar, bi), df_mul(ai, br));
}

// Sky functions shared by all detectors: with e1 = (-sl, cl, 0) and
// e2 = (-sd cl, -sd sl, cd) (sl, cl = sin, cos of ra - gmst; sd, cd of dec),
//   F_+(0) = e1.D.e1 - e2.D.e2 = Dxx b0 + Dyy b1 + Dxy b2 + Dxz b3 + Dyz b4 + Dzz b5,
//   F_x(0) = 2 e1.D.e2 = (Dxx - Dyy) g0 + Dxy g1 + Dxz g2 + Dyz g3,
// b = (sl^2 - sd^2 cl^2, cl^2 - sd^2 sl^2, -2 sl cl (1 + sd^2), 2 sd cd cl,
//      2 sd cd sl, -cd^2),  g = (2 sd sl cl, 2 sd (sl^2 - cl^2), -2 sl cd, 2 cl cd).
struct AntennaBasis {
  df b[6], g[4];
};

RIFT_HELPER void antenna_basis(df sl, df cl, df sd, df cd, AntennaBasis& B) {
  const df sl2 = df_mul(sl, sl), cl2 = df_mul(cl, cl), slcl = df_mul(sl, cl);
  const df sd2 = df_mul(sd, sd), sdcd = df_mul(sd, cd), cd2 = df_mul(cd, cd);
  B.b[0] = df_sub(sl2, df_mul(sd2, cl2));
  B.b[1] = df_sub(cl2, df_mul(sd2, sl2));
  const df t = df_mul(slcl, df_add_f(sd2, 1.f));
  B.b[2] = df{-2.f * t.hi, -2.f * t.lo};
  const df u = df_mul(sdcd, cl), v = df_mul(sdcd, sl);
  B.b[3] = df{2.f * u.hi, 2.f * u.lo};
  B.b[4] = df{2.f * v.hi, 2.f * v.lo};
  B.b[5] = df_neg(cd2);
  const df w = df_mul(sd, slcl);
  B.g[0] = df{2.f * w.hi, 2.f * w.lo};
  const df z = df_mul(sd, df_sub(sl2, cl2));
  B.g[1] = df{2.f * z.hi, 2.f * z.lo};
  const df a = df_mul(sl, cd), c = df_mul(cl, cd);
  B.g[2] = df{-2.f * a.hi, -2.f * a.lo};
  B.g[3] = df{2.f * c.hi, 2.f * c.lo};
}

// acc += a * b for pairs, the hi*hi product exact.
__device__ __forceinline__ void dacc_fma_dd(dacc& acc, df a, df b) {
  const df p = two_prod(a.hi, b.hi);
  const df t = two_sum(acc.s, p.hi);
  acc.s = t.hi;
  float c = __fadd_rn(acc.c, __fadd_rn(t.lo, p.lo));
  c = fmaf(a.hi, b.lo, c);
  acc.c = fmaf(a.lo, b.hi, c);
}

// Head of v on the grid of its own binade: with 2^E <= |v| < 2^(E+1)
// (m = |v| or a larger value), head = v rounded to a multiple of 2^(E-8),
// i.e. at most 10 significant bits, by adding and subtracting 1.5 2^(E+15).
__device__ __forceinline__ float head_constant(float m) {
  const unsigned e = __float_as_uint(m) & 0x7f800000u;
  return __uint_as_float(e + (15u << 23) + 0x400000u);
}

__device__ __forceinline__ float head_of(float v, float C) { return __fsub_rn(__fadd_rn(v, C), C); }

// The sky functions split for the antenna products: (head on the 2^-8 grid,
// tail = rest + lo part); |beta|, |gamma| < 4.
struct AntennaSplit {
  float bh[6], bt[6], gh[4], gt[4];
};

__device__ __forceinline__ void split_antenna_basis(const AntennaBasis& B, AntennaSplit& S) {
  const float C = 49152.0f;  // 1.5 * 2^15: ulp 2^-8
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    S.bh[i] = head_of(B.b[i].hi, C);
    S.bt[i] = __fadd_rn(__fsub_rn(B.b[i].hi, S.bh[i]), B.b[i].lo);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    S.gh[i] = head_of(B.g[i].hi, C);
    S.gt[i] = __fadd_rn(__fsub_rn(B.g[i].hi, S.gh[i]), B.g[i].lo);
  }
}

// x F_k = x e^{2 i psi} (F_+(0) - i F_x(0)) of detector k, with xe = x e^{2 i psi}.
// F_+(0) and F_x(0) by the split product: the detector's coefficients are
// stored as a 10-bit head on the grid 2^(E-9) of their largest magnitude and
// a tail (point.cu); head x head products are exact and their sum of at most
// six stays below 2^22 quanta, so it is exact in FP32; the cross terms are
// >= 2^9 smaller and summed in FP32.
RIFT_HELPER void antenna_df(const MixedTables& T, int k, const AntennaSplit& S, df xer, df xei,
                            df& xFr, df& xFi) {
  float h[12], t[12];
#pragma unroll
  for (int v = 0; v < 3; ++v) {
    const float4 a = T.ah[k][v], b = T.at[k][v];
    h[4 * v] = a.x; h[4 * v + 1] = a.y; h[4 * v + 2] = a.z; h[4 * v + 3] = a.w;
    t[4 * v] = b.x; t[4 * v + 1] = b.y; t[4 * v + 2] = b.z; t[4 * v + 3] = b.w;
  }
  float fp = S.bh[0] * h[0], fpc = 0.f;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    if (i) fp = fmaf(h[i], S.bh[i], fp);
    fpc = fmaf(h[i], S.bt[i], fpc);
    fpc = fmaf(t[i], __fadd_rn(S.bh[i], S.bt[i]), fpc);
  }
  float fx = S.gh[0] * h[6], fxc = 0.f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    if (i) fx = fmaf(h[6 + i], S.gh[i], fx);
    fxc = fmaf(h[6 + i], S.gt[i], fxc);
    fxc = fmaf(t[6 + i], __fadd_rn(S.gh[i], S.gt[i]), fxc);
  }
  // (fp - i fx)(xer + i xei) with the pairs (fp, fpc), (fx, fxc) unnormalised
  {
    const df p1 = two_prod(fp, xer.hi), p2 = two_prod(fx, xei.hi);
    const df sm = two_sum(p1.hi, p2.hi);
    float lo = __fadd_rn(__fadd_rn(p1.lo, p2.lo), sm.lo);
    lo = fmaf(fp, xer.lo, lo);
    lo = fmaf(fpc, xer.hi, lo);
    lo = fmaf(fx, xei.lo, lo);
    lo = fmaf(fxc, xei.hi, lo);
    xFr = fast_two_sum(sm.hi, lo);
  }
  {
    const df p1 = two_prod(fp, xei.hi), p2 = two_prod(-fx, xer.hi);
    const df sm = two_sum(p1.hi, p2.hi);
    float lo = __fadd_rn(__fadd_rn(p1.lo, p2.lo), sm.lo);
    lo = fmaf(fp, xei.lo, lo);
    lo = fmaf(fpc, xei.hi, lo);
    lo = fmaf(-fx, xer.lo, lo);
    lo = fmaf(-fxc, xer.hi, lo);
    xFi = fast_two_sum(sm.hi, lo);
  }
}

// FP32 amplitude of mode i and its derivative with respect to iota (used by
// the adjoint, whose terms multiply the small residual and need only FP32):
// amp = sz^par p(z), d amp/d iota = par z p(z) - sz^(par+1) p'(z) (dz = -sz d iota).
__device__ __forceinline__ void sylm_amp_grad_f(const MixedTables& T, int j, int l, int par,
                                                float z, float sz, float& amp, float& damp) {
  float pz = T.yz[j][l].x, dp = 0.f;
  for (int q = l - 1; q >= 0; --q) {
    dp = fmaf(dp, z, pz);
    pz = fmaf(pz, z, T.yz[j][q].x);
  }
  if (par) {
    amp = sz * pz;
    damp = fmaf(z, pz, -sz * sz * dp);
  } else {
    amp = pz;
    damp = -sz * dp;
  }
}

// d(beta_i)/d(ra), d(beta_i)/d(dec) and the same for gamma (FP32; see AntennaBasis).
struct AntennaBasisGrad {
  float ba[6], bd[6], ga[4], gd[4];
};

__device__ __forceinline__ void antenna_basis_grad(float sl, float cl, float sd, float cd,
                                                   AntennaBasisGrad& G) {
  const float sd2 = sd * sd, slcl = sl * cl, c2 = cl * cl - sl * sl, dd = cd * cd - sd * sd;
  G.ba[0] = 2.f * slcl * (1.f + sd2);
  G.bd[0] = -2.f * sd * cd * cl * cl;
  G.ba[1] = -2.f * slcl * (1.f + sd2);
  G.bd[1] = -2.f * sd * cd * sl * sl;
  G.ba[2] = -2.f * c2 * (1.f + sd2);
  G.bd[2] = -4.f * slcl * sd * cd;
  G.ba[3] = -2.f * sd * cd * sl;
  G.bd[3] = 2.f * dd * cl;
  G.ba[4] = 2.f * sd * cd * cl;
  G.bd[4] = 2.f * dd * sl;
  G.ba[5] = 0.f;
  G.bd[5] = 2.f * cd * sd;
  G.ga[0] = 2.f * sd * c2;
  G.gd[0] = 2.f * cd * slcl;
  G.ga[1] = 8.f * sd * slcl;
  G.gd[1] = -2.f * cd * c2;
  G.ga[2] = -2.f * cl * cd;
  G.gd[2] = 2.f * sl * sd;
  G.ga[3] = -2.f * sl * cd;
  G.gd[3] = -2.f * cl * sd;
}

// The error-free split of a mode value y (|y| < 2): y1 = y rounded to a
// multiple of 2^-8 (9 significant bits), y2 = y - y1 exact.
__device__ __forceinline__ void split_y(float y, float& y1, float& y2) {
  const float C = 49152.0f;  // 1.5 * 2^15: ulp(C) = 2^-8
  y1 = __fsub_rn(__fadd_rn(y, C), C);
  y2 = __fsub_rn(y, y1);
}

struct MixedDraw {
  df lnl;      // lnL, or with DIST the data term K at x = 1
  df R;        // with DIST: the quadratic coefficient R at x = 1 (lnL(x) = K x - R x^2/2)
  int oob;
  double grad[kNpar];
  // with GRAD and DIST (one pass at x = 1): grad = d lnL(1) = dK - dR/2 + ...
  // split as in lnl_mixed_draw, and gradB = dR/2
  double gradB[kNpar];
};

// Distance marginal of one draw from K and R (eq. ap:dexp, eq. ap:dlog);
// ex (if given) receives the node-posterior moments E[x], E[x^2], E[x(1-x)]:
// K^2/(2R) in double-float plus the node sum of dist_lse, in FP32 offsets
// from x* = K/R (see dist_lse in common.cuh for the window rule).
__device__ __forceinline__ df dist_marg_df(const DistParams& dp, df K, df R, float* ex = nullptr) {
  if (!(R.hi > 0.f)) {
    double peak, exd[2];
    const double v = dist_lse(dp, df_to_double(K), df_to_double(R), 0.0, &peak, exd);
    if (ex) {
      ex[0] = (float)exd[0];
      ex[1] = (float)exd[1];
      ex[2] = (float)(exd[0] - exd[1]);
    }
    return df_from_double(v);
  }
  // x* = K / R by one Newton correction of the float quotient
  const float q0 = K.hi / R.hi;
  df pr = two_prod(q0, R.hi);
  pr.lo = fmaf(q0, R.lo, pr.lo);
  const df rem = df_sub(K, pr);
  const df xs = fast_two_sum(q0, rem.hi / R.hi);
  // nearest node by bisection on the hi parts (x decreasing): the bracket
  // x[lo] > xs >= x[hi] narrows to the unique adjacent pair; on a table
  // uniform in ln x it starts from the estimated position when the estimate's
  // bracket holds (two independent loads instead of a chain of ~log2 n)
  int lo = 0, hi = dp.n - 1;
  if (!(xs.hi < dp.xdf[0].x)) {
    hi = 0;
  } else if (!(xs.hi > dp.xdf[dp.n - 1].x)) {
    lo = dp.n - 1;
  } else {
    if (dp.guess) {  // here x[n - 1] < xs.hi < x[0] and x[n - 1] > 0
      const float g = fminf(fmaxf((dp.lnx0 - __logf(xs.hi)) * dp.inv_dlnx, 0.f), (float)(dp.n - 2));
      const int jg = (int)g;
      const int l2 = max(jg - 1, 0), h2 = min(jg + 2, dp.n - 1);
      if (__ldg(&dp.xdf[l2].x) > xs.hi && !(__ldg(&dp.xdf[h2].x) > xs.hi)) {
        lo = l2;
        hi = h2;
      }
    }
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (dp.xdf[mid].x > xs.hi) lo = mid;
      else hi = mid;
    }
  }
  const int j0 = (dp.xdf[lo].x - xs.hi < xs.hi - dp.xdf[hi].x) ? lo : hi;
  // the nearest node's offset qn = R (x_j0 - x*)^2 / 2 in double-float; every
  // node enters relative to it, q_j - qn = R/2 (x_j - x_j0)(x_j + x_j0 - 2 x*)
  // in FP32 (a difference of at most a few tens of nats over the nodes that
  // count), so that a table far from x* (qn large) keeps the precision
  const float2 x0 = __ldg(dp.xdf + j0);
  df d0 = two_sum(x0.x, -xs.hi);
  d0.lo = __fadd_rn(d0.lo, __fsub_rn(x0.y, xs.lo));
  d0 = fast_two_sum(d0.hi, d0.lo);
  const df qn = df_mul(df{0.5f * R.hi, 0.5f * R.lo}, df_mul(d0, d0));
  float m = -CUDART_INF_F, s = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;  // m, t relative to -qn
  const float halfR = 0.5f * R.hi;
  const float lnw_max = (float)dp.lnw_max;
  for (int dir = -1; dir <= 1; dir += 2) {
    int j = dir < 0 ? j0 : j0 + 1;
    if (j < 0 || j >= dp.n) continue;
    // the next node's loads are issued before this node's test (software
    // pipelined: the scan's loads do not wait on its exit test)
    float2 xj = __ldg(dp.xdf + j);
    float lwj = __ldg(dp.lnwf + j);
    for (;;) {
      const int jn = j + dir;
      const bool more = jn >= 0 && jn < dp.n;
      float2 xn = xj;
      float lwn = lwj;
      if (more) {
        xn = __ldg(dp.xdf + jn);
        lwn = __ldg(dp.lnwf + jn);
      }
      const float d = __fadd_rn(__fsub_rn(xj.x, xs.hi), __fsub_rn(xj.y, xs.lo));  // x_j - x*
      const float dr = __fadd_rn(__fsub_rn(xj.x, x0.x), __fsub_rn(xj.y, x0.y));  // x_j - x_j0
      const float q = halfR * dr * __fadd_rn(d, d0.hi);                          // q_j - qn
      if (lnw_max - q < m - 40.f) break;
      const float t = lwj - q;
      const float xq = xj.x * __fsub_rn(1.f, xj.x);  // x (1 - x) without cancellation
      if (t > m) {
        const float r = __expf(m - t);
        s = fmaf(s, r, 1.f);
        s1 = fmaf(s1, r, xj.x);
        s2 = fmaf(s2, r, xj.x * xj.x);
        s3 = fmaf(s3, r, xq);
        m = t;
      } else {
        const float e = t > -CUDART_INF_F ? __expf(t - m) : 0.f;  // a zero-weight node adds 0
        s += e;
        s1 = fmaf(e, xj.x, s1);
        s2 = fmaf(e * xj.x, xj.x, s2);
        s3 = fmaf(e, xq, s3);
      }
      if (!more) break;
      j = jn;
      xj = xn;
      lwj = lwn;
    }
  }
  if (ex) {
    ex[0] = s1 / s;
    ex[1] = s2 / s;
    ex[2] = s3 / s;
  }
  const df peak = df_mul(K, xs);
  return df_add_f(df_sub(df{0.5f * peak.hi, 0.5f * peak.lo}, qn), m + __logf(s));
}

// One draw: lnL, and with GRAD its gradient in (ra, dec, psi, incl, phase, lnD, t).
//
// Adjoint (Sec. II.B): with r_k = e_k - w_k and rho_k = r_k + gm1 w_k,
//   d lnL = sum_k [ (P_k'(f)/dt - r_k . edot_k) dt_k + rho_k . dw_k ],
// the first bracket being w_k . edot_k (computed as the exact polynomial
// slope minus a small residual term); dw_k follows from w_k = Re(xF_k) a1 +
// Im(xF_k) a2: rho_k . dw_k = d Re(xF_k) rho_k.a1 + d Im(xF_k) rho_k.a2 for the
// sky angles, psi and lnD, and (A^T G1 + J^T A^T G2) . dy with
// G1 = sum_k Re(xF_k) rho_k, G2 = sum_k Im(xF_k) rho_k for iota and phase.
// With DIST the template is taken at the distance factor xin (1 for the
// marginal's K and R) instead of D_ref e^{-lnD}.
template <int MM, int RR, bool GRAD, bool DIST = false, bool EXACT = false>
__device__ __forceinline__ MixedDraw lnl_mixed_draw(const PointParams& P, const MixedTables& TB,
                                                    const float4* sA,
                                                    const float* sg, float4* a12s, float4* xfs,
                                                    const DrawsParams& dp, long long i,
                                                    df xin = df{1.f, 0.f}) {
  const float ra = load_param_f(dp, 0, i), dec = load_param_f(dp, 1, i);
  const float psi = load_param_f(dp, 2, i), incl = load_param_f(dp, 3, i);
  const float phi = load_param_f(dp, 4, i), lnD = load_param_f(dp, 5, i);
  const df tc = load_param_df(dp, 6, i);
  const int M = P.M, R = P.R, n = P.n;

  // distance factor x = D_ref e^{-lnD}
  df lx = two_sum(P.ln_dref_hi, -lnD);
  lx.lo = __fadd_rn(lx.lo, P.ln_dref_lo);
  // with distance marginalisation the terms are taken at x = 1
  const df x = DIST ? xin : exp_df(fast_two_sum(lx.hi, lx.lo));

  // sky direction and transverse basis
  df lam = two_sum(ra, -P.gmst_hi);
  lam.lo = __fsub_rn(lam.lo, P.gmst_lo);
  lam = fast_two_sum(lam.hi, lam.lo);
  df sl, cl, sd, cd;
  sincos_df(lam, sl, cl);
  sincos_df(df{dec, 0.f}, sd, cd);
  const df s0 = df_mul(cd, cl), s1 = df_mul(cd, sl), s2 = sd;
  AntennaSplit AS;
  {
    AntennaBasis AB;
    antenna_basis(sl, cl, sd, cd, AB);
    split_antenna_basis(AB, AS);
  }
  df s2p, c2p;
  sincos_df(df{2.f * psi, 0.f}, s2p, c2p);
  const df xer = df_mul(x, c2p), xei = df_mul(x, s2p);
  // x F_k of every detector, kept in this thread's shared-memory slots as
  // (head, tail) pairs on the grid of the larger part (see the template
  // product below), so the sky functions need not stay in registers
  for (int k = 0; k < P.K; ++k) {
    df xFr, xFi;
    antenna_df(TB, k, AS, xer, xei, xFr, xFi);
    const float Cx = head_constant(fmaxf(fabsf(xFr.hi), fabsf(xFi.hi)));
    const float xrh = head_of(xFr.hi, Cx), xih = head_of(xFi.hi, Cx);
    xfs[k * kMixedThreads] = make_float4(xrh, __fadd_rn(__fsub_rn(xFr.hi, xrh), xFr.lo), xih,
                                         __fadd_rn(__fsub_rn(xFi.hi, xih), xFi.lo));
  }
  df sz, z;  // sin and cos of the inclination
  sincos_df(df{incl, 0.f}, sz, z);

  dacc T = dacc_zero();
  dacc Racc = dacc_zero();  // DIST: R = sum_k (|w_k|^2 - sum_r gm1_r w_kr^2)
  // DIST: |w_k|^2 of the direction pairs as the two lanes of a packed
  // compensated sum (sum, error), over all detectors of the draw in the
  // forward pass and per detector in the adjoint (fewer live registers there)
  constexpr bool kW2Draw = DIST && !GRAD;
  float2 w2s = make_float2(0.f, 0.f), w2c = make_float2(0.f, 0.f);
  int oob = 0;
  bool bad = false;
  // gradient accumulators: time-driven parts of (ra, dec, t) as pairs, the rest in FP32
  dacc gt_ra = dacc_zero(), gt_dec = dacc_zero(), gt_t = dacc_zero();
  float g_ra = 0.f, g_dec = 0.f, g_psi = 0.f, g_incl = 0.f, g_phase = 0.f, g_lnd = 0.f;
  // with GRAD and DIST: the same template derivatives weighted by (1 - gm1) w
  constexpr bool TWO = GRAD && DIST;
  float gB_ra = 0.f, gB_dec = 0.f, gB_psi = 0.f, gB_incl = 0.f, gB_phase = 0.f;
  AntennaBasisGrad ABG;
  float dsa[3] = {0.f, 0.f, 0.f}, dsd[3] = {0.f, 0.f, 0.f};
  if (GRAD) {
    antenna_basis_grad(sl.hi, cl.hi, sd.hi, cd.hi, ABG);
    // ds/d ra = (-cd sl, cd cl, 0), ds/d dec = (-sd cl, -sd sl, cd)
    dsa[0] = -cd.hi * sl.hi;
    dsa[1] = cd.hi * cl.hi;
    dsd[0] = -sd.hi * cl.hi;
    dsd[1] = -sd.hi * sl.hi;
    dsd[2] = cd.hi;
  }
  for (int c = 0; c < P.ncls; ++c) {
    // a1 = A y, a2 = A J y by the split product: the products of the 10-bit
    // head of A with the 9-bit head of y are exact and their sum stays below
    // 2^24 quanta, so ex1/ex2 are exact; every other term is ~2^-9 smaller.
    // Directions advance by pairs (r, r + 1) as the two lanes of the packed
    // FMAs (one FFMA2 issues both): ex1[r/2] = (ex1 of r, of r + 1), and
    // likewise ex2, co1, co2
    float2 ex1[RR / 2], ex2[RR / 2], co1[RR / 2], co2[RR / 2];
#pragma unroll
    for (int p = 0; p < RR / 2; ++p) ex1[p] = ex2[p] = co1[p] = co2[p] = make_float2(0.f, 0.f);
    const float4* Ac = sA + (size_t)c * R * M;
    // modes in order of increasing |m| (P.morder): e^{i |m| phi} is reused
    // across modes of equal |m| and stepped by one complex product with
    // e^{i phi} when |m| grows by one; otherwise an anchored sine/cosine
    int prev_am = -1;
    df cm = df{1.f, 0.f}, sm = df{0.f, 0.f}, c1 = df{1.f, 0.f}, s1p = df{0.f, 0.f};
    bool have1 = false;
#if RIFT_MIXED_MODE_UNROLL
#pragma unroll kModeUnroll
#endif
    for (int j = 0; j < M; ++j) {
      const int4 md = TB.mode[j];  // (mode index, m, l, ypar)
      const int m = md.y, am = m < 0 ? -m : m;
      if (am != prev_am) {
        if (have1 && am == prev_am + 1) {
          const df cn = df_sub(df_mul(cm, c1), df_mul(sm, s1p));
          sm = df_add(df_mul(sm, c1), df_mul(cm, s1p));
          cm = cn;
        } else {
          sincos_df(two_prod((float)am, phi), sm, cm);
          if (am == 1) {
            c1 = cm;
            s1p = sm;
            have1 = true;
          }
        }
        prev_am = am;
      }
      const df amp = sylm_amp_df(TB, j, md.z, md.w, z, sz);
      const df yr = df_mul(amp, cm);
      const df yi = m < 0 ? df_neg(df_mul(amp, sm)) : df_mul(amp, sm);
      // y = y1 + y2 with y1 the 9-bit head and y2 = (y.hi - y1) + y.lo
      float yr1, yr2, yi1, yi2;
      split_y(yr.hi, yr1, yr2);
      split_y(yi.hi, yi1, yi2);
      yr2 = __fadd_rn(yr2, yr.lo);
      yi2 = __fadd_rn(yi2, yi.lo);
      const float2 pr1 = make_float2(yr1, yr1), pi1 = make_float2(yi1, yi1);
      const float2 pr2 = make_float2(yr2, yr2), pi2 = make_float2(yi2, yi2);
      const float2 prh = make_float2(yr.hi, yr.hi), pih = make_float2(yi.hi, yi.hi);
      const float2 ni1 = make_float2(-yi1, -yi1), ni2 = make_float2(-yi2, -yi2);
      const float2 nih = make_float2(-yi.hi, -yi.hi);
#pragma unroll
      for (int p = 0; p < RR / 2; ++p) {
        if (EXACT || 2 * p < R) {
          // with t = A[r][a], b = A[r][M + a] as (head, tail), lanes (r, r + 1):
          // hd = (t_h, t_h, b_h, b_h), tl = (t_t, t_t, b_t, b_t);
          // a1_r += t yr + b yi ;  a2_r += b yr - t yi
          const float4 hd = Ac[2 * (p * M + j)], tl = Ac[2 * (p * M + j) + 1];
          const float2 th = make_float2(hd.x, hd.y), bh = make_float2(hd.z, hd.w);
          const float2 tt = make_float2(tl.x, tl.y), bt = make_float2(tl.z, tl.w);
          ex1[p] = __ffma2_rn(th, pr1, ex1[p]);
          ex1[p] = __ffma2_rn(bh, pi1, ex1[p]);
          ex2[p] = __ffma2_rn(bh, pr1, ex2[p]);
          ex2[p] = __ffma2_rn(th, ni1, ex2[p]);
          co1[p] = __ffma2_rn(th, pr2, co1[p]);
          co1[p] = __ffma2_rn(tt, prh, co1[p]);
          co1[p] = __ffma2_rn(bh, pi2, co1[p]);
          co1[p] = __ffma2_rn(bt, pih, co1[p]);
          co2[p] = __ffma2_rn(bh, pr2, co2[p]);
          co2[p] = __ffma2_rn(bt, prh, co2[p]);
          co2[p] = __ffma2_rn(th, ni2, co2[p]);
          co2[p] = __ffma2_rn(tt, nih, co2[p]);
        }
      }
    }
    // a1_r, a2_r as (head, tail) on the grid of the larger of the two exact
    // head sums: the template product below takes head x head exactly; the
    // tail is (ex - head) (exact) + co rounded once, whatever the size of co
    // against ex.  Stored by direction pairs (r, r + 1), r even: slot r =
    // (a1 heads, a1 tails) and slot r + 1 = (a2 heads, a2 tails), each
    // component pair (r, r + 1) adjacent for the packed instructions of the
    // residual loop
    constexpr bool kA12S = A12Smem<RR>::on;
    float4 a12r[kA12S ? 1 : RR];
#pragma unroll
    for (int r = 0; r < RR; r += 2) {
      const int p = r / 2;
      const float2 C2 = make_float2(head_constant(fmaxf(fabsf(ex1[p].x), fabsf(ex2[p].x))),
                                    head_constant(fmaxf(fabsf(ex1[p].y), fabsf(ex2[p].y))));
      const float2 h1 = sub2(__fadd2_rn(ex1[p], C2), C2), h2 = sub2(__fadd2_rn(ex2[p], C2), C2);
      const float2 t1 = __fadd2_rn(sub2(ex1[p], h1), co1[p]);
      const float2 t2 = __fadd2_rn(sub2(ex2[p], h2), co2[p]);
      const float4 qa = make_float4(h1.x, h1.y, t1.x, t1.y);
      const float4 qb = make_float4(h2.x, h2.y, t2.x, t2.y);
      if constexpr (kA12S) {
        a12s[r * kMixedThreads] = qa;
        a12s[(r + 1) * kMixedThreads] = qb;
      } else {
        a12r[r] = qa;
        a12r[r + 1] = qb;
      }
    }
    auto get_a = [&](int r) -> float4 {
      if constexpr (kA12S) {
        return a12s[r * kMixedThreads];
      } else {
        return a12r[r];
      }
    };
    const float* gc = sg + c * R;
    df delay = df{0.f, 0.f};
    // G1, G2 (and G1B, G2B) by direction pairs: .x direction r, .y r + 1
    float2 G1[GRAD ? RR / 2 : 1], G2[GRAD ? RR / 2 : 1];
    float2 G1B[TWO ? RR / 2 : 1], G2B[TWO ? RR / 2 : 1];
    if (GRAD) {
#pragma unroll
      for (int r = 0; r < RR / 2; ++r) G1[r] = G2[r] = make_float2(0.f, 0.f);
    }
    if (TWO) {
#pragma unroll
      for (int r = 0; r < RR / 2; ++r) G1B[r] = G2B[r] = make_float2(0.f, 0.f);
    }
#if RIFT_MIXED_DET_UNROLL
#pragma unroll kDetUnroll
#endif
    const bool hn = P.has_null[c] != 0;  // uniform over the block
    for (int q = P.cls_begin[c]; q < P.cls_begin[c + 1]; ++q) {
      const int k = P.det_order[q];
      const float4 xfq = xfs[k * kMixedThreads];
      const float xrh = xfq.x, xrt = xfq.y, xih = xfq.z, xit = xfq.w;
      const df xFr = df{__fadd_rn(xrh, xrt), 0.f}, xFi = df{__fadd_rn(xih, xit), 0.f};  // FP32 uses
      // arrival time (shared by co-located detectors) and table position
      const float4 ph = TB.pos_hi[k], pl = TB.pos_lo[k];  // (position, t0) pairs
      if (!P.same_pos_prev[q]) delay = dot3_df(ph, pl, s0, s1, s2);
      const df rel = df_add(df_sub(tc, delay), df{-ph.w, -pl.w});
      const df u = df_mul(rel, df{P.inv_dt_hi, P.inv_dt_lo});
      if (!isfinite(u.hi)) {
        bad = true;
        oob += 4;
        continue;
      }
      float jf = floorf(u.hi);
      if (u.hi == jf && u.lo < 0.f) jf -= 1.f;
      const float f = __fadd_rn(__fsub_rn(u.hi, jf), u.lo);
      // the interval's record: j clamped to [-3, n + 1], where every tap
      // outside the table is a zero row of the padded table the coefficients
      // were formed from and the sextic is zero, so the loads need no test
      // (taps outside are only counted)
      {  // taps outside the table: 1 - j below it, j + 3 - n above it (each in [0, 4])
        const float nb = fminf(fmaxf(1.f - jf, 0.f), 4.f);
        const float na = fminf(fmaxf(jf + 3.f - (float)n, 0.f), 4.f);
        oob += (int)fminf(nb + na, 4.f);
      }
      const int jc = (int)fminf(fmaxf(jf, -3.f), (float)(n + 1));
      const float4* Cj = P.erec + ((size_t)k * (n + 5) + (size_t)(jc + 3)) * (size_t)(3 * (R / 2) + 4);
      // 1/2 |e(f)|^2 from the interval's sextic (pairs (c0, c1), (c2, c3),
      // (c4, c5), (c6, -) after the cubic) and, for the adjoint, its slope in
      // f (Horner on both: horner_step, f exact in FP32; both sums absorb
      // unnormalised pairs)
      df half_e2, dhalf = df{0.f, 0.f};
      {
        const float4* pe = Cj + 3 * (R / 2);
        const float4 e01 = __ldg(pe), e23 = __ldg(pe + 1), e45 = __ldg(pe + 2), e6 = __ldg(pe + 3);
        const float2 cf[kPolyDeg + 1] = {make_float2(e01.x, e01.y), make_float2(e01.z, e01.w),
                                         make_float2(e23.x, e23.y), make_float2(e23.z, e23.w),
                                         make_float2(e45.x, e45.y), make_float2(e45.z, e45.w),
                                         make_float2(e6.x, e6.y)};
        df acc = df{cf[kPolyDeg].x, cf[kPolyDeg].y};
#pragma unroll
        for (int p = kPolyDeg - 1; p >= 0; --p) {
          if (GRAD) dhalf = horner_step_f(dhalf, f, acc.hi, acc.lo);
          acc = horner_step_f(acc, f, cf[p].x, cf[p].y);
        }
        half_e2 = acc;
      }
      const float2 f2 = make_float2(f, f), f3 = make_float2(3.f * f, 3.f * f);
      // Per pair of directions: the template w_r = xFr a1_r + xFi a2_r (heads
      // of xF on the grid of its larger part; head x head products of 10 x 10
      // bits and their sum exact, the cross terms >= 2^8 smaller; w kept as
      // the unnormalised pair (exact head sum, FP32 correction)), then the
      // residual r = e(f) - w = (c0.hi - w_head) + (c0.lo + f (c1 + f (c2 + f c3)))
      // - w_tail: the tap row's high part meets the exact head sum of w first
      // (the large terms cancel there), the cubic's f-dependent part and the
      // low parts are FP32 (rounding u |e_i - e_j| as with FP32 tap weights).
      // Both directions of a pair advance together in packed FP32 pairs
      // (FFMA2 / FADD2 / FMUL2 issue two operations each).  The template is
      // formed negated, nw = -w (negation is exact, so every rounding is the
      // one of the unnegated form), which turns e - w into a packed add.
      const float2 nxrh = make_float2(-xrh, -xrh), nxrt = make_float2(-xrt, -xrt);
      const float2 nxih = make_float2(-xih, -xih), nxit = make_float2(-xit, -xit);
      const float2 xFr2 = make_float2(xFr.hi, xFr.hi), xFi2 = make_float2(xFi.hi, xFi.hi);
      const float2 zero2 = make_float2(0.f, 0.f);
      float2 q2p = zero2, nulp = zero2, redp = zero2, g1p = zero2, g2p = zero2, g1Bp = zero2,
             g2Bp = zero2;
      if (!kW2Draw) w2s = w2c = zero2;
#pragma unroll
      for (int r = 0; r < RR; r += 2) {
        if (EXACT || r < R) {
          const float4 qa = get_a(r), qb = get_a(r + 1);  // (a1 | a2) heads, tails of r, r + 1
          const float2 a1h = make_float2(qa.x, qa.y), a1t = make_float2(qa.z, qa.w);
          const float2 a2h = make_float2(qb.x, qb.y), a2t = make_float2(qb.z, qb.w);
          float2 nlo = __fmul2_rn(nxrh, a1t);
          nlo = __ffma2_rn(nxrt, a1h, nlo);
          nlo = __ffma2_rn(nxrt, a1t, nlo);
          nlo = __ffma2_rn(nxih, a2t, nlo);
          nlo = __ffma2_rn(nxit, a2h, nlo);
          nlo = __ffma2_rn(nxit, a2t, nlo);
          const float2 nhi = __ffma2_rn(nxrh, a1h, __fmul2_rn(nxih, a2h));
          // (c0 hi, c0 lo) of directions r, r + 1, then (c1, c2), (c3, -)
          const float4 c0 = __ldg(Cj + 3 * (r / 2)), c12 = __ldg(Cj + 3 * (r / 2) + 1);
          const float4 c3v = __ldg(Cj + 3 * (r / 2) + 2);
          const float2 c1 = make_float2(c12.x, c12.y), c2 = make_float2(c12.z, c12.w);
          const float2 c3 = make_float2(c3v.x, c3v.y);
          float2 hp = __ffma2_rn(c3, f2, c2);
          hp = __ffma2_rn(hp, f2, c1);
          const float2 tl = __ffma2_rn(hp, f2, make_float2(c0.z, c0.w));
          const float2 d0 = __fadd2_rn(make_float2(c0.x, c0.y), nhi);
          const float2 rsv = __fadd2_rn(__fadd2_rn(d0, tl), nlo);
          // the adjoint's de/df = c1 + f (2 c2 + 3 f c3)
          float2 ed = zero2;
          if (GRAD) ed = __ffma2_rn(__ffma2_rn(c3, f3, __fadd2_rn(c2, c2)), f2, c1);
          q2p = __ffma2_rn(rsv, rsv, q2p);
          const float2 nwf = __fadd2_rn(nhi, nlo);  // -w rounded to FP32
          // gm1 is zero unless the class keeps near-null directions: the
          // forward pass skips it then (the adjoint keeps the load, faster there)
          float2 gm = zero2;
          if (GRAD || hn) {
            gm = make_float2(gc[r], gc[r + 1]);
            nulp = __ffma2_rn(__fmul2_rn(gm, nwf), nwf, nulp);
          }
          if (DIST) {  // |w|^2 with the head square exact: lane sums by packed TwoSum
            const df2 p = two_prod2(nhi, nhi);
            const df2 t = two_sum2(w2s, p.hi);
            w2s = t.hi;
            float2 cc = __fadd2_rn(t.lo, p.lo);
            cc = __ffma2_rn(__fadd2_rn(nhi, nhi), nlo, cc);
            cc = __ffma2_rn(nlo, nlo, cc);
            w2c = __fadd2_rn(w2c, cc);
          }
          if (GRAD) {
            redp = __ffma2_rn(rsv, ed, redp);
            // rho = r + gm1 w = r - gm1 nw
            const float2 rho = __ffma2_rn(make_float2(-gm.x, -gm.y), nwf, rsv);
            const float2 a1 = __fadd2_rn(a1h, a1t), a2 = __fadd2_rn(a2h, a2t);
            g1p = __ffma2_rn(rho, a1, g1p);
            g2p = __ffma2_rn(rho, a2, g2p);
            G1[r / 2] = __ffma2_rn(xFr2, rho, G1[r / 2]);
            G2[r / 2] = __ffma2_rn(xFi2, rho, G2[r / 2]);
            if (TWO) {  // dR/2 = sum (1 - gm1) w . dw = sum (gm1 - 1) nw . dw
              const float2 rhoB = __fmul2_rn(make_float2(__fsub_rn(gm.x, 1.f), __fsub_rn(gm.y, 1.f)),
                                             nwf);
              g1Bp = __ffma2_rn(rhoB, a1, g1Bp);
              g2Bp = __ffma2_rn(rhoB, a2, g2Bp);
              G1B[r / 2] = __ffma2_rn(xFr2, rhoB, G1B[r / 2]);
              G2B[r / 2] = __ffma2_rn(xFi2, rhoB, G2B[r / 2]);
            }
          }
        }
      }
      const float q2 = __fadd_rn(q2p.x, q2p.y), nul = __fadd_rn(nulp.x, nulp.y);
      const float red = __fadd_rn(redp.x, redp.y);
      const float g1 = __fadd_rn(g1p.x, g1p.y), g2 = __fadd_rn(g2p.x, g2p.y);
      const float g1B = __fadd_rn(g1Bp.x, g1Bp.y), g2B = __fadd_rn(g2Bp.x, g2Bp.y);
      dacc_add(T, half_e2);
      dacc_add(T, df{-0.5f * q2, 0.f});
      if (P.has_null[c] && !DIST) dacc_add(T, df{0.5f * nul, 0.f});
      if (DIST) {
        // K_k = e.w = 1/2|e|^2 + 1/2|w|^2 - 1/2|e - w|^2 (the first and last are in T
        // already); R_k = |w|^2 - sum_r gm1_r w_r^2
        if (!kW2Draw) {
          const df w2t = two_sum(w2s.x, w2s.y);
          const df w2d = fast_two_sum(w2t.hi, __fadd_rn(w2t.lo, __fadd_rn(w2c.x, w2c.y)));
          dacc_add(T, df{0.5f * w2d.hi, 0.5f * w2d.lo});
          dacc_add(Racc, w2d);
        }
        if (P.has_null[c]) dacc_add(Racc, df{-nul, 0.f});
      }
      if (GRAD) {
        // time: d lnL_k / d t_k = (P'(f) - r . edot dt) / dt
        const df dtk = df_mul(df_add_f(dhalf, -red), df{P.inv_dt_hi, P.inv_dt_lo});
        const float dka = -(ph.x * dsa[0] + ph.y * dsa[1]);
        const float dkd = -(ph.x * dsd[0] + ph.y * dsd[1] + ph.z * dsd[2]);
        dacc_add(gt_t, dtk);
        dacc_add(gt_ra, df_mul_f(dtk, dka));
        dacc_add(gt_dec, df_mul_f(dtk, dkd));
        // antenna: d(xF) = x e^{2 i psi} (dF+ - i dFx), d/d psi (xF) = 2 i xF
        float dfpa = 0.f, dfpd = 0.f, dfxa = 0.f, dfxd = 0.f;
        float ac[12];  // the antenna coefficients in FP32 (head + tail)
#pragma unroll
        for (int v = 0; v < 3; ++v) {
          const float4 a4 = TB.ah[k][v], b4 = TB.at[k][v];
          ac[4 * v] = a4.x + b4.x;
          ac[4 * v + 1] = a4.y + b4.y;
          ac[4 * v + 2] = a4.z + b4.z;
          ac[4 * v + 3] = a4.w + b4.w;
        }
#pragma unroll
        for (int u = 0; u < 6; ++u) {
          dfpa = fmaf(ac[u], ABG.ba[u], dfpa);
          dfpd = fmaf(ac[u], ABG.bd[u], dfpd);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          dfxa = fmaf(ac[6 + u], ABG.ga[u], dfxa);
          dfxd = fmaf(ac[6 + u], ABG.gd[u], dfxd);
        }
        // (dfp - i dfx)(xer + i xei)
        const float dxra = dfpa * xer.hi + dfxa * xei.hi, dxia = dfpa * xei.hi - dfxa * xer.hi;
        const float dxrd = dfpd * xer.hi + dfxd * xei.hi, dxid = dfpd * xei.hi - dfxd * xer.hi;
        g_ra = fmaf(dxra, g1, fmaf(dxia, g2, g_ra));
        g_dec = fmaf(dxrd, g1, fmaf(dxid, g2, g_dec));
        g_psi = fmaf(-2.f * xFi.hi, g1, fmaf(2.f * xFr.hi, g2, g_psi));
        g_lnd = fmaf(-xFr.hi, g1, fmaf(-xFi.hi, g2, g_lnd));
        if (TWO) {
          gB_ra = fmaf(dxra, g1B, fmaf(dxia, g2B, gB_ra));
          gB_dec = fmaf(dxrd, g1B, fmaf(dxid, g2B, gB_dec));
          gB_psi = fmaf(-2.f * xFi.hi, g1B, fmaf(2.f * xFr.hi, g2B, gB_psi));
        }
      }
    }
    if (GRAD) {
      // iota and phase through the modes: H = A^T G1 + J^T A^T G2 (FP32)
      const float4* Ac2 = sA + (size_t)c * R * M;
      const float ci = z.hi, si = sz.hi;
      float cmf = 1.f, smf = 0.f;
      int prev = -1;
      for (int j = 0; j < M; ++j) {
        const int4 md = TB.mode[j];  // (mode index, m, l, ypar)
        float h1t = 0.f, h1b = 0.f, h2t = 0.f, h2b = 0.f;
        float k1t = 0.f, k1b = 0.f, k2t = 0.f, k2b = 0.f;
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          if (EXACT || r < R) {
            // heads (t_h, t_h, b_h, b_h) and tails of the pair (r, r + 1)
            const float4 hd = Ac2[2 * ((r / 2) * M + j)], tl = Ac2[2 * ((r / 2) * M + j) + 1];
            const bool odd = r & 1;
            const float ath = odd ? hd.y + tl.y : hd.x + tl.x;
            const float abh = odd ? hd.w + tl.w : hd.z + tl.z;
            const float g1r = odd ? G1[r / 2].y : G1[r / 2].x;
            const float g2r = odd ? G2[r / 2].y : G2[r / 2].x;
            h1t = fmaf(g1r, ath, h1t);
            h1b = fmaf(g1r, abh, h1b);
            h2t = fmaf(g2r, ath, h2t);
            h2b = fmaf(g2r, abh, h2b);
            if (TWO) {
              const float g1Br = odd ? G1B[r / 2].y : G1B[r / 2].x;
              const float g2Br = odd ? G2B[r / 2].y : G2B[r / 2].x;
              k1t = fmaf(g1Br, ath, k1t);
              k1b = fmaf(g1Br, abh, k1b);
              k2t = fmaf(g2Br, ath, k2t);
              k2b = fmaf(g2Br, abh, k2b);
            }
          }
        }
        const float Hre = h1t + h2b, Him = h1b - h2t;
        const float HreB = k1t + k2b, HimB = k1b - k2t;
        const int m = md.y, am = m < 0 ? -m : m;
        if (am != prev) {
          sincosf((float)am * phi, &smf, &cmf);
          prev = am;
        }
        const float sgn = m < 0 ? -1.f : 1.f;
        float amp, damp;
        sylm_amp_grad_f(TB, j, md.z, md.w, ci, si, amp, damp);
        const float yre = amp * cmf, yim = sgn * amp * smf;
        g_phase = fmaf((float)m, fmaf(-yim, Hre, yre * Him), g_phase);
        g_incl = fmaf(damp * cmf, Hre, fmaf(sgn * damp * smf, Him, g_incl));
        if (TWO) {
          gB_phase = fmaf((float)m, fmaf(-yim, HreB, yre * HimB), gB_phase);
          gB_incl = fmaf(damp * cmf, HreB, fmaf(sgn * damp * smf, HimB, gB_incl));
        }
      }
    }
  }
  if (kW2Draw) {  // 1/2 |w|^2 into K and |w|^2 into R, summed over every detector
    const df w2t = two_sum(w2s.x, w2s.y);
    const df w2d = fast_two_sum(w2t.hi, __fadd_rn(w2t.lo, __fadd_rn(w2c.x, w2c.y)));
    dacc_add(T, df{0.5f * w2d.hi, 0.5f * w2d.lo});
    dacc_add(Racc, w2d);
  }
  MixedDraw o;
  o.lnl = dacc_result(T);
  o.R = dacc_result(Racc);
  if (bad) o.lnl = df{CUDART_NAN_F, 0.f};
  o.oob = oob;
  if (GRAD) {
    const df a = dacc_result(gt_ra), b = dacc_result(gt_dec), t = dacc_result(gt_t);
    o.grad[0] = (double)a.hi + (double)a.lo + (double)g_ra;
    o.grad[1] = (double)b.hi + (double)b.lo + (double)g_dec;
    o.grad[2] = g_psi;
    o.grad[3] = g_incl;
    o.grad[4] = g_phase;
    o.grad[5] = g_lnd;
    o.grad[6] = (double)t.hi + (double)t.lo;
    if (bad)
      for (int p = 0; p < kNpar; ++p) o.grad[p] = CUDART_NAN;
    if (TWO) {
      o.gradB[0] = gB_ra;
      o.gradB[1] = gB_dec;
      o.gradB[2] = gB_psi;
      o.gradB[3] = gB_incl;
      o.gradB[4] = gB_phase;
      o.gradB[5] = 0.0;
      o.gradB[6] = 0.0;
    }
  }
  return o;
}

// Stages the whitening matrices of all classes into shared memory in split
// form, by direction pairs (r, r + 1) with r even (R is even: the tables are
// padded to the kernel's width): entry (pair, j < M) is two float4,
// (t_h[r], t_h[r+1], b_h[r], b_h[r+1]) and (t_t[r], t_t[r+1], b_t[r], b_t[r+1]),
// with (t_h, t_t) the (head, tail) of A[r][a] and (b_h, b_t) of A[r][M + a],
// for mode a = morder[j] (modes in the kernels' order of increasing |m|; the
// direction pairs feed the packed FMAs of the mat-vec), head = A_hi rounded
// to a multiple of 2^-9 of a power of two >= max_a |A[r][a]| (10 significant
// bits; the error-free product of lnl_mixed_draw relies on it), tail =
// (A_hi - head) + A_lo rounded to FP32; then gm1.  Whole block.
__device__ __forceinline__ void stage_split_A(const PointParams& P, float4* smem4) {
  const int R = P.R, D = P.D, M = P.M, ncls = P.ncls;
  float* sAf = reinterpret_cast<float*>(smem4);
  float* sg = reinterpret_cast<float*>(smem4 + split_a_f4(ncls, R, M));
  for (int t = threadIdx.x; t < ncls * R; t += blockDim.x) {
    const float2* row = P.A + (size_t)t * D;
    float mx = 0.f;
    for (int a = 0; a < D; ++a) mx = fmaxf(mx, fabsf(__ldg(row + a).x));
    int e = 0;
    frexpf(mx, &e);  // mx < 2^e
    const float C = ldexpf(1.5f, e + 14);  // ulp(C) = 2^(e - 9)
    // row t = c R + r: pair t / 2, lane t % 2 within it
    float* dst = sAf + (size_t)(t >> 1) * M * 8 + (t & 1);
    for (int j = 0; j < M; ++j) {
      const int a = P.morder[j];
      const float2 v = __ldg(row + a), u = __ldg(row + M + a);
      const float hv = __fsub_rn(__fadd_rn(v.x, C), C);
      const float hu = __fsub_rn(__fadd_rn(u.x, C), C);
      const float tv = __fadd_rn(__fsub_rn(v.x, hv), v.y), tu = __fadd_rn(__fsub_rn(u.x, hu), u.y);
      float* e8 = dst + (size_t)j * 8;
      e8[0] = hv;
      e8[2] = hu;
      e8[4] = tv;
      e8[6] = tu;
    }
    sg[t] = __ldg(P.gm1 + t);
  }
}

template <int MM, int RR, bool LSE, bool GRAD = false, bool DIST = false>
__global__ void __launch_bounds__(128, GRAD ? RIFT_MIXED_MIN_BLOCKS_GRAD : RIFT_MIXED_MIN_BLOCKS)
    lnl_mixed_kernel(const __grid_constant__ PointParams P, DrawsParams dp,
                     double* __restrict__ lnl_out, LseState* __restrict__ partials,
                     unsigned long long* __restrict__ oob_count,
                     double* __restrict__ grad_out = nullptr, DistParams dist = DistParams{}) {
  // The point's parameters are a kernel parameter (constant bank, read with
  // warp-uniform addresses; 7.4 KB, within the 32 KB parameter limit), so
  // they need neither shared memory nor staging.
  extern __shared__ float4 smem4[];
  __shared__ MixedTables T;
  stage_split_A(P, smem4);
  stage_tables(P, T);
  __syncthreads();
  const float4* sA = smem4;
  const float* sg = reinterpret_cast<const float*>(smem4 + split_a_f4(P.ncls, P.R, P.M));
  float4* a12s = a12_slice<RR>(smem4, P.ncls, P.R, P.M);
  float4* xfs = xf_slice<RR>(smem4, P.ncls, P.R, P.M);
  ThreadLse st = tlse_init();
  int oob = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  // the LSE update of a draw is applied during the next draw (its loads in
  // flight), so that its dependent chain does not stall the warp at the end
  // of every iteration
  bool pend = false;
  df pend_l = df{0.f, 0.f};
  float pend_w = 0.f;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    float lw = 0.f;
    if (LSE && dp.logw)
      lw = dp.f64 ? (float)__ldcs((const double*)dp.logw + i) : __ldcs((const float*)dp.logw + i);
    if (LSE && pend) tlse_push_lw(st, pend_l, pend_w);
    MixedDraw o;
    if (DIST && GRAD) {
      // distance-marginal gradient in one pass at x = 1: with lnL(x) = K x -
      // R x^2/2, the pass gives gA = dK - dR/2 (the adjoint at x = 1) and
      // gB = dR/2, and E[x] dK - E[x^2] dR/2 = E[x] gA + E[x(1 - x)] gB
      // (the lnD slot is 0)
      o = lnl_mixed_draw<MM, RR, true, true, true>(P, T, sA, sg, a12s, xfs, dp, i);
      float ex[3] = {1.f, 1.f, 0.f};
      const df marg = isnan(o.lnl.hi) ? o.lnl : dist_marg_df(dist, o.lnl, o.R, ex);
      for (int p = 0; p < kNpar; ++p) o.grad[p] = ex[0] * o.grad[p] + ex[2] * o.gradB[p];
      o.grad[5] = 0.0;
      o.lnl = marg;
    } else {
      o = lnl_mixed_draw<MM, RR, GRAD, DIST, true>(P, T, sA, sg, a12s, xfs, dp, i);
      if (DIST) o.lnl = isnan(o.lnl.hi) ? o.lnl : dist_marg_df(dist, o.lnl, o.R);
    }
    oob += o.oob;
    if (GRAD) {
      if (lnl_out) lnl_out[i] = (double)o.lnl.hi + (double)o.lnl.lo;
#pragma unroll
      for (int p = 0; p < kNpar; ++p) grad_out[(size_t)p * dp.n + i] = o.grad[p];
    } else if (!LSE) {
      lnl_out[i] = (double)o.lnl.hi + (double)o.lnl.lo;
    } else {
      pend = true;
      pend_l = o.lnl;
      pend_w = lw;
    }
  }
  if (LSE && pend) tlse_push_lw(st, pend_l, pend_w);
  if (LSE) block_lse_write(st, partials + blockIdx.x);
  if (oob_count) {
    for (int off = 16; off > 0; off >>= 1) oob += __shfl_down_sync(0xffffffffu, oob, off);
    if ((threadIdx.x & 31) == 0 && oob) atomicAdd(oob_count, (unsigned long long)oob);
  }
}

// Bytes of the per-point image (the split whitening, gm1 and the staged
// tables) that the warp-per-draw kernel copies flat.
__host__ __device__ inline size_t image_bytes(int ncls, int R, int M) {
  return split_a_bytes(ncls, R, M) + ((sizeof(MixedTables) + 15) & ~(size_t)15);
}

// Builds the image once per point: the block stages the tables into shared
// memory exactly as the kernels do, then writes that memory out.
__global__ void __launch_bounds__(128) image_kernel(const __grid_constant__ PointParams P,
                                                    float4* __restrict__ img, int nf4) {
  extern __shared__ float4 smem4[];
  for (int t = threadIdx.x; t < nf4; t += blockDim.x) smem4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  stage_split_A(P, smem4);
  MixedTables& T = *reinterpret_cast<MixedTables*>(reinterpret_cast<char*>(smem4) +
                                                    split_a_bytes(P.ncls, P.R, P.M));
  stage_tables(P, T);
  __syncthreads();
  for (int t = threadIdx.x; t < nf4; t += blockDim.x) img[t] = smem4[t];
}

// Resident blocks per SM of `kern` at `smem` bytes of dynamic shared memory on
// the current device, with the kernel's shared-memory attribute set on first
// use: both are cached per (kernel, device, block size, shared memory), keyed
// by the kernel's address (every instantiation of a kernel template has the
// same function type), so a launch costs no attribute or occupancy call once
// a point's shape has been seen.
template <typename KernelT>
int cached_blocks_per_sm(KernelT kern, int threads, size_t smem) {
  struct Entry {
    const void* fn;
    int dev, threads, nb;
    size_t smem;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  static std::vector<std::pair<const void*, int>> attr_set;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
  const void* fn = reinterpret_cast<const void*>(kern);
  std::lock_guard<std::mutex> lock(mu);
  for (const Entry& e : cache)
    if (e.fn == fn && e.dev == dev && e.threads == threads && e.smem == smem) return e.nb;
  bool have_attr = false;
  for (const auto& a : attr_set) have_attr |= (a.first == fn && a.second == dev);
  if (!have_attr) {
    cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    attr_set.emplace_back(fn, dev);
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem) != cudaSuccess || nb < 1)
    nb = 1;
  nb = nb < kMaxPartialsPerSM ? nb : kMaxPartialsPerSM;
  cache.push_back(Entry{fn, dev, threads, nb, smem});
  return nb;
}

#include "lnl_warp.cuh"

template <int MM, int RR, bool GRAD>
cudaError_t launch_warp_k(const PointParams& hp, const DrawsParams& dp, double* lnl_out,
                          double* grad_out, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = warp_smem_bytes<MM, RR>(hp.ncls, hp.R, hp.M);
  auto kern = lnl_warp_kernel<MM, RR, GRAD>;
  const long long need = (dp.n + kWarpDrawsPerBlock - 1) / kWarpDrawsPerBlock;
  const long long cap = (long long)device_sms() * cached_blocks_per_sm(kern, 32 * kWarpDrawWarps, smem);
  const int blocks = (int)(need < cap ? need : cap);
  // with programmatic stream serialisation: the kernel's prologue (the
  // point's image into shared memory) overlaps the previous kernel, which
  // matters in a chain of sampler calls; the kernel waits for that kernel
  // (griddepcontrol.wait) before it reads the draws or writes anything
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(32 * kWarpDrawWarps);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, hp, dp, lnl_out, grad_out);
}

// Serves lnL (GRAD false) or lnL and its gradient with one warp per draw when
// the batch is small (at most small_batch_max() draws) and the point's
// scratch fits; returns false to leave the call to the per-thread kernels.
template <int MM, bool GRAD>
bool try_warp(const PointParams& hp, const DrawsParams& dp, double* lnl_out, double* grad_out,
              cudaStream_t st, cudaError_t* e) {
  if (dp.n > small_batch_max() || hp.K > kMaxDet || (hp.R != MM && hp.R != 2 * MM) || !hp.img)
    return false;
  const bool wide = hp.R > MM;
  const size_t smem = wide ? warp_smem_bytes<MM, 2 * MM>(hp.ncls, hp.R, hp.M)
                           : warp_smem_bytes<MM, MM>(hp.ncls, hp.R, hp.M);
  if (smem > 200 * 1024) return false;
  *e = wide ? launch_warp_k<MM, 2 * MM, GRAD>(hp, dp, lnl_out, grad_out, st)
            : launch_warp_k<MM, MM, GRAD>(hp, dp, lnl_out, grad_out, st);
  return true;
}

template <int MM, int RR, bool LSE>
cudaError_t launch_mixed_k(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                           double* lnl_out, LseState* partials, unsigned long long* oob,
                           int* blocks, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = mixed_smem_bytes<RR>(hp.ncls, hp.R, hp.M, hp.K);
  *blocks = grid_cap(device_sms() * cached_blocks_per_sm(lnl_mixed_kernel<MM, RR, LSE>, 128, smem),
                     dp.n, 128);
  lnl_mixed_kernel<MM, RR, LSE><<<*blocks, 128, smem, st>>>(hp, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

template <int MM, int RR, bool LSE>
cudaError_t launch_mixed_dist_k(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                const DistParams& dist, double* lnl_out, LseState* partials,
                                unsigned long long* oob, int* blocks, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = mixed_smem_bytes<RR>(hp.ncls, hp.R, hp.M, hp.K);
  auto kern = lnl_mixed_kernel<MM, RR, LSE, false, true>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  *blocks = grid_cap(grid_for(kern, 128, smem), dp.n, 128);
  kern<<<*blocks, 128, smem, st>>>(hp, dp, lnl_out, partials, oob, nullptr, dist);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_mixed_dist_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                 const DistParams& dist, double* lnl_out, LseState* partials,
                                 unsigned long long* oob, int* blocks, cudaStream_t st) {
  const bool wide = hp.R > MM;
  if (partials)
    return wide ? launch_mixed_dist_k<MM, 2 * MM, true>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st)
                : launch_mixed_dist_k<MM, MM, true>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  return wide ? launch_mixed_dist_k<MM, 2 * MM, false>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st)
              : launch_mixed_dist_k<MM, MM, false>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
}

template <int MM, int RR>
cudaError_t launch_mixed_mr(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                            double* lnl_out, LseState* partials, unsigned long long* oob,
                            int* blocks, cudaStream_t st) {
  if (partials) return launch_mixed_k<MM, RR, true>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_mixed_k<MM, RR, false>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

template <int MM>
cudaError_t launch_mixed_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                            double* lnl_out, LseState* partials, unsigned long long* oob,
                            int* blocks, cudaStream_t st) {
  cudaError_t e;
  if (!partials && !oob && try_warp<MM, false>(hp, dp, lnl_out, nullptr, st, &e)) {
    *blocks = 0;
    return e;
  }
  if (hp.R <= MM) return launch_mixed_mr<MM, MM>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_mixed_mr<MM, 2 * MM>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

template <int MM, int RR>
cudaError_t launch_mixed_grad_mr(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                 double* lnl_out, double* grad_out, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = mixed_smem_bytes<RR>(hp.ncls, hp.R, hp.M, hp.K);
  const int blocks = grid_cap(
      device_sms() * cached_blocks_per_sm(lnl_mixed_kernel<MM, RR, false, true>, 128, smem), dp.n, 128);
  lnl_mixed_kernel<MM, RR, false, true><<<blocks, 128, smem, st>>>(hp, dp, lnl_out, nullptr, nullptr,
                                                                   grad_out);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_mixed_grad_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                 double* lnl_out, double* grad_out, cudaStream_t st) {
  cudaError_t e;
  if (try_warp<MM, true>(hp, dp, lnl_out, grad_out, st, &e)) return e;
  if (hp.R <= MM) return launch_mixed_grad_mr<MM, MM>(hp, dP, dp, lnl_out, grad_out, st);
  return launch_mixed_grad_mr<MM, 2 * MM>(hp, dP, dp, lnl_out, grad_out, st);
}

template <int MM, int RR>
cudaError_t launch_mixed_grad_dist_mr(const PointParams& hp, const PointParams* dP,
                                      const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                      double* grad_out, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = mixed_smem_bytes<RR>(hp.ncls, hp.R, hp.M, hp.K);
  auto kern = lnl_mixed_kernel<MM, RR, false, true, true>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  const int blocks = grid_cap(grid_for(kern, 128, smem), dp.n, 128);
  kern<<<blocks, 128, smem, st>>>(hp, dp, lnl_out, nullptr, nullptr, grad_out, dist);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_mixed_grad_dist_mm(const PointParams& hp, const PointParams* dP,
                                      const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                      double* grad_out, cudaStream_t st) {
  if (hp.R <= MM) return launch_mixed_grad_dist_mr<MM, MM>(hp, dP, dp, dist, lnl_out, grad_out, st);
  return launch_mixed_grad_dist_mr<MM, 2 * MM>(hp, dP, dp, dist, lnl_out, grad_out, st);
}

template <int MM, int RR, bool LSE>
cudaError_t launch_mixed_k_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                               double* lnl_out, LseState* partials, unsigned long long* oob,
                               int sms, int* blocks, cudaStream_t st) {
  if (hp.R != RR) return cudaErrorInvalidValue;  // tables are padded to RR
  const size_t smem = mixed_smem_bytes<RR>(hp.ncls, hp.R, hp.M, hp.K);
  cudaFuncSetAttribute(lnl_mixed_kernel<MM, RR, LSE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       200 * 1024);
  *blocks = grid_cap(grid_for_sms(lnl_mixed_kernel<MM, RR, LSE>, 128, smem, sms), dp.n, 128);
  lnl_mixed_kernel<MM, RR, LSE><<<*blocks, 128, smem, st>>>(hp, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_mixed_mm_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                double* lnl_out, LseState* partials, unsigned long long* oob,
                                int sms, int* blocks, cudaStream_t st) {
  const bool wide = hp.R > MM;
  if (partials)
    return wide ? launch_mixed_k_sms<MM, 2 * MM, true>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st)
                : launch_mixed_k_sms<MM, MM, true>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  return wide ? launch_mixed_k_sms<MM, 2 * MM, false>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st)
              : launch_mixed_k_sms<MM, MM, false>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
}


// Persistent kernel of rift_ile_batch: resident blocks take (point, tile)
// items from the queue with an atomic ticket, restage the point's tables when
// the point changes, and leave one LSE state per item.  No block waits on
// another: a block stops when the ticket passes the end of the queue.
template <int MM, int RR>
__global__ void __launch_bounds__(128, RIFT_MIXED_MIN_BLOCKS)
    lnz_batch_kernel(const PointParams* const* __restrict__ pts, const DrawsParams* __restrict__ dps,
                     const BatchItem* __restrict__ items, int n_items, unsigned int* __restrict__ head,
                     LseState* __restrict__ partials, unsigned long long* __restrict__ oob_count) {
  __shared__ PointParams P;
  __shared__ MixedTables T;
  __shared__ DrawsParams sdp;
  __shared__ int s_item;
  extern __shared__ float4 smem4[];
  int cur = -1;
  int oob = 0;
  for (;;) {
    if (threadIdx.x == 0) s_item = (int)atomicAdd(head, 1u);
    __syncthreads();
    const int item = s_item;
    if (item >= n_items) break;
    const BatchItem it = items[item];
    if (it.point != cur) {
      stage_point(P, pts[it.point]);
      if (threadIdx.x == 0) sdp = dps[it.point];
      __syncthreads();
      stage_split_A(P, smem4);
      stage_tables(P, T);
      __syncthreads();
      cur = it.point;
    }
    const float4* sA = smem4;
    const float* sg = reinterpret_cast<const float*>(smem4 + split_a_f4(P.ncls, P.R, P.M));
    float4* a12s = a12_slice<RR>(smem4, P.ncls, P.R, P.M);
    float4* xfs = xf_slice<RR>(smem4, P.ncls, P.R, P.M);
    ThreadLse st = tlse_init();
    const long long end = it.begin + it.count;
    bool pend = false;  // deferred LSE update, as in lnl_mixed_kernel
    df pend_l = df{0.f, 0.f};
    float pend_w = 0.f;
    for (long long i = it.begin + threadIdx.x; i < end; i += blockDim.x) {
      float lw = 0.f;
      if (sdp.logw) lw = sdp.f64 ? (float)__ldcs((const double*)sdp.logw + i) : __ldcs((const float*)sdp.logw + i);
      if (pend) tlse_push_lw(st, pend_l, pend_w);
      MixedDraw o = lnl_mixed_draw<MM, RR, false, false, true>(P, T, sA, sg, a12s, xfs, sdp, i);
      oob += o.oob;
      pend = true;
      pend_l = o.lnl;
      pend_w = lw;
    }
    if (pend) tlse_push_lw(st, pend_l, pend_w);
    block_lse_write(st, partials + item);  // ends with every thread past its use of s_item
    __syncthreads();
  }
  if (oob_count) {
    for (int off = 16; off > 0; off >>= 1) oob += __shfl_down_sync(0xffffffffu, oob, off);
    if ((threadIdx.x & 31) == 0 && oob) atomicAdd(oob_count, (unsigned long long)oob);
  }
}

template <int MM>
BatchKernelFn pick_batch_kernel(int R) {
  // every point of a group has exactly the compiled width (tables padded)
  if (R == MM) return lnz_batch_kernel<MM, MM>;
  if (R == 2 * MM) return lnz_batch_kernel<MM, 2 * MM>;
  return nullptr;
}


}  // namespace

// ---- the per-mode-count entry points (explicitly instantiated by the
// lnl_mixed_m*.cu translation units, dispatched in lnl_mixed.cu)

template <int MM>
cudaError_t mixed_lnl(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                      double* lnl_out, LseState* partials, unsigned long long* oob, int* blocks,
                      cudaStream_t st) {
  return launch_mixed_mm<MM>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

template <int MM>
cudaError_t mixed_lnl_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                          double* lnl_out, LseState* partials, unsigned long long* oob, int sms,
                          int* blocks, cudaStream_t st) {
  return launch_mixed_mm_sms<MM>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
}

template <int MM>
cudaError_t mixed_dist(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                       const DistParams& dist, double* lnl_out, LseState* partials,
                       unsigned long long* oob, int* blocks, cudaStream_t st) {
  return launch_mixed_dist_mm<MM>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
}

template <int MM>
cudaError_t mixed_grad(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                       double* lnl_out, double* grad_out, cudaStream_t st) {
  return launch_mixed_grad_mm<MM>(hp, dP, dp, lnl_out, grad_out, st);
}

template <int MM>
cudaError_t mixed_grad_dist(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                            const DistParams& dist, double* lnl_out, double* grad_out,
                            cudaStream_t st) {
  return launch_mixed_grad_dist_mm<MM>(hp, dP, dp, dist, lnl_out, grad_out, st);
}

template <int MM>
BatchKernelFn mixed_batch_kernel(int R) {
  return pick_batch_kernel<MM>(R);
}

// Dynamic shared memory of the batch kernel mixed_batch_kernel<MM>(R) for a
// point with ncls classes of width Rp, Mp modes and Kp detectors.
template <int MM>
size_t mixed_batch_smem(int R, int ncls, int Rp, int Mp, int Kp) {
  return R == MM ? mixed_smem_bytes<MM>(ncls, Rp, Mp, Kp) : mixed_smem_bytes<2 * MM>(ncls, Rp, Mp, Kp);
}

template <int MM>
int mixed_upload_anchors(const float4* sincos_tab, const float2* exp_tab) {
  int rc = check_cuda(cudaMemcpyToSymbol(g_anchor, sincos_tab, sizeof(g_anchor)), "anchor table upload");
  if (!rc) rc = check_cuda(cudaMemcpyToSymbol(g_exp_anchor, exp_tab, sizeof(g_exp_anchor)), "exp table upload");
  return rc;
}

template <int MM>
int mixed_image(const PointParams& hp, float4** img, int* nf4, cudaStream_t st) {
  const size_t bytes = image_bytes(hp.ncls, hp.R, hp.M);
  *nf4 = (int)(bytes / 16);
  *img = nullptr;
  if (bytes > 200 * 1024) return RIFT_ILE_OK;  // no image: the warp kernel is not used then
  int rc = check_cuda(cudaMalloc((void**)img, bytes), "point image allocation");
  if (rc) return rc;
  cudaFuncSetAttribute(image_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  image_kernel<<<1, 128, bytes, st>>>(hp, *img, *nf4);
  return check_cuda(cudaGetLastError(), "point image kernel");
}

#define RIFT_INSTANTIATE_MIXED(MM)                                                              \
  template cudaError_t mixed_lnl<MM>(const PointParams&, const PointParams*, const DrawsParams&, \
                                     double*, LseState*, unsigned long long*, int*, cudaStream_t); \
  template cudaError_t mixed_lnl_sms<MM>(const PointParams&, const PointParams*,                 \
                                         const DrawsParams&, double*, LseState*,                 \
                                         unsigned long long*, int, int*, cudaStream_t);          \
  template cudaError_t mixed_dist<MM>(const PointParams&, const PointParams*, const DrawsParams&, \
                                      const DistParams&, double*, LseState*, unsigned long long*, \
                                      int*, cudaStream_t);                                        \
  template cudaError_t mixed_grad<MM>(const PointParams&, const PointParams*, const DrawsParams&, \
                                      double*, double*, cudaStream_t);                            \
  template cudaError_t mixed_grad_dist<MM>(const PointParams&, const PointParams*,                \
                                           const DrawsParams&, const DistParams&, double*,        \
                                           double*, cudaStream_t);                                \
  template BatchKernelFn mixed_batch_kernel<MM>(int);                                             \
  template size_t mixed_batch_smem<MM>(int, int, int, int, int);                                       \
  template int mixed_upload_anchors<MM>(const float4*, const float2*);                         \
  template int mixed_image<MM>(const PointParams&, float4**, int*, cudaStream_t);

}  // namespace rift
