// FP32-mixed likelihood of the composite-index response (Sec. III,
// eq. slowrot:lnL:Decomposed), included after lnl_mixed_impl.cuh by the
// mode-count translation units lnl_mixed_m4/m10/m16.cu (which share its anchor
// tables and double-float helpers); the host side is comp_mixed.cu.
//
// One thread per draw.  Per class of detectors the whitening built by
// rift_ile_comp_mixed_build gives, per detector,
//     lnL_k = 1/2 |e_k(t_k)|^2 - 1/2 |e_k(t_k) - w_k|^2,
//     w_k,r = sum_a (Re C~^k_a a1_a,r + Im C~^k_a a2_a,r),
//     a1_a,r + i a2_a,r = sum_i (t_a,r,i + i b_a,r,i) conj(Y_i),
// (t, b) the Re and Im columns of block a of whitening row r, the x factor
// folded into the coefficients.  The precision design is the static mixed
// path's: the coefficients C~, the harmonics, the arrival times and 1/2|e|^2
// are double-float; a1, a2 and w are formed by error-free split products
// (10-bit heads whose products and sums are exact in FP32, the remaining
// terms >= 2^8 smaller summed in FP32); only the residual e - w is FP32.
//
// Loop order: the coefficients x C~^k_a of every detector (as head/tail
// pairs on the grid of the detector's largest) and each detector's table
// position go to this thread's slots in shared memory; the harmonics stay in
// registers as mode pairs (j, j + 1), which are the lanes of the packed
// FFMA2 instructions of the a1/a2 sums.  Then, per class and pair of
// directions (r, r + 1): for each response index a the two rows of a1_a, a2_a,
// their split, and their products with the coefficients of up to
// kCompMixedKG detectors; then those detectors' residuals from the table
// interval's cubic coefficients.
#pragma once
#include "comp.cuh"

namespace rift {
namespace {

struct cdf {
  df re, im;
};

// a b with the real and imaginary parts in the two lanes of packed pairs
// (the operations of cmul_df, hence the same result, in half the issue slots).
__device__ __forceinline__ cdf cdf_mul(const cdf& a, const cdf& b) {
  const df2 p = df_mul2(df2_make(a.re, a.re), df2_make(b.re, b.im));
  const df2 q = df_mul2(df2_make(a.im, a.im), df2_make(b.im, b.re));
  const df2 r = df_add2(p, df2{make_float2(-q.hi.x, q.hi.y), make_float2(-q.lo.x, q.lo.y)});
  return cdf{df2_x(r), df2_y(r)};
}
__device__ __forceinline__ cdf cdf_conj(const cdf& a) { return cdf{a.re, df_neg(a.im)}; }
__device__ __forceinline__ cdf cdf_scale(const cdf& a, df s) {
  return cdf{df_mul(a.re, s), df_mul(a.im, s)};
}
__device__ __forceinline__ cdf cdf_add(const cdf& a, const cdf& b) {
  return cdf{df_add(a.re, b.re), df_add(a.im, b.im)};
}
__device__ __forceinline__ df df_of(float2 v) { return df{v.x, v.y}; }
__device__ __forceinline__ df df_half(df a) { return df{0.5f * a.hi, 0.5f * a.lo}; }

// The anchored sine/cosine as a real call: the kernel takes it at up to a
// dozen sites per draw, and one body keeps its code within the instruction
// cache.
__device__ __noinline__ void sincos_df_call(df a, df& s, df& c) { sincos_df(a, s, c); }

// Slot s of this thread (stride: the block size): c / sigma_a (a power of
// two, so the scaling is exact), and the running largest component.
__device__ __forceinline__ void slot_put(float4* base, int s, int bd, float isg, const cdf& c,
                                         float& mx) {
  const float4 v = make_float4(c.re.hi * isg, c.re.lo * isg, c.im.hi * isg, c.im.lo * isg);
  base[(size_t)s * bd] = v;
  mx = fmaxf(mx, fmaxf(fabsf(v.x), fabsf(v.z)));
}

// Sky quantities of one draw shared by its detectors (double-float).
struct CompSky {
  df sl, cl, sd, cd;  // of ra - gmst and dec
  df s[3];            // unit vector towards the source
  cdf xe2p;           // x e^{2 i psi}
};

// x C~^k_a of a detector under Earth rotation (eq. slowrot:Fharm,
// eq. slowrot:delay, eq. slowrot:master, eq. slowrot:postphase), composite
// order a = (p, n), into slots k na + a; returns the largest |component|.
// With al = (1 + sin dec)/2, be = (1 - sin dec)/2, the five sidereal harmonics
// of the antenna factor are A_-2 = al^2 (r1 + i r2), A_2 = be^2 (r1 - i r2),
// A_-1 = al cos(dec) (r3 - i r4), A_1 = -be cos(dec) (r3 + i r4),
// A_0 = 2 al be r5 - cos(dec)^2 r6 (r = Dyy - Dxx, 2 Dxy, 2 Dxz, 2 Dyz,
// Dxx + Dyy, Dzz), and C_(0,n) = e^{2 i psi} A_n e^{i n g}, g = gmst - ra.
__device__ __noinline__ float rot_coeffs(const CompMixed& C, int k, const CompSky& S,
                                         const cdf* G, df f0a, df f0b, df tk, float4* slot,
                                         int bd, float2* ep_out) {
  const float2* rc = C.rc[k];
  const df r1 = df_of(rc[0]), r2 = df_of(rc[1]), r3 = df_of(rc[2]), r4 = df_of(rc[3]);
  const df r5 = df_of(rc[4]), r6 = df_of(rc[5]);
  cdf C0[5];
  C0[0] = cdf_mul(G[0], cdf{r1, r2});
  C0[4] = cdf_mul(G[4], cdf{r1, df_neg(r2)});
  C0[1] = cdf_mul(G[1], cdf{r3, df_neg(r4)});
  {
    const cdf t = cdf_mul(G[3], cdf{r3, r4});
    C0[3] = cdf{df_neg(t.re), df_neg(t.im)};
  }
  C0[2] = cdf_scale(S.xe2p, df_sub(df_mul(f0a, r5), df_mul(f0b, r6)));
  // post-phase step e^{i Omega t_k}
  cdf ep;
  sincos_df_call(df_mul(df{C.omega_hi, C.omega_lo}, tk), ep.im, ep.re);
  const cdf epc = cdf_conj(ep);
  if (ep_out) *ep_out = make_float2(ep.re.hi, ep.im.hi);
  float mx = 0.f;
  if (C.p_max == 0) {  // Path A: C~_(0,n) = C_(0,n) e^{i n Omega t_k}, n = -2..2
    const cdf e2 = cdf_mul(ep, ep);
    const float* isg = C.inv_sigma;
    const int off = k * C.na;
    slot_put(slot, off, bd, isg[0], cdf_mul(C0[0], cdf_conj(e2)), mx);
    slot_put(slot, off + 1, bd, isg[1], cdf_mul(C0[1], epc), mx);
    slot_put(slot, off + 2, bd, isg[2], C0[2], mx);
    slot_put(slot, off + 3, bd, isg[3], cdf_mul(C0[3], ep), mx);
    slot_put(slot, off + 4, bd, isg[4], cdf_mul(C0[4], e2), mx);
    return mx;
  }
  // drift harmonics of -(t_k(t) - t_k(0)): with w = (x + i y) e^{i g},
  // E_-1 = cos(dec) conj(w)/2, E_0 = -cos(dec) Re w, E_1 = cos(dec) w/2
  cdf E[3];
  if (C.p_max > 0) {
    const cdf eg = cdf{S.cl, df_neg(S.sl)};
    const float4 ph = C.pos_hi[k], pl = C.pos_lo[k];
    const cdf w = cdf_mul(cdf{df{ph.x, pl.x}, df{ph.y, pl.y}}, eg);
    const df hc = df_half(S.cd);
    E[0] = cdf{df_mul(hc, w.re), df_neg(df_mul(hc, w.im))};
    E[1] = cdf{df_neg(df_mul(S.cd, w.re)), df{0.f, 0.f}};
    E[2] = cdf{df_mul(hc, w.re), df_mul(hc, w.im)};
  }
  cdf P[2 * RIFT_ILE_MAX_ROT_PMAX + 1];  // harmonics of (-dt)^p, index m + p
  P[0] = cdf{df{1.f, 0.f}, df{0.f, 0.f}};
  int off = k * C.na;
  for (int p = 0; p <= C.p_max; ++p) {
    if (p > 0) {
      cdf Pn[2 * RIFT_ILE_MAX_ROT_PMAX + 1];
      for (int j = 0; j < 2 * p + 1; ++j) {
        cdf acc = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
        for (int e = 0; e < 3; ++e) {
          const int src = j - e;
          if (src >= 0 && src < 2 * p - 1) acc = cdf_add(acc, cdf_mul(P[src], E[e]));
        }
        Pn[j] = acc;
      }
      for (int j = 0; j < 2 * p + 1; ++j) P[j] = Pn[j];
    }
    const df inv_fact = df{C.inv_fact[p], 0.f};
    // e^{i nn Omega t_k} from nn = -(2 + p)
    cdf ph = epc;
    for (int q = 1; q < 2 + p; ++q) ph = cdf_mul(ph, epc);
    const int width = 2 * (2 + p) + 1;
    for (int j = 0; j < width; ++j) {
      const int nn = j - (2 + p);
      cdf acc = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
      for (int n = -2; n <= 2; ++n) {
        const int m = nn - n;
        if (m >= -p && m <= p) acc = cdf_add(acc, p ? cdf_mul(C0[n + 2], P[m + p]) : C0[n + 2]);
      }
      if (p) acc = cdf_scale(acc, inv_fact);
      slot_put(slot, off + j, bd, C.inv_sigma[off + j - k * C.na], cdf_mul(acc, ph), mx);
      ph = cdf_mul(ph, ep);
    }
    off += width;
  }
  return mx;
}

// x b^k_p = x/2 [(X.s)^p (m.X)^2 - (Y.s)^p (m.Y)^2] (eq. fsize:bp), p = 0..p_max,
// with (m.X)^2 = e^{2 i psi} (e1.X - i e2.X)^2, into slots k na + p.
__device__ __noinline__ float arm_coeffs(const CompMixed& C, int k, const CompSky& S,
                                         float4* slot, int bd) {
  const float2* rc = C.rc[k];
  cdf q[2];
  df u[2];
  for (int v = 0; v < 2; ++v) {
    const df X0 = df_of(rc[3 * v]), X1 = df_of(rc[3 * v + 1]), X2 = df_of(rc[3 * v + 2]);
    const df ax = df_sub(df_mul(S.cl, X1), df_mul(S.sl, X0));  // e1 . X
    const df hx = df_add(df_mul(S.cl, X0), df_mul(S.sl, X1));
    const df bx = df_sub(df_mul(S.cd, X2), df_mul(S.sd, hx));  // e2 . X
    u[v] = df_add(df_mul(S.cd, hx), df_mul(S.sd, X2));          // s . X
    const df ab = df_mul(ax, bx);
    const cdf sq = cdf{df_sub(df_mul(ax, ax), df_mul(bx, bx)), df{-2.f * ab.hi, -2.f * ab.lo}};
    q[v] = cdf_mul(S.xe2p, sq);
  }
  df px = df{0.5f, 0.f}, py = df{0.5f, 0.f};
  float mx = 0.f;
  for (int p = 0; p <= C.p_max; ++p) {
    const cdf t = cdf{df_sub(df_mul(px, q[0].re), df_mul(py, q[1].re)),
                      df_sub(df_mul(px, q[0].im), df_mul(py, q[1].im))};
    slot_put(slot, k * C.na + p, bd, C.inv_sigma[p], t, mx);
    px = df_mul(px, u[0]);
    py = df_mul(py, u[1]);
  }
  return mx;
}

// ---- the adjoint's coefficient terms (FP32: they multiply the residual)

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float dotf2(float2 a, float2 b) { return fmaf(a.x, b.x, a.y * b.y); }

struct CompSkyF {
  float sl, cl, sd, cd;  // of ra - gmst and dec
  float2 xe2p;           // x e^{2 i psi}
};

// Adds sum_a (d C~_a / d theta) . rho_a / sigma_a of detector k for theta = ra,
// dec, t_c (rho_a = (r . a1_a, r . a2_a) with the scaled a-values, slot k na + a;
// ep = e^{i Omega t_k}, dtk_* = d t_k / d ra, d dec).
// Rotation: C_(0,n) = x e^{2 i psi} A_n(dec) e^{i n g} with d/d ra = -i n C_(0,n)
// (g = gmst - ra) and d/d dec through A_n; the drift harmonics move with
// w = (x + i y) e^{i g} and cos(dec); d P^(p) = d P^(p-1) * E + P^(p-1) * d E;
// the post-phase adds i nn Omega (d t_k / d theta) C~ and is the t_c term.
// Finite arms: b_p through the arm projections of e1, e2 and s.
__device__ __noinline__ void comp_coeff_grad_contract(const CompMixed& C, int k, const CompSkyF& S,
                                                      float2 ep, float dtk_ra, float dtk_dec,
                                                      const float2* rho, int bd, float& g_ra,
                                                      float& g_dec, float& g_tc) {
  const int na = C.na;
  const float2* rc = C.rc[k];
  const float sl = S.sl, cl = S.cl, sd = S.sd, cd = S.cd;
  if (C.kind == RIFT_ILE_RESP_FINITE_ARM) {
    // e1 = (-sl, cl, 0), e2 = (-sd cl, -sd sl, cd), s = (cd cl, cd sl, sd) and
    // their ra, dec derivatives
    float q2[2][2], dq[2][2][2], u[2], du[2][2];  // per arm: q (complex), dq/d(ra, dec), u, du
    for (int v = 0; v < 2; ++v) {
      const float X0 = rc[3 * v].x, X1 = rc[3 * v + 1].x, X2 = rc[3 * v + 2].x;
      const float a = -sl * X0 + cl * X1, b = -sd * (cl * X0 + sl * X1) + cd * X2;
      u[v] = cd * (cl * X0 + sl * X1) + sd * X2;
      const float da[2] = {-cl * X0 - sl * X1, 0.f};
      const float db[2] = {sd * (sl * X0 - cl * X1), -cd * (cl * X0 + sl * X1) - sd * X2};
      du[v][0] = cd * (-sl * X0 + cl * X1);
      du[v][1] = -sd * (cl * X0 + sl * X1) + cd * X2;
      const float2 q = cmulf(S.xe2p, make_float2(a * a - b * b, -2.f * a * b));
      q2[v][0] = q.x;
      q2[v][1] = q.y;
      for (int j = 0; j < 2; ++j) {
        const float2 d = cmulf(S.xe2p, cmulf(make_float2(2.f * a, -2.f * b), make_float2(da[j], -db[j])));
        dq[v][j][0] = d.x;
        dq[v][j][1] = d.y;
      }
    }
    float px = 0.5f, py = 0.5f, pxm = 0.f, pym = 0.f;  // u^p / 2 and p u^(p-1) / 2
    for (int p = 0; p < na; ++p) {
      const float2 r = rho[(size_t)(k * na + p) * bd];
      const float isg = C.inv_sigma[p];
      float g[2];
      for (int j = 0; j < 2; ++j) {
        const float cx = pxm * du[0][j], cy = pym * du[1][j];
        const float dre = cx * q2[0][0] + px * dq[0][j][0] - cy * q2[1][0] - py * dq[1][j][0];
        const float dim = cx * q2[0][1] + px * dq[0][j][1] - cy * q2[1][1] - py * dq[1][j][1];
        g[j] = isg * fmaf(dre, r.x, dim * r.y);
      }
      g_ra += g[0];
      g_dec += g[1];
      pxm = (float)(p + 1) * px;
      pym = (float)(p + 1) * py;
      px *= u[0];
      py *= u[1];
    }
    return;
  }
  const float r1 = rc[0].x, r2 = rc[1].x, r3 = rc[2].x, r4 = rc[3].x, r5 = rc[4].x, r6 = rc[5].x;
  const float al = 0.5f * (1.f + sd), be = 0.5f * (1.f - sd), dal = 0.5f * cd, dbe = -0.5f * cd;
  const float dcd = -sd;
  float2 A[5], dA[5];
  A[0] = make_float2(al * al * r1, al * al * r2);
  dA[0] = make_float2(2.f * al * dal * r1, 2.f * al * dal * r2);
  A[4] = make_float2(be * be * r1, -be * be * r2);
  dA[4] = make_float2(2.f * be * dbe * r1, -2.f * be * dbe * r2);
  A[1] = make_float2(al * cd * r3, -al * cd * r4);
  {
    const float f = dal * cd + al * dcd;
    dA[1] = make_float2(f * r3, -f * r4);
  }
  A[3] = make_float2(-be * cd * r3, -be * cd * r4);
  {
    const float f = dbe * cd + be * dcd;
    dA[3] = make_float2(-f * r3, -f * r4);
  }
  A[2] = make_float2(2.f * al * be * r5 - cd * cd * r6, 0.f);
  dA[2] = make_float2(2.f * (dal * be + al * dbe) * r5 - 2.f * cd * dcd * r6, 0.f);
  const float2 eg = make_float2(cl, -sl);
  float2 egn[5];
  egn[2] = make_float2(1.f, 0.f);
  egn[3] = eg;
  egn[4] = cmulf(eg, eg);
  egn[1] = conjf2(eg);
  egn[0] = conjf2(egn[4]);
  float2 C0[5], dC0[2][5];
  for (int j = 0; j < 5; ++j) {
    const float n = (float)(j - 2);
    C0[j] = cmulf(cmulf(S.xe2p, A[j]), egn[j]);
    dC0[0][j] = make_float2(n * C0[j].y, -n * C0[j].x);  // -i n C0
    dC0[1][j] = cmulf(cmulf(S.xe2p, dA[j]), egn[j]);
  }
  float2 E[3], dE[2][3];
  if (C.p_max > 0) {
    const float2 w = cmulf(make_float2(C.pos_hi[k].x, C.pos_hi[k].y), eg);
    E[0] = make_float2(0.5f * cd * w.x, -0.5f * cd * w.y);
    E[1] = make_float2(-cd * w.x, 0.f);
    E[2] = make_float2(0.5f * cd * w.x, 0.5f * cd * w.y);
    dE[0][0] = make_float2(-E[0].y, E[0].x);
    dE[0][1] = make_float2(-cd * w.y, 0.f);
    dE[0][2] = make_float2(E[2].y, -E[2].x);
    dE[1][0] = make_float2(0.5f * dcd * w.x, -0.5f * dcd * w.y);
    dE[1][1] = make_float2(-dcd * w.x, 0.f);
    dE[1][2] = make_float2(0.5f * dcd * w.x, 0.5f * dcd * w.y);
  }
  const float om = C.omega_hi;
  const float dtk[2] = {dtk_ra, dtk_dec};
  float2 P[2 * RIFT_ILE_MAX_ROT_PMAX + 1], dP[2][2 * RIFT_ILE_MAX_ROT_PMAX + 1];
  P[0] = make_float2(1.f, 0.f);
  dP[0][0] = dP[1][0] = make_float2(0.f, 0.f);
  int off = 0;
  for (int p = 0; p <= C.p_max; ++p) {
    if (p > 0) {
      float2 Pn[2 * RIFT_ILE_MAX_ROT_PMAX + 1], dPn[2][2 * RIFT_ILE_MAX_ROT_PMAX + 1];
      for (int j = 0; j < 2 * p + 1; ++j) {
        float2 acc = make_float2(0.f, 0.f), d0 = acc, d1 = acc;
        for (int e = 0; e < 3; ++e) {
          const int src = j - e;
          if (src >= 0 && src < 2 * p - 1) {
            const float2 t = cmulf(P[src], E[e]);
            acc.x += t.x;
            acc.y += t.y;
            const float2 a0 = cmulf(dP[0][src], E[e]), b0 = cmulf(P[src], dE[0][e]);
            const float2 a1 = cmulf(dP[1][src], E[e]), b1 = cmulf(P[src], dE[1][e]);
            d0.x += a0.x + b0.x;
            d0.y += a0.y + b0.y;
            d1.x += a1.x + b1.x;
            d1.y += a1.y + b1.y;
          }
        }
        Pn[j] = acc;
        dPn[0][j] = d0;
        dPn[1][j] = d1;
      }
      for (int j = 0; j < 2 * p + 1; ++j) {
        P[j] = Pn[j];
        dP[0][j] = dPn[0][j];
        dP[1][j] = dPn[1][j];
      }
    }
    const float inv_fact = C.inv_fact[p];
    float2 ph = make_float2(1.f, 0.f);
    for (int q = 0; q < 2 + p; ++q) ph = cmulf(ph, conjf2(ep));
    const int width = 2 * (2 + p) + 1;
    for (int j = 0; j < width; ++j) {
      const int nn = j - (2 + p);
      float2 acc = make_float2(0.f, 0.f), d0 = acc, d1 = acc;
      for (int n = -2; n <= 2; ++n) {
        const int m = nn - n;
        if (m >= -p && m <= p) {
          const float2 t = cmulf(C0[n + 2], P[m + p]);
          acc.x += t.x;
          acc.y += t.y;
          const float2 a0 = cmulf(dC0[0][n + 2], P[m + p]), b0 = cmulf(C0[n + 2], dP[0][m + p]);
          const float2 a1 = cmulf(dC0[1][n + 2], P[m + p]), b1 = cmulf(C0[n + 2], dP[1][m + p]);
          d0.x += a0.x + b0.x;
          d0.y += a0.y + b0.y;
          d1.x += a1.x + b1.x;
          d1.y += a1.y + b1.y;
        }
      }
      const float2 c = cmulf(make_float2(acc.x * inv_fact, acc.y * inv_fact), ph);
      const float2 ct = make_float2(-(float)nn * om * c.y, (float)nn * om * c.x);  // i nn Omega c
      const float2 dra = cmulf(make_float2(d0.x * inv_fact, d0.y * inv_fact), ph);
      const float2 ddec = cmulf(make_float2(d1.x * inv_fact, d1.y * inv_fact), ph);
      const int a = off + j;
      const float2 r = rho[(size_t)(k * na + a) * bd];
      const float isg = C.inv_sigma[a];
      g_ra += isg * dotf2(make_float2(fmaf(dtk[0], ct.x, dra.x), fmaf(dtk[0], ct.y, dra.y)), r);
      g_dec += isg * dotf2(make_float2(fmaf(dtk[1], ct.x, ddec.x), fmaf(dtk[1], ct.y, ddec.y)), r);
      g_tc += isg * dotf2(ct, r);
      ph = cmulf(ph, ep);
    }
    off += width;
  }
}

// This thread's adjoint slots (stride: the block size): rho_(k,a) = (r . a1,
// r . a2) summed over the directions, the current direction pair's a-values,
// and d lnL / d(Re Y, Im Y) of the mode pairs.
struct CompGradSlots {
  float2* rho;  // [K na]
  float4* af;   // [na] (a1 row 0, a1 row 1, a2 row 0, a2 row 1)
  float4* dy;   // [JP] (d Re Y lanes, d Im Y lanes)
};

// Table slots per detector: (position f in the interval, the interval, and
// for the adjoint the slope of 1/2 |e|^2 as a pair), then (adjoint)
// (d t_k / d ra, d t_k / d dec, r . de/du) and e^{i Omega t_k}.
template <bool GRAD>
constexpr int comp_tap_slots() { return GRAD ? 3 : 1; }

// The adjoint's last pass over a draw's detectors and modes: the arrival-time
// terms (d/dt 1/2 |e_k|^2 - r_k . de_k/dt) d t_k (double-float), the coefficient
// terms through rho (psi: d C~ = 2 i C~ d psi; lnD: d C~ = -C~ d lnD; sky and
// t_c by comp_coeff_grad_contract), and the harmonic terms from d lnL / d Y
// with Y_j = amp_j(iota) e^{i m phase} (FP32 amplitude and its iota slope).
template <int MM>
__device__ __noinline__ void comp_mixed_grad_tail(const CompMixed& C, const CompSkyF S,
                                                  const float4* tslot, const float4* cslot,
                                                  const CompGradSlots gs, float incl, float phi,
                                                  bool bad, double* gout) {
  constexpr int TS = comp_tap_slots<true>();
  const int bd = blockDim.x, K = C.K, na = C.na;
  dacc gt_ra = dacc_zero(), gt_dec = dacc_zero(), gt_t = dacc_zero();
  float g_ra = 0.f, g_dec = 0.f, g_tc = 0.f, g_psi = 0.f, g_lnd = 0.f;
  for (int k = 0; k < K; ++k) {
    const float4 t1 = tslot[(size_t)(TS * k) * bd], t3 = tslot[(size_t)(TS * k + 1) * bd];
    const float4 t4 = tslot[(size_t)(TS * k + 2) * bd];
    const df dtk = df_mul(df_add_f(df{t1.z, t1.w}, -t3.z), df{C.inv_dt_hi, C.inv_dt_lo});
    dacc_add(gt_t, dtk);
    dacc_add(gt_ra, df_mul_f(dtk, t3.x));
    dacc_add(gt_dec, df_mul_f(dtk, t3.y));
    comp_coeff_grad_contract(C, k, S, make_float2(t4.x, t4.y), t3.x, t3.y, gs.rho, bd, g_ra, g_dec,
                             g_tc);
    for (int a = 0; a < na; ++a) {
      const size_t e = (size_t)(k * na + a) * bd;
      const float4 cs = cslot[e];
      const float cre = cs.x + cs.z, cim = cs.y + cs.w;
      const float2 r = gs.rho[e];
      g_psi = fmaf(2.f, fmaf(cre, r.y, -cim * r.x), g_psi);
      g_lnd -= fmaf(cre, r.x, cim * r.y);
    }
  }
  float g_incl = 0.f, g_phase = 0.f, si, ci;
  sincosf(incl, &si, &ci);
  for (int j = 0; j < C.M; ++j) {
    const float4 y4 = gs.dy[(size_t)(j / 2) * bd];
    const float Hre = (j & 1) ? y4.y : y4.x, Him = (j & 1) ? y4.w : y4.z;
    const int4 md = C.mode[j];
    const int m = md.y, l = md.z;
    float pz = C.yz[j][l].x, dpz = 0.f;
    for (int q = l - 1; q >= 0; --q) {
      dpz = fmaf(dpz, ci, pz);
      pz = fmaf(pz, ci, C.yz[j][q].x);
    }
    float amp, damp;  // d/d iota through z = cos(iota): dz = -sin(iota) d iota
    if (md.w) {
      amp = si * pz;
      damp = fmaf(ci, pz, -si * si * dpz);
    } else {
      amp = pz;
      damp = -si * dpz;
    }
    float sm, cm;
    sincosf((float)m * phi, &sm, &cm);
    const float yre = amp * cm, yim = amp * sm;
    g_phase = fmaf((float)m, fmaf(-yim, Hre, yre * Him), g_phase);
    g_incl = fmaf(damp * cm, Hre, fmaf(damp * sm, Him, g_incl));
  }
  const df a = dacc_result(gt_ra), b = dacc_result(gt_dec), t = dacc_result(gt_t);
  gout[0] = (double)a.hi + (double)a.lo + (double)g_ra;
  gout[1] = (double)b.hi + (double)b.lo + (double)g_dec;
  gout[2] = g_psi;
  gout[3] = g_incl;
  gout[4] = g_phase;
  gout[5] = g_lnd;
  gout[6] = (double)t.hi + (double)t.lo + (double)g_tc;
  if (bad)
    for (int p = 0; p < kNpar; ++p) gout[p] = CUDART_NAN;
}

__device__ __forceinline__ CompSkyF comp_sky_f(const CompSky& S) {
  CompSkyF f;
  f.sl = S.sl.hi;
  f.cl = S.cl.hi;
  f.sd = S.sd.hi;
  f.cd = S.cd.hi;
  f.xe2p = make_float2(S.xe2p.re.hi, S.xe2p.im.hi);
  return f;
}

// One draw of the composite FP32-mixed likelihood.  B: split whitening (shared
// or global), AG: head constants of a1, a2; cslot/tslot: this thread's slots.
// With GRAD also d lnL / d (ra, dec, psi, incl, phase, lnD, t) into gout: the
// chain rule of the FP64 adjoint taken in the whitened coordinates,
//   d lnL = sum_k [(d/dt 1/2 |e_k|^2 - r_k . de_k/dt) d t_k + r_k . d w_k],
// with r_k = e_k - w_k; d w_k splits into the coefficient derivatives
// (contracted with rho) and the harmonic derivatives (through d lnL / d Y).
// Those terms multiply the residual and are FP32; the arrival-time slope of
// 1/2 |e|^2 is double-float.
template <int MM, bool GRAD>
__device__ __forceinline__ df comp_mixed_draw(const CompMixed& C, const float4* __restrict__ B,
                                              const float* __restrict__ AG, float4* cslot,
                                              float4* tslot, const CompGradSlots& gs,
                                              const DrawsParams& dp, long long i, int& oob,
                                              double* gout) {
  constexpr int JPM = MM / 2;
  constexpr int TS = comp_tap_slots<GRAD>();
  const int bd = blockDim.x;
  const float ra = load_param_f(dp, 0, i), dec = load_param_f(dp, 1, i);
  const float psi = load_param_f(dp, 2, i), incl = load_param_f(dp, 3, i);
  const float phi = load_param_f(dp, 4, i), lnD = load_param_f(dp, 5, i);
  const df tc = load_param_df(dp, 6, i);
  const int K = C.K, M = C.M, na = C.na, R = C.R, n = C.n;

  df lx = two_sum(C.ln_dref_hi, -lnD);
  lx.lo = __fadd_rn(lx.lo, C.ln_dref_lo);
  const df x = exp_df(fast_two_sum(lx.hi, lx.lo));

  CompSky S;
  {
    df lam = two_sum(ra, -C.gmst_hi);
    lam.lo = __fsub_rn(lam.lo, C.gmst_lo);
    lam = fast_two_sum(lam.hi, lam.lo);
    sincos_df_call(lam, S.sl, S.cl);
    sincos_df_call(df{dec, 0.f}, S.sd, S.cd);
    S.s[0] = df_mul(S.cd, S.cl);
    S.s[1] = df_mul(S.cd, S.sl);
    S.s[2] = S.sd;
    df s2p, c2p;
    sincos_df_call(df{2.f * psi, 0.f}, s2p, c2p);
    S.xe2p = cdf{df_mul(x, c2p), df_mul(x, s2p)};
  }

  // ---- shared rotation factors: G_n = x e^{2 i psi} e^{i n g} f_n (n != 0)
  cdf G[5];
  df f0a = df{0.f, 0.f}, f0b = df{0.f, 0.f};
  if (C.kind == RIFT_ILE_RESP_ROTATION) {
    const df al = df_half(df_add_f(S.sd, 1.f)), be = df_half(df_add_f(df_neg(S.sd), 1.f));
    const cdf eg = cdf{S.cl, df_neg(S.sl)};  // e^{i g}
    const cdf e2g = cdf_mul(eg, eg);
    G[3] = cdf_scale(cdf_mul(S.xe2p, eg), df_mul(be, S.cd));
    G[4] = cdf_scale(cdf_mul(S.xe2p, e2g), df_mul(be, be));
    G[1] = cdf_scale(cdf_mul(S.xe2p, cdf_conj(eg)), df_mul(al, S.cd));
    G[0] = cdf_scale(cdf_mul(S.xe2p, cdf_conj(e2g)), df_mul(al, al));
    const df ab = df_mul(al, be);
    f0a = df{2.f * ab.hi, 2.f * ab.lo};
    f0b = df_mul(S.cd, S.cd);
  }

  // ---- per detector: arrival time, table position, 1/2 |e|^2,
  // and the coefficients (df pairs first, then split on the detector's grid)
  dacc T = dacc_zero();
  bool bad = false;
  for (int k = 0; k < K; ++k) {
    const float4 ph = C.pos_hi[k], pl = C.pos_lo[k];
    const df delay = dot3_df(ph, pl, S.s[0], S.s[1], S.s[2]);
    const df tk = df_sub(tc, delay);
    float2 ep = make_float2(1.f, 0.f);
    const float mx = (C.kind == RIFT_ILE_RESP_ROTATION)
                         ? rot_coeffs(C, k, S, G, f0a, f0b, tk, cslot, bd, GRAD ? &ep : nullptr)
                         : arm_coeffs(C, k, S, cslot, bd);
    {
      // heads on the grid 2^(E-8) of the largest component (one step coarser
      // for more than 16 response indices, so that the 2 na head products of a
      // direction stay below 2^24 quanta)
      float Cx = head_constant(mx);
      if (na > 16) Cx *= 2.f;
      for (int a = 0; a < na; ++a) {
        float4* p = cslot + (size_t)(k * na + a) * bd;
        const float4 v = *p;
        const float rh = head_of(v.x, Cx), ih = head_of(v.z, Cx);
        *p = make_float4(rh, ih, __fadd_rn(__fsub_rn(v.x, rh), v.y),
                         __fadd_rn(__fsub_rn(v.z, ih), v.w));
      }
    }
    const df rel = df_add(tk, df{-ph.w, -pl.w});
    const df u = df_mul(rel, df{C.inv_dt_hi, C.inv_dt_lo});
    df dhalf = df{0.f, 0.f};
    float f = 0.f;
    int jc = -3;  // zero coefficients: a detector without a finite position adds nothing but NaN
    if (!isfinite(u.hi)) {
      bad = true;
      oob += 4;
    } else {
      float jf = floorf(u.hi);
      if (u.hi == jf && u.lo < 0.f) jf -= 1.f;
      f = __fadd_rn(__fsub_rn(u.hi, jf), u.lo);
      if (jf >= -2.f && jf <= (float)n) {
        const float2* pc = C.epoly + ((size_t)k * (n + 3) + (size_t)((int)jf + 2)) * (kPolyDeg + 1);
        float2 cf = __ldg(pc + kPolyDeg);
        df acc = df{cf.x, cf.y};
#pragma unroll
        for (int p = kPolyDeg - 1; p >= 0; --p) {
          if (GRAD) dhalf = horner_step_f(dhalf, f, acc.hi, acc.lo);  // the slope: d f + acc
          cf = __ldg(pc + p);
          acc = horner_step_f(acc, f, cf.x, cf.y);
        }
        dacc_add(T, acc);
      }
      const float nb = fminf(fmaxf(1.f - jf, 0.f), 4.f);
      const float nab = fminf(fmaxf(jf + 3.f - (float)n, 0.f), 4.f);
      oob += (int)fminf(nb + nab, 4.f);
      jc = (int)fminf(fmaxf(jf, -3.f), (float)(n + 1));
    }
    tslot[(size_t)(TS * k) * bd] = make_float4(f, __int_as_float(jc), dhalf.hi, dhalf.lo);
    if (GRAD) {
      // d t_k / d ra = -pos . ds/d ra, d t_k / d dec = -pos . ds/d dec
      const float sl = S.sl.hi, cl = S.cl.hi, sd = S.sd.hi, cd = S.cd.hi;
      const float dka = -(ph.x * (-cd * sl) + ph.y * (cd * cl));
      const float dkd = -(ph.x * (-sd * cl) + ph.y * (-sd * sl) + ph.z * cd);
      tslot[(size_t)(TS * k + 1) * bd] = make_float4(dka, dkd, 0.f, 0.f);
      tslot[(size_t)(TS * k + 2) * bd] = make_float4(ep.x, ep.y, 0.f, 0.f);
      for (int a = 0; a < na; ++a) gs.rho[(size_t)(k * na + a) * bd] = make_float2(0.f, 0.f);
    }
  }
  if (GRAD)
    for (int q = 0; q < JPM; ++q) gs.dy[(size_t)q * bd] = make_float4(0.f, 0.f, 0.f, 0.f);

  // ---- harmonics in visiting order j, split: (head on 2^-8, tail with the
  // low part); lanes (j even, j odd) of pair j / 2
  float2 Yr1[JPM], Yi1[JPM], Yr2[JPM], Yi2[JPM], Yrh[JPM], Yih[JPM];
#pragma unroll
  for (int q = 0; q < JPM; ++q)
    Yr1[q] = Yi1[q] = Yr2[q] = Yi2[q] = Yrh[q] = Yih[q] = make_float2(0.f, 0.f);
  {
    df sz, z;
    sincos_df_call(df{incl, 0.f}, sz, z);
    int prev_am = -1;
    df cm = df{1.f, 0.f}, sm = df{0.f, 0.f}, c1 = df{1.f, 0.f}, s1p = df{0.f, 0.f};
    bool have1 = false;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      if (j < M) {
        const int4 md = C.mode[j];
        const int m = md.y, am = m < 0 ? -m : m;
        if (am != prev_am) {
          if (have1 && am == prev_am + 1) {
            const df cn = df_sub(df_mul(cm, c1), df_mul(sm, s1p));
            sm = df_add(df_mul(sm, c1), df_mul(cm, s1p));
            cm = cn;
          } else {
            sincos_df_call(two_prod((float)am, phi), sm, cm);
            if (am == 1) {
              c1 = cm;
              s1p = sm;
              have1 = true;
            }
          }
          prev_am = am;
        }
        // the harmonic amplitude by Horner in cos(iota) (see sylm_amp_df)
        const int l = md.z;
        float2 c = C.yz[j][l];
        df acc = df{c.x, c.y};
        for (int q = l - 1; q >= 0; --q) {
          c = C.yz[j][q];
          acc = horner_step(acc, z, c.x, c.y);
        }
        const df amp = md.w ? df_mul(acc, sz) : fast_two_sum(acc.hi, acc.lo);
        const df yr = df_mul(amp, cm);
        const df yi = m < 0 ? df_neg(df_mul(amp, sm)) : df_mul(amp, sm);
        float yr1, yr2, yi1, yi2;
        split_y(yr.hi, yr1, yr2);
        split_y(yi.hi, yi1, yi2);
        yr2 = __fadd_rn(yr2, yr.lo);
        yi2 = __fadd_rn(yi2, yi.lo);
        if (j & 1) {
          Yr1[j / 2].y = yr1; Yi1[j / 2].y = yi1; Yr2[j / 2].y = yr2; Yi2[j / 2].y = yi2;
          Yrh[j / 2].y = yr.hi; Yih[j / 2].y = yi.hi;
        } else {
          Yr1[j / 2].x = yr1; Yi1[j / 2].x = yi1; Yr2[j / 2].x = yr2; Yi2[j / 2].x = yi2;
          Yrh[j / 2].x = yr.hi; Yih[j / 2].x = yi.hi;
        }
      }
    }
  }

  // ---- the r loop
  float2 q2p = make_float2(0.f, 0.f);
  const size_t bstride_a = (size_t)R * JPM * 3;  // float4 per response index
  for (int c = 0; c < C.ncls; ++c) {
    for (int g0 = C.cls_begin[c]; g0 < C.cls_begin[c + 1]; g0 += kCompMixedKG) {
      const int nk = min(kCompMixedKG, C.cls_begin[c + 1] - g0);
      int kd[kCompMixedKG];
#pragma unroll
      for (int kk = 0; kk < kCompMixedKG; ++kk) kd[kk] = C.det_order[kk < nk ? g0 + kk : g0];
      float red[kCompMixedKG];  // r . de/du of the group's detectors
#pragma unroll
      for (int kk = 0; kk < kCompMixedKG; ++kk) red[kk] = 0.f;
      for (int r0 = 0; r0 < R; r0 += 2) {
        float2 whp[kCompMixedKG][2], wcp[kCompMixedKG][2];
        float2 rsk[kCompMixedKG];
#pragma unroll
        for (int kk = 0; kk < kCompMixedKG; ++kk)
          whp[kk][0] = whp[kk][1] = wcp[kk][0] = wcp[kk][1] = make_float2(0.f, 0.f);
        const float4* Bc = B + (size_t)c * na * bstride_a + (size_t)r0 * JPM * 3;
        const float* AGc = AG + (size_t)c * R + r0;
        for (int a = 0; a < na; ++a) {
          const float4* Ba = Bc + (size_t)a * bstride_a;
          float2 e1[2], e2[2], c1[2], c2[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) e1[h] = e2[h] = c1[h] = c2[h] = make_float2(0.f, 0.f);
#pragma unroll
          for (int jp = 0; jp < JPM; ++jp) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              // (t_h, b_h), (-t_h, t_t), (b_t, -t_t) of modes (2 jp, 2 jp + 1), row r0 + h
              const float4 u0 = Ba[(h * JPM + jp) * 3], u1 = Ba[(h * JPM + jp) * 3 + 1];
              const float4 u2 = Ba[(h * JPM + jp) * 3 + 2];
              const float2 Th = make_float2(u0.x, u0.y), Bh = make_float2(u0.z, u0.w);
              const float2 nTh = make_float2(u1.x, u1.y), Tt = make_float2(u1.z, u1.w);
              const float2 Bt = make_float2(u2.x, u2.y), nTt = make_float2(u2.z, u2.w);
              // a1 += t yr + b yi ;  a2 += b yr - t yi (heads exact, the rest in c)
              e1[h] = __ffma2_rn(Th, Yr1[jp], e1[h]);
              e1[h] = __ffma2_rn(Bh, Yi1[jp], e1[h]);
              e2[h] = __ffma2_rn(Bh, Yr1[jp], e2[h]);
              e2[h] = __ffma2_rn(nTh, Yi1[jp], e2[h]);
              c1[h] = __ffma2_rn(Th, Yr2[jp], c1[h]);
              c1[h] = __ffma2_rn(Bh, Yi2[jp], c1[h]);
              c1[h] = __ffma2_rn(Tt, Yrh[jp], c1[h]);
              c1[h] = __ffma2_rn(Bt, Yih[jp], c1[h]);
              c2[h] = __ffma2_rn(Bh, Yr2[jp], c2[h]);
              c2[h] = __ffma2_rn(nTh, Yi2[jp], c2[h]);
              c2[h] = __ffma2_rn(Bt, Yrh[jp], c2[h]);
              c2[h] = __ffma2_rn(nTt, Yih[jp], c2[h]);
            }
          }
          // per row: (a1, a2) exact head sums (the two mode lanes added),
          // heads on the row's fixed grid (common to every a, so that the
          // head products below share one quantum), tails, and FP32 values
          float2 ah[2], at[2], af[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const float2 ex = __fadd2_rn(make_float2(e1[h].x, e2[h].x), make_float2(e1[h].y, e2[h].y));
            const float2 co = __fadd2_rn(make_float2(c1[h].x, c2[h].x), make_float2(c1[h].y, c2[h].y));
            const float g = AGc[h];
            const float2 G2 = make_float2(g, g);
            ah[h] = sub2(__fadd2_rn(ex, G2), G2);
            at[h] = __fadd2_rn(sub2(ex, ah[h]), co);
            af[h] = __fadd2_rn(ah[h], at[h]);
          }
          if (GRAD) gs.af[(size_t)a * bd] = make_float4(af[0].x, af[1].x, af[0].y, af[1].y);
          // w_k += Re C a1 + Im C a2 as lanes (Re, Im): heads exact, tails in FP32
#pragma unroll
          for (int kk = 0; kk < kCompMixedKG; ++kk) {
            if (kk < nk) {
              const float4 cs = cslot[(size_t)(kd[kk] * na + a) * bd];
              const float2 Ch = make_float2(cs.x, cs.y), Ct = make_float2(cs.z, cs.w);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                whp[kk][h] = __ffma2_rn(Ch, ah[h], whp[kk][h]);
                wcp[kk][h] = __ffma2_rn(Ch, at[h], wcp[kk][h]);
                wcp[kk][h] = __ffma2_rn(Ct, af[h], wcp[kk][h]);
              }
            }
          }
        }
        // residuals of rows r0, r0 + 1 from the interval's cubic,
        // r = (c0.hi + nhi) + (c0.lo + f (c1 + f (c2 + f c3))) + nlo with
        // -w = nhi + nlo (nhi the exact head sum), as in the static path
#pragma unroll
        for (int kk = 0; kk < kCompMixedKG; ++kk) {
          if (kk < nk) {
            const int k = kd[kk];
            const float4 t0 = tslot[(size_t)(TS * k) * bd];
            const int jc = __float_as_int(t0.y);
            const float2 f2 = make_float2(t0.x, t0.x);
            const float2 nhi = make_float2(-__fadd_rn(whp[kk][0].x, whp[kk][0].y),
                                           -__fadd_rn(whp[kk][1].x, whp[kk][1].y));
            const float2 nlo = make_float2(-__fadd_rn(wcp[kk][0].x, wcp[kk][0].y),
                                           -__fadd_rn(wcp[kk][1].x, wcp[kk][1].y));
            const float4* Cj =
                C.ecub + (((size_t)k * (n + 5) + (size_t)(jc + 3)) * (R / 2) + r0 / 2) * 3;
            const float4 c0 = __ldg(Cj), c12 = __ldg(Cj + 1), c3v = __ldg(Cj + 2);
            const float2 c1 = make_float2(c12.x, c12.y), c2 = make_float2(c12.z, c12.w);
            const float2 c3 = make_float2(c3v.x, c3v.y);
            float2 hp = __ffma2_rn(c3, f2, c2);
            hp = __ffma2_rn(hp, f2, c1);
            const float2 tl = __ffma2_rn(hp, f2, make_float2(c0.z, c0.w));
            const float2 d0 = __fadd2_rn(make_float2(c0.x, c0.y), nhi);
            const float2 rsv = __fadd2_rn(__fadd2_rn(d0, tl), nlo);
            float2 ed = make_float2(0.f, 0.f);  // de/df = c1 + f (2 c2 + 3 f c3)
            if (GRAD)
              ed = __ffma2_rn(__ffma2_rn(c3, make_float2(3.f * t0.x, 3.f * t0.x), __fadd2_rn(c2, c2)),
                              f2, c1);
            q2p = __ffma2_rn(rsv, rsv, q2p);
            if (GRAD) {
              rsk[kk] = rsv;
              red[kk] = fmaf(rsv.x, ed.x, fmaf(rsv.y, ed.y, red[kk]));
            }
          } else if (GRAD) {
            rsk[kk] = make_float2(0.f, 0.f);
          }
        }
        if (GRAD) {
          // per response index: rho_(k,a) += (r . a1_a, r . a2_a) and, with
          // G = sum_k C~'_k r_k, d lnL / d Y += G (t + i b) conj-linear terms:
          // d/d Re Y_i += G1 t_i + G2 b_i,  d/d Im Y_i += G1 b_i - G2 t_i
          for (int a = 0; a < na; ++a) {
            const float4 av = gs.af[(size_t)a * bd];
            float2 G1 = make_float2(0.f, 0.f), G2 = make_float2(0.f, 0.f);
#pragma unroll
            for (int kk = 0; kk < kCompMixedKG; ++kk) {
              if (kk < nk) {
                const size_t e = (size_t)(kd[kk] * na + a) * bd;
                const float4 cs = cslot[e];
                const float cre = cs.x + cs.z, cim = cs.y + cs.w;
                G1 = __ffma2_rn(make_float2(cre, cre), rsk[kk], G1);
                G2 = __ffma2_rn(make_float2(cim, cim), rsk[kk], G2);
                float2 rh = gs.rho[e];
                rh.x = fmaf(rsk[kk].x, av.x, fmaf(rsk[kk].y, av.y, rh.x));
                rh.y = fmaf(rsk[kk].x, av.z, fmaf(rsk[kk].y, av.w, rh.y));
                gs.rho[e] = rh;
              }
            }
            const float4* Ba = Bc + (size_t)a * bstride_a;
            for (int jp = 0; jp < JPM; ++jp) {
              const float4 y4 = gs.dy[(size_t)jp * bd];
              float2 dyr = make_float2(y4.x, y4.y), dyi = make_float2(y4.z, y4.w);
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const float4 u0 = Ba[(h * JPM + jp) * 3], u1 = Ba[(h * JPM + jp) * 3 + 1];
                const float4 u2 = Ba[(h * JPM + jp) * 3 + 2];
                const float2 tf = __fadd2_rn(make_float2(u0.x, u0.y), make_float2(u1.z, u1.w));
                const float2 bf = __fadd2_rn(make_float2(u0.z, u0.w), make_float2(u2.x, u2.y));
                const float g1 = h ? G1.y : G1.x, g2 = h ? G2.y : G2.x;
                dyr = __ffma2_rn(make_float2(g1, g1), tf, dyr);
                dyr = __ffma2_rn(make_float2(g2, g2), bf, dyr);
                dyi = __ffma2_rn(make_float2(g1, g1), bf, dyi);
                dyi = __ffma2_rn(make_float2(-g2, -g2), tf, dyi);
              }
              gs.dy[(size_t)jp * bd] = make_float4(dyr.x, dyr.y, dyi.x, dyi.y);
            }
          }
        }
      }
      if (GRAD) {
#pragma unroll
        for (int kk = 0; kk < kCompMixedKG; ++kk)
          if (kk < nk) tslot[(size_t)(TS * kd[kk] + 1) * bd].z = red[kk];
      }
    }
  }
  dacc_fma_ff(T, -0.5f, __fadd_rn(q2p.x, q2p.y));
  df out = dacc_result(T);
  if (bad) out = df{CUDART_NAN_F, 0.f};
  if (GRAD) comp_mixed_grad_tail<MM>(C, comp_sky_f(S), tslot, cslot, gs, incl, phi, bad, gout);
  return out;
}

// MINB: the resident blocks per SM the registers are sized for (2, or 3 where
// shared memory admits three blocks: up to ten modes that fits without spills).
template <int MM, bool BSMEM, bool LSE, int MINB>
__global__ void __launch_bounds__(kCompMixedThreads, MINB)
    comp_mixed_kernel(const __grid_constant__ CompMixed C, DrawsParams dp,
                      double* __restrict__ lnl_out, LseState* __restrict__ partials,
                      unsigned long long* __restrict__ oob_count) {
  extern __shared__ float4 smem4[];
  const size_t nb = BSMEM ? comp_mixed_b_f4(C) : 0, ng = comp_mixed_ag_f4(C);
  if constexpr (BSMEM)
    for (size_t q = threadIdx.x; q < nb; q += blockDim.x) smem4[q] = __ldg(C.Bs + q);
  float* sAG = reinterpret_cast<float*>(smem4 + nb);
  for (size_t q = threadIdx.x; q < (size_t)C.ncls * C.R; q += blockDim.x)
    sAG[q] = __ldg(C.agrid + q);
  __syncthreads();
  const float4* B = BSMEM ? smem4 : C.Bs;
  float4* cslot = smem4 + nb + ng + threadIdx.x;
  float4* tslot = cslot + (size_t)C.K * C.na * blockDim.x;
  ThreadLse st = tlse_init();
  int oob = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    float lw = 0.f;
    if (LSE && dp.logw)
      lw = dp.f64 ? (float)__ldcs((const double*)dp.logw + i) : __ldcs((const float*)dp.logw + i);
    const df l = comp_mixed_draw<MM, false>(C, B, sAG, cslot, tslot, CompGradSlots{}, dp, i, oob,
                                            nullptr);
    if (LSE)
      tlse_push_lw(st, l, lw);
    else
      lnl_out[i] = (double)l.hi + (double)l.lo;
  }
  if (LSE) block_lse_write(st, partials + blockIdx.x);
  if (oob_count) {
    for (int off = 16; off > 0; off >>= 1) oob += __shfl_down_sync(0xffffffffu, oob, off);
    if ((threadIdx.x & 31) == 0 && oob) atomicAdd(oob_count, (unsigned long long)oob);
  }
}

// Resident blocks per SM of a composite mixed kernel at (block size, shared
// memory), cached per (kernel, device, shape); the kernel's shared-memory
// attribute is set once to the device's opt-in maximum less its static shared
// memory.
template <typename KernelT>
cudaError_t comp_blocks_per_sm(KernelT kern, int threads, size_t smem, int* per_sm) {
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
    if (e.fn == fn && e.dev == dev && e.threads == threads && e.smem == smem) {
      *per_sm = e.nb;
      return cudaSuccess;
    }
  bool have_attr = false;
  for (const auto& a : attr_set) have_attr |= (a.first == fn && a.second == dev);
  if (!have_attr) {
    int optin = 0;
    cudaFuncAttributes fa;
    cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               optin - (int)fa.sharedSizeBytes);
    if (e != cudaSuccess) return e;
    attr_set.emplace_back(fn, dev);
  }
  int nb = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
  if (e != cudaSuccess) return e;
  if (nb < 1) return cudaErrorInvalidConfiguration;
  nb = nb < kMaxPartialsPerSM ? nb : kMaxPartialsPerSM;
  cache.push_back(Entry{fn, dev, threads, nb, smem});
  *per_sm = nb;
  return cudaSuccess;
}

template <int MM, bool BSMEM, bool LSE, int MINB>
cudaError_t launch_comp_mixed_k(const CompMixed& C, int threads, const DrawsParams& dp,
                                double* lnl_out, LseState* partials, unsigned long long* oob,
                                int* blocks, cudaStream_t st) {
  auto kern = comp_mixed_kernel<MM, BSMEM, LSE, MINB>;
  const size_t smem = comp_mixed_smem(C, BSMEM, threads);
  int per_sm = 0;
  const cudaError_t e = comp_blocks_per_sm(kern, threads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  *blocks = grid_cap(device_sms() * per_sm, dp.n, threads);
  kern<<<*blocks, threads, smem, st>>>(C, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

// lnL (when lnl_out is non-NULL) and its gradient, grad_out[7][n]; the slots
// of comp_mixed_thread_f4(C, true) per thread after the coefficient and tap
// slots.
template <int MM, bool BSMEM>
__global__ void __launch_bounds__(kCompMixedThreads, 2)
    comp_mixed_grad_kernel(const __grid_constant__ CompMixed C, DrawsParams dp,
                           double* __restrict__ lnl_out, double* __restrict__ grad_out) {
  extern __shared__ float4 smem4[];
  const size_t nb = BSMEM ? comp_mixed_b_f4(C) : 0, ng = comp_mixed_ag_f4(C);
  if constexpr (BSMEM)
    for (size_t q = threadIdx.x; q < nb; q += blockDim.x) smem4[q] = __ldg(C.Bs + q);
  float* sAG = reinterpret_cast<float*>(smem4 + nb);
  for (size_t q = threadIdx.x; q < (size_t)C.ncls * C.R; q += blockDim.x)
    sAG[q] = __ldg(C.agrid + q);
  __syncthreads();
  const float4* B = BSMEM ? smem4 : C.Bs;
  const size_t bd = blockDim.x, kna = (size_t)C.K * C.na;
  float4* cslot = smem4 + nb + ng + threadIdx.x;
  float4* tslot = cslot + kna * bd;
  float4* gbase = smem4 + nb + ng + (kna + (size_t)comp_tap_slots<true>() * C.K) * bd;
  CompGradSlots gs;
  gs.rho = reinterpret_cast<float2*>(gbase) + threadIdx.x;
  gs.af = gbase + ((kna + 1) / 2) * bd + threadIdx.x;
  gs.dy = gs.af + (size_t)C.na * bd;
  int oob = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    double g[kNpar];
    const df l = comp_mixed_draw<MM, true>(C, B, sAG, cslot, tslot, gs, dp, i, oob, g);
    if (lnl_out) lnl_out[i] = (double)l.hi + (double)l.lo;
#pragma unroll
    for (int p = 0; p < kNpar; ++p) grad_out[(size_t)p * dp.n + i] = g[p];
  }
}

template <int MM, bool BSMEM>
cudaError_t launch_comp_mixed_grad_k(const CompMixed& C, int threads, const DrawsParams& dp,
                                     double* lnl_out, double* grad_out, cudaStream_t st) {
  auto kern = comp_mixed_grad_kernel<MM, BSMEM>;
  const size_t smem = comp_mixed_smem(C, BSMEM, threads, true);
  int per_sm = 0;
  const cudaError_t e = comp_blocks_per_sm(kern, threads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  const int blocks = grid_cap(device_sms() * per_sm, dp.n, threads);
  kern<<<blocks, threads, smem, st>>>(C, dp, lnl_out, grad_out);
  return cudaGetLastError();
}

template <int MM, int MINB>
cudaError_t comp_mixed_lnl_b(const CompMixed& C, bool bsmem, int threads, const DrawsParams& dp,
                             double* lnl_out, LseState* partials, unsigned long long* oob,
                             int* blocks, cudaStream_t st) {
  if (partials)
    return bsmem ? launch_comp_mixed_k<MM, true, true, MINB>(C, threads, dp, lnl_out, partials, oob, blocks, st)
                 : launch_comp_mixed_k<MM, false, true, MINB>(C, threads, dp, lnl_out, partials, oob, blocks, st);
  return bsmem ? launch_comp_mixed_k<MM, true, false, MINB>(C, threads, dp, lnl_out, partials, oob, blocks, st)
               : launch_comp_mixed_k<MM, false, false, MINB>(C, threads, dp, lnl_out, partials, oob, blocks, st);
}

}  // namespace

// Entry point of one mode-count bucket (explicitly instantiated by the
// lnl_mixed_m4/m10/m16 translation units, dispatched in comp_mixed.cu): B is
// staged in shared memory when bsmem; `threads` per block (128, 64 or 32);
// the kernel variant sized for minb resident blocks per SM (3 only up to ten
// modes, else 2).
template <int MM>
cudaError_t comp_mixed_lnl(const CompMixed& C, bool bsmem, int threads, int minb,
                           const DrawsParams& dp, double* lnl_out, LseState* partials,
                           unsigned long long* oob, int* blocks, cudaStream_t st) {
  if constexpr (MM <= 10) {
    if (minb == 3)
      return comp_mixed_lnl_b<MM, 3>(C, bsmem, threads, dp, lnl_out, partials, oob, blocks, st);
  }
  return comp_mixed_lnl_b<MM, 2>(C, bsmem, threads, dp, lnl_out, partials, oob, blocks, st);
}

// The adjoint's entry point of one bucket (launch shape chosen by the build
// for comp_mixed_smem(C, bsmem, threads, true)).
template <int MM>
cudaError_t comp_mixed_grad(const CompMixed& C, bool bsmem, int threads, const DrawsParams& dp,
                            double* lnl_out, double* grad_out, cudaStream_t st) {
  return bsmem ? launch_comp_mixed_grad_k<MM, true>(C, threads, dp, lnl_out, grad_out, st)
               : launch_comp_mixed_grad_k<MM, false>(C, threads, dp, lnl_out, grad_out, st);
}

// Registers per thread of the adjoint kernel (grad) or of the fused lnZ kernel
// variant sized for minb blocks per SM of one bucket (the larger of the
// staged and unstaged variants; 0 on error, or when the bucket has no such
// variant), for the build's choice of launch shape.
template <int MM>
int comp_mixed_regs(bool grad, int minb) {
  cudaFuncAttributes a, b;
  cudaError_t e = cudaErrorInvalidValue;
  if (grad) {
    e = cudaFuncGetAttributes(&a, comp_mixed_grad_kernel<MM, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&b, comp_mixed_grad_kernel<MM, false>);
  } else if (minb == 2) {
    e = cudaFuncGetAttributes(&a, comp_mixed_kernel<MM, true, true, 2>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&b, comp_mixed_kernel<MM, false, true, 2>);
  } else if constexpr (MM <= 10) {
    if (minb == 3) {
      e = cudaFuncGetAttributes(&a, comp_mixed_kernel<MM, true, true, 3>);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&b, comp_mixed_kernel<MM, false, true, 3>);
    }
  }
  if (e != cudaSuccess) return 0;
  return a.numRegs > b.numRegs ? a.numRegs : b.numRegs;
}

#define RIFT_INSTANTIATE_COMP_MIXED(MM)                                                        \
  template cudaError_t comp_mixed_lnl<MM>(const CompMixed&, bool, int, int, const DrawsParams&, \
                                          double*, LseState*, unsigned long long*, int*,         \
                                          cudaStream_t);                                         \
  template cudaError_t comp_mixed_grad<MM>(const CompMixed&, bool, int, const DrawsParams&,     \
                                           double*, double*, cudaStream_t);                      \
  template int comp_mixed_regs<MM>(bool, int);

}  // namespace rift
