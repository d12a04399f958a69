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
// pairs on the grid of the detector's largest) and each detector's tap
// weights go to this thread's slots in shared memory; the harmonics stay in
// registers as mode pairs (j, j + 1), which are the lanes of the packed
// FFMA2 instructions of the a1/a2 sums.  Then, per class and pair of
// directions (r, r + 1): for each response index a the two rows of a1_a, a2_a,
// their split, and their products with the coefficients of up to
// kCompMixedKG detectors; then those detectors' residuals over the four taps.
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
                                         int bd) {
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

// One draw of the composite FP32-mixed likelihood.  B: split whitening (shared
// or global), AG: head constants of a1, a2; cslot/tslot: this thread's slots.
template <int MM>
__device__ __forceinline__ df comp_mixed_draw(const CompMixed& C, const float4* __restrict__ B,
                                              const float* __restrict__ AG, float4* cslot,
                                              float4* tslot, const DrawsParams& dp, long long i,
                                              int& oob) {
  constexpr int JPM = MM / 2;
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

  // ---- per detector: arrival time, table position, 1/2 |e|^2, tap weights,
  // and the coefficients (df pairs first, then split on the detector's grid)
  dacc T = dacc_zero();
  bool bad = false;
  for (int k = 0; k < K; ++k) {
    const float4 ph = C.pos_hi[k], pl = C.pos_lo[k];
    df delay = df_mul(df{ph.x, pl.x}, S.s[0]);
    delay = df_add(delay, df_mul(df{ph.y, pl.y}, S.s[1]));
    delay = df_add(delay, df_mul(df{ph.z, pl.z}, S.s[2]));
    const df tk = df_sub(tc, delay);
    const float mx = (C.kind == RIFT_ILE_RESP_ROTATION)
                         ? rot_coeffs(C, k, S, G, f0a, f0b, tk, cslot, bd)
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
    float4 w4 = make_float4(0.f, 0.f, 0.f, 0.f);
    float nsig = 0.f;
    int jc = -3;  // zero rows: a detector without a finite position adds nothing but NaN
    if (!isfinite(u.hi)) {
      bad = true;
      oob += 4;
    } else {
      float jf = floorf(u.hi);
      if (u.hi == jf && u.lo < 0.f) jf -= 1.f;
      const float f = __fadd_rn(__fsub_rn(u.hi, jf), u.lo);
      if (jf >= -2.f && jf <= (float)n) {
        const float2* pc = C.epoly + ((size_t)k * (n + 3) + (size_t)((int)jf + 2)) * (kPolyDeg + 1);
        float2 cf = __ldg(pc + kPolyDeg);
        df acc = df{cf.x, cf.y};
#pragma unroll
        for (int p = kPolyDeg - 1; p >= 0; --p) {
          cf = __ldg(pc + p);
          df pr = two_prod(acc.hi, f);
          pr.lo = fmaf(acc.lo, f, pr.lo);
          const df sm2 = two_sum(pr.hi, cf.x);
          acc = fast_two_sum(sm2.hi, __fadd_rn(__fadd_rn(pr.lo, sm2.lo), cf.y));
        }
        dacc_add(T, acc);
      }
      const float fa = f + 1.f, fc = f - 1.f, fd = f - 2.f;
      w4.x = -(f * fc * fd) * (1.f / 6.f);
      w4.y = (fa * fc * fd) * 0.5f;
      w4.z = -(fa * f * fd) * 0.5f;
      w4.w = (fa * f * fc) * (1.f / 6.f);
      const df ws = df_add(two_sum(w4.x, w4.y), two_sum(w4.z, w4.w));
      nsig = -__fadd_rn(__fsub_rn(ws.hi, 1.f), ws.lo);
      const float nb = fminf(fmaxf(1.f - jf, 0.f), 4.f);
      const float nab = fminf(fmaxf(jf + 3.f - (float)n, 0.f), 4.f);
      oob += (int)fminf(nb + nab, 4.f);
      jc = (int)fminf(fmaxf(jf, -3.f), (float)(n + 1));
    }
    tslot[(size_t)(2 * k) * bd] = w4;
    tslot[(size_t)(2 * k + 1) * bd] = make_float4(nsig, __int_as_float(jc), 0.f, 0.f);
  }

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
          df pr = two_prod(acc.hi, z.hi);
          pr.lo = fmaf(acc.hi, z.lo, fmaf(acc.lo, z.hi, pr.lo));
          const df sm2 = two_sum(pr.hi, c.x);
          acc = fast_two_sum(sm2.hi, __fadd_rn(__fadd_rn(pr.lo, sm2.lo), c.y));
        }
        const df amp = md.w ? df_mul(acc, sz) : acc;
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
      for (int r0 = 0; r0 < R; r0 += 2) {
        float2 whp[kCompMixedKG][2], wcp[kCompMixedKG][2];
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
        // residuals of rows r0, r0 + 1: r = sum_i wt_i (e_i - w) - sigma (e_j - w)
        // with -w = nhi + nlo (nhi the exact head sum), as in the static path
#pragma unroll
        for (int kk = 0; kk < kCompMixedKG; ++kk) {
          if (kk < nk) {
            const int k = kd[kk];
            const float4 w4 = tslot[(size_t)(2 * k) * bd];
            const float4 t1 = tslot[(size_t)(2 * k + 1) * bd];
            const int jc = __float_as_int(t1.y);
            const float2 nhi = make_float2(-__fadd_rn(whp[kk][0].x, whp[kk][0].y),
                                           -__fadd_rn(whp[kk][1].x, whp[kk][1].y));
            const float2 nlo = make_float2(-__fadd_rn(wcp[kk][0].x, wcp[kk][0].y),
                                           -__fadd_rn(wcp[kk][1].x, wcp[kk][1].y));
            const float2* Ej =
                C.ehat + ((size_t)k * (n + 2 * kEhatPad) + kEhatPad + (ptrdiff_t)(jc - 1)) * R + r0;
            const float wt[4] = {w4.x, w4.y, w4.z, w4.w};
            float2 rs = make_float2(0.f, 0.f);
#pragma unroll
            for (int tap = 0; tap < 4; ++tap) {
              const float4 e4 = __ldg(reinterpret_cast<const float4*>(Ej + (size_t)tap * R));
              const float2 d = __fadd2_rn(__fadd2_rn(make_float2(e4.x, e4.y), nhi),
                                          make_float2(e4.z, e4.w));
              rs = __ffma2_rn(make_float2(wt[tap], wt[tap]), d, rs);
              if (tap == 1) rs = __ffma2_rn(make_float2(t1.x, t1.x), d, rs);
            }
            const float2 rsv = __fadd2_rn(rs, nlo);
            q2p = __ffma2_rn(rsv, rsv, q2p);
          }
        }
      }
    }
  }
  dacc_fma_ff(T, -0.5f, __fadd_rn(q2p.x, q2p.y));
  df out = dacc_result(T);
  if (bad) out = df{CUDART_NAN_F, 0.f};
  return out;
}

template <int MM, bool BSMEM, bool LSE>
__global__ void __launch_bounds__(kCompMixedThreads, 2)
    comp_mixed_kernel(const __grid_constant__ CompMixed C, DrawsParams dp,
                      double* __restrict__ lnl_out, LseState* __restrict__ partials,
                      unsigned long long* __restrict__ oob_count) {
  extern __shared__ float4 smem4[];
  const size_t nb = BSMEM ? comp_mixed_b_f4(C) : 0, ng = comp_mixed_ag_f4(C);
  if (BSMEM)
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
      lw = dp.f64 ? (float)__ldg((const double*)dp.logw + i) : __ldg((const float*)dp.logw + i);
    const df l = comp_mixed_draw<MM>(C, B, sAG, cslot, tslot, dp, i, oob);
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

template <int MM, bool BSMEM, bool LSE>
cudaError_t launch_comp_mixed_k(const CompMixed& C, int threads, const DrawsParams& dp,
                                double* lnl_out, LseState* partials, unsigned long long* oob,
                                int* blocks, cudaStream_t st) {
  auto kern = comp_mixed_kernel<MM, BSMEM, LSE>;
  const size_t smem = comp_mixed_smem(C, BSMEM, threads);
  // the shared-memory attribute (the device's opt-in maximum) once per device,
  // the occupancy once per (device, shared-memory size, block size)
  static std::mutex mu;
  static bool attr_set[64] = {false};
  static size_t last_smem[64] = {0};
  static int last_threads[64] = {0}, last_nb[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  int per_sm = 0;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!attr_set[dev]) {
      // the opt-in maximum less the kernel's static shared memory
      int optin = 0;
      cudaFuncAttributes fa;
      cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
      if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 optin - (int)fa.sharedSizeBytes);
      if (e != cudaSuccess) return e;
      attr_set[dev] = true;
    }
    if (last_nb[dev] == 0 || last_smem[dev] != smem || last_threads[dev] != threads) {
      int nb = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, threads, smem);
      if (e != cudaSuccess) return e;
      if (nb < 1) return cudaErrorInvalidConfiguration;
      last_nb[dev] = nb < kMaxPartialsPerSM ? nb : kMaxPartialsPerSM;
      last_smem[dev] = smem;
      last_threads[dev] = threads;
    }
    per_sm = last_nb[dev];
  }
  *blocks = grid_cap(device_sms() * per_sm, dp.n, threads);
  kern<<<*blocks, threads, smem, st>>>(C, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

}  // namespace

// Entry point of one mode-count bucket (explicitly instantiated by the
// lnl_mixed_m4/m10/m16 translation units, dispatched in comp_mixed.cu): B is
// staged in shared memory when bsmem; `threads` per block (128, 64 or 32).
template <int MM>
cudaError_t comp_mixed_lnl(const CompMixed& C, bool bsmem, int threads, const DrawsParams& dp,
                           double* lnl_out, LseState* partials, unsigned long long* oob,
                           int* blocks, cudaStream_t st) {
  if (partials)
    return bsmem ? launch_comp_mixed_k<MM, true, true>(C, threads, dp, lnl_out, partials, oob, blocks, st)
                 : launch_comp_mixed_k<MM, false, true>(C, threads, dp, lnl_out, partials, oob, blocks, st);
  return bsmem ? launch_comp_mixed_k<MM, true, false>(C, threads, dp, lnl_out, partials, oob, blocks, st)
               : launch_comp_mixed_k<MM, false, false>(C, threads, dp, lnl_out, partials, oob, blocks, st);
}

#define RIFT_INSTANTIATE_COMP_MIXED(MM)                                                        \
  template cudaError_t comp_mixed_lnl<MM>(const CompMixed&, bool, int, const DrawsParams&,      \
                                          double*, LseState*, unsigned long long*, int*,         \
                                          cudaStream_t);

}  // namespace rift
