// FP32-mixed lnL and gradient with two warps per draw, for the small batches
// a gradient-based extrinsic sampler issues (the paper's warm-likelihood
// regime, App. H): included by lnl_mixed_impl.cuh inside its anonymous
// namespace, so it shares that file's double-float helpers.
//
// The arithmetic is the one of lnl_mixed_draw (whitened residual, double-float
// template, packed pairs), rearranged so that a pair of warps shares one draw:
// role 0 takes the sky, the detectors and the sums, role 1 the harmonics, the
// mat-vec and the adjoint's mode terms, so that the two independent branches
// after the angles run at once; within a warp each phase runs on its active
// lanes, and the phases hand their results on through the pair's slice of
// shared memory, the two warps meeting at named barriers:
//   1  role 0, lanes 0..3: sine/cosine of ra - gmst, dec, 2 psi, iota (no
//      table: quadrant reduction and Taylor series in double-float); lanes
//      4..15: of |m| phi for |m| = 1..12; every lane the distance factor
//      (the exponential, also without a table)
//   4a role 0, lane k < K: the arrival time and table position; the interval
//      polynomial's coefficients loaded and the interval's cubic coefficients
//      prefetched into L1, in flight during phase 2
//   2  role 0: the sky direction and x e^{2 i psi}; lanes 0..5 the six
//      products of the sky sines and cosines, lanes 0..9 the ten antenna-basis
//      terms from them, split for the exact products
//   3  role 1, lane j < M: the harmonic of mode j, split for the exact
//      products; lane (c, r): row r of the class-c mat-vec a1 = A y, a2 = A J y
//   4  role 0, lane k < K: x F_k, 1/2 |e|^2 and its slope, the detector's
//      antenna derivatives (phases 4a, 2 and 4 run while role 1 runs phase 3)
//   5  role 0, lane (k, direction pair): the template, the residual from the
//      interval's cubic and the pair's shares of |r|^2, r . edot, rho . a1,
//      rho . a2
//   6  role 1, lane (c, r): G1_r, G2_r of the class; role 0, lane k: the
//      detector's terms of lnL and of the gradient, summed over the detectors
//      by a fixed shuffle tree (compensated pairs merged exactly)
//   7  role 1, lane (c, j): the iota and phi_ref derivatives through mode j,
//      summed over the lanes by a fixed shuffle tree, and written out by its
//      lane 0 (while role 0 runs the second half of phase 6 and phase 8)
//   8  role 0, lanes 0..3, 6, 7: lnL and the other five gradient outputs
// The per-point tables (split whitening, gm1, detector and mode tables) are
// copied flat from the point's image at block start.
// Reductions run in fixed orders, so results are reproducible; they differ
// from the one-thread-per-draw kernel's by rounding only (e^{i |m| phi} is
// taken by the sine/cosine for every |m| rather than by recurrence, and the
// direction sums are grouped differently).
#pragma once

constexpr int kWarpDrawWarps = 4;  // warps per block
constexpr int kWarpDrawsPerBlock = kWarpDrawWarps / 2;  // two warps per draw

template <int MM, int RR>
struct WarpScratch {
  float4 ang[16];                  // (sin hi, sin lo, cos hi, cos lo): lam, dec, 2 psi, iota, |m| phi
  float2 x;                        // distance factor (hi, lo)
  float2 base[12];                 // sl, cl, sd, cd, sl^2, cl^2, sl cl, sd^2, sd cd, cd^2, 1, 0
  float2 bs[10];                   // antenna basis beta_0..5, gamma_0..3 as (head, tail)
  float4 ys[MM];                   // (yr1, yr2, yi1, yi2) of visited mode j
  float2 yh[MM];                   // (yr.hi, yi.hi)
  float4 a12[kMaxDet][RR];         // class c, direction r: (a1 head, a1 tail, a2 head, a2 tail)
  float4 xf[kMaxDet];              // x F_k: (re head, re tail, im head, im tail)
  float fpos[kMaxDet];             // position in the table interval
  int jc[kMaxDet];
  int bad[kMaxDet];
  float2 he2[kMaxDet], dhe2[kMaxDet];  // 1/2 |e|^2 and its slope in f (hi, lo)
  float4 dx[kMaxDet];              // d(x F_k)/d ra (re, im), d(x F_k)/d dec (re, im)
  float2 dk[kMaxDet];              // d t_k / d ra, d t_k / d dec
  float4 part[kMaxDet][RR / 2];    // per (k, pair): |r|^2, null term, r.edot, rho.a1
  float part5[kMaxDet][RR / 2];    // per (k, pair): rho.a2
  float2 gp[kMaxDet][RR];          // per (k, r): (Re xF_k rho_r, Im xF_k rho_r)
  float2 G[kMaxDet][RR];           // per class c, direction r: (G1, G2)
  float4 out[8];                   // lnL and the gradient as (hi, lo, extra, bad flag)
};

// Antenna-basis term i (beta_0..5, gamma_0..3, see antenna_basis) as
// kappa (X Y + sigma Z W) over the values of WarpScratch::base:
// (X, Y, Z, W, sigma + 1, kappa + 2) packed as bytes.
// Operand codes of the ten antenna-basis terms over WarpScratch::base
// (0 sl, 1 cl, 2 sd, 3 cd, 4 sl^2, 5 cl^2, 6 sl cl, 7 sd^2, 8 sd cd, 9 cd^2,
// 10 one, 11 zero): X | Y<<4 | Z<<8 | W<<12 | (sigma+1)<<16 | (kappa+2)<<20
// for the term kappa (X Y + sigma Z W).  Copied into shared memory at block
// start, so that each lane reads its own code without a branch.
__host__ __device__ constexpr unsigned basis_code(int i) {
  return i == 0 ? (4u | 10u << 4 | 7u << 8 | 5u << 12 | 0u << 16 | 3u << 20)      // sl^2 - sd^2 cl^2
         : i == 1 ? (5u | 10u << 4 | 7u << 8 | 4u << 12 | 0u << 16 | 3u << 20)    // cl^2 - sd^2 sl^2
         : i == 2 ? (6u | 10u << 4 | 6u << 8 | 7u << 12 | 2u << 16 | 0u << 20)    // -2 (sl cl + sl cl sd^2)
         : i == 3 ? (8u | 1u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 4u << 20)   // 2 sd cd cl
         : i == 4 ? (8u | 0u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 4u << 20)   // 2 sd cd sl
         : i == 5 ? (9u | 10u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 1u << 20)  // -cd^2
         : i == 6 ? (2u | 6u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 4u << 20)   // 2 sd sl cl
         : i == 7 ? (2u | 4u << 4 | 2u << 8 | 5u << 12 | 0u << 16 | 4u << 20)     // 2 (sd sl^2 - sd cl^2)
         : i == 8 ? (0u | 3u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 0u << 20)   // -2 sl cd
                  : (1u | 3u << 4 | 11u << 8 | 11u << 12 | 1u << 16 | 4u << 20);  // 2 cl cd
}

// sylm_amp_df with the Horner loop unrolled to the largest degree (steps
// beyond the mode's degree are skipped), so its coefficient reads issue
// together.
__device__ __forceinline__ df sylm_amp_df_unrolled(const MixedTables& T, int j, int l, int par, df z,
                                                   df sz) {
  float2 cq[kMaxEll + 1];
#pragma unroll
  for (int q = 0; q <= kMaxEll; ++q) cq[q] = T.yz[j][q];
  df acc = df{0.f, 0.f};
  bool started = false;
#pragma unroll
  for (int q = kMaxEll; q >= 0; --q) {
    if (q > l) continue;
    if (!started) {
      acc = df{cq[q].x, cq[q].y};
      started = true;
      continue;
    }
    acc = horner_step(acc, z, cq[q].x, cq[q].y);
  }
  return par ? df_mul(acc, sz) : fast_two_sum(acc.hi, acc.lo);
}

// Sine and cosine of a double-float angle without a table, for the
// latency-bound warp kernel (the anchored form waits on a dependent table
// load): a = 2 pi k + q pi/2 + d with |d| <= pi/4 (the 2 pi and pi/2 products
// exact or double-float), then sin d = d S(d^2), cos d = C(d^2) by their
// Taylor series to d^15 and d^16 (truncation < 1e-16 on |d| <= pi/4), the
// terms of order u^4 and up (u = d^2, each < 3e-6) by FP32 Horner, the four
// lowest by double-float Horner; absolute error ~1e-14, far below the
// template's 1e-10 budget.  The quadrant q then swaps and negates.
__device__ __forceinline__ df horner_df_step(df acc, df u, float ch, float cl) {
  // acc u + c with the high-part product exact
  df pr = two_prod(acc.hi, u.hi);
  pr.lo = fmaf(acc.hi, u.lo, fmaf(acc.lo, u.hi, pr.lo));
  const df sm = two_sum(pr.hi, ch);
  return fast_two_sum(sm.hi, __fadd_rn(__fadd_rn(pr.lo, sm.lo), cl));
}

__device__ __forceinline__ void sincos_df_notable(df a, df& s_out, df& c_out) {
  const float kTwoPiHi = 6.28318548202514648f;
  const float kTwoPiLo = -1.7484555314695172e-07f;
  const float kHalfPiHi = 1.57079637050628662f;
  const float kHalfPiLo = -4.37113900018624283e-08f;
  const float k = rintf(a.hi * 0.159154943091895336f);
  df kp = two_prod(k, kTwoPiHi);
  kp.lo = fmaf(k, kTwoPiLo, kp.lo);
  const df r = df_sub_reduce(a, kp);
  const float q = rintf(r.hi * 0.636619772367581343f);  // -2..2
  const df d = df_sub_reduce(r, df{q * kHalfPiHi, q * kHalfPiLo});  // q pi/2 exact in the pair
  df u = two_prod(d.hi, d.hi);
  u.lo = fmaf(2.f * d.hi, d.lo, u.lo);
  u = fast_two_sum(u.hi, u.lo);
  // 1/(2j+1)! and 1/(2j)! with alternating signs, as (hi, lo) pairs
  constexpr double s1 = -1.0 / 6, s2 = 1.0 / 120, s3 = -1.0 / 5040, s4 = 1.0 / 362880,
                   s5 = -1.0 / 39916800, s6 = 1.0 / 6227020800.0, s7 = -1.0 / 1307674368000.0;
  constexpr double c1 = -0.5, c2 = 1.0 / 24, c3 = -1.0 / 720, c4 = 1.0 / 40320,
                   c5 = -1.0 / 3628800, c6 = 1.0 / 479001600, c7 = -1.0 / 87178291200.0,
                   c8 = 1.0 / 20922789888000.0;
  const float uh = u.hi;
  float ts = fmaf(fmaf(fmaf((float)s7, uh, (float)s6), uh, (float)s5), uh, (float)s4);
  float tc = fmaf(fmaf(fmaf(fmaf((float)c8, uh, (float)c7), uh, (float)c6), uh, (float)c5), uh,
                  (float)c4);
  df S = df{ts, 0.f}, Cc = df{tc, 0.f};
  S = horner_df_step(S, u, (float)s3, (float)(s3 - (double)(float)s3));
  S = horner_df_step(S, u, (float)s2, (float)(s2 - (double)(float)s2));
  S = horner_df_step(S, u, (float)s1, (float)(s1 - (double)(float)s1));
  S = horner_df_step(S, u, 1.f, 0.f);
  Cc = horner_df_step(Cc, u, (float)c3, (float)(c3 - (double)(float)c3));
  Cc = horner_df_step(Cc, u, (float)c2, (float)(c2 - (double)(float)c2));
  Cc = horner_df_step(Cc, u, (float)c1, 0.f);
  Cc = horner_df_step(Cc, u, 1.f, 0.f);
  const df sd = df_mul(d, S);
  // quadrant: (sin, cos) of d + q pi/2
  const int qi = (int)q & 3;
  df so = sd, co = Cc;
  if (qi == 1) {
    so = Cc;
    co = df_neg(sd);
  } else if (qi == 2) {
    so = df_neg(sd);
    co = df_neg(Cc);
  } else if (qi == 3) {
    so = df_neg(Cc);
    co = sd;
  }
  s_out = so;
  c_out = co;
}

// e^a for a double-float a without a table: a = k ln2 + r, |r| <= ln2/2 (k ln2
// as a pair), e^r by its Taylor series to r^13 (truncation < 2e-16), the terms
// of order r^5 and up by FP32 Horner, the five lowest by double-float Horner;
// then the exact scaling by 2^k.  Relative error ~1e-14.
__device__ __forceinline__ df exp_df_notable(df a) {
  const float kLn2Hi = 0.693147182464599609f;
  const float kLn2Lo = -1.904654323148236e-09f;
  const float k = rintf(a.hi * 1.44269504088896341f);
  df kp = two_prod(k, kLn2Hi);
  kp.lo = fmaf(k, kLn2Lo, kp.lo);
  const df r = df_sub_reduce(a, kp);
  const float rh = r.hi;
  constexpr double e5 = 1.0 / 120, e6 = 1.0 / 720, e7 = 1.0 / 5040, e8 = 1.0 / 40320,
                   e9 = 1.0 / 362880, e10 = 1.0 / 3628800, e11 = 1.0 / 39916800,
                   e12 = 1.0 / 479001600, e13 = 1.0 / 6227020800.0;
  constexpr double e2 = 0.5, e3 = 1.0 / 6, e4 = 1.0 / 24;
  float t = fmaf((float)e13, rh, (float)e12);
  t = fmaf(t, rh, (float)e11);
  t = fmaf(t, rh, (float)e10);
  t = fmaf(t, rh, (float)e9);
  t = fmaf(t, rh, (float)e8);
  t = fmaf(t, rh, (float)e7);
  t = fmaf(t, rh, (float)e6);
  t = fmaf(t, rh, (float)e5);
  df E = df{t, 0.f};
  E = horner_df_step(E, r, (float)e4, (float)(e4 - (double)(float)e4));
  E = horner_df_step(E, r, (float)e3, (float)(e3 - (double)(float)e3));
  E = horner_df_step(E, r, (float)e2, 0.f);
  E = horner_df_step(E, r, 1.f, 0.f);
  E = horner_df_step(E, r, 1.f, 0.f);
  const int ki = (int)k;
  return df{ldexpf(E.hi, ki), ldexpf(E.lo, ki)};
}

// Merge of two compensated accumulators (the sum of their values).
__device__ __forceinline__ dacc dacc_merge(dacc a, dacc b) {
  const df t = two_sum(a.s, b.s);
  return dacc{t.hi, __fadd_rn(__fadd_rn(a.c, b.c), t.lo)};
}

template <int MM, int RR>
__host__ __device__ inline size_t warp_smem_bytes(int ncls, int R, int M) {
  // the point's image (split whitening, gm1, staged tables), then one
  // scratch slice per warp
  return image_bytes(ncls, R, M) + (size_t)kWarpDrawsPerBlock * sizeof(WarpScratch<MM, RR>);
}

template <int MM, int RR, bool GRAD>
__global__ void __launch_bounds__(32 * kWarpDrawWarps)
    lnl_warp_kernel(const __grid_constant__ PointParams P, DrawsParams dp,
                    double* __restrict__ lnl_out, double* __restrict__ grad_out) {
  extern __shared__ float4 smem4[];
  __shared__ unsigned s_basis[10];
  if (threadIdx.x < 10) s_basis[threadIdx.x] = basis_code(threadIdx.x);
  // the point's image into shared memory by asynchronous copies, waited for
  // once the first draw's angles (which need neither) are under way
  {
    const unsigned sbase = (unsigned)__cvta_generic_to_shared(smem4);
    for (int t = threadIdx.x; t < P.img_f4; t += blockDim.x)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * (unsigned)t),
                   "l"(P.img + t)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  // programmatic dependent launch (the host launches this kernel with it):
  // the point's image and parameters are immutable once the point exists, so
  // the copies above may overlap the previous kernel in the stream; the draws
  // (possibly that kernel's output) are read, and the outputs written, only
  // after it has completed.  The next kernel may likewise begin its prologue.
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  asm volatile("griddepcontrol.wait;" ::: "memory");
  const float4* sA = smem4;
  const float* sg = reinterpret_cast<const float*>(smem4 + split_a_f4(P.ncls, P.R, P.M));
  const MixedTables& T = *reinterpret_cast<const MixedTables*>(
      reinterpret_cast<const char*>(smem4) + split_a_bytes(P.ncls, P.R, P.M));
  const size_t aoff = (size_t)P.img_f4 * 16;
  // two warps per draw: role 0 takes the sky, the detectors and the sums, role
  // 1 the harmonics, the mat-vec and the mode terms of the adjoint; the pair
  // meets at named barriers (id 1 + pair, 64 threads)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pair = warp >> 1, role = warp & 1;
  WarpScratch<MM, RR>& W =
      reinterpret_cast<WarpScratch<MM, RR>*>(reinterpret_cast<char*>(smem4) + aoff)[pair];
  auto pair_sync = [&]() { asm volatile("bar.sync %0, 64;" ::"r"(1 + pair) : "memory"); };
  const int K = P.K, M = P.M, n = P.n, ncls = P.ncls;
  constexpr int NP = RR / 2;  // direction pairs

  // ---- 1 (a function of the draw): the sines and cosines, and the
  // distance factor; leaves the draw's t_c in tc
  df tc;
  auto angles = [&](long long i) {
    const float ra = load_param_f(dp, 0, i), dec = load_param_f(dp, 1, i);
    const float psi = load_param_f(dp, 2, i), incl = load_param_f(dp, 3, i);
    const float phi = load_param_f(dp, 4, i), lnD = load_param_f(dp, 5, i);
    tc = load_param_df(dp, 6, i);
    // every lane takes the exponential in the same instruction stream as its
    // sine and cosine (both without tables: no dependent load)
    df lx = two_sum(P.ln_dref_hi, -lnD);
    lx.lo = __fadd_rn(lx.lo, P.ln_dref_lo);
    const df x = exp_df_notable(fast_two_sum(lx.hi, lx.lo));
    {
      df a;
      if (lane == 0) {
        a = two_sum(ra, -P.gmst_hi);
        a.lo = __fsub_rn(a.lo, P.gmst_lo);
        a = fast_two_sum(a.hi, a.lo);
      } else if (lane == 1) {
        a = df{dec, 0.f};
      } else if (lane == 2) {
        a = df{2.f * psi, 0.f};
      } else if (lane == 3) {
        a = df{incl, 0.f};
      } else {
        a = two_prod((float)(lane - 3), phi);
      }
      df s, c;
      // lanes 4.. take |m| phi for |m| = lane - 3 (beyond the point's largest
      // |m| a spare angle; no loop over the modes' constants on this path)
      sincos_df_notable(a, s, c);
      if (lane < 16) W.ang[lane] = make_float4(s.hi, s.lo, c.hi, c.lo);
      if (lane == 31) W.x = make_float2(x.hi, x.lo);
    }
    __syncwarp();
  };

  const long long i0 = blockIdx.x * (long long)kWarpDrawsPerBlock + pair;
  const long long stride = (long long)gridDim.x * kWarpDrawsPerBlock;
  if (i0 < dp.n && role == 0) angles(i0);  // uniform over the warp
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();

  for (long long i = i0; i < dp.n; i += stride) {
    if (i != i0) {
      if (role == 0) angles(i);
      pair_sync();
    }

    // ---- 2: sky direction, antenna basis (every lane), x e^{2 i psi}
    const float4 a0 = W.ang[0], a1v = W.ang[1], a2v = W.ang[2], a3v = W.ang[3];
    const df sl{a0.x, a0.y}, cl{a0.z, a0.w}, sd{a1v.x, a1v.y}, cd{a1v.z, a1v.w};
    const df s2p{a2v.x, a2v.y}, c2p{a2v.z, a2v.w}, sz{a3v.x, a3v.y}, z{a3v.z, a3v.w};
    const df x{W.x.x, W.x.y};
    const df s0 = df_mul(cd, cl), s1 = df_mul(cd, sl), s2 = sd;
    const df xer = df_mul(x, c2p), xei = df_mul(x, s2p);
    // ---- 4a: role 0, lane k < K: the arrival time and table position, so
    // that the interval polynomial's coefficients and the cubic's are in
    // flight while phase 2 forms the antenna basis
    float4 ph = make_float4(0.f, 0.f, 0.f, 0.f), pl = ph;
    int bad = 0, jck = 0;
    float f = 0.f, jf = 0.f;
    bool inpoly = false;
    float2 cf[kPolyDeg + 1];
    if (role == 0 && lane < K) {
      const int k = lane;
      ph = T.pos_hi[k];
      pl = T.pos_lo[k];
      const df delay = dot3_df(ph, pl, s0, s1, s2);
      const df rel = df_add(df_sub(tc, delay), df{-ph.w, -pl.w});
      const df u = df_mul(rel, df{P.inv_dt_hi, P.inv_dt_lo});
      bad = isfinite(u.hi) ? 0 : 1;
      if (!bad) {
        jf = floorf(u.hi);
        if (u.hi == jf && u.lo < 0.f) jf -= 1.f;
        f = __fadd_rn(__fsub_rn(u.hi, jf), u.lo);
      }
      jck = (int)fminf(fmaxf(jf, -3.f), (float)(n + 1));
      // the interval's record: the sextic loaded now (zero outside the
      // table), the cubic coefficients before it prefetched into L1 for the
      // residual phase
      const float4* rec = P.erec + ((size_t)k * (n + 5) + (size_t)(jck + 3)) * (3 * (RR / 2) + 4);
      inpoly = !bad;
      if (inpoly) {
        const float4* pe = rec + 3 * (RR / 2);
        const float4 e01 = __ldg(pe), e23 = __ldg(pe + 1), e45 = __ldg(pe + 2), e6 = __ldg(pe + 3);
        cf[0] = make_float2(e01.x, e01.y);
        cf[1] = make_float2(e01.z, e01.w);
        cf[2] = make_float2(e23.x, e23.y);
        cf[3] = make_float2(e23.z, e23.w);
        cf[4] = make_float2(e45.x, e45.y);
        cf[5] = make_float2(e45.z, e45.w);
        cf[6] = make_float2(e6.x, e6.y);
      }
      {
        const char* cb = reinterpret_cast<const char*>(rec);
        constexpr int kBytes = (RR / 2) * 48;
        for (int off = 0; off < kBytes; off += 128)
          asm volatile("prefetch.global.L1 [%0];" ::"l"(cb + off));
        asm volatile("prefetch.global.L1 [%0];" ::"l"(cb + kBytes - 16));
      }
    }

    if (role == 0) {
      // the antenna basis: six products on lanes 0..5, ten terms on lanes 0..9
      if (lane < 6) {
        // (sl, sl), (cl, cl), (sl, cl), (sd, sd), (sd, cd), (cd, cd)
        const df u = lane < 2 ? (lane == 0 ? sl : cl) : lane == 2 ? sl : lane == 5 ? cd : sd;
        const df v = lane == 0 ? sl : lane < 3 ? cl : lane == 3 ? sd : cd;
        const df pr = df_mul(u, v);
        W.base[4 + lane] = make_float2(pr.hi, pr.lo);
      } else if (lane < 10) {
        const df b = lane == 6 ? sl : lane == 7 ? cl : lane == 8 ? sd : cd;
        W.base[lane - 6] = make_float2(b.hi, b.lo);
      } else if (lane == 10) {
        W.base[10] = make_float2(1.f, 0.f);
        W.base[11] = make_float2(0.f, 0.f);
      }
      __syncwarp();
      if (lane < 10) {
        const unsigned code = s_basis[lane];
        const int X = (int)(code & 15u), Y = (int)((code >> 4) & 15u);
        const int Z = (int)((code >> 8) & 15u), Wd = (int)((code >> 12) & 15u);
        const float sig = (float)((int)((code >> 16) & 15u) - 1);
        const float kap = (float)((int)((code >> 20) & 15u) - 2);
        const float2 bx = W.base[X], by = W.base[Y], bz = W.base[Z], bw = W.base[Wd];
        const df p1 = df_mul(df{bx.x, bx.y}, df{by.x, by.y});
        const df p2 = df_mul(df{bz.x, bz.y}, df{bw.x, bw.y});
        const df q = df_add(p1, df{sig * p2.hi, sig * p2.lo});
        // kappa is 0, +-1 or +-2: the scaling is exact; then the split of
        // split_antenna_basis (head on the 2^-8 grid, tail = rest + low part)
        const float qh = kap * q.hi, ql = kap * q.lo;
        const float h = head_of(qh, 49152.0f);
        W.bs[lane] = make_float2(h, __fadd_rn(__fsub_rn(qh, h), ql));
      }
    }

    if (role == 1) {
      // ---- 3a: lane j < M: the harmonic of mode j (visiting order), split
      if (lane < M) {
        const int4 md = T.mode[lane];  // (mode index, m, l, ypar)
        const int m = md.y, am = m < 0 ? -m : m;
        df cm{1.f, 0.f}, sm{0.f, 0.f};
        if (am > 0) {
          const float4 e = W.ang[3 + am];
          sm = df{e.x, e.y};
          cm = df{e.z, e.w};
        }
        const df amp = sylm_amp_df_unrolled(T, lane, md.z, md.w, z, sz);
        const df yr = df_mul(amp, cm);
        const df yi = m < 0 ? df_neg(df_mul(amp, sm)) : df_mul(amp, sm);
        float yr1, yr2, yi1, yi2;
        split_y(yr.hi, yr1, yr2);
        split_y(yi.hi, yi1, yi2);
        W.ys[lane] = make_float4(yr1, __fadd_rn(yr2, yr.lo), yi1, __fadd_rn(yi2, yi.lo));
        W.yh[lane] = make_float2(yr.hi, yi.hi);
      }
      __syncwarp();
      // ---- 3b: lane (c, r): row r of class c's mat-vec, packed as in the per-thread kernel
      for (int it = lane; it < ncls * RR; it += 32) {
        const int c = it / RR, r = it - c * RR;
        const float4* Ac = sA + (size_t)c * RR * M + (size_t)(r / 2) * M * 2;
        const bool odd = r & 1;
        float2 ex = make_float2(0.f, 0.f), co = make_float2(0.f, 0.f);
  #pragma unroll
        for (int j = 0; j < MM; ++j) {
          if (j >= M) break;
          const float4 y = W.ys[j];
          const float2 yh = W.yh[j];
          // this direction's lane of the pair's heads and tails (t = A[r][a],
          // b = A[r][M + a]): ap = (t_h, b_h, t_t, b_t), an = (b_h, -t_h, b_t, -t_t)
          const float4 hp = Ac[2 * j], tp = Ac[2 * j + 1];
          const float th = odd ? hp.y : hp.x, bh = odd ? hp.w : hp.z;
          const float tt = odd ? tp.y : tp.x, bt = odd ? tp.w : tp.z;
          const float4 ap = make_float4(th, bh, tt, bt), an = make_float4(bh, -th, bt, -tt);
          ex = __ffma2_rn(make_float2(ap.x, ap.y), make_float2(y.x, y.x), ex);
          ex = __ffma2_rn(make_float2(an.x, an.y), make_float2(y.z, y.z), ex);
          co = __ffma2_rn(make_float2(ap.x, ap.y), make_float2(y.y, y.y), co);
          co = __ffma2_rn(make_float2(ap.z, ap.w), make_float2(yh.x, yh.x), co);
          co = __ffma2_rn(make_float2(an.x, an.y), make_float2(y.w, y.w), co);
          co = __ffma2_rn(make_float2(an.z, an.w), make_float2(yh.y, yh.y), co);
        }
        // heads on the grid of the larger exact head sum, tails (ex - head) + co
        // (as in the per-thread kernel)
        const float C = head_constant(fmaxf(fabsf(ex.x), fabsf(ex.y)));
        const float2 C2 = make_float2(C, C);
        const float2 hd = sub2(__fadd2_rn(ex, C2), C2);
        const float2 tl = __fadd2_rn(sub2(ex, hd), co);
        W.a12[c][r] = make_float4(hd.x, tl.x, hd.y, tl.y);
      }
    }

    if (role == 0) {
      // ---- 4: lane k < K (the arrival time and the table loads of phase 4a):
      // the antenna factor, 1/2|e|^2, the derivatives
      if (lane < K) {
        const int k = lane;
        AntennaSplit AS;
  #pragma unroll
        for (int q = 0; q < 6; ++q) {
          AS.bh[q] = W.bs[q].x;
          AS.bt[q] = W.bs[q].y;
        }
  #pragma unroll
        for (int q = 0; q < 4; ++q) {
          AS.gh[q] = W.bs[6 + q].x;
          AS.gt[q] = W.bs[6 + q].y;
        }
        df xFr, xFi;
        antenna_df(T, k, AS, xer, xei, xFr, xFi);
        const float Cx = head_constant(fmaxf(fabsf(xFr.hi), fabsf(xFi.hi)));
        const float xrh = head_of(xFr.hi, Cx), xih = head_of(xFi.hi, Cx);
        W.xf[k] = make_float4(xrh, __fadd_rn(__fsub_rn(xFr.hi, xrh), xFr.lo), xih,
                              __fadd_rn(__fsub_rn(xFi.hi, xih), xFi.lo));
        if (GRAD) {
          AntennaBasisGrad ABG;
          antenna_basis_grad(sl.hi, cl.hi, sd.hi, cd.hi, ABG);
          float dfpa = 0.f, dfpd = 0.f, dfxa = 0.f, dfxd = 0.f;
          float ac[12];
  #pragma unroll
          for (int v = 0; v < 3; ++v) {
            const float4 a4 = T.ah[k][v], b4 = T.at[k][v];
            ac[4 * v] = a4.x + b4.x;
            ac[4 * v + 1] = a4.y + b4.y;
            ac[4 * v + 2] = a4.z + b4.z;
            ac[4 * v + 3] = a4.w + b4.w;
          }
  #pragma unroll
          for (int q = 0; q < 6; ++q) {
            dfpa = fmaf(ac[q], ABG.ba[q], dfpa);
            dfpd = fmaf(ac[q], ABG.bd[q], dfpd);
          }
  #pragma unroll
          for (int q = 0; q < 4; ++q) {
            dfxa = fmaf(ac[6 + q], ABG.ga[q], dfxa);
            dfxd = fmaf(ac[6 + q], ABG.gd[q], dfxd);
          }
          W.dx[k] = make_float4(dfpa * xer.hi + dfxa * xei.hi, dfpa * xei.hi - dfxa * xer.hi,
                                dfpd * xer.hi + dfxd * xei.hi, dfpd * xei.hi - dfxd * xer.hi);
          // ds/d ra = (-cd sl, cd cl, 0), ds/d dec = (-sd cl, -sd sl, cd)
          W.dk[k] = make_float2(-(ph.x * (-cd.hi * sl.hi) + ph.y * (cd.hi * cl.hi)),
                                -(ph.x * (-sd.hi * cl.hi) + ph.y * (-sd.hi * sl.hi) + ph.z * cd.hi));
        }
        // 1/2 |e(f)|^2 from the interval polynomial (zero when no tap is in the
        // table) and its slope in f, Horner on both as in the per-thread kernel
        df half_e2 = df{0.f, 0.f}, dhalf = df{0.f, 0.f};
        if (inpoly) {
          df acc = df{cf[kPolyDeg].x, cf[kPolyDeg].y};
          df dacc_p = df{0.f, 0.f};
  #pragma unroll
          for (int p = kPolyDeg - 1; p >= 0; --p) {
            if (GRAD) dacc_p = horner_step_f(dacc_p, f, acc.hi, acc.lo);
            acc = horner_step_f(acc, f, cf[p].x, cf[p].y);
          }
          half_e2 = acc;
          dhalf = dacc_p;
        }
        W.fpos[k] = f;
        W.jc[k] = jck;
        W.bad[k] = bad;
        W.he2[k] = make_float2(half_e2.hi, half_e2.lo);
        W.dhe2[k] = make_float2(dhalf.hi, dhalf.lo);
      }
      __syncwarp();
    }
    pair_sync();  // a12 from role 1, the detectors' tables from role 0

    if (role == 0) {
      // ---- 5: lane (k, pair): the residual of two directions (packed, as in
      // the per-thread kernel's loop body)
      for (int it = lane; it < K * NP; it += 32) {
        const int k = it / NP, pr = it - k * NP, r = 2 * pr;
        if (W.bad[k]) continue;
        const int c = P.cls_of[k];
        const float4 xfq = W.xf[k];
        const float2 nxrh = make_float2(-xfq.x, -xfq.x), nxrt = make_float2(-xfq.y, -xfq.y);
        const float2 nxih = make_float2(-xfq.z, -xfq.z), nxit = make_float2(-xfq.w, -xfq.w);
        const float4 qa0 = W.a12[c][r], qa1 = W.a12[c][r + 1];
        const float2 a1h = make_float2(qa0.x, qa1.x), a1t = make_float2(qa0.y, qa1.y);
        const float2 a2h = make_float2(qa0.z, qa1.z), a2t = make_float2(qa0.w, qa1.w);
        float2 nlo = __fmul2_rn(nxrh, a1t);
        nlo = __ffma2_rn(nxrt, a1h, nlo);
        nlo = __ffma2_rn(nxrt, a1t, nlo);
        nlo = __ffma2_rn(nxih, a2t, nlo);
        nlo = __ffma2_rn(nxit, a2h, nlo);
        nlo = __ffma2_rn(nxit, a2t, nlo);
        const float2 nhi = __ffma2_rn(nxrh, a1h, __fmul2_rn(nxih, a2h));
        // the interval's cubic e(f) = c0 + f (c1 + f (c2 + f c3)) (as in the
        // per-thread kernel): c0.hi meets the exact head of w first
        const float fk = W.fpos[k];
        const float2 f2 = make_float2(fk, fk);
        const float4* Cj = P.erec + ((size_t)k * (n + 5) + (size_t)(W.jc[k] + 3)) * (3 * (RR / 2) + 4) + 3 * pr;
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
          ed = __ffma2_rn(__ffma2_rn(c3, make_float2(3.f * fk, 3.f * fk), __fadd2_rn(c2, c2)), f2, c1);
        const float2 q2 = __fmul2_rn(rsv, rsv);
        const float2 nwf = __fadd2_rn(nhi, nlo);
        float2 gm = make_float2(0.f, 0.f), nul = make_float2(0.f, 0.f);
        const float* gc = sg + c * RR;
        if (GRAD || P.has_null[c]) {
          gm = make_float2(gc[r], gc[r + 1]);
          nul = __fmul2_rn(__fmul2_rn(gm, nwf), nwf);
        }
        float4 pt = make_float4(__fadd_rn(q2.x, q2.y), __fadd_rn(nul.x, nul.y), 0.f, 0.f);
        if (GRAD) {
          const float2 red = __fmul2_rn(rsv, ed);
          const float2 rho = __ffma2_rn(make_float2(-gm.x, -gm.y), nwf, rsv);
          const float2 g1 = __fmul2_rn(rho, __fadd2_rn(a1h, a1t));
          const float2 g2 = __fmul2_rn(rho, __fadd2_rn(a2h, a2t));
          pt.z = __fadd_rn(red.x, red.y);
          pt.w = __fadd_rn(g1.x, g1.y);
          W.part5[k][pr] = __fadd_rn(g2.x, g2.y);
          const float xFr = __fadd_rn(xfq.x, xfq.y), xFi = __fadd_rn(xfq.z, xfq.w);
          W.gp[k][r] = make_float2(xFr * rho.x, xFi * rho.x);
          W.gp[k][r + 1] = make_float2(xFr * rho.y, xFi * rho.y);
        }
        W.part[k][pr] = pt;
      }
      __syncwarp();
    }
    pair_sync();  // the residual terms

    // ---- 6: role 1, lane (c, r): G1_r, G2_r of class c over its detectors in
    // order; role 0, lane k: the detector's terms
    if (GRAD && role == 1) {
      for (int it = lane; it < ncls * RR; it += 32) {
        const int c = it / RR, r = it - c * RR;
        float g1 = 0.f, g2 = 0.f;
        for (int q = P.cls_begin[c]; q < P.cls_begin[c + 1]; ++q) {
          const int k = P.det_order[q];
          if (W.bad[k]) continue;
          const float2 v = W.gp[k][r];
          g1 += v.x;
          g2 += v.y;
        }
        W.G[c][r] = make_float2(g1, g2);
      }
    }
    // lane k's terms (zero on lanes without a detector or with a bad one)
    dacc tk = dacc_zero(), gk_t = dacc_zero(), gk_ra = dacc_zero(), gk_dec = dacc_zero();
    float gk[4] = {0.f, 0.f, 0.f, 0.f};  // ra, dec, psi, lnD through the antenna factor
    int badk = 0;
    if (role == 0) {
      if (lane < K) badk = W.bad[lane];
      if (lane < K && !badk) {
        const int k = lane, c = P.cls_of[k];
        float q2 = 0.f, nul = 0.f, red = 0.f, g1 = 0.f, g2 = 0.f;
  #pragma unroll
        for (int pr = 0; pr < NP; ++pr) {
          const float4 v = W.part[k][pr];
          q2 += v.x;
          nul += v.y;
          if (GRAD) {
            red += v.z;
            g1 += v.w;
            g2 += W.part5[k][pr];
          }
        }
        const float2 he = W.he2[k];
        dacc_add(tk, df{he.x, he.y});
        dacc_add(tk, df{-0.5f * q2, 0.f});
        if (P.has_null[c]) dacc_add(tk, df{0.5f * nul, 0.f});
        if (GRAD) {
          const float2 dh = W.dhe2[k];
          const df dtk = df_mul(df_add_f(df{dh.x, dh.y}, -red), df{P.inv_dt_hi, P.inv_dt_lo});
          const float2 dkk = W.dk[k];
          const df dra = df_mul_f(dtk, dkk.x), ddec = df_mul_f(dtk, dkk.y);
          gk_t = dacc{dtk.hi, dtk.lo};
          gk_ra = dacc{dra.hi, dra.lo};
          gk_dec = dacc{ddec.hi, ddec.lo};
          const float4 d = W.dx[k];
          const float4 xfq = W.xf[k];
          const float xFr = __fadd_rn(xfq.x, xfq.y), xFi = __fadd_rn(xfq.z, xfq.w);
          gk[0] = fmaf(d.x, g1, d.y * g2);
          gk[1] = fmaf(d.z, g1, d.w * g2);
          gk[2] = fmaf(-2.f * xFi, g1, 2.f * xFr * g2);
          gk[3] = fmaf(-xFr, g1, -xFi * g2);
        }
      }
      // the sums over detectors: a fixed shuffle tree over lanes 0..7 (the
      // levels whose upper half holds no detector only add zeros: skipped)
  #pragma unroll
      for (int off = 4; off > 0; off >>= 1) {
        if (off >= K) continue;  // uniform over the warp
        dacc o;
        o.s = __shfl_down_sync(0xffffffffu, tk.s, off, 8);
        o.c = __shfl_down_sync(0xffffffffu, tk.c, off, 8);
        tk = dacc_merge(tk, o);
        badk |= __shfl_down_sync(0xffffffffu, badk, off, 8);
        if (GRAD) {
          o.s = __shfl_down_sync(0xffffffffu, gk_t.s, off, 8);
          o.c = __shfl_down_sync(0xffffffffu, gk_t.c, off, 8);
          gk_t = dacc_merge(gk_t, o);
          o.s = __shfl_down_sync(0xffffffffu, gk_ra.s, off, 8);
          o.c = __shfl_down_sync(0xffffffffu, gk_ra.c, off, 8);
          gk_ra = dacc_merge(gk_ra, o);
          o.s = __shfl_down_sync(0xffffffffu, gk_dec.s, off, 8);
          o.c = __shfl_down_sync(0xffffffffu, gk_dec.c, off, 8);
          gk_dec = dacc_merge(gk_dec, o);
  #pragma unroll
          for (int q = 0; q < 4; ++q) gk[q] += __shfl_down_sync(0xffffffffu, gk[q], off, 8);
        }
      }
    }
    __syncwarp();
    if (GRAD && role == 1) {
      // ---- 7: role 1, lane (c, j): iota and phi_ref through mode j of class c
      float gph = 0.f, gin = 0.f;
      for (int it = lane; it < ncls * M; it += 32) {
        const int c = it / M, j = it - c * M;
        const float4* Ac2 = sA + (size_t)c * RR * M;
        float h1t = 0.f, h1b = 0.f, h2t = 0.f, h2b = 0.f;
#pragma unroll
        for (int r = 0; r < RR; ++r) {
          // heads (t_h, t_h, b_h, b_h) and tails of the pair (r, r + 1)
          const float4 hp = Ac2[2 * ((r / 2) * M + j)], tp = Ac2[2 * ((r / 2) * M + j) + 1];
          const float ath = (r & 1) ? hp.y + tp.y : hp.x + tp.x;
          const float abh = (r & 1) ? hp.w + tp.w : hp.z + tp.z;
          const float2 g = W.G[c][r];
          h1t = fmaf(g.x, ath, h1t);
          h1b = fmaf(g.x, abh, h1b);
          h2t = fmaf(g.y, ath, h2t);
          h2b = fmaf(g.y, abh, h2b);
        }
        const float Hre = h1t + h2b, Him = h1b - h2t;
        const int4 md = T.mode[j];
        const int m = md.y, am = m < 0 ? -m : m;
        float cmf = 1.f, smf = 0.f;
        if (am > 0) {
          const float4 e = W.ang[3 + am];
          smf = e.x;
          cmf = e.z;
        }
        const float sgn = m < 0 ? -1.f : 1.f;
        float amp, damp;
        sylm_amp_grad_f(T, j, md.z, md.w, z.hi, sz.hi, amp, damp);
        const float yre = amp * cmf, yim = sgn * amp * smf;
        gph = fmaf((float)m, fmaf(-yim, Hre, yre * Him), gph);
        gin = fmaf(damp * cmf, Hre, fmaf(sgn * damp * smf, Him, gin));
      }
      // a fixed shuffle tree over the 32 lanes (levels above the lanes that
      // hold terms only add zeros: skipped)
      const int nact = ncls * M < 32 ? ncls * M : 32;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) {
        if (off >= nact) continue;  // uniform over the warp
        gph += __shfl_down_sync(0xffffffffu, gph, off);
        gin += __shfl_down_sync(0xffffffffu, gin, off);
      }
      // role 1 writes its two outputs itself (the draw is NaN if any
      // detector's arrival time was not finite), while role 0 forms the rest
      if (lane == 0) {
        int badany = 0;
        for (int k = 0; k < K; ++k) badany |= W.bad[k];
        grad_out[(size_t)3 * dp.n + i] = badany ? CUDART_NAN : (double)gin;
        grad_out[(size_t)4 * dp.n + i] = badany ? CUDART_NAN : (double)gph;
      }
    }

    // ---- 8: lane 0 holds the sums; lanes 0..3, 6, 7 then form one output each
    // in FP64 (a warp-wide FP64 instruction costs the same for one lane or
    // eight; the iota and phase outputs come from role 1)
    if (role == 0 && lane == 0) {
      const df lnl = dacc_result(tk);
      W.out[0] = make_float4(lnl.hi, lnl.lo, 0.f, __int_as_float(badk));
      if (GRAD) {
        const df a = dacc_result(gk_ra), b = dacc_result(gk_dec), t = dacc_result(gk_t);
        W.out[1] = make_float4(a.hi, a.lo, gk[0], 0.f);
        W.out[2] = make_float4(b.hi, b.lo, gk[1], 0.f);
        W.out[3] = make_float4(gk[2], 0.f, 0.f, 0.f);
        W.out[6] = make_float4(gk[3], 0.f, 0.f, 0.f);
        W.out[7] = make_float4(t.hi, t.lo, 0.f, 0.f);
      }
    }
    __syncwarp();
    if (role == 0 && lane < (GRAD ? 8 : 1) && lane != 4 && lane != 5) {
      const float4 o = W.out[lane];
      const bool bad = __float_as_int(W.out[0].w) != 0;
      const double v = bad ? CUDART_NAN : (double)o.x + (double)o.y + (double)o.z;
      if (lane == 0) {
        if (lnl_out) lnl_out[i] = v;
      } else {
        grad_out[(size_t)(lane - 1) * dp.n + i] = v;
      }
    }
    pair_sync();  // the scratch is reused by the pair's next draw
  }
}
