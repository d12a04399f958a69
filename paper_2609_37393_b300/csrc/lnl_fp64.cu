// FP64 likelihood kernels: eq. def:lnL:Decomposed evaluated term by term in
// IEEE double, one draw per thread.  This is the plain reference path of the
// library (the FP32-mixed kernels are measured against it on the same GPU).
//
// Per draw: source direction and transverse basis from (ra - gmst, dec);
// F_k = F_+ - i F_x with F_+ = p.D.p - q.D.q, F_x = 2 p.D.q; t_k = t_c - x_k.s;
// -2Y_lm(iota, phi) from the Wigner-d polynomial of the point; Q_{k,lm}(t_k) by
// the four-point Lagrange cubic on the table; then
//   T_d = x Re sum_k conj(F_k) sum_lm conj(Y_lm) Q_{k,lm}(t_k)
//   T_q = x^2/4 sum_k [|F_k|^2 Y^+ U_k Y + Re(F_k^2 Y^T V_k Y)]
// with the Hermitian and symmetric forms summed over i <= j pairs.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "common.cuh"
#include "kernels.h"

namespace rift {
namespace {

struct Fp64Out {
  double lnl;
  double td, tq;  // data sum and quadratic sum at x = 1: lnL(x) = x td - x^2 tq / 4
  int oob;
};

template <int MM>
__device__ __forceinline__ Fp64Out lnl_fp64_draw(const PointParams& P, const double2* sUV,
                                                 const DrawsParams& dp, long long i) {
  const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
  const double psi = load_param_d(dp, 2, i), incl = load_param_d(dp, 3, i);
  const double phi = load_param_d(dp, 4, i), lnD = load_param_d(dp, 5, i);
  const double tc = load_param_d(dp, 6, i);
  const int K = P.K, M = P.M;
  const double x = P.d_ref * exp(-lnD);
  double sl, cl, sd, cd;
  sincos(ra - P.gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  const double s[3] = {cd * cl, cd * sl, sd};
  const double e1[3] = {-sl, cl, 0.0};
  const double e2[3] = {-sd * cl, -sd * sl, cd};
  double s2p, c2p;
  sincos(2.0 * psi, &s2p, &c2p);

  double yr[MM], yi[MM];
  {
    double sh, ch, sp, cp;
    sincos(0.5 * incl, &sh, &ch);
    sincos(phi, &sp, &cp);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      yr[m] = yi[m] = 0.0;
      if (m < M) sylm_eval<double>(P, m, ch, sh, cp, sp, P.ycoef[m], yr[m], yi[m]);
    }
  }

  // quadratic forms a_k = Y^+ U_k Y (real) and b_k = Y^T V_k Y, all detectors
  double a[kMaxDet], br[kMaxDet], bi[kMaxDet];
#pragma unroll
  for (int k = 0; k < kMaxDet; ++k) a[k] = br[k] = bi[k] = 0.0;
#pragma unroll
  for (int m = 0; m < MM; ++m) {
#pragma unroll
    for (int n = m; n < MM; ++n) {
      if (n < M) {
        const double f = (m == n) ? 1.0 : 2.0;
        // p = conj(Y_m) Y_n, q = Y_m Y_n
        const double pr = yr[m] * yr[n] + yi[m] * yi[n];
        const double pi = yr[m] * yi[n] - yi[m] * yr[n];
        const double qr = yr[m] * yr[n] - yi[m] * yi[n];
        const double qi = yr[m] * yi[n] + yi[m] * yr[n];
#pragma unroll
        for (int k = 0; k < kMaxDet; ++k) {
          if (k < K) {
            const double2 u = sUV[(k * M + m) * M + n];
            const double2 v = sUV[K * M * M + (k * M + m) * M + n];
            a[k] = fma(f, pr * u.x - pi * u.y, a[k]);
            br[k] = fma(f, qr * v.x - qi * v.y, br[k]);
            bi[k] = fma(f, qr * v.y + qi * v.x, bi[k]);
          }
        }
      }
    }
  }

  double td = 0.0, tq = 0.0;
  int oob = 0;
  for (int k = 0; k < K; ++k) {
    const double* D = P.resp[k];
    const double fa = quad3(D, e1, e1), fb = quad3(D, e2, e2), fc = quad3(D, e1, e2);
    // F(psi) = (F_+(0) - i F_x(0)) e^{2 i psi}, F_+(0) = e1.D.e1 - e2.D.e2, F_x(0) = 2 e1.D.e2
    const double f0r = fa - fb, f0i = -2.0 * fc;
    const double Fr = f0r * c2p - f0i * s2p, Fi = f0r * s2p + f0i * c2p;
    const double tk = tc - (P.pos[k][0] * s[0] + P.pos[k][1] * s[1] + P.pos[k][2] * s[2]);
    const double u = (tk - P.t0[k]) * P.inv_dt;
    const double jf = floor(u);
    double w[4], dw[4];
    lagrange4_d(u - jf, w, dw);
    double gr = 0.0, gi = 0.0;  // sum_lm conj(Y) Q(t_k)
    if (isfinite(u)) {
      const long long j0 = (long long)jf - 1;
#pragma unroll
      for (int tap = 0; tap < 4; ++tap) {
        const long long j = j0 + tap;
        if (j < 0 || j >= P.n) {
          ++oob;
          continue;
        }
        double qr[MM], qi[MM];
        if (P.q_c128) {
          const double2* row = (const double2*)P.Q + ((long long)k * P.n + j) * M;
#pragma unroll
          for (int m = 0; m < MM; ++m)
            if (m < M) {
              double2 q = __ldg(row + m);
              qr[m] = q.x;
              qi[m] = q.y;
            }
        } else {
          const float2* row = (const float2*)P.Q + ((long long)k * P.n + j) * M;
#pragma unroll
          for (int m = 0; m < MM; ++m)
            if (m < M) {
              float2 q = __ldg(row + m);
              qr[m] = q.x;
              qi[m] = q.y;
            }
        }
        double sr = 0.0, si = 0.0;
#pragma unroll
        for (int m = 0; m < MM; ++m)
          if (m < M) {
            sr += yr[m] * qr[m] + yi[m] * qi[m];
            si += yr[m] * qi[m] - yi[m] * qr[m];
          }
        gr = fma(w[tap], sr, gr);
        gi = fma(w[tap], si, gi);
      }
    } else {
      gr = gi = CUDART_NAN;
    }
    td += Fr * gr + Fi * gi;  // Re(conj(F) G)
    double ak = 0.0, bkr = 0.0, bki = 0.0;
#pragma unroll
    for (int kk = 0; kk < kMaxDet; ++kk)
      if (kk == k) {
        ak = a[kk];
        bkr = br[kk];
        bki = bi[kk];
      }
    const double F2r = Fr * Fr - Fi * Fi, F2i = 2.0 * Fr * Fi;
    tq += (Fr * Fr + Fi * Fi) * ak + (F2r * bkr - F2i * bki);
  }
  Fp64Out o;
  o.lnl = x * td - 0.25 * x * x * tq;
  o.td = td;
  o.tq = tq;
  o.oob = oob;
  return o;
}

template <int MM, bool LSE, bool DIST = false>
__global__ void __launch_bounds__(256) lnl_fp64_kernel(const PointParams* __restrict__ gP,
                                                       DrawsParams dp, double* __restrict__ lnl_out,
                                                       LseState* __restrict__ partials,
                                                       unsigned long long* __restrict__ oob_count,
                                                       DistParams dist = DistParams{}) {
  __shared__ PointParams P;
  extern __shared__ double2 sUV[];
  stage_point(P, gP);
  __syncthreads();
  {
    const int nuv = 2 * P.K * P.M * P.M;
    for (int t = threadIdx.x; t < nuv; t += blockDim.x) sUV[t] = __ldg(P.U + t);  // U then V
  }
  __syncthreads();
  ThreadLse64 st = tlse64_init();
  int oob = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    Fp64Out o = lnl_fp64_draw<MM>(P, sUV, dp, i);
    oob += o.oob;
    if (DIST && !isnan(o.lnl)) {
      // lnL(x) = K x - R x^2/2 with K = td, R = tq/2 (eq. ap:dexp), summed on the nodes
      const double K = o.td, Rq = 0.5 * o.tq;
      double peak;
      const double nodes = dist_lse(dist, K, Rq, Rq > 0.0 ? K / Rq : 0.0, &peak);
      o.lnl = peak + nodes;
    }
    if (!LSE) {
      lnl_out[i] = o.lnl;
    } else {
      tlse64_push(st, o.lnl + load_logw_d(dp, i));
    }
  }
  if (LSE) block_lse64_write(st, partials + blockIdx.x);
  if (oob_count) {
    for (int off = 16; off > 0; off >>= 1) oob += __shfl_down_sync(0xffffffffu, oob, off);
    if ((threadIdx.x & 31) == 0 && oob) atomicAdd(oob_count, (unsigned long long)oob);
  }
}

template <int MM, bool LSE>
cudaError_t launch_fp64_dist_k(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                               const DistParams& dist, double* lnl_out, LseState* partials,
                               unsigned long long* oob, int* blocks, cudaStream_t st) {
  const size_t smem = (size_t)2 * hp.K * hp.M * hp.M * sizeof(double2);
  auto kern = lnl_fp64_kernel<MM, LSE, true>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  *blocks = grid_cap(grid_for(kern, 256, smem), dp.n, 256);
  kern<<<*blocks, 256, smem, st>>>(dP, dp, lnl_out, partials, oob, dist);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_fp64_dist_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                const DistParams& dist, double* lnl_out, LseState* partials,
                                unsigned long long* oob, int* blocks, cudaStream_t st) {
  if (partials) return launch_fp64_dist_k<MM, true>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  return launch_fp64_dist_k<MM, false>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
}

template <int MM, bool LSE>
cudaError_t launch_fp64_k(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                          double* lnl_out, LseState* partials, unsigned long long* oob,
                          int* blocks, cudaStream_t st) {
  const size_t smem = (size_t)2 * hp.K * hp.M * hp.M * sizeof(double2);
  cudaFuncSetAttribute(lnl_fp64_kernel<MM, LSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  *blocks = grid_cap(grid_for(lnl_fp64_kernel<MM, LSE>, 256, smem), dp.n, 256);
  lnl_fp64_kernel<MM, LSE><<<*blocks, 256, smem, st>>>(dP, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_fp64_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                           double* lnl_out, LseState* partials, unsigned long long* oob,
                           int* blocks, cudaStream_t st) {
  if (partials) return launch_fp64_k<MM, true>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_fp64_k<MM, false>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

// ---------------------------------------------------------------- gradient

// lnL and d lnL / d(ra, dec, psi, iota, phase, lnD, t_c) of one draw in FP64,
// the chain rule of eq. def:lnL:Decomposed written out:
//   T_d = x sum_k Re(conj F_k G_k), G_k = sum_lm conj(Y_lm) Q_k,lm(t_k),
//   T_q = x^2/4 sum_k [|F_k|^2 a_k + Re(F_k^2 b_k)], a_k = Y^+ U_k Y, b_k = Y^T V_k Y,
// with dF_k from the derivatives of the transverse basis, dY/d phase = i m Y,
// dY/d iota from the Wigner-d polynomial, dQ/dt from the cubic's slope, and
// da_k = 2 Re(dY^+ U_k Y), db_k = 2 dY^T V_k Y (U Hermitian, V symmetric as
// eq. QUV makes them).
// With raw != NULL the x-free sums are also returned: raw[0] = T_d/x,
// raw[1] = 4 T_q/x^2, raw[2..8] = their derivatives of T_d/x, raw[9..15] of
// 4 T_q / x^2 (slot 5, lnD, excluded).
template <int MM>
__device__ __forceinline__ double lnl_fp64_grad_draw(const PointParams& P, const double2* sUV,
                                                     const DrawsParams& dp, long long i,
                                                     double g[kNpar], double* raw = nullptr) {
  const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
  const double psi = load_param_d(dp, 2, i), incl = load_param_d(dp, 3, i);
  const double phi = load_param_d(dp, 4, i), lnD = load_param_d(dp, 5, i);
  const double tc = load_param_d(dp, 6, i);
  const int K = P.K, M = P.M;
  const double x = P.d_ref * exp(-lnD);
  double sl, cl, sd, cd;
  sincos(ra - P.gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  const double s[3] = {cd * cl, cd * sl, sd};
  const double ds_ra[3] = {-cd * sl, cd * cl, 0.0};
  const double ds_dec[3] = {-sd * cl, -sd * sl, cd};
  const double e1[3] = {-sl, cl, 0.0};
  const double e2[3] = {-sd * cl, -sd * sl, cd};
  const double de1_ra[3] = {-cl, -sl, 0.0};
  const double de2_ra[3] = {sd * sl, -sd * cl, 0.0};
  const double de2_dec[3] = {-cd * cl, -cd * sl, -sd};
  double s2p, c2p;
  sincos(2.0 * psi, &s2p, &c2p);

  double yr[MM], yi[MM], dyr[MM], dyi[MM];
  {
    double sh, ch, sp, cp;
    sincos(0.5 * incl, &sh, &ch);
    sincos(phi, &sp, &cp);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      yr[m] = yi[m] = dyr[m] = dyi[m] = 0.0;
      if (m < M) {
        sylm_eval<double>(P, m, ch, sh, cp, sp, P.ycoef[m], yr[m], yi[m]);
        const int em = P.em[m];
        const double damp = sylm_damp_dincl(P, m, ch, sh);
        double er = 1.0, ei = 0.0;
        const int am = em < 0 ? -em : em;
        for (int u = 0; u < am; ++u) {
          const double nr = er * cp - ei * sp, ni = er * sp + ei * cp;
          er = nr;
          ei = ni;
        }
        if (em < 0) ei = -ei;
        dyr[m] = damp * er;
        dyi[m] = damp * ei;
      }
    }
  }

  double td = 0.0, tq = 0.0;
  double gd[kNpar], gq[kNpar];
#pragma unroll
  for (int p = 0; p < kNpar; ++p) gd[p] = gq[p] = 0.0;
  for (int k = 0; k < K; ++k) {
    const double* D = P.resp[k];
    // F(0) = e1.D.e1 - e2.D.e2 - 2 i e1.D.e2 and its ra, dec derivatives
    const double f0r = quad3(D, e1, e1) - quad3(D, e2, e2), f0i = -2.0 * quad3(D, e1, e2);
    const double f0r_ra = 2.0 * quad3(D, de1_ra, e1) - 2.0 * quad3(D, de2_ra, e2);
    const double f0i_ra = -2.0 * (quad3(D, de1_ra, e2) + quad3(D, e1, de2_ra));
    const double f0r_dec = -2.0 * quad3(D, de2_dec, e2);
    const double f0i_dec = -2.0 * quad3(D, e1, de2_dec);
    const double Fr = f0r * c2p - f0i * s2p, Fi = f0r * s2p + f0i * c2p;
    const double Fr_ra = f0r_ra * c2p - f0i_ra * s2p, Fi_ra = f0r_ra * s2p + f0i_ra * c2p;
    const double Fr_dec = f0r_dec * c2p - f0i_dec * s2p, Fi_dec = f0r_dec * s2p + f0i_dec * c2p;
    const double Fr_psi = -2.0 * Fi, Fi_psi = 2.0 * Fr;
    const double tk = tc - (P.pos[k][0] * s[0] + P.pos[k][1] * s[1] + P.pos[k][2] * s[2]);
    const double dt_ra = -(P.pos[k][0] * ds_ra[0] + P.pos[k][1] * ds_ra[1]);
    const double dt_dec = -(P.pos[k][0] * ds_dec[0] + P.pos[k][1] * ds_dec[1] + P.pos[k][2] * ds_dec[2]);
    const double u = (tk - P.t0[k]) * P.inv_dt;
    const double jf = floor(u);
    double w[4], dw[4];
    lagrange4_d(u - jf, w, dw);
    // G = sum conj(Y) Q, Gt = sum conj(Y) dQ/dt, Gi = sum conj(dY_iota) Q, Gp = sum conj(dY_phase) Q
    double Gr = 0, Gi_ = 0, Gtr = 0, Gti = 0, Gir = 0, Gii = 0, Gpr = 0, Gpi = 0;
    if (isfinite(u)) {
      const long long j0 = (long long)jf - 1;
      for (int tap = 0; tap < 4; ++tap) {
        const long long j = j0 + tap;
        if (j < 0 || j >= P.n) continue;
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          if (m < M) {
            double qr, qi;
            if (P.q_c128) {
              const double2 q = __ldg((const double2*)P.Q + ((long long)k * P.n + j) * M + m);
              qr = q.x;
              qi = q.y;
            } else {
              const float2 q = __ldg((const float2*)P.Q + ((long long)k * P.n + j) * M + m);
              qr = q.x;
              qi = q.y;
            }
            const double wq = w[tap], dq = dw[tap] * P.inv_dt;
            const double cr = yr[m] * qr + yi[m] * qi, ci = yr[m] * qi - yi[m] * qr;  // conj(Y) Q
            Gr = fma(wq, cr, Gr);
            Gi_ = fma(wq, ci, Gi_);
            Gtr = fma(dq, cr, Gtr);
            Gti = fma(dq, ci, Gti);
            Gir = fma(wq, dyr[m] * qr + dyi[m] * qi, Gir);
            Gii = fma(wq, dyr[m] * qi - dyi[m] * qr, Gii);
            const double em = (double)P.em[m];  // dY/d phase = i m Y: conj = -i m conj(Y)
            Gpr = fma(wq, em * ci, Gpr);
            Gpi = fma(wq, -em * cr, Gpi);
          }
        }
      }
    } else {
      Gr = CUDART_NAN;
    }
    // data term and its derivatives: Re(conj(A) B) = Ar Br + Ai Bi
    const double dre = Fr * Gr + Fi * Gi_;
    td += dre;
    const double dt_term = Fr * Gtr + Fi * Gti;
    gd[0] += Fr_ra * Gr + Fi_ra * Gi_ + dt_term * dt_ra;
    gd[1] += Fr_dec * Gr + Fi_dec * Gi_ + dt_term * dt_dec;
    gd[2] += Fr_psi * Gr + Fi_psi * Gi_;
    gd[3] += Fr * Gir + Fi * Gii;
    gd[4] += Fr * Gpr + Fi * Gpi;
    gd[6] += dt_term;
    // quadratic forms: rows (U Y)_m and (V Y)_m formed on the fly
    const double2* Uk = sUV + (size_t)k * M * M;
    const double2* Vk = sUV + (size_t)K * M * M + (size_t)k * M * M;
    double a = 0, da_i = 0, da_p = 0, br = 0, bi = 0, dbi_r = 0, dbi_i = 0, dbp_r = 0, dbp_i = 0;
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      if (m < M) {
        double uyr = 0, uyi = 0, vyr = 0, vyi = 0;
#pragma unroll
        for (int n2 = 0; n2 < MM; ++n2) {
          if (n2 < M) {
            const double2 uu = Uk[m * M + n2], vv = Vk[m * M + n2];
            uyr += uu.x * yr[n2] - uu.y * yi[n2];
            uyi += uu.x * yi[n2] + uu.y * yr[n2];
            vyr += vv.x * yr[n2] - vv.y * yi[n2];
            vyi += vv.x * yi[n2] + vv.y * yr[n2];
          }
        }
        const double em = (double)P.em[m];
        const double pyr = -em * yi[m], pyi = em * yr[m];  // dY/d phase
        a += yr[m] * uyr + yi[m] * uyi;                    // Re(conj(Y) UY)
        da_i += 2.0 * (dyr[m] * uyr + dyi[m] * uyi);
        da_p += 2.0 * (pyr * uyr + pyi * uyi);
        br += yr[m] * vyr - yi[m] * vyi;                   // Y (VY)
        bi += yr[m] * vyi + yi[m] * vyr;
        dbi_r += 2.0 * (dyr[m] * vyr - dyi[m] * vyi);
        dbi_i += 2.0 * (dyr[m] * vyi + dyi[m] * vyr);
        dbp_r += 2.0 * (pyr * vyr - pyi * vyi);
        dbp_i += 2.0 * (pyr * vyi + pyi * vyr);
      }
    }
    const double F2 = Fr * Fr + Fi * Fi, F2r = Fr * Fr - Fi * Fi, F2i = 2.0 * Fr * Fi;
    tq += F2 * a + (F2r * br - F2i * bi);
    // d(|F|^2) = 2 Re(conj F dF);  d(F^2 b) = 2 F dF b
    auto quad_dF = [&](double dFr, double dFi) {
      const double dF2 = 2.0 * (Fr * dFr + Fi * dFi);
      const double pr = 2.0 * (Fr * dFr - Fi * dFi), pi = 2.0 * (Fr * dFi + Fi * dFr);  // 2 F dF
      return dF2 * a + (pr * br - pi * bi);
    };
    gq[0] += quad_dF(Fr_ra, Fi_ra);
    gq[1] += quad_dF(Fr_dec, Fi_dec);
    gq[2] += quad_dF(Fr_psi, Fi_psi);
    gq[3] += F2 * da_i + (F2r * dbi_r - F2i * dbi_i);
    gq[4] += F2 * da_p + (F2r * dbp_r - F2i * dbp_i);
  }
  const double q4 = 0.25 * x * x;
#pragma unroll
  for (int p = 0; p < kNpar; ++p) g[p] = x * gd[p] - q4 * gq[p];
  g[5] = -x * td + 2.0 * q4 * tq;
  if (raw) {
    raw[0] = td;
    raw[1] = tq;
    for (int p = 0; p < kNpar; ++p) {
      raw[2 + p] = gd[p];
      raw[9 + p] = gq[p];
    }
  }
  return x * td - q4 * tq;
}

template <int MM, bool DIST = false>
__global__ void __launch_bounds__(256) grad_fp64_kernel(const PointParams* __restrict__ gP,
                                                        DrawsParams dp, double* __restrict__ lnl_out,
                                                        double* __restrict__ grad_out,
                                                        DistParams dist = DistParams{}) {
  __shared__ PointParams P;
  extern __shared__ double2 sUV[];
  stage_point(P, gP);
  __syncthreads();
  {
    const int nuv = 2 * P.K * P.M * P.M;
    for (int t = threadIdx.x; t < nuv; t += blockDim.x) sUV[t] = __ldg(P.U + t);
  }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    double g[kNpar];
    double v;
    if (DIST) {
      // lnL(x) = K x - R x^2 / 2 with K = T_d/x, R = T_q/(2 x^2) ... in raw
      // sums: K = raw[0], R = raw[1]/2; gradient E[x] dK - E[x^2] dR / 2
      double raw[16];
      const double v0 = lnl_fp64_grad_draw<MM>(P, sUV, dp, i, g, raw);
      const double K = raw[0], Rq = 0.5 * raw[1];
      double peak, ex[2] = {0.0, 0.0};
      const double nodes = dist_lse(dist, K, Rq, Rq > 0.0 ? K / Rq : 0.0, &peak, ex);
      v = isnan(v0) ? v0 : peak + nodes;
      for (int p = 0; p < kNpar; ++p) g[p] = ex[0] * raw[2 + p] - 0.25 * ex[1] * raw[9 + p];
      g[5] = 0.0;
    } else {
      v = lnl_fp64_grad_draw<MM>(P, sUV, dp, i, g);
    }
    if (lnl_out) lnl_out[i] = v;
#pragma unroll
    for (int p = 0; p < kNpar; ++p) grad_out[(size_t)p * dp.n + i] = g[p];
  }
}

template <int MM>
cudaError_t launch_grad_fp64_mm(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                double* lnl_out, double* grad_out, cudaStream_t st) {
  const size_t smem = (size_t)2 * hp.K * hp.M * hp.M * sizeof(double2);
  cudaFuncSetAttribute(grad_fp64_kernel<MM>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  const int blocks = grid_cap(grid_for(grad_fp64_kernel<MM>, 256, smem), dp.n, 256);
  grad_fp64_kernel<MM><<<blocks, 256, smem, st>>>(dP, dp, lnl_out, grad_out);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_grad_fp64_dist_mm(const PointParams& hp, const PointParams* dP,
                                     const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                     double* grad_out, cudaStream_t st) {
  const size_t smem = (size_t)2 * hp.K * hp.M * hp.M * sizeof(double2);
  auto kern = grad_fp64_kernel<MM, true>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  const int blocks = grid_cap(grid_for(kern, 256, smem), dp.n, 256);
  kern<<<blocks, 256, smem, st>>>(dP, dp, lnl_out, grad_out, dist);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_grad_fp64_dist(const PointParams& hp, const PointParams* dP,
                                  const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                  double* grad_out, cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_grad_fp64_dist_mm<2>(hp, dP, dp, dist, lnl_out, grad_out, st);
  if (M <= 4) return launch_grad_fp64_dist_mm<4>(hp, dP, dp, dist, lnl_out, grad_out, st);
  if (M <= 6) return launch_grad_fp64_dist_mm<6>(hp, dP, dp, dist, lnl_out, grad_out, st);
  if (M <= 8) return launch_grad_fp64_dist_mm<8>(hp, dP, dp, dist, lnl_out, grad_out, st);
  if (M <= 10) return launch_grad_fp64_dist_mm<10>(hp, dP, dp, dist, lnl_out, grad_out, st);
  if (M <= 12) return launch_grad_fp64_dist_mm<12>(hp, dP, dp, dist, lnl_out, grad_out, st);
  return launch_grad_fp64_dist_mm<16>(hp, dP, dp, dist, lnl_out, grad_out, st);
}

cudaError_t launch_grad_fp64(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                             double* lnl_out, double* grad_out, cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_grad_fp64_mm<2>(hp, dP, dp, lnl_out, grad_out, st);
  if (M <= 4) return launch_grad_fp64_mm<4>(hp, dP, dp, lnl_out, grad_out, st);
  if (M <= 6) return launch_grad_fp64_mm<6>(hp, dP, dp, lnl_out, grad_out, st);
  if (M <= 8) return launch_grad_fp64_mm<8>(hp, dP, dp, lnl_out, grad_out, st);
  if (M <= 10) return launch_grad_fp64_mm<10>(hp, dP, dp, lnl_out, grad_out, st);
  if (M <= 12) return launch_grad_fp64_mm<12>(hp, dP, dp, lnl_out, grad_out, st);
  return launch_grad_fp64_mm<16>(hp, dP, dp, lnl_out, grad_out, st);
}

namespace {
}  // namespace

cudaError_t launch_lnl_fp64_dist(const PointParams& hp, const PointParams* dP,
                                 const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                 LseState* partials, unsigned long long* oob, int* blocks,
                                 cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_fp64_dist_mm<2>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  if (M <= 4) return launch_fp64_dist_mm<4>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  if (M <= 6) return launch_fp64_dist_mm<6>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  if (M <= 8) return launch_fp64_dist_mm<8>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  if (M <= 10) return launch_fp64_dist_mm<10>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  if (M <= 12) return launch_fp64_dist_mm<12>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
  return launch_fp64_dist_mm<16>(hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
}

cudaError_t launch_lnl_fp64(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                            double* lnl_out, LseState* partials, unsigned long long* oob,
                            int* blocks, cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_fp64_mm<2>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 4) return launch_fp64_mm<4>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 6) return launch_fp64_mm<6>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 8) return launch_fp64_mm<8>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 10) return launch_fp64_mm<10>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 12) return launch_fp64_mm<12>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_fp64_mm<16>(hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

namespace {

template <int MM, bool LSE>
cudaError_t launch_fp64_k_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                              double* lnl_out, LseState* partials, unsigned long long* oob,
                              int sms, int* blocks, cudaStream_t st) {
  const size_t smem = (size_t)2 * hp.K * hp.M * hp.M * sizeof(double2);
  cudaFuncSetAttribute(lnl_fp64_kernel<MM, LSE>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  *blocks = grid_cap(grid_for_sms(lnl_fp64_kernel<MM, LSE>, 256, smem, sms), dp.n, 256);
  lnl_fp64_kernel<MM, LSE><<<*blocks, 256, smem, st>>>(dP, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_fp64_mm_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                               double* lnl_out, LseState* partials, unsigned long long* oob,
                               int sms, int* blocks, cudaStream_t st) {
  if (partials) return launch_fp64_k_sms<MM, true>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  return launch_fp64_k_sms<MM, false>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
}

}  // namespace

cudaError_t launch_lnl_fp64_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                double* lnl_out, LseState* partials, unsigned long long* oob,
                                int sms, int* blocks, cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_fp64_mm_sms<2>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  if (M <= 4) return launch_fp64_mm_sms<4>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  if (M <= 6) return launch_fp64_mm_sms<6>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  if (M <= 8) return launch_fp64_mm_sms<8>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  if (M <= 10) return launch_fp64_mm_sms<10>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  if (M <= 12) return launch_fp64_mm_sms<12>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
  return launch_fp64_mm_sms<16>(hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
}

}  // namespace rift
