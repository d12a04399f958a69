// Adjoint of the composite-index likelihood (Sec. III with the chain rule of
// Sec. II.B), FP64, one draw per thread: lnL and d lnL / d(ra, dec, psi,
// incl, phase, lnD, t_c).
//
// Coefficients.  The derivatives of C~^k_a are carried analytically beside
// the values:
// * psi: every coefficient is proportional to e^{2 i psi}, so dC~ = 2i C~;
// * t_c: only through the post-phase, dC~_(p,n) = i n Omega C~ (rotation);
// * ra: C_(0,n) is proportional to e^{i n g}, g = gmst - ra, so dC_(0,n) =
//   -i n C_(0,n); the drift harmonics move with w = (x + i y) e^{i g}; the
//   powers of the drift follow dP^(p) = dP^(p-1) * E + P^(p-1) * dE; the
//   arrival time adds i n Omega (dt_k/d ra) C~;
// * dec: the five bilinear forms through (1 +- sin dec)/2 and cos dec, the
//   drift through cos dec, the arrival time as for ra;
// * finite arms: b_p from the derivatives of the arm projections of e1, e2, s.
// Harmonics: dY/d phase = i m Y, dY/d incl from the Goldberg sum.
//
// Data term: per response index a the tap sums of conj(Y) Q, of conj(Y) dQ/dt
// (the cubic's slope), and of conj(dY) Q for incl and phase.
// Quadratic term: T = sum_{a <= b} z_a^T S_ab z_b over the stored blocks (S the
// folded real form, off-diagonal blocks doubled), so that
// dT = sum_{a <= b} (dz_a . S_ab z_b + dz_b . S_ab^T z_a).  With
// u = S_ab z_b and v = S_ab^T z_a written as complex M-vectors, dz . u =
// Re(conj(dC_a) sum_i conj(Y_i) u_i) for a coefficient parameter and
// Re(conj(C_a) sum_i conj(dY_i) u_i) for a harmonic one, so each block costs
// two M x 2M matrix-vector products and a few complex dot products.
#include <cuda_runtime.h>
#include <math_constants.h>

#include "comp.cuh"
#include "common.cuh"
#include "kernels.h"

namespace rift {
namespace {

constexpr int kPsi = 2, kRa = 0, kDec = 1, kTc = 3;  // slots of dC: ra, dec, psi, t_c
constexpr int kClassCoefGrad = 64;  // detectors x response indices kept for the class pass

// C~^k_a and dC~^k_a / d(ra, dec, psi, t_c) of one detector.
__device__ void comp_coeffs_grad(const CompParams& C, int k, const CompDraw& g, double tk,
                                 double dtk_ra, double dtk_dec, double2* out, double2 (*dout)[4]) {
  const int na = C.na;
  if (C.kind == RIFT_ILE_RESP_FINITE_ARM) {
    const double* X = C.armx[k];
    const double* Yv = C.army[k];
    const double ax = dot3(g.e1, X), bx = dot3(g.e2, X), ux = dot3(g.s, X);
    const double ay = dot3(g.e1, Yv), by = dot3(g.e2, Yv), uy = dot3(g.s, Yv);
    // derivatives of (a, b, u) for ra and dec
    const double dax[2] = {dot3(g.de1_ra, X), 0.0}, dbx[2] = {dot3(g.de2_ra, X), dot3(g.de2_dec, X)};
    const double dux[2] = {dot3(g.ds_ra, X), dot3(g.ds_dec, X)};
    const double day[2] = {dot3(g.de1_ra, Yv), 0.0}, dby[2] = {dot3(g.de2_ra, Yv), dot3(g.de2_dec, Yv)};
    const double duy[2] = {dot3(g.ds_ra, Yv), dot3(g.ds_dec, Yv)};
    const double2 e2p = make_double2(g.c2p, g.s2p);
    // q = e^{2 i psi} (a - i b)^2, dq = e^{2 i psi} 2 (a - i b)(da - i db)
    const double2 qx = cmul(e2p, make_double2(ax * ax - bx * bx, -2.0 * ax * bx));
    const double2 qy = cmul(e2p, make_double2(ay * ay - by * by, -2.0 * ay * by));
    double2 dqx[2], dqy[2];
    for (int j = 0; j < 2; ++j) {
      dqx[j] = cmul(e2p, cmul(make_double2(2.0 * ax, -2.0 * bx), make_double2(dax[j], -dbx[j])));
      dqy[j] = cmul(e2p, cmul(make_double2(2.0 * ay, -2.0 * by), make_double2(day[j], -dby[j])));
    }
    double px = 0.5, py = 0.5, pxm = 0.0, pym = 0.0;  // u^p / 2 and p u^(p-1) / 2
    for (int p = 0; p < na; ++p) {
      out[p] = make_double2(px * qx.x - py * qy.x, px * qx.y - py * qy.y);
      for (int j = 0; j < 2; ++j) {
        const double cx = pxm * dux[j], cy = pym * duy[j];
        dout[p][j] = make_double2(cx * qx.x + px * dqx[j].x - cy * qy.x - py * dqy[j].x,
                                  cx * qx.y + px * dqx[j].y - cy * qy.y - py * dqy[j].y);
      }
      dout[p][kPsi] = make_double2(-2.0 * out[p].y, 2.0 * out[p].x);
      dout[p][kTc] = make_double2(0.0, 0.0);
      pxm = (p + 1) * px;
      pym = (p + 1) * py;
      px *= ux;
      py *= uy;
    }
    return;
  }
  const double* D = C.resp[k];  // xx, xy, xz, yy, yz, zz
  const double sd = g.sd, cd = g.cd;
  const double al = 0.5 * (1.0 + sd), be = 0.5 * (1.0 - sd);
  const double dal = 0.5 * cd, dbe = -0.5 * cd, dcd = -sd;  // d/d dec
  double2 A[5], dA[5];  // n = -2..2 before e^{2 i psi}; dA = d/d dec
  A[0] = make_double2(al * al * (D[3] - D[0]), 2.0 * al * al * D[1]);
  dA[0] = make_double2(2.0 * al * dal * (D[3] - D[0]), 4.0 * al * dal * D[1]);
  A[4] = make_double2(be * be * (D[3] - D[0]), -2.0 * be * be * D[1]);
  dA[4] = make_double2(2.0 * be * dbe * (D[3] - D[0]), -4.0 * be * dbe * D[1]);
  A[1] = make_double2(2.0 * al * cd * D[2], -2.0 * al * cd * D[4]);
  {
    const double f = 2.0 * (dal * cd + al * dcd);
    dA[1] = make_double2(f * D[2], -f * D[4]);
  }
  A[3] = make_double2(-2.0 * be * cd * D[2], -2.0 * be * cd * D[4]);
  {
    const double f = 2.0 * (dbe * cd + be * dcd);
    dA[3] = make_double2(-f * D[2], -f * D[4]);
  }
  A[2] = make_double2(2.0 * al * be * (D[0] + D[3]) - cd * cd * D[5], 0.0);
  dA[2] = make_double2(2.0 * (dal * be + al * dbe) * (D[0] + D[3]) - 2.0 * cd * dcd * D[5], 0.0);
  const double2 eg = make_double2(g.cg, g.sg);
  const double2 e2p = make_double2(g.c2p, g.s2p);
  double2 egn[5];  // e^{i n g}, n = -2..2
  egn[2] = make_double2(1.0, 0.0);
  egn[3] = eg;
  egn[4] = cmul(eg, eg);
  egn[1] = make_double2(eg.x, -eg.y);
  egn[0] = make_double2(egn[4].x, -egn[4].y);
  double2 C0[5], dC0[2][5];  // dC0[0]: d/d ra, dC0[1]: d/d dec
  for (int j = 0; j < 5; ++j) {
    const int n = j - 2;
    C0[j] = cmul(cmul(e2p, A[j]), egn[j]);
    dC0[0][j] = make_double2(n * C0[j].y, -n * C0[j].x);  // -i n C0
    dC0[1][j] = cmul(cmul(e2p, dA[j]), egn[j]);
  }
  // drift harmonics m = -1, 0, 1 and their ra, dec derivatives
  const double* x = C.pos[k];
  const double2 w = cmul(make_double2(x[0], x[1]), eg);
  const double2 E[3] = {make_double2(0.5 * cd * w.x, -0.5 * cd * w.y), make_double2(-cd * w.x, 0.0),
                        make_double2(0.5 * cd * w.x, 0.5 * cd * w.y)};
  const double2 dE[2][3] = {
      {make_double2(-E[0].y, E[0].x), make_double2(-cd * w.y, 0.0), make_double2(E[2].y, -E[2].x)},
      {make_double2(0.5 * dcd * w.x, -0.5 * dcd * w.y), make_double2(-dcd * w.x, 0.0),
       make_double2(0.5 * dcd * w.x, 0.5 * dcd * w.y)}};
  double so, co;
  sincos(C.omega * tk, &so, &co);
  const double2 ep = make_double2(co, so);
  const double dtk[2] = {dtk_ra, dtk_dec};
  double2 P[2 * RIFT_ILE_MAX_ROT_PMAX + 1], dP[2][2 * RIFT_ILE_MAX_ROT_PMAX + 1];
  P[0] = make_double2(1.0, 0.0);
  dP[0][0] = dP[1][0] = make_double2(0.0, 0.0);
  int off = 0;
  double inv_fact = 1.0;
  for (int p = 0; p <= C.p_max; ++p) {
    if (p > 0) {
      inv_fact /= (double)p;
      double2 Pn[2 * RIFT_ILE_MAX_ROT_PMAX + 1], dPn[2][2 * RIFT_ILE_MAX_ROT_PMAX + 1];
      for (int j = 0; j < 2 * p + 1; ++j) {
        double2 acc = make_double2(0.0, 0.0), dacc[2] = {acc, acc};
        for (int e = 0; e < 3; ++e) {
          const int src = j - e;
          if (src >= 0 && src < 2 * p - 1) {
            const double2 t = cmul(P[src], E[e]);
            acc.x += t.x;
            acc.y += t.y;
            for (int v = 0; v < 2; ++v) {
              const double2 t1 = cmul(dP[v][src], E[e]), t2 = cmul(P[src], dE[v][e]);
              dacc[v].x += t1.x + t2.x;
              dacc[v].y += t1.y + t2.y;
            }
          }
        }
        Pn[j] = acc;
        dPn[0][j] = dacc[0];
        dPn[1][j] = dacc[1];
      }
      for (int j = 0; j < 2 * p + 1; ++j) {
        P[j] = Pn[j];
        dP[0][j] = dPn[0][j];
        dP[1][j] = dPn[1][j];
      }
    }
    const int width = 2 * (2 + p) + 1;
    double2 ph = make_double2(1.0, 0.0);
    for (int q = 0; q < 2 + p; ++q) ph = cmul(ph, make_double2(ep.x, -ep.y));
    for (int j = 0; j < width; ++j) {
      const int nn = j - (2 + p);
      double2 acc = make_double2(0.0, 0.0), dacc[2] = {acc, acc};
      for (int n = -2; n <= 2; ++n) {
        const int m = nn - n;
        if (m >= -p && m <= p) {
          const double2 t = cmul(C0[n + 2], P[m + p]);
          acc.x += t.x;
          acc.y += t.y;
          for (int v = 0; v < 2; ++v) {
            const double2 t1 = cmul(dC0[v][n + 2], P[m + p]), t2 = cmul(C0[n + 2], dP[v][m + p]);
            dacc[v].x += t1.x + t2.x;
            dacc[v].y += t1.y + t2.y;
          }
        }
      }
      const double2 c = cmul(make_double2(acc.x * inv_fact, acc.y * inv_fact), ph);
      out[off + j] = c;
      // i nn Omega c: the post-phase's t_k derivative
      const double2 ct = make_double2(-nn * C.omega * c.y, nn * C.omega * c.x);
      for (int v = 0; v < 2; ++v) {
        const double2 d = cmul(make_double2(dacc[v].x * inv_fact, dacc[v].y * inv_fact), ph);
        dout[off + j][v] = make_double2(d.x + dtk[v] * ct.x, d.y + dtk[v] * ct.y);
      }
      dout[off + j][kPsi] = make_double2(-2.0 * c.y, 2.0 * c.x);
      dout[off + j][kTc] = ct;
      ph = cmul(ph, ep);
    }
    off += width;
  }
}

// lnL of one draw and its gradient g[7] (ra, dec, psi, incl, phase, lnD, t_c).
template <int MM>
__device__ double comp_grad_draw(const CompParams& C, const PointParams& P, const DrawsParams& dp,
                                 long long i, double gout[kNpar]) {
  const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
  const double psi = load_param_d(dp, 2, i), incl = load_param_d(dp, 3, i);
  const double phi = load_param_d(dp, 4, i), lnD = load_param_d(dp, 5, i);
  const double tc = load_param_d(dp, 6, i);
  const int M = C.M, na = C.na, A = C.A;
  const double x = C.d_ref * exp(-lnD);
  const CompDraw g = comp_geometry(C, ra, dec, psi);

  // Y, dY/d incl, dY/d phase (= i m Y)
  double yr[MM], yi[MM], ir[MM], ii[MM], pr[MM], pi[MM];
  {
    double sh, ch, sp, cp;
    sincos(0.5 * incl, &sh, &ch);
    sincos(phi, &sp, &cp);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      yr[m] = yi[m] = ir[m] = ii[m] = pr[m] = pi[m] = 0.0;
      if (m < M) {
        sylm_eval<double>(P, m, ch, sh, cp, sp, P.ycoef[m], yr[m], yi[m]);
        const double damp = sylm_damp_dincl(P, m, ch, sh);
        double er = 1.0, ei = 0.0;  // e^{i m phi}
        const int em = P.em[m], am = em < 0 ? -em : em;
        for (int u = 0; u < am; ++u) {
          const double nr = er * cp - ei * sp, ni = er * sp + ei * cp;
          er = nr;
          ei = ni;
        }
        if (em < 0) ei = -ei;
        ir[m] = damp * er;
        ii[m] = damp * ei;
        pr[m] = -em * yi[m];
        pi[m] = em * yr[m];
      }
    }
  }

  double td = 0.0, tq = 0.0, gd[kNpar], gq[kNpar];
  // coefficients of all detectors kept locally: the quadratic forms are then
  // formed once per detector class (below)
  const bool by_class = C.K * na <= kClassCoefGrad;
  double2 cfs[kClassCoefGrad], dcfs[kClassCoefGrad][4];
  bool bad = false;  // an arrival time that is not finite
#pragma unroll
  for (int p = 0; p < kNpar; ++p) gd[p] = gq[p] = 0.0;
  for (int k = 0; k < C.K; ++k) {
    const double tk = tc - dot3(C.pos[k], g.s);
    const double dtk_ra = -dot3(C.pos[k], g.ds_ra), dtk_dec = -dot3(C.pos[k], g.ds_dec);
    double2 cf[kMaxRespIdx], dcf[kMaxRespIdx][4];
    comp_coeffs_grad(C, k, g, tk, dtk_ra, dtk_dec, cf, dcf);

    // data term
    const double u = (tk - C.t0[k]) * C.inv_dt;
    if (!isfinite(u)) {
      bad = true;
    } else {
      const double jf = floor(u);
      double w[4], dw[4];
      lagrange4_d(u - jf, w, dw);
      const long long j0 = (long long)jf - 1;
      for (int a = 0; a < na; ++a) {
        double2 G0 = make_double2(0.0, 0.0), Gt = G0, Gi = G0, Gp = G0;
#pragma unroll
        for (int tap = 0; tap < 4; ++tap) {
          const long long j = j0 + tap;
          if (j < 0 || j >= C.n) continue;
          const double2* row = C.Q + ((long long)k * C.n + j) * A + (long long)a * M;
          const double wq = w[tap], dq = dw[tap] * C.inv_dt;
#pragma unroll
          for (int m = 0; m < MM; ++m)
            if (m < M) {
              const double2 q = __ldg(row + m);
              const double cr = yr[m] * q.x + yi[m] * q.y, ci = yr[m] * q.y - yi[m] * q.x;
              G0.x = fma(wq, cr, G0.x);
              G0.y = fma(wq, ci, G0.y);
              Gt.x = fma(dq, cr, Gt.x);
              Gt.y = fma(dq, ci, Gt.y);
              Gi.x = fma(wq, ir[m] * q.x + ii[m] * q.y, Gi.x);
              Gi.y = fma(wq, ir[m] * q.y - ii[m] * q.x, Gi.y);
              Gp.x = fma(wq, pr[m] * q.x + pi[m] * q.y, Gp.x);
              Gp.y = fma(wq, pr[m] * q.y - pi[m] * q.x, Gp.y);
            }
        }
        // Re(conj(c) G) = c.x G.x + c.y G.y
        const double2 c = cf[a];
        td += c.x * G0.x + c.y * G0.y;
        const double slope = c.x * Gt.x + c.y * Gt.y;
        gd[0] += dcf[a][kRa].x * G0.x + dcf[a][kRa].y * G0.y + dtk_ra * slope;
        gd[1] += dcf[a][kDec].x * G0.x + dcf[a][kDec].y * G0.y + dtk_dec * slope;
        gd[2] += dcf[a][kPsi].x * G0.x + dcf[a][kPsi].y * G0.y;
        gd[3] += c.x * Gi.x + c.y * Gi.y;
        gd[4] += c.x * Gp.x + c.y * Gp.y;
        gd[6] += dcf[a][kTc].x * G0.x + dcf[a][kTc].y * G0.y + slope;
      }
    }

    if (by_class) {
      for (int a = 0; a < na; ++a) {
        cfs[k * na + a] = cf[a];
        for (int v = 0; v < 4; ++v) dcfs[k * na + a][v] = dcf[a][v];
      }
      continue;
    }
    // quadratic term over the block pairs a <= b
    const double* Gk = C.G + (size_t)C.cls_of[k] * C.nblk * 4 * M * M;
    int blk = 0;
    for (int a = 0; a < na; ++a) {
      double ar[MM], ai[MM];
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        ar[m] = cf[a].x * yr[m] - cf[a].y * yi[m];
        ai[m] = cf[a].x * yi[m] + cf[a].y * yr[m];
      }
      double ur[MM], ui[MM];  // sum_b S_ab z_b (Re rows, Im rows)
#pragma unroll
      for (int m = 0; m < MM; ++m) ur[m] = ui[m] = 0.0;
      for (int b = a; b < na; ++b, ++blk) {
        double br[MM], bi[MM];
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          br[m] = cf[b].x * yr[m] - cf[b].y * yi[m];
          bi[m] = cf[b].x * yi[m] + cf[b].y * yr[m];
        }
        const double* Gb = Gk + (size_t)blk * 4 * M * M;
        double vr[MM], vi[MM];  // S_ab^T z_a
#pragma unroll
        for (int m = 0; m < MM; ++m) vr[m] = vi[m] = 0.0;
#pragma unroll
        for (int r = 0; r < MM; ++r) {
          if (r < M) {
            double t1 = 0.0, t2 = 0.0;
#pragma unroll
            for (int c = 0; c < MM; ++c) {
              if (c < M) {
                const double g00 = __ldg(Gb + r * M + c), g01 = __ldg(Gb + M * M + r * M + c);
                const double g10 = __ldg(Gb + 2 * M * M + r * M + c);
                const double g11 = __ldg(Gb + 3 * M * M + r * M + c);
                t1 = fma(g00, br[c], t1);
                t1 = fma(g01, bi[c], t1);
                t2 = fma(g10, br[c], t2);
                t2 = fma(g11, bi[c], t2);
                vr[c] = fma(g00, ar[r], vr[c]);
                vr[c] = fma(g10, ai[r], vr[c]);
                vi[c] = fma(g01, ar[r], vi[c]);
                vi[c] = fma(g11, ai[r], vi[c]);
              }
            }
            ur[r] += t1;
            ui[r] += t2;
            tq = fma(ar[r], t1, tq);
            tq = fma(ai[r], t2, tq);
          }
        }
        // dz_b . v: gamma = sum conj(Y) v~ (and with dY for incl, phase)
        double2 gy = make_double2(0.0, 0.0), gyi = gy, gyp = gy;
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          gy.x += yr[m] * vr[m] + yi[m] * vi[m];
          gy.y += yr[m] * vi[m] - yi[m] * vr[m];
          gyi.x += ir[m] * vr[m] + ii[m] * vi[m];
          gyi.y += ir[m] * vi[m] - ii[m] * vr[m];
          gyp.x += pr[m] * vr[m] + pi[m] * vi[m];
          gyp.y += pr[m] * vi[m] - pi[m] * vr[m];
        }
        gq[0] += dcf[b][kRa].x * gy.x + dcf[b][kRa].y * gy.y;
        gq[1] += dcf[b][kDec].x * gy.x + dcf[b][kDec].y * gy.y;
        gq[2] += dcf[b][kPsi].x * gy.x + dcf[b][kPsi].y * gy.y;
        gq[6] += dcf[b][kTc].x * gy.x + dcf[b][kTc].y * gy.y;
        gq[3] += cf[b].x * gyi.x + cf[b].y * gyi.y;
        gq[4] += cf[b].x * gyp.x + cf[b].y * gyp.y;
      }
      // dz_a . u
      double2 gy = make_double2(0.0, 0.0), gyi = gy, gyp = gy;
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        gy.x += yr[m] * ur[m] + yi[m] * ui[m];
        gy.y += yr[m] * ui[m] - yi[m] * ur[m];
        gyi.x += ir[m] * ur[m] + ii[m] * ui[m];
        gyi.y += ir[m] * ui[m] - ii[m] * ur[m];
        gyp.x += pr[m] * ur[m] + pi[m] * ui[m];
        gyp.y += pr[m] * ui[m] - pi[m] * ur[m];
      }
      gq[0] += dcf[a][kRa].x * gy.x + dcf[a][kRa].y * gy.y;
      gq[1] += dcf[a][kDec].x * gy.x + dcf[a][kDec].y * gy.y;
      gq[2] += dcf[a][kPsi].x * gy.x + dcf[a][kPsi].y * gy.y;
      gq[6] += dcf[a][kTc].x * gy.x + dcf[a][kTc].y * gy.y;
      gq[3] += cf[a].x * gyi.x + cf[a].y * gyi.y;
      gq[4] += cf[a].x * gyp.x + cf[a].y * gyp.y;
    }
  }
  if (by_class) {
    // With v_0 = y = (Re Y, Im Y), v_1 = Jy = (-Im Y, Re Y), z_a = sum_p c^p_a v_p
    // (c^0 = Re C_a, c^1 = Im C_a), so per block and class the forms
    // S^pq = v_p^T G v_q and, for incl and phase, v_p'^T G v_q + v_p^T G v_q'
    // carry the whole quadratic term and its derivatives.
    for (int cc = 0; cc < C.ncls; ++cc) {
      const double* Gc = C.G + (size_t)cc * C.nblk * 4 * M * M;
      int blk = 0;
      for (int a = 0; a < na; ++a) {
        for (int b = a; b < na; ++b, ++blk) {
          const double* Gb = Gc + (size_t)blk * 4 * M * M;
          // rows of G v_q (g) and of G^T v_p (h), q, p in {0, 1}
          double S[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, Ti[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
          double Tp[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
#pragma unroll
          for (int r = 0; r < MM; ++r) {
            if (r < M) {
              double g[2][2] = {{0.0, 0.0}, {0.0, 0.0}};  // [q][Re row, Im row]
              double hh[2][2] = {{0.0, 0.0}, {0.0, 0.0}}; // [p][Re col, Im col] of G^T v_p at r
#pragma unroll
              for (int c = 0; c < MM; ++c) {
                if (c < M) {
                  const double g00 = __ldg(Gb + r * M + c), g01 = __ldg(Gb + M * M + r * M + c);
                  const double g10 = __ldg(Gb + 2 * M * M + r * M + c);
                  const double g11 = __ldg(Gb + 3 * M * M + r * M + c);
                  // G v_0, G v_1 at rows (Re r, Im r)
                  g[0][0] = fma(g00, yr[c], fma(g01, yi[c], g[0][0]));
                  g[0][1] = fma(g10, yr[c], fma(g11, yi[c], g[0][1]));
                  g[1][0] = fma(g01, yr[c], fma(-g00, yi[c], g[1][0]));
                  g[1][1] = fma(g11, yr[c], fma(-g10, yi[c], g[1][1]));
                  // G^T v_0, G^T v_1 at columns (Re r, Im r): sum over rows c
                  const double t00 = __ldg(Gb + c * M + r), t01 = __ldg(Gb + M * M + c * M + r);
                  const double t10 = __ldg(Gb + 2 * M * M + c * M + r);
                  const double t11 = __ldg(Gb + 3 * M * M + c * M + r);
                  hh[0][0] = fma(t00, yr[c], fma(t10, yi[c], hh[0][0]));
                  hh[0][1] = fma(t01, yr[c], fma(t11, yi[c], hh[0][1]));
                  hh[1][0] = fma(t10, yr[c], fma(-t00, yi[c], hh[1][0]));
                  hh[1][1] = fma(t11, yr[c], fma(-t01, yi[c], hh[1][1]));
                }
              }
              // v_p (and its incl, phase derivatives) at rows (Re r, Im r)
              const double vr[2][2] = {{yr[r], yi[r]}, {-yi[r], yr[r]}};
              const double vi[2][2] = {{ir[r], ii[r]}, {-ii[r], ir[r]}};
              const double vp[2][2] = {{pr[r], pi[r]}, {-pi[r], pr[r]}};
#pragma unroll
              for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) {
                  S[pp][qq] = fma(vr[pp][0], g[qq][0], fma(vr[pp][1], g[qq][1], S[pp][qq]));
                  // v_p'^T G v_q + v_p^T G v_q' = v_p' . g_q + v_q' . h_p
                  Ti[pp][qq] = fma(vi[pp][0], g[qq][0], fma(vi[pp][1], g[qq][1], Ti[pp][qq]));
                  Ti[pp][qq] = fma(vi[qq][0], hh[pp][0], fma(vi[qq][1], hh[pp][1], Ti[pp][qq]));
                  Tp[pp][qq] = fma(vp[pp][0], g[qq][0], fma(vp[pp][1], g[qq][1], Tp[pp][qq]));
                  Tp[pp][qq] = fma(vp[qq][0], hh[pp][0], fma(vp[qq][1], hh[pp][1], Tp[pp][qq]));
                }
            }
          }
          for (int k = 0; k < C.K; ++k) {
            if (C.cls_of[k] != cc) continue;
            const double2 ca = cfs[k * na + a], cb = cfs[k * na + b];
            const double pa[2] = {ca.x, ca.y}, pb[2] = {cb.x, cb.y};
            double val = 0.0, vi_ = 0.0, vp_ = 0.0;
#pragma unroll
            for (int pp = 0; pp < 2; ++pp)
#pragma unroll
              for (int qq = 0; qq < 2; ++qq) {
                val = fma(pa[pp] * pb[qq], S[pp][qq], val);
                vi_ = fma(pa[pp] * pb[qq], Ti[pp][qq], vi_);
                vp_ = fma(pa[pp] * pb[qq], Tp[pp][qq], vp_);
              }
            tq += val;
            gq[3] += vi_;
            gq[4] += vp_;
            const int slot[4] = {0, 1, 2, 6};
#pragma unroll
            for (int v = 0; v < 4; ++v) {
              const double2 da = dcfs[k * na + a][v], db = dcfs[k * na + b][v];
              const double qa[2] = {da.x, da.y}, qb[2] = {db.x, db.y};
              double d = 0.0;
#pragma unroll
              for (int pp = 0; pp < 2; ++pp)
#pragma unroll
                for (int qq = 0; qq < 2; ++qq) d = fma(qa[pp] * pb[qq] + pa[pp] * qb[qq], S[pp][qq], d);
              gq[slot[v]] += d;
            }
          }
        }
      }
    }
  }
  const double q4 = 0.25 * x * x;
#pragma unroll
  for (int p = 0; p < kNpar; ++p) gout[p] = x * gd[p] - q4 * gq[p];
  gout[5] = -x * td + 2.0 * q4 * tq;
  if (bad) {
#pragma unroll
    for (int p = 0; p < kNpar; ++p) gout[p] = CUDART_NAN;
    return CUDART_NAN;
  }
  return x * td - q4 * tq;
}

template <int MM>
__global__ void __launch_bounds__(kCompThreads) comp_grad_kernel(const __grid_constant__ CompParams C,
                                                                 const PointParams* __restrict__ gP,
                                                                 DrawsParams dp,
                                                                 double* __restrict__ lnl_out,
                                                                 double* __restrict__ grad_out) {
  __shared__ PointParams P;
  stage_point(P, gP);
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    double g[kNpar];
    const double l = comp_grad_draw<MM>(C, P, dp, i, g);
    if (lnl_out) lnl_out[i] = l;
#pragma unroll
    for (int p = 0; p < kNpar; ++p) grad_out[p * dp.n + i] = g[p];
  }
}

template <int MM>
cudaError_t launch_comp_grad_mm(const CompParams& C, const PointParams* dP, const DrawsParams& dp,
                                double* lnl_out, double* grad_out, cudaStream_t st) {
  const int blocks = grid_cap(grid_for(comp_grad_kernel<MM>, kCompThreads, 0), dp.n, kCompThreads);
  comp_grad_kernel<MM><<<blocks, kCompThreads, 0, st>>>(C, dP, dp, lnl_out, grad_out);
  return cudaGetLastError();
}

cudaError_t launch_comp_grad(const CompParams& C, const PointParams* dP, const DrawsParams& dp,
                             double* lnl_out, double* grad_out, cudaStream_t st) {
  const int M = C.M;
  if (M <= 2) return launch_comp_grad_mm<2>(C, dP, dp, lnl_out, grad_out, st);
  if (M <= 4) return launch_comp_grad_mm<4>(C, dP, dp, lnl_out, grad_out, st);
  if (M <= 6) return launch_comp_grad_mm<6>(C, dP, dp, lnl_out, grad_out, st);
  if (M <= 8) return launch_comp_grad_mm<8>(C, dP, dp, lnl_out, grad_out, st);
  if (M <= 10) return launch_comp_grad_mm<10>(C, dP, dp, lnl_out, grad_out, st);
  if (M <= 12) return launch_comp_grad_mm<12>(C, dP, dp, lnl_out, grad_out, st);
  return launch_comp_grad_mm<16>(C, dP, dp, lnl_out, grad_out, st);
}

}  // namespace
}  // namespace rift

using namespace rift;

extern "C" int rift_ile_comp_lnL_grad(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                      double* lnL_out, double* grad_out, void* stream) {
  if (!cp) {
    rift_ile_set_error("composite point is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int rc = validate_draws(draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!grad_out) {
    rift_ile_set_error("rift_ile_comp_lnL_grad: grad_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  return check_cuda(launch_comp_grad(cp->host, cp->dev_base, draws_params(draws), lnL_out, grad_out,
                                     (cudaStream_t)stream),
                    "rift_ile_comp_lnL_grad launch");
}
