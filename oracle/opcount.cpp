// opcount.cpp -- the arithmetic of the extrinsic likelihood, counted.
//
// TEST INFRASTRUCTURE, like rift_oracle.c: only the tests and the script that
// freezes the counts (oracle/freeze_flops.py) load it.  It shares nothing with
// the CUDA library.
//
// A plain FP64 evaluation of one draw, step by step in the order of the
// method, with every floating-point operation on per-draw values counted:
//   sky geometry, polarisation basis, antenna factor F_k and arrival time t_k
//                                                   (Sec. II.A, eq. fsize:FA at f -> 0)
//   the harmonics -2Y_lm(iota, phi_ref) by Goldberg's sum           (eq. strain_mode)
//   Q_{k,lm}(t_k) by the four-point Lagrange cubic               (eq. q-time-pregrid)
//   the data term x Re sum_k conj(F_k) sum_lm conj(Y_lm) Q_klm(t_k)
//   the quadratic term (x^2/4) sum_k [|F_k|^2 Y^dag U_k Y + Re(F_k^2 Y^T V_k Y)]
//     through the products P_ij = conj(Y_i) Y_j and S_ij = Y_i Y_j of i <= j,
//     formed once per draw and shared by the detectors  (eq. def:lnL:Decomposed)
//   lnL = data - quadratic term, and the online log-sum-exp update of lnZ
//                                                   (eq. lnL:MonteCarlo, eq. neff)
//   the gradient in (ra, dec, psi, iota, phi_ref, lnD, t_c) by the chain rule:
//     forward derivatives of F_k, t_k, Y and the cubic's slope, and for the
//     quadratic term the adjoint of the P/S step: with
//     Ubar = sum_k |F_k|^2 U_k and Vbar = sum_k F_k^2 V_k, the iota and phi_ref
//     derivatives are 2 Re(dY^dag Ubar Y) and 2 Re(dY^T Vbar Y)        (Sec. II.B)
//   the distance marginal K x_j - R x_j^2/2 + ln w_j summed over the nodes,
//     and its gradient E[x] dK - E[x^2] dR/2                (eq. ap:dexp, eq. ap:dlog)
//
// Counting rules: an add, subtract or multiply is one flop, so a multiply-add
// is two; a divide is one flop (also counted apart); sin, cos, exp and log are
// special-function calls, counted apart and not as flops; sign changes,
// copies, comparisons, floor and indexing are free.  Values fixed per point
// (Goldberg's coefficients with their normalisation, 1/dt, the nodes' x_j,
// x_j^2 and ln w_j) are set up beforehand and not counted.  Structural zeros
// (the east vector has no z component) are not multiplied.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <vector>

extern "C" {
#include "rift_oracle.h"
}

namespace {

struct Counts {
  long long add = 0, mul = 0, div = 0, special = 0;
};
Counts g_cnt;  // single-threaded by design

struct Num {
  double v;
  Num() : v(0.0) {}
  Num(double x) : v(x) {}  // NOLINT: constants enter uncounted
};
inline Num operator+(Num a, Num b) { ++g_cnt.add; return Num(a.v + b.v); }
inline Num operator-(Num a, Num b) { ++g_cnt.add; return Num(a.v - b.v); }
inline Num operator*(Num a, Num b) { ++g_cnt.mul; return Num(a.v * b.v); }
inline Num operator/(Num a, Num b) { ++g_cnt.div; return Num(a.v / b.v); }
inline Num operator-(Num a) { return Num(-a.v); }
inline Num& operator+=(Num& a, Num b) { a = a + b; return a; }
inline Num& operator-=(Num& a, Num b) { a = a - b; return a; }
inline Num nsin(Num a) { ++g_cnt.special; return Num(std::sin(a.v)); }
inline Num ncos(Num a) { ++g_cnt.special; return Num(std::cos(a.v)); }
inline Num nexp(Num a) { ++g_cnt.special; return Num(std::exp(a.v)); }
inline Num nlog(Num a) { ++g_cnt.special; return Num(std::log(a.v)); }

struct Cx {
  Num re, im;
};
inline Cx cmul(Cx a, Cx b) { return Cx{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
// conj(a) b
inline Cx cmulc(Cx a, Cx b) { return Cx{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }
inline Cx cadd(Cx a, Cx b) { return Cx{a.re + b.re, a.im + b.im}; }
inline Cx cscale(Num s, Cx a) { return Cx{s * a.re, s * a.im}; }
// Re(conj(a) b)
inline Num re_cmulc(Cx a, Cx b) { return a.re * b.re + a.im * b.im; }
// Re(a b)
inline Num re_cmul(Cx a, Cx b) { return a.re * b.re - a.im * b.im; }

double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}
double binom(int n, int k) {
  if (k < 0 || k > n || n < 0) return 0.0;
  return factorial(n) / (factorial(k) * factorial(n - k));
}

// One term coef c^k s^j of Goldberg's sum for -2Y_lm(theta, 0) with
// c = cos(theta/2), s = sin(theta/2); the normalisation is folded into coef.
struct Term {
  double coef;
  int k, j;
};

struct Setup {
  int K = 0, M = 0, lmax = 0, mmax = 0;
  std::vector<std::vector<Term>> terms;  // per mode
  double inv_dt = 0.0;
};

Setup make_setup(const ora_point* P) {
  Setup S;
  S.K = P->K;
  S.M = P->M;
  S.inv_dt = 1.0 / P->dt;
  const int s = -2;
  S.terms.resize(P->M);
  for (int i = 0; i < P->M; ++i) {
    const int l = P->ell[i], m = P->em[i];
    S.lmax = std::max(S.lmax, l);
    S.mmax = std::max(S.mmax, std::abs(m));
    const double norm = ((m & 1) ? -1.0 : 1.0) *
                        std::sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1) /
                                  (4.0 * M_PI * factorial(l + s) * factorial(l - s)));
    for (int r = 0; r <= l - s; ++r) {
      double coef = binom(l - s, r) * binom(l + s, r + s - m);
      if (coef == 0.0) continue;
      if ((l - r - s) & 1) coef = -coef;
      const int k = 2 * r + s - m;
      S.terms[i].push_back(Term{norm * coef, k, 2 * l - k});
    }
  }
  return S;
}

// Per-draw quantities of one detector needed by the gradient.
struct DetState {
  Cx F, dF_ra, dF_dec;
  Num dt_ra, dt_dec;
  Num A;  // Y^dag U_k Y (real)
  Cx B;   // Y^T V_k Y
  Cx G, Gt, G_incl, G_phi;
};

// lnL of one draw at distance factor x (x_fixed > 0: that value; else
// D_ref e^{-lnD}), and with grad != nullptr its gradient; td/tq receive the
// data and quadratic terms.
Num draw_lnl(const ora_point* P, const Setup& S, const double* th, double x_fixed, double* grad,
             Num* td_out, Num* tq_out, Num* dtd_out, Num* dtq_out) {
  const int K = S.K, M = S.M;
  const bool G = grad != nullptr || dtd_out != nullptr;
  const Num ra = th[ORA_RA], dec = th[ORA_DEC], psi = th[ORA_PSI], incl = th[ORA_INCL];
  const Num phi = th[ORA_PHASE], lnD = th[ORA_LND], tc = th[ORA_TC];
  // distance factor
  const Num x = x_fixed > 0.0 ? Num(x_fixed) : Num(P->d_ref) * nexp(-lnD);

  // sky direction s, east e1 = (-sl, cl, 0), north e2 = (-sd cl, -sd sl, cd)
  const Num lam = ra - Num(P->gmst);
  const Num sl = nsin(lam), cl = ncos(lam), sd = nsin(dec), cd = ncos(dec);
  const Num sdcl = sd * cl, sdsl = sd * sl;
  const Num s[3] = {cd * cl, cd * sl, sd};
  const Num e1[2] = {-sl, cl};
  const Num e2[3] = {-sdcl, -sdsl, cd};
  const Num cp = ncos(psi), sp = nsin(psi);
  const Num p[3] = {cp * e1[0] + sp * e2[0], cp * e1[1] + sp * e2[1], sp * e2[2]};
  const Num q[3] = {cp * e2[0] - sp * e1[0], cp * e2[1] - sp * e1[1], cp * e2[2]};
  // their derivatives (gradient only): d e1/d ra = (-cl, -sl, 0), d e2/d ra =
  // (sd sl, -sd cl, 0), d e2/d dec = (-cd cl, -cd sl, -sd), d e1/d dec = 0
  Num ds_ra[2], dp_ra[2], dq_ra[2], dp_dec[3], dq_dec[3];
  if (G) {
    ds_ra[0] = -s[1];
    ds_ra[1] = s[0];
    dp_ra[0] = sp * sdsl - cp * cl;
    dp_ra[1] = -(cp * sl) - sp * sdcl;
    dq_ra[0] = cp * sdsl + sp * cl;
    dq_ra[1] = sp * sl - cp * sdcl;
    dp_dec[0] = -(sp * s[0]);
    dp_dec[1] = -(sp * s[1]);
    dp_dec[2] = -(sp * sd);
    dq_dec[0] = -(cp * s[0]);
    dq_dec[1] = -(cp * s[1]);
    dq_dec[2] = -(cp * sd);
  }

  // harmonics: powers of c = cos(iota/2), s = sin(iota/2), e^{i m phi}
  const Num h = Num(0.5) * incl;
  const Num ch = ncos(h), sh = nsin(h);
  std::vector<Num> cpow(2 * S.lmax + 2), spow(2 * S.lmax + 2);
  cpow[0] = 1.0;
  spow[0] = 1.0;
  cpow[1] = ch;
  spow[1] = sh;
  for (int a = 2; a <= 2 * S.lmax + 1; ++a) {
    cpow[a] = cpow[a - 1] * ch;
    spow[a] = spow[a - 1] * sh;
  }
  std::vector<Cx> eim(S.mmax + 1);
  eim[0] = Cx{1.0, 0.0};
  if (S.mmax >= 1) eim[1] = Cx{ncos(phi), nsin(phi)};
  for (int a = 2; a <= S.mmax; ++a) eim[a] = cmul(eim[a - 1], eim[1]);
  std::vector<Cx> Y(M), dY_incl(M);
  for (int i = 0; i < M; ++i) {
    Num amp = 0.0, damp = 0.0;
    bool first = true;
    for (const Term& t : S.terms[i]) {
      const Num v = Num(t.coef) * (cpow[t.k] * spow[t.j]);
      amp = first ? v : amp + v;
      if (G) {
        // d/d iota [c^k s^j] = (j c^(k+1) s^(j-1) - k c^(k-1) s^(j+1)) / 2
        Num dv = 0.0;
        bool dfirst = true;
        if (t.j > 0) {
          dv = Num(0.5 * t.coef * t.j) * (cpow[t.k + 1] * spow[t.j - 1]);
          dfirst = false;
        }
        if (t.k > 0) {
          const Num w = Num(0.5 * t.coef * t.k) * (cpow[t.k - 1] * spow[t.j + 1]);
          dv = dfirst ? -w : dv - w;
        }
        damp = first ? dv : damp + dv;
      }
      first = false;
    }
    const int m = P->em[i], am = std::abs(m);
    const Cx e = m < 0 ? Cx{eim[am].re, -eim[am].im} : eim[am];
    Y[i] = am == 0 ? Cx{amp, 0.0} : cscale(amp, e);
    if (G) dY_incl[i] = am == 0 ? Cx{damp, 0.0} : cscale(damp, e);
  }

  // quadratic-term products of i <= j, shared by the detectors
  std::vector<Cx> Pm(M * M), Sm(M * M);
  for (int i = 0; i < M; ++i) {
    Pm[i * M + i] = Cx{Y[i].re * Y[i].re + Y[i].im * Y[i].im, 0.0};
    Sm[i * M + i] = cmul(Y[i], Y[i]);
    for (int j = i + 1; j < M; ++j) {
      Pm[i * M + j] = cmulc(Y[i], Y[j]);
      Sm[i * M + j] = cmul(Y[i], Y[j]);
    }
  }

  std::vector<DetState> D(K);
  Num td = 0.0, tq = 0.0;
  Num gtd[ORA_NPAR], gtq[ORA_NPAR];
  for (int k = 0; k < K; ++k) {
    DetState& ds = D[k];
    const double* R = P->resp + 6 * k;
    const double* xk = P->pos + 3 * k;
    // D v for the symmetric response tensor (xx, xy, xz, yy, yz, zz)
    auto Dv = [&](const Num* v, Num* out) {
      out[0] = Num(R[0]) * v[0] + Num(R[1]) * v[1] + Num(R[2]) * v[2];
      out[1] = Num(R[1]) * v[0] + Num(R[3]) * v[1] + Num(R[4]) * v[2];
      out[2] = Num(R[2]) * v[0] + Num(R[4]) * v[1] + Num(R[5]) * v[2];
    };
    auto dot3 = [](const Num* a, const Num* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; };
    auto dot2 = [](const Num* a, const Num* b) { return a[0] * b[0] + a[1] * b[1]; };
    Num Dp[3], Dq[3];
    Dv(p, Dp);
    Dv(q, Dq);
    const Num Fp = dot3(p, Dp) - dot3(q, Dq);
    const Num Fx = Num(2.0) * dot3(p, Dq);
    ds.F = Cx{Fp, -Fx};
    const Num xn[3] = {xk[0], xk[1], xk[2]};
    const Num tk = tc - dot3(xn, s);
    if (G) {
      // d(p.D.p) = 2 dp.D p; d(p.D.q) = dp.D q + dq.D p (D symmetric)
      const Num dFp_ra = Num(2.0) * (dot2(dp_ra, Dp) - dot2(dq_ra, Dq));
      const Num dFx_ra = Num(2.0) * (dot2(dp_ra, Dq) + dot2(dq_ra, Dp));
      const Num dFp_dec = Num(2.0) * (dot3(dp_dec, Dp) - dot3(dq_dec, Dq));
      const Num dFx_dec = Num(2.0) * (dot3(dp_dec, Dq) + dot3(dq_dec, Dp));
      ds.dF_ra = Cx{dFp_ra, -dFx_ra};
      ds.dF_dec = Cx{dFp_dec, -dFx_dec};
      ds.dt_ra = -(Num(xk[0]) * ds_ra[0] + Num(xk[1]) * ds_ra[1]);
      const Num ds_dec[3] = {-sdcl, -sdsl, cd};
      ds.dt_dec = -dot3(xn, ds_dec);
    }

    // four-point Lagrange cubic on taps j-1 .. j+2 (taps outside read zero)
    const Num u = (tk - Num(P->t0[k])) * Num(S.inv_dt);
    const double jf = std::floor(u.v);
    const Num f = u - Num(jf);
    const Num a = f + Num(1.0), c = f - Num(1.0), d = f - Num(2.0);
    const Num cd_ = c * d, af = a * f;
    const Num w[4] = {Num(-1.0 / 6.0) * (f * cd_), Num(0.5) * (a * cd_), Num(-0.5) * (af * d),
                      Num(1.0 / 6.0) * (af * c)};
    Num dw[4];
    if (G) {
      // d w_i / dt = (d w_i / df) / dt
      const Num fd = f * d, fc = f * c, ad = a * d, ac = a * c;
      dw[0] = Num(-S.inv_dt / 6.0) * (cd_ + fd + fc);
      dw[1] = Num(0.5 * S.inv_dt) * (cd_ + ad + ac);
      dw[2] = Num(-0.5 * S.inv_dt) * (fd + ad + af);
      dw[3] = Num(S.inv_dt / 6.0) * (fc + ac + af);
    }
    const long j0 = (long)jf - 1;
    std::vector<Cx> Qk(M), dQk(M);
    for (int i = 0; i < M; ++i) {
      Cx acc{0.0, 0.0}, dacc{0.0, 0.0};
      for (int tap = 0; tap < 4; ++tap) {
        const long jj = j0 + tap;
        double qr = 0.0, qi = 0.0;
        if (jj >= 0 && jj < P->n) {
          qr = P->Q[((size_t)k * P->n + jj) * M * 2 + 2 * i];
          qi = P->Q[((size_t)k * P->n + jj) * M * 2 + 2 * i + 1];
        }
        const Cx term = cscale(w[tap], Cx{qr, qi});
        acc = tap ? cadd(acc, term) : term;
        if (G) {
          const Cx dterm = cscale(dw[tap], Cx{qr, qi});
          dacc = tap ? cadd(dacc, dterm) : dterm;
        }
      }
      Qk[i] = acc;
      dQk[i] = dacc;
    }

    // data term: Re conj(F) sum_i conj(Y_i) Q_i
    std::vector<Cx> yq(M);
    for (int i = 0; i < M; ++i) {
      yq[i] = cmulc(Y[i], Qk[i]);
      ds.G = i ? cadd(ds.G, yq[i]) : yq[i];
    }
    const Num tdk = re_cmulc(ds.F, ds.G);
    td = k ? td + tdk : tdk;

    // quadratic term through P and S
    Num Adiag = 0.0, Aoff = 0.0;
    Cx Bdiag{0.0, 0.0}, Boff{0.0, 0.0};
    bool fd1 = true, fo1 = true;
    for (int i = 0; i < M; ++i) {
      const double* Ui = P->U + ((size_t)k * M * M + (size_t)i * M) * 2;
      const double* Vi = P->V + ((size_t)k * M * M + (size_t)i * M) * 2;
      const Num ad = Num(Ui[2 * i]) * Pm[i * M + i].re;
      const Cx bd = cmul(Cx{Vi[2 * i], Vi[2 * i + 1]}, Sm[i * M + i]);
      Adiag = fd1 ? ad : Adiag + ad;
      Bdiag = fd1 ? bd : cadd(Bdiag, bd);
      fd1 = false;
      for (int j = i + 1; j < M; ++j) {
        const Num ao = re_cmul(Cx{Ui[2 * j], Ui[2 * j + 1]}, Pm[i * M + j]);
        const Cx bo = cmul(Cx{Vi[2 * j], Vi[2 * j + 1]}, Sm[i * M + j]);
        Aoff = fo1 ? ao : Aoff + ao;
        Boff = fo1 ? bo : cadd(Boff, bo);
        fo1 = false;
      }
    }
    ds.A = Adiag + Num(2.0) * Aoff;
    ds.B = cadd(Bdiag, cscale(Num(2.0), Boff));
    const Num fr2 = ds.F.re * ds.F.re, fi2 = ds.F.im * ds.F.im;
    const Num F2 = fr2 + fi2;
    const Cx FF{fr2 - fi2, Num(2.0) * (ds.F.re * ds.F.im)};
    const Num tqk = F2 * ds.A + re_cmul(FF, ds.B);
    tq = k ? tq + tqk : tqk;

    if (G) {
      // data-term derivatives
      bool phi_first = true;
      for (int i = 0; i < M; ++i) {
        const Cx gt = cmulc(Y[i], dQk[i]);
        const Cx gi = cmulc(dY_incl[i], Qk[i]);
        ds.Gt = i ? cadd(ds.Gt, gt) : gt;
        ds.G_incl = i ? cadd(ds.G_incl, gi) : gi;
        // conj(i m Y) Q = -i m conj(Y) Q
        if (P->em[i] != 0) {
          const Num mm = (double)P->em[i];
          const Cx gp{mm * yq[i].im, -(mm * yq[i].re)};
          ds.G_phi = phi_first ? gp : cadd(ds.G_phi, gp);
          phi_first = false;
        }
      }
      const Num ft = re_cmulc(ds.F, ds.Gt);
      Num c_td[ORA_NPAR];
      c_td[ORA_RA] = re_cmulc(ds.dF_ra, ds.G) + ft * ds.dt_ra;
      c_td[ORA_DEC] = re_cmulc(ds.dF_dec, ds.G) + ft * ds.dt_dec;
      // d F / d psi = 2 i F: Re(conj(2 i F) G) = 2 Im(conj(F) G)
      c_td[ORA_PSI] = Num(2.0) * (ds.F.re * ds.G.im - ds.F.im * ds.G.re);
      c_td[ORA_INCL] = re_cmulc(ds.F, ds.G_incl);
      c_td[ORA_PHASE] = re_cmulc(ds.F, ds.G_phi);
      c_td[ORA_TC] = ft;
      // quadratic-term derivatives through F: d|F|^2 = 2 Re(conj F dF), d F^2 = 2 F dF
      Num c_tq[3];
      const Cx dFs[3] = {ds.dF_ra, ds.dF_dec, Cx{-(Num(2.0) * ds.F.im), Num(2.0) * ds.F.re}};
      for (int v = 0; v < 3; ++v) {
        const Num dF2 = Num(2.0) * re_cmulc(ds.F, dFs[v]);
        const Cx dFF = cscale(Num(2.0), cmul(ds.F, dFs[v]));
        c_tq[v] = dF2 * ds.A + re_cmul(dFF, ds.B);
      }
      for (int v : {ORA_RA, ORA_DEC, ORA_PSI, ORA_INCL, ORA_PHASE, ORA_TC})
        gtd[v] = k ? gtd[v] + c_td[v] : c_td[v];
      for (int v = 0; v < 3; ++v) gtq[v] = k ? gtq[v] + c_tq[v] : c_tq[v];
    }
  }

  if (G) {
    // iota and phi_ref through Y: the adjoint of the P/S step
    std::vector<Cx> Ub(M * M), Vb(M * M);
    for (int k = 0; k < K; ++k) {
      const Num fr2 = D[k].F.re * D[k].F.re, fi2 = D[k].F.im * D[k].F.im;
      const Num F2 = fr2 + fi2;
      const Cx FF{fr2 - fi2, Num(2.0) * (D[k].F.re * D[k].F.im)};
      for (int i = 0; i < M; ++i)
        for (int j = i; j < M; ++j) {
          const double* u = P->U + ((size_t)k * M * M + (size_t)i * M + j) * 2;
          const double* v = P->V + ((size_t)k * M * M + (size_t)i * M + j) * 2;
          const Cx uu = i == j ? Cx{F2 * Num(u[0]), 0.0} : cscale(F2, Cx{u[0], u[1]});
          const Cx vv = cmul(FF, Cx{v[0], v[1]});
          Ub[i * M + j] = k ? cadd(Ub[i * M + j], uu) : uu;
          Vb[i * M + j] = k ? cadd(Vb[i * M + j], vv) : vv;
        }
    }
    // (Ubar Y)_i = sum_j Ubar_ij Y_j with Ubar_ji = conj(Ubar_ij); (Vbar Y) likewise, Vbar symmetric
    std::vector<Cx> UY(M), VY(M);
    for (int i = 0; i < M; ++i) {
      for (int j = 0; j < M; ++j) {
        const Cx ub = j >= i ? Ub[i * M + j] : Cx{Ub[j * M + i].re, -Ub[j * M + i].im};
        const Cx vb = j >= i ? Vb[i * M + j] : Vb[j * M + i];
        const Cx tu = cmul(ub, Y[j]), tv = cmul(vb, Y[j]);
        UY[i] = j ? cadd(UY[i], tu) : tu;
        VY[i] = j ? cadd(VY[i], tv) : tv;
      }
    }
    Num s_incl = 0.0, s_phi = 0.0;
    for (int i = 0; i < M; ++i) {
      // dY/d phi = i m Y
      const Num mm = (double)P->em[i];
      const Cx dYp{-(mm * Y[i].im), mm * Y[i].re};
      const Num ti = re_cmulc(dY_incl[i], UY[i]) + re_cmul(dY_incl[i], VY[i]);
      const Num tp = re_cmulc(dYp, UY[i]) + re_cmul(dYp, VY[i]);
      s_incl = i ? s_incl + ti : ti;
      s_phi = i ? s_phi + tp : tp;
    }
    gtq[ORA_INCL] = Num(2.0) * s_incl;
    gtq[ORA_PHASE] = Num(2.0) * s_phi;
  }

  // at x = 1 (the distance marginal's K and R) nothing is multiplied by x
  const bool unit = x_fixed == 1.0;
  const Num Td = unit ? td : x * td;
  const Num x2q = unit ? Num(0.25) : Num(0.25) * (x * x);
  const Num Tq = x2q * tq;
  const Num lnl = Td - Tq;
  if (td_out) *td_out = Td;
  if (tq_out) *tq_out = Tq;
  if (G) {
    if (!unit)
      for (int v : {ORA_RA, ORA_DEC, ORA_PSI, ORA_INCL, ORA_PHASE, ORA_TC}) gtd[v] = x * gtd[v];
    for (int v : {ORA_RA, ORA_DEC, ORA_PSI, ORA_INCL, ORA_PHASE}) gtq[v] = x2q * gtq[v];
    gtq[ORA_TC] = 0.0;
    if (dtd_out)
      for (int v = 0; v < ORA_NPAR; ++v) dtd_out[v] = v == ORA_LND ? Num(0.0) : gtd[v];
    if (dtq_out)
      for (int v = 0; v < ORA_NPAR; ++v) dtq_out[v] = v == ORA_LND ? Num(0.0) : gtq[v];
    if (grad) {
      for (int v : {ORA_RA, ORA_DEC, ORA_PSI, ORA_INCL, ORA_PHASE}) grad[v] = (gtd[v] - gtq[v]).v;
      grad[ORA_TC] = gtd[ORA_TC].v;
      // x = D_ref e^{-lnD}: d T_d / d lnD = -T_d, d T_q / d lnD = -2 T_q
      grad[ORA_LND] = (Num(2.0) * Tq - Td).v;
    }
  }
  return lnl;
}

}  // namespace

extern "C" {

// Evaluates `which` over N draws (theta [N][7], one after the other, one
// thread) and returns in counts[4] the totals (add/sub, mul, div, special):
//   0  lnL and the online log-sum-exp of lnL + ln w (logw may be NULL);
//      values[i] = lnL, lse[3] = (max, sum e, sum e^2) of the online update
//   1  lnL and its gradient (values, grad [N][7])
//   2  the distance-marginalised lnL over the node table
//   3  the distance-marginalised lnL and its gradient
// Returns 0, or -1 for an unknown `which`.
int ora_count_ops(const ora_point* P, const double* theta, int64_t N, const double* logw,
                  const double* x_nodes, const double* lnw_nodes, int n_nodes, int which,
                  double* values, double* grad, double* lse, long long* counts) {
  if (which < 0 || which > 3) return -1;
  const Setup S = make_setup(P);
  g_cnt = Counts();
  std::vector<double> x2(n_nodes > 0 ? n_nodes : 0);
  for (int j = 0; j < n_nodes; ++j) x2[j] = x_nodes[j] * x_nodes[j];
  Num m = -INFINITY, s = 0.0, s2 = 0.0;
  for (int64_t i = 0; i < N; ++i) {
    const double* th = theta + (size_t)i * ORA_NPAR;
    if (which == 0 || which == 1) {
      const Num lnl = draw_lnl(P, S, th, 0.0, which == 1 ? grad + (size_t)i * ORA_NPAR : nullptr,
                               nullptr, nullptr, nullptr, nullptr);
      values[i] = lnl.v;
      if (which == 0) {
        // online log-sum-exp with the running maximum m
        const Num v = logw ? lnl + Num(logw[i]) : lnl;
        if (v.v > m.v) {
          const Num r = std::isfinite(m.v) ? nexp(m - v) : Num(0.0);
          s = s * r + Num(1.0);
          s2 = s2 * (r * r) + Num(1.0);
          m = v;
        } else {
          const Num e = nexp(v - m);
          s += e;
          s2 += e * e;
        }
      }
    } else {
      // K = T_d(x = 1), R = 2 T_q(x = 1): lnL(x) = K x - R x^2 / 2
      Num Td, Tq, dTd[ORA_NPAR], dTq[ORA_NPAR];
      const bool g = which == 3;
      draw_lnl(P, S, th, 1.0, nullptr, &Td, &Tq, g ? dTd : nullptr, g ? dTq : nullptr);
      const Num halfR = Tq;  // R / 2
      std::vector<Num> v(n_nodes);
      double vmax = -INFINITY;
      for (int j = 0; j < n_nodes; ++j) {
        v[j] = Td * Num(x_nodes[j]) - halfR * Num(x2[j]) + Num(lnw_nodes[j]);
        vmax = std::max(vmax, v[j].v);
      }
      Num se = 0.0, s1 = 0.0, sx2 = 0.0;
      for (int j = 0; j < n_nodes; ++j) {
        const Num e = nexp(v[j] - Num(vmax));
        se = j ? se + e : e;
        if (g) {
          s1 = j ? s1 + e * Num(x_nodes[j]) : e * Num(x_nodes[j]);
          sx2 = j ? sx2 + e * Num(x2[j]) : e * Num(x2[j]);
        }
      }
      values[i] = (Num(vmax) + nlog(se)).v;
      if (g) {
        const Num ex = s1 / se, ex2 = sx2 / se;
        double* gi = grad + (size_t)i * ORA_NPAR;
        for (int p = 0; p < ORA_NPAR; ++p)
          gi[p] = p == ORA_LND ? 0.0 : (ex * dTd[p] - ex2 * dTq[p]).v;
      }
    }
  }
  if (lse) {
    lse[0] = m.v;
    lse[1] = s.v;
    lse[2] = s2.v;
  }
  counts[0] = g_cnt.add;
  counts[1] = g_cnt.mul;
  counts[2] = g_cnt.div;
  counts[3] = g_cnt.special;
  return 0;
}

}  // extern "C"
