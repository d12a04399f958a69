/* rift_oracle.c -- plain FP64 CPU oracle of the extrinsic-marginalised
 * likelihood of RIFT ("Scaling RIFT 1", Sec. II.A-II.C, App. E-F).
 *
 * TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load this file.  It shares no code, header, table
 * or constant with the CUDA library: it is written directly from the paper's
 * equations, one draw at a time, in double precision, with no blocking,
 * fusion or reordering beyond what the equations state.
 *
 * What it computes, and where each step comes from:
 *   - sky direction, polarisation basis, antenna factor F_k = F_+ - i F_x and
 *     arrival time t_k = t_c - x_k . s                      (Sec. II.A, eq. 5-6 text)
 *   - spin-weighted harmonics -2Y_lm(iota, phi_ref), Goldberg's sum      (eq. strain_mode)
 *   - Q_{k,lm}(t_k) from the fine table by four-point Lagrange cubic C_3
 *     (eq. q-time-pregrid), or by the direct Fourier sum of eq. QUV ("exact-Q")
 *   - lnL of eq. def:lnL:Decomposed: the data term minus the U/V quadratic term
 *   - the analytic gradient of that lnL by the chain rule           (Sec. II.B)
 *   - lnZ = LSE_i(lnL_i + ln w_i) - ln N, its delta-method error and n_eff
 *                                            (eq. lnL:MonteCarlo, eq. neff)
 *   - distance marginalisation on a log-uniform lnD node table
 *                                            (eq. ap:dexp, eq. ap:dlog)
 *
 * Readings of points the paper leaves open (listed with reasons in the
 * design notes of the repository):
 *   - s points from the geocentre TO the source; t_k = t_c - x_k . s.
 *   - polarisation basis e1 = d s/d(ra) normalised (east), e2 = north;
 *     p = cos(psi) e1 + sin(psi) e2, q = -sin(psi) e1 + cos(psi) e2;
 *     F_+ = p.D.p - q.D.q, F_x = 2 p.D.q, so that F(psi) = exp(2 i psi) F(0).
 *   - -2Y_lm(iota, phi_ref) literally, Condon-Shortley phase.
 *   - the U term is taken as a real number (Re of the Hermitian form).
 *   - C_3 is the four-point Lagrange cubic on taps j-1..j+2 with
 *     j = floor((t - t0)/dt); taps outside [0, n) read as zero and are counted.
 *   - the paper prints no lnL value for a reproducible input, so no absolute
 *     value is compared; every function here is pinned by the closed forms,
 *     invariants, limits and brute-force checks of the oracle tests.
 */
#include "rift_oracle.h"

#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

typedef double complex cplx;

/* ---------------------------------------------------------------- geometry */

/* Source direction s (towards the source) and the transverse basis (e1, e2)
 * in Earth-fixed coordinates; lam = ra - gmst is the Earth-fixed longitude. */
void ora_sky_basis(double ra, double dec, double gmst, double s[3], double e1[3], double e2[3]) {
  double lam = ra - gmst;
  s[0] = cos(dec) * cos(lam);
  s[1] = cos(dec) * sin(lam);
  s[2] = sin(dec);
  e1[0] = -sin(lam);
  e1[1] = cos(lam);
  e1[2] = 0.0;
  e2[0] = -sin(dec) * cos(lam);
  e2[1] = -sin(dec) * sin(lam);
  e2[2] = cos(dec);
}

/* a^T D b for the symmetric response tensor stored as xx, xy, xz, yy, yz, zz. */
static double quad_form(const double D[6], const double a[3], const double b[3]) {
  double Db0 = D[0] * b[0] + D[1] * b[1] + D[2] * b[2];
  double Db1 = D[1] * b[0] + D[3] * b[1] + D[4] * b[2];
  double Db2 = D[2] * b[0] + D[4] * b[1] + D[5] * b[2];
  return a[0] * Db0 + a[1] * Db1 + a[2] * Db2;
}

/* Complex antenna factor F = F_+ - i F_x for basis vectors (e1, e2). */
static cplx antenna_from_basis(const double D[6], const double e1[3], const double e2[3],
                               double psi) {
  double p[3], q[3];
  for (int i = 0; i < 3; ++i) {
    p[i] = cos(psi) * e1[i] + sin(psi) * e2[i];
    q[i] = -sin(psi) * e1[i] + cos(psi) * e2[i];
  }
  double fp = quad_form(D, p, p) - quad_form(D, q, q);
  double fx = 2.0 * quad_form(D, p, q);
  return fp - I * fx;
}

/* Derivative of F along a change (de1, de2) of the basis vectors. */
static cplx antenna_basis_derivative(const double D[6], const double e1[3], const double e2[3],
                                     const double de1[3], const double de2[3], double psi) {
  double p[3], q[3], dp[3], dq[3];
  for (int i = 0; i < 3; ++i) {
    p[i] = cos(psi) * e1[i] + sin(psi) * e2[i];
    q[i] = -sin(psi) * e1[i] + cos(psi) * e2[i];
    dp[i] = cos(psi) * de1[i] + sin(psi) * de2[i];
    dq[i] = -sin(psi) * de1[i] + cos(psi) * de2[i];
  }
  /* D is symmetric, so d(p.D.p) = 2 dp.D.p and d(p.D.q) = dp.D.q + p.D.dq. */
  double dfp = 2.0 * quad_form(D, dp, p) - 2.0 * quad_form(D, dq, q);
  double dfx = 2.0 * (quad_form(D, dp, q) + quad_form(D, p, dq));
  return dfp - I * dfx;
}

void ora_antenna(const double resp[6], double ra, double dec, double psi, double gmst,
                 double* f_re, double* f_im) {
  double s[3], e1[3], e2[3];
  ora_sky_basis(ra, dec, gmst, s, e1, e2);
  cplx F = antenna_from_basis(resp, e1, e2, psi);
  *f_re = creal(F);
  *f_im = cimag(F);
}

double ora_delay(const double pos[3], double ra, double dec, double gmst, double tc) {
  double s[3], e1[3], e2[3];
  ora_sky_basis(ra, dec, gmst, s, e1, e2);
  return tc - (pos[0] * s[0] + pos[1] * s[1] + pos[2] * s[2]);
}

/* ------------------------------------------------- spin-weighted harmonics */

static double factorial(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

static double binom(int n, int k) {
  if (k < 0 || k > n || n < 0) return 0.0;
  return factorial(n) / (factorial(k) * factorial(n - k));
}

/* Goldberg et al. (1967):
 *   sY_lm = (-1)^m sqrt[(l+m)!(l-m)!(2l+1) / (4 pi (l+s)!(l-s)!)]
 *           sum_r C(l-s, r) C(l+s, r+s-m) (-1)^(l-r-s) e^{i m phi}
 *           sin^{2l}(theta/2) cot^{2r+s-m}(theta/2),
 * written with c = cos(theta/2), sn = sin(theta/2) as c^k sn^(2l-k),
 * k = 2r + s - m.  With deriv != 0 the theta-derivative is returned. */
static cplx sylm_impl(int s, int l, int m, double theta, double phi, int deriv) {
  if (l < abs(s) || l < abs(m)) return 0.0;
  double norm = ((m & 1) ? -1.0 : 1.0) *
                sqrt(factorial(l + m) * factorial(l - m) * (2 * l + 1) /
                     (4.0 * M_PI * factorial(l + s) * factorial(l - s)));
  double c = cos(0.5 * theta), sn = sin(0.5 * theta);
  double sum = 0.0;
  for (int r = 0; r <= l - s; ++r) {
    double coef = binom(l - s, r) * binom(l + s, r + s - m);
    if (coef == 0.0) continue;
    if ((l - r - s) & 1) coef = -coef;
    int k = 2 * r + s - m;
    int j = 2 * l - k;
    double term;
    if (!deriv) {
      term = pow(c, k) * pow(sn, j);
    } else {
      /* d/dtheta [c^k sn^j] = 1/2 [-k c^(k-1) sn^(j+1) + j c^(k+1) sn^(j-1)] */
      double a = (k > 0) ? -k * pow(c, k - 1) * pow(sn, j + 1) : 0.0;
      double b = (j > 0) ? j * pow(c, k + 1) * pow(sn, j - 1) : 0.0;
      term = 0.5 * (a + b);
    }
    sum += coef * term;
  }
  return norm * sum * cexp(I * m * phi);
}

void ora_sylm(int s, int l, int m, double theta, double phi, double* re, double* im) {
  cplx y = sylm_impl(s, l, m, theta, phi, 0);
  *re = creal(y);
  *im = cimag(y);
}

void ora_sylm_dtheta(int s, int l, int m, double theta, double phi, double* re, double* im) {
  cplx y = sylm_impl(s, l, m, theta, phi, 1);
  *re = creal(y);
  *im = cimag(y);
}

/* ------------------------------------------------------ Q interpolation C_3 */

/* Four-point Lagrange cubic through nodes -1, 0, 1, 2 at offset f in [0, 1),
 * and its derivative with respect to f (product rule, written out). */
static void lagrange4(double f, double w[4], double dw[4]) {
  double a = f + 1.0, b = f, c = f - 1.0, d = f - 2.0;
  w[0] = -(b * c * d) / 6.0;
  w[1] = (a * c * d) / 2.0;
  w[2] = -(a * b * d) / 2.0;
  w[3] = (a * b * c) / 6.0;
  dw[0] = -(c * d + b * d + b * c) / 6.0;
  dw[1] = (c * d + a * d + a * c) / 2.0;
  dw[2] = -(b * d + a * d + a * b) / 2.0;
  dw[3] = (b * c + a * c + a * b) / 6.0;
}

/* Q(t) for all M modes of one detector from its table q[n][M][2]; dout (may
 * be NULL) receives dQ/dt.  Returns the number of taps outside [0, n). */
int ora_qinterp(const double* q, int n, int M, double t0, double dt, double t, double* out,
                double* dout) {
  double u = (t - t0) / dt;
  double jf = floor(u);
  double f = u - jf;
  double w[4], dw[4];
  lagrange4(f, w, dw);
  int oob = 0;
  for (int i = 0; i < M; ++i) {
    out[2 * i] = out[2 * i + 1] = 0.0;
    if (dout) dout[2 * i] = dout[2 * i + 1] = 0.0;
  }
  for (int tap = 0; tap < 4; ++tap) {
    double jj = jf - 1.0 + tap;
    if (!(jj >= 0.0 && jj < (double)n)) {
      ++oob;
      continue;
    }
    const double* row = q + (size_t)((long)jj) * M * 2;
    for (int i = 0; i < M; ++i) {
      out[2 * i] += w[tap] * row[2 * i];
      out[2 * i + 1] += w[tap] * row[2 * i + 1];
      if (dout) {
        dout[2 * i] += dw[tap] * row[2 * i] / dt;
        dout[2 * i + 1] += dw[tap] * row[2 * i + 1] / dt;
      }
    }
  }
  return oob;
}

/* Exact-Q: the direct Fourier sum of eq. QUV at time t (and its t-derivative). */
static void exact_q_sum(const ora_point* P, int k, double t, cplx* out, cplx* dout) {
  for (int i = 0; i < P->M; ++i) {
    cplx acc = 0.0, dacc = 0.0;
    for (int n = 0; n < P->nf; ++n) {
      double w = P->wgt[(size_t)k * P->nf + n];
      if (w == 0.0) continue;
      double f = P->freq[n];
      cplx h = P->hlm[((size_t)i * P->nf + n) * 2] + I * P->hlm[((size_t)i * P->nf + n) * 2 + 1];
      cplx d = P->dk[((size_t)k * P->nf + n) * 2] + I * P->dk[((size_t)k * P->nf + n) * 2 + 1];
      cplx term = w * cexp(2.0 * M_PI * I * f * t) * conj(h) * d;
      acc += term;
      dacc += 2.0 * M_PI * I * f * term;
    }
    out[i] = acc;
    if (dout) dout[i] = dacc;
  }
}

/* ------------------------------------------------------------ likelihood */

#define ORA_MAX_M 32

/* Data term T_d and quadratic term T_q of eq. def:lnL:Decomposed at distance
 * factor x = D_ref/D, and (if dTd/dTq are non-NULL) their derivatives with
 * respect to ra, dec, psi, iota, phi_ref, t_c at fixed x (slots 0..4, 6;
 * slot 5 is left zero: the lnD dependence enters only through x). */
static int ora_terms(const ora_point* P, const double* th, double x, int exact_q, double* Td,
                     double* Tq, double dTd[ORA_NPAR], double dTq[ORA_NPAR]) {
  const int M = P->M;
  double ra = th[ORA_RA], dec = th[ORA_DEC], psi = th[ORA_PSI];
  double incl = th[ORA_INCL], phi = th[ORA_PHASE], tc = th[ORA_TC];
  double s[3], e1[3], e2[3];
  ora_sky_basis(ra, dec, P->gmst, s, e1, e2);
  double lam = ra - P->gmst;
  /* Derivatives of s, e1, e2 with respect to ra and dec. */
  double ds_ra[3] = {-cos(dec) * sin(lam), cos(dec) * cos(lam), 0.0};
  double ds_dec[3] = {-sin(dec) * cos(lam), -sin(dec) * sin(lam), cos(dec)};
  double de1_ra[3] = {-cos(lam), -sin(lam), 0.0};
  double de1_dec[3] = {0.0, 0.0, 0.0};
  double de2_ra[3] = {sin(dec) * sin(lam), -sin(dec) * cos(lam), 0.0};
  double de2_dec[3] = {-cos(dec) * cos(lam), -cos(dec) * sin(lam), -sin(dec)};

  cplx Y[ORA_MAX_M], dY_incl[ORA_MAX_M], dY_phi[ORA_MAX_M];
  for (int i = 0; i < M; ++i) {
    Y[i] = sylm_impl(-2, P->ell[i], P->em[i], incl, phi, 0);
    dY_incl[i] = sylm_impl(-2, P->ell[i], P->em[i], incl, phi, 1);
    dY_phi[i] = I * P->em[i] * Y[i];
  }

  int oob = 0;
  double td = 0.0, tq = 0.0;
  double gtd[ORA_NPAR] = {0}, gtq[ORA_NPAR] = {0};
  for (int k = 0; k < P->K; ++k) {
    const double* D = P->resp + 6 * k;
    const double* xk = P->pos + 3 * k;
    cplx F = antenna_from_basis(D, e1, e2, psi);
    cplx dF_ra = antenna_basis_derivative(D, e1, e2, de1_ra, de2_ra, psi);
    cplx dF_dec = antenna_basis_derivative(D, e1, e2, de1_dec, de2_dec, psi);
    cplx dF_psi = 2.0 * I * F;
    double tk = tc - (xk[0] * s[0] + xk[1] * s[1] + xk[2] * s[2]);
    double dtk_ra = -(xk[0] * ds_ra[0] + xk[1] * ds_ra[1] + xk[2] * ds_ra[2]);
    double dtk_dec = -(xk[0] * ds_dec[0] + xk[1] * ds_dec[1] + xk[2] * ds_dec[2]);

    cplx Qh[ORA_MAX_M], dQh[ORA_MAX_M];
    if (exact_q) {
      exact_q_sum(P, k, tk, Qh, dQh);
    } else {
      double qb[2 * ORA_MAX_M], dqb[2 * ORA_MAX_M];
      oob += ora_qinterp(P->Q + (size_t)k * P->n * M * 2, P->n, M, P->t0[k], P->dt, tk, qb, dqb);
      for (int i = 0; i < M; ++i) {
        Qh[i] = qb[2 * i] + I * qb[2 * i + 1];
        dQh[i] = dqb[2 * i] + I * dqb[2 * i + 1];
      }
    }

    /* Data term: x Re sum_lm (F Y_lm)^* Q_lm(t_k). */
    cplx G = 0.0, Gt = 0.0, G_incl = 0.0, G_phi = 0.0;
    for (int i = 0; i < M; ++i) {
      G += conj(Y[i]) * Qh[i];
      Gt += conj(Y[i]) * dQh[i];
      G_incl += conj(dY_incl[i]) * Qh[i];
      G_phi += conj(dY_phi[i]) * Qh[i];
    }
    td += creal(conj(F) * G);
    gtd[ORA_RA] += creal(conj(dF_ra) * G) + creal(conj(F) * Gt) * dtk_ra;
    gtd[ORA_DEC] += creal(conj(dF_dec) * G) + creal(conj(F) * Gt) * dtk_dec;
    gtd[ORA_PSI] += creal(conj(dF_psi) * G);
    gtd[ORA_INCL] += creal(conj(F) * G_incl);
    gtd[ORA_PHASE] += creal(conj(F) * G_phi);
    gtd[ORA_TC] += creal(conj(F) * Gt);

    /* Quadratic term: |F|^2 Y^dag U Y + Re(F^2 Y^T V Y), and the parts
     * needed for its derivatives. */
    const double* Uk = P->U + (size_t)k * M * M * 2;
    const double* Vk = P->V + (size_t)k * M * M * 2;
    cplx A = 0.0, B = 0.0, A_incl = 0.0, B_incl = 0.0, A_phi = 0.0, B_phi = 0.0;
    for (int i = 0; i < M; ++i) {
      for (int j = 0; j < M; ++j) {
        cplx u = Uk[(i * M + j) * 2] + I * Uk[(i * M + j) * 2 + 1];
        cplx v = Vk[(i * M + j) * 2] + I * Vk[(i * M + j) * 2 + 1];
        A += conj(Y[i]) * Y[j] * u;
        B += Y[i] * Y[j] * v;
        A_incl += (conj(dY_incl[i]) * Y[j] + conj(Y[i]) * dY_incl[j]) * u;
        B_incl += (dY_incl[i] * Y[j] + Y[i] * dY_incl[j]) * v;
        A_phi += (conj(dY_phi[i]) * Y[j] + conj(Y[i]) * dY_phi[j]) * u;
        B_phi += (dY_phi[i] * Y[j] + Y[i] * dY_phi[j]) * v;
      }
    }
    double F2 = creal(F * conj(F));
    tq += F2 * creal(A) + creal(F * F * B);
    gtq[ORA_RA] += 2.0 * creal(conj(F) * dF_ra) * creal(A) + creal(2.0 * F * dF_ra * B);
    gtq[ORA_DEC] += 2.0 * creal(conj(F) * dF_dec) * creal(A) + creal(2.0 * F * dF_dec * B);
    gtq[ORA_PSI] += 2.0 * creal(conj(F) * dF_psi) * creal(A) + creal(2.0 * F * dF_psi * B);
    gtq[ORA_INCL] += F2 * creal(A_incl) + creal(F * F * B_incl);
    gtq[ORA_PHASE] += F2 * creal(A_phi) + creal(F * F * B_phi);
  }
  *Td = x * td;
  *Tq = 0.25 * x * x * tq;
  if (dTd) {
    for (int p = 0; p < ORA_NPAR; ++p) dTd[p] = x * gtd[p];
    dTd[ORA_LND] = 0.0;
  }
  if (dTq) {
    for (int p = 0; p < ORA_NPAR; ++p) dTq[p] = 0.25 * x * x * gtq[p];
    dTq[ORA_LND] = 0.0;
    dTq[ORA_TC] = 0.0;
  }
  return oob;
}

/* --------------------------------------------------------------- threading */

int ora_nthreads_default(void) {
  long n = sysconf(_SC_NPROCESSORS_ONLN);
  return n > 0 ? (int)n : 1;
}

typedef struct {
  const ora_point* P;
  const double* theta;
  int64_t begin, end;
  int exact_q;
  int mode; /* 0: lnL, 1: grad, 2: dist-marg lnL, 3: dist-marg grad */
  const double* x_nodes;
  const double* lnw_nodes;
  int n_nodes;
  double *lnL, *Td, *Tq, *grad;
  int64_t oob;
} ora_job;

static double lse_nodes(double K, double R, const double* xn, const double* lnw, int nn,
                        double* weights);

static void* ora_worker(void* arg) {
  ora_job* J = (ora_job*)arg;
  const ora_point* P = J->P;
  for (int64_t i = J->begin; i < J->end; ++i) {
    const double* th = J->theta + (size_t)i * ORA_NPAR;
    if (J->mode == 0 || J->mode == 1) {
      double x = P->d_ref * exp(-th[ORA_LND]);
      double td, tq, dtd[ORA_NPAR], dtq[ORA_NPAR];
      J->oob += ora_terms(P, th, x, J->exact_q, &td, &tq, J->mode ? dtd : NULL,
                          J->mode ? dtq : NULL);
      if (J->lnL) J->lnL[i] = td - tq;
      if (J->Td) J->Td[i] = td;
      if (J->Tq) J->Tq[i] = tq;
      if (J->mode == 1) {
        double* g = J->grad + (size_t)i * ORA_NPAR;
        for (int p = 0; p < ORA_NPAR; ++p) g[p] = dtd[p] - dtq[p];
        /* x = D_ref exp(-lnD): d T_d/d lnD = -T_d, d T_q/d lnD = -2 T_q. */
        g[ORA_LND] = -td + 2.0 * tq;
      }
    } else {
      /* Distance marginalised: lnL(x) = K x - R x^2 / 2 with K = T_d(x=1),
       * R = 2 T_q(x=1) (eq. ap:dexp), summed over the node table. */
      double td, tq, dtd[ORA_NPAR], dtq[ORA_NPAR];
      int want_grad = (J->mode == 3);
      J->oob += ora_terms(P, th, 1.0, 0, &td, &tq, want_grad ? dtd : NULL, want_grad ? dtq : NULL);
      double K = td, R = 2.0 * tq;
      double* wts = want_grad ? (double*)malloc(sizeof(double) * J->n_nodes) : NULL;
      double val = lse_nodes(K, R, J->x_nodes, J->lnw_nodes, J->n_nodes, wts);
      J->lnL[i] = val;
      if (want_grad) {
        double ex = 0.0, ex2 = 0.0; /* posterior means of x and x^2 over the nodes */
        for (int j = 0; j < J->n_nodes; ++j) {
          ex += wts[j] * J->x_nodes[j];
          ex2 += wts[j] * J->x_nodes[j] * J->x_nodes[j];
        }
        double* g = J->grad + (size_t)i * ORA_NPAR;
        for (int p = 0; p < ORA_NPAR; ++p) g[p] = ex * dtd[p] - ex2 * dtq[p];
        g[ORA_LND] = 0.0;
        free(wts);
      }
    }
  }
  return NULL;
}

/* Splits the draws over nthreads POSIX threads; returns the total count of
 * Q taps that fell outside their tables. */
static int64_t run_jobs(ora_job proto, int64_t N, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  if ((int64_t)nthreads > N) nthreads = (int)(N > 0 ? N : 1);
  ora_job jobs[256];
  pthread_t tid[256];
  for (int t = 0; t < nthreads; ++t) {
    jobs[t] = proto;
    jobs[t].begin = N * t / nthreads;
    jobs[t].end = N * (t + 1) / nthreads;
    jobs[t].oob = 0;
  }
  for (int t = 1; t < nthreads; ++t) pthread_create(&tid[t], NULL, ora_worker, &jobs[t]);
  ora_worker(&jobs[0]);
  for (int t = 1; t < nthreads; ++t) pthread_join(tid[t], NULL);
  int64_t oob = 0;
  for (int t = 0; t < nthreads; ++t) oob += jobs[t].oob;
  return oob;
}

void ora_lnL_batch(const ora_point* P, const double* theta, int64_t N, int exact_q, int nthreads,
                   double* lnL, double* Td, double* Tq, int64_t* oob) {
  ora_job j;
  memset(&j, 0, sizeof(j));
  j.P = P;
  j.theta = theta;
  j.exact_q = exact_q;
  j.mode = 0;
  j.lnL = lnL;
  j.Td = Td;
  j.Tq = Tq;
  int64_t total = run_jobs(j, N, nthreads);
  if (oob) *oob = total;
}

void ora_grad_batch(const ora_point* P, const double* theta, int64_t N, int exact_q, int nthreads,
                    double* lnL, double* grad) {
  ora_job j;
  memset(&j, 0, sizeof(j));
  j.P = P;
  j.theta = theta;
  j.exact_q = exact_q;
  j.mode = 1;
  j.lnL = lnL;
  j.grad = grad;
  run_jobs(j, N, nthreads);
}

/* ------------------------------------------------------------------ lnZ */

/* Pairwise (recursive halving) sum, so that rounding grows as log N. */
static double pairwise_sum(const double* v, int64_t n) {
  if (n <= 8) {
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) s += v[i];
    return s;
  }
  int64_t h = n / 2;
  return pairwise_sum(v, h) + pairwise_sum(v + h, n - h);
}

/* lnZ = ln[(1/N) sum_i exp(lnL_i + ln w_i)]  (eq. lnL:MonteCarlo with
 * w_i = p/p_s), the delta-method standard error of lnZ,
 *   sigma = sqrt(max(0, sum w^2 / (sum w)^2 - 1/N)),
 * and n_eff = sum w / max w (eq. neff).  logw may be NULL (w = 1). */
void ora_lnZ(const double* lnL, const double* logw, int64_t N, double out[3]) {
  if (N <= 0) {
    out[0] = -INFINITY;
    out[1] = NAN;
    out[2] = 0.0;
    return;
  }
  double m = -INFINITY;
  int any_nan = 0;
  for (int64_t i = 0; i < N; ++i) {
    double v = lnL[i] + (logw ? logw[i] : 0.0);
    if (isnan(v)) any_nan = 1;
    if (v > m) m = v;
  }
  if (any_nan) {
    out[0] = out[1] = out[2] = NAN;
    return;
  }
  if (!isfinite(m)) {
    out[0] = m;
    out[1] = NAN;
    out[2] = 0.0;
    return;
  }
  double* e = (double*)malloc(sizeof(double) * (size_t)N);
  double* e2 = (double*)malloc(sizeof(double) * (size_t)N);
  for (int64_t i = 0; i < N; ++i) {
    double v = lnL[i] + (logw ? logw[i] : 0.0);
    e[i] = exp(v - m);
    e2[i] = exp(2.0 * (v - m));
  }
  double s = pairwise_sum(e, N);
  double s2 = pairwise_sum(e2, N);
  free(e);
  free(e2);
  out[0] = m + log(s) - log((double)N);
  double var = s2 / (s * s) - 1.0 / (double)N;
  out[1] = sqrt(var > 0.0 ? var : 0.0);
  out[2] = s; /* the largest weight is exp(m - m) = 1 */
}

/* --------------------------------------------------- distance marginalisation */

/* LSE_j [K x_j - R x_j^2 / 2 + lnw_j]; optional normalised node weights. */
static double lse_nodes(double K, double R, const double* xn, const double* lnw, int nn,
                        double* weights) {
  double m = -INFINITY;
  for (int j = 0; j < nn; ++j) {
    double v = K * xn[j] - 0.5 * R * xn[j] * xn[j] + lnw[j];
    if (v > m) m = v;
  }
  double s = 0.0;
  for (int j = 0; j < nn; ++j) {
    double v = K * xn[j] - 0.5 * R * xn[j] * xn[j] + lnw[j];
    double e = exp(v - m);
    if (weights) weights[j] = e;
    s += e;
  }
  if (weights)
    for (int j = 0; j < nn; ++j) weights[j] /= s;
  return m + log(s);
}

/* Log-uniform node table of eq. ap:dlog: spacing in ln d of at most
 * c(tol)/rho_max with c(tol) = pi sqrt(2 / ln(2/tol)), over [d_min, d_max];
 * trapezoid weights in ln d; prior p(d) = 3 d^2 / (d_max^3 - d_min^3)
 * (uniform in Euclidean volume).  Node j carries x_j = d_ref/d_j and
 * lnw_j = ln(trapezoid weight) + ln p(d_j) + ln d_j (the Jacobian of d -> ln d).
 * Returns the node count, or -1 if it exceeds max_nodes. */
int ora_dist_nodes(double d_min, double d_max, double d_ref, double tol, double rho_max,
                   int max_nodes, double* x_nodes, double* lnw_nodes) {
  double c = M_PI * sqrt(2.0 / log(2.0 / tol));
  double span = log(d_max) - log(d_min);
  int n_int = (int)ceil(span / (c / rho_max));
  if (n_int < 1) n_int = 1;
  int nn = n_int + 1;
  if (nn > max_nodes) return -1;
  double h = span / n_int;
  double lnZp = log(3.0) - log(d_max * d_max * d_max - d_min * d_min * d_min);
  for (int j = 0; j < nn; ++j) {
    double lnd = log(d_min) + j * h;
    double d = exp(lnd);
    double wtrap = (j == 0 || j == nn - 1) ? 0.5 * h : h;
    x_nodes[j] = d_ref / d;
    lnw_nodes[j] = log(wtrap) + lnZp + 2.0 * lnd + lnd;
  }
  return nn;
}

void ora_lnL_distmarg_batch(const ora_point* P, const double* theta, int64_t N,
                            const double* x_nodes, const double* lnw_nodes, int n_nodes,
                            int nthreads, double* lnL) {
  ora_job j;
  memset(&j, 0, sizeof(j));
  j.P = P;
  j.theta = theta;
  j.mode = 2;
  j.x_nodes = x_nodes;
  j.lnw_nodes = lnw_nodes;
  j.n_nodes = n_nodes;
  j.lnL = lnL;
  run_jobs(j, N, nthreads);
}

void ora_grad_distmarg_batch(const ora_point* P, const double* theta, int64_t N,
                             const double* x_nodes, const double* lnw_nodes, int n_nodes,
                             int nthreads, double* lnL, double* grad) {
  ora_job j;
  memset(&j, 0, sizeof(j));
  j.P = P;
  j.theta = theta;
  j.mode = 3;
  j.x_nodes = x_nodes;
  j.lnw_nodes = lnw_nodes;
  j.n_nodes = n_nodes;
  j.lnL = lnL;
  j.grad = grad;
  run_jobs(j, N, nthreads);
}
