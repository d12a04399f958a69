/* rift_oracle.h -- plain FP64 CPU oracle of the extrinsic likelihood (test
 * infrastructure only; see rift_oracle.c). */
#ifndef RIFT_ORACLE_H
#define RIFT_ORACLE_H
#include <stdint.h>

/* One intrinsic point: everything the factored likelihood needs.
 * Complex arrays are interleaved (re, im) doubles. */
typedef struct {
  int K;                /* detectors */
  int M;                /* modes */
  int n;                /* samples per Q series */
  const int* ell;       /* [M] */
  const int* em;        /* [M] */
  const double* Q;      /* [K][n][M][2]  Q_{k,lm}(t0_k + j dt) */
  const double* t0;     /* [K] time of sample 0, seconds relative to t_ref */
  double dt;            /* table spacing, seconds */
  const double* U;      /* [K][M][M][2]  U_{k,i,j} = <h_i|h_j>_k */
  const double* V;      /* [K][M][M][2]  V_{k,i,j} = <h_i^*|h_j>_k */
  const double* pos;    /* [K][3] detector positions, light-seconds, Earth-fixed */
  const double* resp;   /* [K][6] response tensor xx, xy, xz, yy, yz, zz */
  double gmst;          /* Greenwich mean sidereal time, rad */
  double d_ref;         /* reference distance of the modes (same unit as D) */
  /* Exact-Q mode (used when the caller asks for it; NULL otherwise):
   * Q_{k,lm}(t) = sum_n wgt[k][n] exp(2 pi i f_n t) conj(hlm[lm][n]) dk[k][n]. */
  int nf;
  const double* freq;   /* [nf] two-sided grid, Hz */
  const double* wgt;    /* [K][nf]  2 df / S_k(|f_n|), 0 outside the band */
  const double* hlm;    /* [M][nf][2] */
  const double* dk;     /* [K][nf][2] */
} ora_point;

/* Parameter order of a draw: */
enum { ORA_RA = 0, ORA_DEC, ORA_PSI, ORA_INCL, ORA_PHASE, ORA_LND, ORA_TC, ORA_NPAR };

void ora_sky_basis(double ra, double dec, double gmst, double s[3], double e1[3], double e2[3]);
void ora_antenna(const double resp[6], double ra, double dec, double psi, double gmst,
                 double* f_re, double* f_im);
double ora_delay(const double pos[3], double ra, double dec, double gmst, double tc);
void ora_sylm(int s, int l, int m, double theta, double phi, double* re, double* im);
void ora_sylm_dtheta(int s, int l, int m, double theta, double phi, double* re, double* im);
int ora_qinterp(const double* q, int n, int M, double t0, double dt, double t, double* out,
                double* dout);

void ora_lnL_batch(const ora_point* P, const double* theta, int64_t N, int exact_q,
                   int nthreads, double* lnL, double* Td, double* Tq, int64_t* oob);
void ora_grad_batch(const ora_point* P, const double* theta, int64_t N, int exact_q,
                    int nthreads, double* lnL, double* grad);
void ora_lnZ(const double* lnL, const double* logw, int64_t N, double out[3]);
void ora_lnL_distmarg_batch(const ora_point* P, const double* theta, int64_t N,
                            const double* x_nodes, const double* lnw_nodes, int n_nodes,
                            int nthreads, double* lnL);
void ora_grad_distmarg_batch(const ora_point* P, const double* theta, int64_t N,
                             const double* x_nodes, const double* lnw_nodes, int n_nodes,
                             int nthreads, double* lnL, double* grad);
int ora_dist_nodes(double d_min, double d_max, double d_ref, double tol, double rho_max,
                   int max_nodes, double* x_nodes, double* lnw_nodes);
int ora_nthreads_default(void);

#endif
