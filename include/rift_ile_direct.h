/* rift_ile_direct.h -- direct marginalisation inside the likelihood
 * ("Scaling RIFT 1", arXiv 2609.37393, eq. direct_marginalization, App. F),
 * C ABI, FP64.
 *
 * For each draw of the sampled coordinates (ra, dec, incl, t_c) the library
 * returns
 *
 *   ln L_dir = ln int dphi dpsi dx p(phi) p(psi) p_x(x) exp[lnL(phi, psi, x)]
 *
 * with lnL(x) = K x - R x^2 / 2 (eq. ap:dexp), K and R the data term and the
 * model norm of eq. def:lnL:Decomposed at x = d_ref / D = 1.  At the draw's
 * arrival time K and R are finite trigonometric polynomials in (phi, psi)
 * (eq. ap:angleharm): their harmonic coefficients are formed per draw from the
 * factored likelihood (F_k(psi) = e^{2 i psi} F_k(0), Y_lm(phi) = e^{i m phi}
 * Y_lm(0)), which is the exact reconstruction ERAI performs, and the
 * exponential is integrated on an n_phi x n_psi periodic trapezoid grid over
 * [0, 2 pi) x [0, pi) (uniform priors).  At each grid point the distance is
 * integrated by adaptive Gauss-Hermite (eq. ap:dgh) about x* = K/R with width
 * R^(-1/2) (eq. ap:dpeak), n_gh nodes, prior uniform in volume on
 * [d_min, d_max]: p_x(x) = 3 d_ref^3 x^-4 / (d_max^3 - d_min^3) on
 * [d_ref/d_max, d_ref/d_min].  Grid points whose largest possible
 * contribution is more than 60 nat below the best point's are skipped.
 *
 * With n_t > 0 the geocentric time is integrated as well, by the
 * fixed-spacing rule of eq. ap:tfixed on the window [t_lo, t_hi] (the draw's
 * t is then ignored); the harmonic model is rebuilt at every time node
 * before any integration, as App. F.1 requires; or by the band-limited rule
 * (t_up) or the peak-local rule (t_local) below.
 *
 * The draw's psi, phase and lnD are ignored.  A draw whose distance nodes all
 * fall outside the prior gets -inf.  Ownership and errors as in rift_ile.h;
 * asynchronous on `stream`.  Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA.
 */
#ifndef RIFT_ILE_DIRECT_H
#define RIFT_ILE_DIRECT_H
#include "rift_ile.h"

#ifdef __cplusplus
extern "C" {
#endif

#define RIFT_ILE_MAX_GH 64

typedef struct {
  int32_t n_phi;  /* phase nodes over [0, 2 pi), >= 1; spacing should resolve the peak */
  int32_t n_psi;  /* polarisation nodes over [0, pi), >= 1; n_phi n_psi <= 2^26 */
  int32_t n_gh;   /* Gauss-Hermite nodes in x, 1..RIFT_ILE_MAX_GH */
  double d_min;   /* distance prior range, same unit as d_ref */
  double d_max;
  int32_t n_t;    /* 0: use each draw's t; else time nodes of the fixed-spacing rule */
  double t_lo;    /* time window (seconds, n_t > 0): midpoints t_lo + (j + 1/2) h, */
  double t_hi;    /* h = (t_hi - t_lo) / n_t, uniform prior on the window */
  int32_t t_up;   /* 0 or 1: the fixed-spacing rule (eq. ap:tfixed) on the n_t
                   * midpoints.  > 1 (needs n_t in 1..1024, n_t t_up <= 2^20):
                   * the band-limited full-window rule of eq. ap:tband -- the
                   * data coefficients (linear in Q) are formed at the n_t
                   * midpoints, carried to t_up fine midpoints per interval,
                   * t_lo + (f + 1/2) h / t_up, by sum_j c(t_j) sinc((t_f -
                   * t_j) / h) over the window, sinc(x) = sin(pi x)/(pi x),
                   * and the angles and distance are integrated at every fine
                   * node (weight 1 / (n_t t_up)).  The call then allocates a
                   * stream-ordered scratch of n_t * 17 complex doubles per
                   * resident warp and frees it before returning.  The stencil
                   * is truncated at the window: place the window so that the
                   * correlation has decayed at its ends. */
  int32_t precision; /* RIFT_ILE_FP64 (0): every step in double.  RIFT_ILE_FP32_MIXED:
                   * the harmonic model, K, R, K^2/(2R), the Gauss-Hermite
                   * abscissae and their prior-range test stay in double; the
                   * prior-weighted sum sum_i w_i (x_i / x_lo)^-4 runs in
                   * float (relative error ~1e-6, i.e. ~1e-6 in ln L_dir);
                   * needs d_max / d_min <= 1e9. */
  int32_t t_local; /* 0: off.  1 (needs t_up >= 2, n_t t_up <= 65536): the
                   * peak-local rule of eq. ap:tlocal on the band-limited
                   * rule's fine nodes.  Per draw the envelope
                   * U(t) = 1/2 sum_k |e_k(t_k)|^2 (the data of each detector
                   * projected on its template span, from the point's whitened
                   * tables; U bounds the angular-and-distance integrand at t
                   * by Cauchy-Schwarz and is attained at a noise-free
                   * injection) is taken at every fine node; its maxima within
                   * ln(1/t_tol) + ln(n_t t_up) of the largest get a width
                   * sigma_t^2 = h_f^2 / (2 U_m - U_{m-1} - U_{m+1}) (h_f the
                   * fine spacing; the end nodes mirror their neighbour); the
                   * fine nodes within t_c sigma_t of a maximum are integrated,
                   * the others bounded together by ln R = LSE(U) -
                   * ln(n_t t_up).  If ln R exceeds ln(t_tol) plus the kept
                   * value, or a maximum is flat or there are more than 64, every
                   * fine node is integrated (the band-limited rule).  The
                   * scratch grows by 12 bytes per fine node and 1 KB per
                   * resident warp. */
  double t_c;     /* neighbourhood half-width in units of sigma_t (e.g. 16) */
  double t_tol;   /* relative tolerance of the skipped remainder, in (0, 1) */
  int32_t t_mirror; /* 0: the fine coefficients by the truncated sinc sum of
                   * eq. ap:tband.  1 (needs t_up >= 2): by the mirrored series
                   * -- the n_t window samples reflected about the window's ends
                   * (period 2 n_t h, continuous), its trigonometric interpolant
                   * with harmonics |k| < n_t at the fine midpoints:
                   * sum_j c(t_j) [D(t_f - t_j) + D(t_f + t_j - 2 t_lo)],
                   * D(z h) = sin((2 n_t - 1) pi z / (2 n_t)) /
                   * (2 n_t sin(pi z / (2 n_t))); exact for series the reflection
                   * continues smoothly, equal to the pregrid construction of
                   * eq. q-time-pregrid applied to the window. */
} rift_ile_direct_rule;

/* ln L_dir per draw into DEVICE out[n] (double). */
int rift_ile_lnL_direct(const rift_ile_point* pt, const rift_ile_draws* draws,
                        const rift_ile_direct_rule* rule, double* out, void* stream);

/* The Monte Carlo evidence over the sampled coordinates with the direct
 * marginal as the integrand: the LSE state (see rift_ile_lse) of
 * ln L_dir_i + ln w_i over the draws (eq. lnL:MonteCarlo), written to DEVICE
 * state_out without a host synchronisation; `scratch` is DEVICE [n] doubles
 * for the per-draw values (may alias nothing else).  Errors as
 * rift_ile_lnL_direct. */
int rift_ile_lnZ_direct_state(const rift_ile_point* pt, const rift_ile_draws* draws,
                              const rift_ile_direct_rule* rule, double* scratch,
                              rift_ile_lse* state_out, void* stream);

/* The Gauss-Hermite rule the kernel uses (weight e^{-x^2}): HOST x[n], w[n]. */
int rift_ile_gauss_hermite(int32_t n, double* x, double* w);

#ifdef __cplusplus
}
#endif
#endif
