/* rift_ile_response.h -- composite-index response of the extrinsic likelihood
 * ("Scaling RIFT 1", arXiv 2609.37393, Sec. III), C ABI, FP64 path.
 *
 * When the detector response depends on time (Earth rotation, Sec. III.A) or
 * on frequency (arms long against the wavelength, Sec. III.B), the template
 * of detector k is a short sum of sky-independent elementary templates
 * chi^(a)_lm times analytic coefficients C~^k_a (eq. slowrot:master, eq.
 * fsize:factorization), and the likelihood keeps the static form with the
 * mode index widened to the composite index A = (a, lm)
 * (eq. slowrot:lnL:Decomposed):
 *
 *   lnL = x Re sum_k sum_A conj(c_kA) Q_{k,A}(t_k)
 *       - x^2/4 sum_k [c_k^+ U_k c_k + Re(c_k^T V_k c_k)],   c_kA = C~^k_a Y_lm,
 *
 * with x = d_ref e^{-lnD}, t_k = t_c - x_k . s and Y_lm = -2Y_lm(incl, phase)
 * as in rift_ile.h, and Q, U, V the products of eq. slowrot:QUV over the bank
 * {chi^(a)_lm}, built by the caller.
 *
 * Coefficients computed per draw by the library:
 *
 *   RIFT_ILE_RESP_ROTATION (Paths A and B; a = (p, n), p = 0..p_max,
 *   n = -(2+p)..(2+p)).  With g = gmst - ra and the five sidereal harmonics
 *   A_n(dec, psi) of the static antenna factor of rift_ile.h,
 *   F_k(gmst + Omega t) = sum_{n=-2..2} A_n e^{i n (g + Omega t)}
 *   (eq. slowrot:Fharm), and the three harmonics of the arrival-time drift
 *   -(t_k(t) - t_k(0)) (eq. slowrot:delay), C^k_(p,n) is the coefficient of
 *   e^{i n Omega t} in F_k(t) (-(t_k(t) - t_k(0)))^p / p!; then
 *   C~ = C e^{i n Omega t_k} (arrival-time post-phase, eq. slowrot:postphase).
 *   The elementary templates are chi^(p,n)_lm(t) = e^{i n Omega t} d^p h_lm/dt^p
 *   in the template's own time, t = 0 at the reference time.  p_max = 0 is
 *   Path A; Omega = 0 gives back the static likelihood.
 *
 *   RIFT_ILE_RESP_FINITE_ARM (Path D; a = p, p = 0..p_max).
 *   C~^k_p = b^k_p = 1/2 [(X.s)^p eps:XX - (Y.s)^p eps:YY] (eq. fsize:bp), with
 *   X, Y the unit arm vectors of detector k, s the unit vector towards the
 *   source and eps = eps_+ - i eps_x the complex polarisation tensor, so that
 *   b^k_0 is the static antenna factor.  The frequency weights W_p and the
 *   common light-crossing delay belong to the bank.
 *
 * Composite index order: A = a * M + i, i the mode, a as listed above.
 *
 * Ownership and errors as in rift_ile.h: the caller owns every buffer it
 * passes; rift_ile_comp_create copies Q (device to device) and what it needs
 * from the host arrays into an object the library owns until
 * rift_ile_comp_destroy.  Calls are asynchronous on the caller's stream
 * except rift_ile_comp_create and rift_ile_comp_lnZ_state, which synchronise.
 * Every entry point returns 0 or a negative RIFT_ILE_ERR_* code with a
 * thread-local message (rift_ile_last_error).
 */
#ifndef RIFT_ILE_RESPONSE_H
#define RIFT_ILE_RESPONSE_H
#include "rift_ile.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RIFT_ILE_RESP_ROTATION = 1,  /* Earth rotation: Paths A (p_max = 0) and B */
  RIFT_ILE_RESP_FINITE_ARM = 2 /* long arms: Path D */
} rift_ile_resp_kind;

#define RIFT_ILE_MAX_ROT_PMAX 3   /* rotation: at most 32 response indices */
#define RIFT_ILE_MAX_ARM_PMAX 15  /* finite arms: at most 16 response indices */
#define RIFT_ILE_MAX_COMP 256     /* composite dimension n_index * M */

/* One intrinsic point with a composite response.
 *   kind, p_max   response and truncation order (limits above)
 *   omega         sidereal rate, rad/s (ROTATION; may be 0)
 *   arm_x, arm_y  HOST [K][3] unit arm vectors, Earth-fixed (FINITE_ARM; may
 *                 be NULL for ROTATION)
 *   Q             DEVICE [K][q_len][n_comp] complex128 (re, im interleaved):
 *                 Q_{k,A}(q_t0[k] + j q_dt), n_comp = n_index * M
 *   U, V          HOST [K][n_comp][n_comp][2] double: <chi_A|chi_B>_k and
 *                 <chi_A^*|chi_B>_k
 *   the other fields as in rift_ile_point_desc; det_resp is required for
 *   ROTATION and may be NULL for FINITE_ARM (the arms define the response). */
typedef struct {
  int32_t n_det;
  int32_t n_modes;
  const int32_t* ell;
  const int32_t* em;
  int32_t kind;
  int32_t p_max;
  double omega;
  const double* arm_x;
  const double* arm_y;
  const double* Q;
  int32_t q_len;
  const double* q_t0;
  double q_dt;
  const double* U;
  const double* V;
  const double* det_pos;
  const double* det_resp;
  double gmst;
  double d_ref;
} rift_ile_comp_desc;

typedef struct rift_ile_comp rift_ile_comp; /* opaque, library-owned */

/* Number of response indices a for (kind, p_max): (p_max + 1)(p_max + 5) for
 * ROTATION, p_max + 1 for FINITE_ARM; a negative error code if unsupported. */
int rift_ile_comp_n_index(int32_t kind, int32_t p_max);

/* Validates the description, copies Q, folds U and V into one real quadratic
 * form per detector, and uploads the constants.  Runs on `stream` and
 * synchronises it.  Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA, ALLOC. */
int rift_ile_comp_create(const rift_ile_comp_desc* desc, rift_ile_comp** out, void* stream);
int rift_ile_comp_destroy(rift_ile_comp* cp);

/* The coefficients C~^k_a of every draw: DEVICE coef_out[n][K][n_index]
 * complex128 (re, im interleaved), on `stream`.  Errors: INVALID_ARG, CUDA. */
int rift_ile_comp_coeffs(const rift_ile_comp* cp, const rift_ile_draws* draws, double* coef_out,
                         void* stream);

/* lnL per draw into DEVICE lnL_out[n] (double), FP64, on `stream`.
 * Errors: INVALID_ARG, SHAPE, CUDA. */
int rift_ile_comp_lnL(const rift_ile_comp* cp, const rift_ile_draws* draws, double* lnL_out,
                      void* stream);

/* lnL (DEVICE [n], may be NULL) and d lnL / d theta into DEVICE grad_out
 * [7][n] (double; parameter-major: ra, dec, psi, incl, phase, lnD, t), FP64,
 * on `stream`: the chain rule of Sec. II.B through the coefficients C~^k_a
 * (their angle and arrival-time derivatives in closed form), the harmonics
 * and the slope of the table cubic.  A draw whose arrival time is not finite
 * gets NaN throughout.  Errors: INVALID_ARG, CUDA. */
int rift_ile_comp_lnL_grad(const rift_ile_comp* cp, const rift_ile_draws* draws, double* lnL_out,
                           double* grad_out, void* stream);

/* LSE state of the draws (fused lnL -> LSE, FP64), to HOST *state; synchronises.
 * Taps outside the table read zero and are counted (rift_ile_last_oob). */
int rift_ile_comp_lnZ_state(const rift_ile_comp* cp, const rift_ile_draws* draws,
                            rift_ile_lse* state, void* stream);

/* The same state written to DEVICE state_out (one rift_ile_lse) without a host
 * synchronisation. */
int rift_ile_comp_lnZ_state_async(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                  rift_ile_lse* state_out, void* stream);

/* ---- FP32-mixed form (eq. slowrot:lnL:Decomposed in whitened coordinates).
 *
 * rift_ile_comp_mixed_build prepares it: for each class of detectors with
 * identical U, V the real quadratic form G of the term above (over
 * z = (Re c, Im c), 2 n_comp dimensions) is diagonalised on the host (cyclic
 * Jacobi), and the eigen-directions with eigenvalue > tol * (the largest) are
 * kept.  In those coordinates (whitened data e_k(t) = V^T b(t) / s, template
 * w_k = s V^T z) each detector contributes 1/2 |e_k|^2 - 1/2 |e_k - w_k|^2, the
 * form of the static FP32-mixed path (rift_ile.h), with
 *   w_k = sum_a (Re C~^k_a a1_a + Im C~^k_a a2_a), a1_a + i a2_a = B_a conj(Y)
 * (B_a the whitening's columns of response index a, shared by a class).  The
 * coefficients, harmonics, arrival times and 1/2|e|^2 are double-float; a1,
 * a2 and w use error-free split products; the residual e - w is FP32.  The
 * dropped directions' share of lnL, sum_r (b_r zeta_r - lam_r zeta_r^2 / 2)
 * over them (zeta_r = x v_r . z, b_r = v_r . b), is left out: it is the part
 * of the interpolated data outside the bank's numerical span (about 1e-5 nat
 * within 50 nat of the peak for tol = 1e-14 on a 3G-network SNR-600 point).
 * The build copies nothing from the caller; it runs on `stream` and
 * synchronises it; a second call rebuilds with the new tol.
 * Errors: INVALID_ARG (tol outside (0, 1)), UNSUPPORTED (a form that is not
 * positive, or has an eigenvalue below -max(tol, 1e-10) * the largest; more
 * detectors x response indices than shared memory holds), ALLOC, CUDA. */
int rift_ile_comp_mixed_build(rift_ile_comp* cp, double tol, void* stream);

/* out[0] = the whitened width R the kernels use (kept directions padded to
 * even), out[1] = the largest kept count of a class, out[2] = classes,
 * out[3] = threads per block; all zero before rift_ile_comp_mixed_build. */
int rift_ile_comp_mixed_info(const rift_ile_comp* cp, int32_t out[4]);

/* lnL per draw into DEVICE lnL_out[n] (double), FP32-mixed, on `stream`;
 * draws float32 or float64.  A draw whose arrival time is not finite gets NaN.
 * Errors: INVALID_ARG (also: the mixed form is not built), SHAPE, CUDA. */
int rift_ile_comp_lnL_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws, double* lnL_out,
                            void* stream);

/* lnL (DEVICE [n], may be NULL) and d lnL / d theta into DEVICE grad_out [7][n]
 * (double; parameter-major: ra, dec, psi, incl, phase, lnD, t) from the
 * FP32-mixed form, on `stream`: the chain rule of rift_ile_comp_lnL_grad taken
 * in the whitened coordinates.  lnL is the value rift_ile_comp_lnL_mixed gives;
 * the terms of the gradient that multiply the residual e_k - w_k (coefficient
 * and harmonic derivatives) are FP32, the slope of 1/2 |e_k|^2 in t_k is
 * double-float.  A draw whose arrival time is not finite gets NaN throughout.
 * Errors: INVALID_ARG (also: the mixed form is not built, grad_out NULL),
 * UNSUPPORTED (the adjoint's per-thread slots exceed the device's shared
 * memory), CUDA. */
int rift_ile_comp_lnL_grad_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                 double* lnL_out, double* grad_out, void* stream);

/* LSE state of the draws (fused lnL -> LSE, FP32-mixed lnL, FP64 combine) to
 * HOST *state; synchronises; out-of-table taps as rift_ile_comp_lnZ_state. */
int rift_ile_comp_lnZ_state_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                  rift_ile_lse* state, void* stream);

/* The same state written to DEVICE state_out without a host synchronisation. */
int rift_ile_comp_lnZ_state_mixed_async(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                        rift_ile_lse* state_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
