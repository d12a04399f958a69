/* rift_ile_precompute.h -- GPU precompute of the per-point products of
 * eq. QUV ("Scaling RIFT 1", arXiv 2609.37393, Sec. II.A; the fine-table
 * pregrid of eq. q-time-pregrid), C ABI, FP64.
 *
 * On a two-sided uniform frequency grid f_q = (q - (nf - 1)/2) df, q < nf
 * (nf odd, so that -f_q is the grid entry nf - 1 - q), with inner-product
 * weights w_k(f_q) (2 df / S_k(|f|) inside the band, 0 outside):
 *
 *   Q_{k,lm}(t) = sum_q w_k(f_q) e^{2 pi i f_q t} conj(h_lm(f_q)) d_k(f_q)
 *   U_{k,ij}    = sum_q w_k(f_q) conj(h_i(f_q)) h_j(f_q)
 *   V_{k,ij}    = sum_q w_k(f_q) h_i(-f_q) h_j(f_q)
 *
 * Q is produced on the table t = q_t0[k] + j q_dt, j < q_len, by one
 * zero-padded inverse FFT of length nfft = 1 / (df q_dt) per (detector, mode)
 * (cuFFT, double complex, batched): the frequency series times
 * e^{2 pi i f t0} is scattered to the FFT bins f / df mod nfft, which makes
 * sample j of the transform exactly the sum above at t0 + j dt.  U and V are
 * block reductions in a fixed order (bitwise reproducible) over the pairs
 * i <= j, the rest filled by U_ji = conj(U_ij) and V_ji = V_ij: the weights
 * must be even in f (w_k(-f) = w_k(f), as for a one-sided noise curve).
 *
 * Requirements: 1 / (df q_dt) within 1e-9 of an integer nfft >= max(nf,
 * q_len); nf odd; K <= RIFT_ILE_MAX_DET, M <= RIFT_ILE_MAX_MODES.
 * Ownership: the caller owns every buffer; the call allocates its FFT work
 * buffer (K M nfft complex doubles) stream-ordered and frees it before
 * returning, and keeps one cuFFT plan per (device, nfft, batch) until
 * rift_ile_release.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA (cuFFT failures included),
 * ALLOC.
 */
#ifndef RIFT_ILE_PRECOMPUTE_H
#define RIFT_ILE_PRECOMPUTE_H
#include "rift_ile.h"

#ifdef __cplusplus
extern "C" {
#endif

/*   hlm   DEVICE [M][nf] complex128 (re, im interleaved): the mode spectra
 *   dk    DEVICE [K][nf] complex128: the data of each detector
 *   wgt   DEVICE [K][nf] double: inner-product weights
 *   q_t0  HOST [K] time of table sample 0, seconds
 *   q_dtype  RIFT_ILE_C64 or RIFT_ILE_C128: element type of Q_out */
typedef struct {
  int32_t n_det;
  int32_t n_modes;
  int32_t nf;
  double df;
  const double* hlm;
  const double* dk;
  const double* wgt;
  const double* q_t0;
  double q_dt;
  int32_t q_len;
  int32_t q_dtype;
} rift_ile_precompute_desc;

/* Q_out: DEVICE [K][q_len][M] complex (q_dtype); U_out, V_out: DEVICE
 * [K][M][M] complex128.  Any of the three may be NULL to skip it. */
int rift_ile_precompute(const rift_ile_precompute_desc* desc, void* Q_out, double* U_out,
                        double* V_out, void* stream);

/* The widened bank of Earth-rotation templates of Sec. III.A,
 * chi^(p,n)_lm = M_n h_lm^(p) (eq. slowrot:master), built as Appendix B
 * describes: the p-th time derivative as the weight (2 pi i f)^p on the
 * frequency grid, then the sidereal modulation e^{i n Omega t} applied as a
 * linear phase in the time domain through one DFT round trip over the grid's
 * period 1/df (times centred on the reference time, t_j = j' / (nf df),
 * j' in [-(nf-1)/2, (nf-1)/2]).  Composite order as in rift_ile_response.h:
 * row a * M + i with a = (p, n), p = 0..p_max, n = -(2+p)..(2+p).
 *   hlm       DEVICE [M][nf] complex128 on the two-sided grid (nf odd)
 *   bank_out  DEVICE [n_index * M][nf] complex128
 * Allocates its work buffers stream-ordered and frees them before returning;
 * asynchronous on `stream`.  Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA,
 * ALLOC. */
int rift_ile_rotation_bank(const double* hlm, int32_t n_modes, int32_t nf, double df,
                           double omega, int32_t p_max, double* bank_out, void* stream);

/* The finite-arm bank of Sec. III.B (Path D): chi^(p)_lm(f) =
 * e^{-2 pi i f T} W_p(pi f T) h_lm(f), p = 0..p_max (eq. fsize:factorization),
 * with W_p the Taylor coefficients in u of the residual arm transfer D^(u, x)
 * (eq. fsize:Wp), taken by a 64-point Cauchy integral over |u| = 1 (D^ is
 * entire in u) for each frequency; T is the detector's one-way light time
 * L / c, seconds.  Rows p * M + i of bank_out DEVICE [(p_max + 1) M][nf]
 * complex128.  Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA. */
int rift_ile_arm_bank(const double* hlm, int32_t n_modes, int32_t nf, double df, double T,
                      int32_t p_max, double* bank_out, void* stream);

/* The fine table of eq. q-time-pregrid from a native-rate one: per
 * (detector, mode) series q_j = Q(t0 + j h), j < n, the reflected series
 * q_0 .. q_{n-1}, q_{n-1} .. q_0 of length 2n (its periodic extension is
 * continuous), its DFT, the coefficients zero-padded to length 2 r n (the
 * Z_r of eq. q-time-pregrid: frequencies 0 .. n-1 first, -(n-1) .. -1 last,
 * zeros between; the reflected series has no Nyquist component), and the
 * inverse DFT scaled by 1/(2n): sample m is the trigonometric interpolant
 * of the reflected series at t0 + m h / r, and the fine table passes
 * through every native sample (m = r j).  The first r (n - 1) + 1 samples,
 * the native window, are written.  The four-point cubic of the likelihood
 * kernels then reads the fine table (eq. ap:q-pregrid-rate: h = 1/4096 s,
 * r = 8 gives 32 768 Hz).  Two batched cuFFT transforms (lengths 2n and
 * 2rn, K M series each) in FP64.
 *   Q_native  DEVICE [K][n][M] complex, q_dtype_in RIFT_ILE_C64 or RIFT_ILE_C128
 *   Q_fine    DEVICE [K][r (n - 1) + 1][M] complex, q_dtype_out likewise
 * Requirements: K, M >= 1, K M <= 4096, n >= 1, 1 <= r <= 64,
 * 2 r n <= 2^27.  Ownership: the caller owns both tables (they must not
 * overlap); the call allocates its two FFT work buffers (K M 2n and
 * K M 2rn complex doubles) stream-ordered and frees them before returning,
 * and keeps one cuFFT plan per (device, length, batch) until
 * rift_ile_release.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA (cuFFT failures included),
 * ALLOC. */
int rift_ile_pregrid(const void* Q_native, int32_t n_det, int32_t n_modes, int32_t n,
                     int32_t q_dtype_in, int32_t r, void* Q_fine, int32_t q_dtype_out,
                     void* stream);

#ifdef __cplusplus
}
#endif
#endif
