/* rift_ile.h -- C ABI of the extrinsic-marginalised likelihood (ILE) stage of
 * RIFT ("Scaling RIFT 1", arXiv 2609.37393), for one NVIDIA B300 (sm_103a).
 *
 * What the library computes (Sec. II.A-II.C of the paper):
 *
 *   lnL(theta) = x Re sum_k sum_lm (F_k Y_lm)^* Q_{k,lm}(t_k)
 *              - x^2/4 sum_k sum_{lm,l'm'} [ |F_k|^2 Y_lm^* Y_l'm' U_{k,lm,l'm'}
 *                                            + Re(F_k^2 Y_lm Y_l'm' V_{k,lm,l'm'}) ]
 *                                                        (eq. def:lnL:Decomposed)
 *   with theta = (ra, dec, psi, incl, phase, lnD, t_c), x = D_ref/D = D_ref e^{-lnD},
 *   F_k = F_+ - i F_x the antenna factor of detector k, t_k = t_c - x_k . s its
 *   arrival time, Y_lm = -2Y_lm(incl, phase), and Q_{k,lm}(t) read from a fine
 *   uniform table by the four-point cubic C_3 (eq. q-time-pregrid);
 *
 *   lnZ = ln[(1/N) sum_i exp(lnL_i + ln w_i)], w_i = p(theta_i)/p_s(theta_i)
 *                                         (eq. lnL:MonteCarlo), with its
 *   delta-method standard error and n_eff = sum w / max w (eq. neff);
 *
 *   the gradient of lnL with respect to the seven extrinsic parameters
 *   (Sec. II.B), and the distance-marginalised lnL on a log-uniform lnD node
 *   table (eq. ap:dexp, eq. ap:dlog).
 *
 * Conventions.  Times are seconds relative to a reference time chosen by the
 * caller; angles are radians; positions are light-seconds in an Earth-fixed
 * frame; the source direction s points from the geocentre to the source;
 * the polarisation basis is e1 = (-sin lam, cos lam, 0), e2 = (-sin dec cos lam,
 * -sin dec sin lam, cos dec) with lam = ra - gmst, p = cos psi e1 + sin psi e2,
 * q = -sin psi e1 + cos psi e2, F_+ = p.D.p - q.D.q, F_x = 2 p.D.q; the Q cubic
 * is the Lagrange cubic on taps j-1..j+2, j = floor((t - t0_k)/dt), and taps
 * outside the table read as zero (they are counted, see rift_ile_last_oob).
 *
 * Ownership.  The caller owns every buffer it passes.  rift_ile_point_create
 * copies what it needs (device-to-device for Q) into a point object that the
 * library owns until rift_ile_point_destroy.  Calls are asynchronous on the
 * caller's stream unless stated; the host-scalar forms of lnZ synchronise.
 *
 * Errors.  Every entry point returns 0 on success or a negative RIFT_ILE_ERR_*
 * code; rift_ile_last_error() gives a thread-local message.  Non-finite draws
 * give a NaN lnL for that draw, not an error.
 */
#ifndef RIFT_ILE_H
#define RIFT_ILE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  RIFT_ILE_OK = 0,
  RIFT_ILE_ERR_INVALID_ARG = -1, /* null pointer, bad enum, non-finite scalar */
  RIFT_ILE_ERR_SHAPE = -2,       /* inconsistent sizes */
  RIFT_ILE_ERR_UNSUPPORTED = -3, /* K, M or l outside the compiled limits */
  RIFT_ILE_ERR_CUDA = -4,        /* a CUDA call failed; message carries its text */
  RIFT_ILE_ERR_TIMEOUT = -5,     /* a bounded device wait expired */
  RIFT_ILE_ERR_ALLOC = -6        /* device or host allocation failed */
};

#define RIFT_ILE_MAX_DET 8    /* K */
#define RIFT_ILE_MAX_MODES 16 /* M */
#define RIFT_ILE_MAX_ELL 8    /* l of every mode */
#define RIFT_ILE_NPAR 7       /* ra, dec, psi, incl, phase, lnD, t */

typedef enum {
  RIFT_ILE_FP64 = 0,      /* every step in IEEE double */
  RIFT_ILE_FP32_MIXED = 1 /* FP32 template, double-float contractions */
} rift_ile_precision;

typedef enum { RIFT_ILE_F32 = 0, RIFT_ILE_F64 = 1 } rift_ile_dtype;
typedef enum { RIFT_ILE_C64 = 0, RIFT_ILE_C128 = 1 } rift_ile_cdtype;

/* One intrinsic point: the precomputed products of eq. QUV and the network.
 *   Q      DEVICE [K][q_len][M] complex (re, im interleaved), float (C64) or
 *          double (C128): Q_{k,lm}(q_t0[k] + j q_dt), j = 0..q_len-1 (eq. QUV,
 *          sampled on the fine table of eq. q-time-pregrid)
 *   U, V   HOST [K][M][M][2] double: U_{k,i,j} = <h_i|h_j>_k (Hermitian),
 *          V_{k,i,j} = <h_i^*|h_j>_k (complex symmetric)  (eq. QUV)
 *   ell,em HOST [M] mode indices, 2 <= l <= RIFT_ILE_MAX_ELL, |m| <= l
 *   det_pos  HOST [K][3] detector positions, light-seconds
 *   det_resp HOST [K][6] response tensors D_k: xx, xy, xz, yy, yz, zz
 *   q_t0   HOST [K] time of table sample 0, seconds
 *   gmst   Greenwich sidereal angle at the reference time, rad
 *   d_ref  the reference distance of the modes (same unit as e^{lnD}) */
typedef struct {
  int32_t n_det;
  int32_t n_modes;
  const int32_t* ell;
  const int32_t* em;
  const void* Q;
  int32_t q_dtype;
  int32_t q_len;
  const double* q_t0;
  double q_dt;
  const double* U;
  const double* V;
  const double* det_pos;
  const double* det_resp;
  double gmst;
  double d_ref;
} rift_ile_point_desc;

typedef struct rift_ile_point rift_ile_point; /* opaque, library-owned */

/* Extrinsic draws: DEVICE structure-of-arrays, each [n] of `dtype`; logw
 * (ln p - ln p_s per draw) may be NULL (all zero). */
typedef struct {
  const void* ra;
  const void* dec;
  const void* psi;
  const void* incl;
  const void* phase;
  const void* lnD;
  const void* t;
  const void* logw;
  int64_t n;
  int32_t dtype;
} rift_ile_draws;

/* Prepares a point for evaluation: validates the description, copies Q,
 * builds the constant tables of both precisions (for FP32_MIXED: the
 * eigen-decomposition of each detector's real quadratic form and the
 * whitened, double-float Q table; see the design notes).  Runs on `stream`
 * (a cudaStream_t, NULL = legacy default stream) and synchronises it.
 * Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA, ALLOC. */
int rift_ile_point_create(const rift_ile_point_desc* desc, rift_ile_point** out, void* stream);
int rift_ile_point_destroy(rift_ile_point* pt);

/* Shape of a prepared point (HOST out[6]): K, M, table length, the whitened
 * dimension R (the rank of the quadratic form of eq. def:lnL:Decomposed in
 * real coordinates; M for aligned-spin mode pairs), the number of detector
 * classes (detectors with identical U and V) and whether any class kept its
 * near-null directions.  Errors: INVALID_ARG. */
int rift_ile_point_info(const rift_ile_point* pt, int32_t out[6]);

/* lnL per draw (eq. def:lnL:Decomposed) into DEVICE lnL_out[n] (double), on
 * `stream`, asynchronous.  Errors: INVALID_ARG, SHAPE, CUDA. */
int rift_ile_lnL(const rift_ile_point* pt, const rift_ile_draws* draws, rift_ile_precision prec,
                 double* lnL_out, void* stream);

/* lnL (DEVICE [n], may be NULL) and d lnL / d theta into DEVICE grad_out
 * [7][n] (double; parameter-major: ra, dec, psi, incl, phase, lnD, t), on
 * `stream`, asynchronous.  Sec. II.B. */
int rift_ile_lnL_grad(const rift_ile_point* pt, const rift_ile_draws* draws,
                      rift_ile_precision prec, double* lnL_out, double* grad_out, void* stream);

/* Log-sum-exp state of a set of draws: m = max_i (lnL_i + ln w_i),
 * s = sum_i exp(lnL_i + ln w_i - m), s2 = sum_i exp(2 (lnL_i + ln w_i - m)),
 * n = number of draws.  States of disjoint draw sets merge exactly (see
 * rift_ile_lnZ_merge); lnZ = m + ln s - ln n, sigma_lnZ = sqrt(max(0,
 * s2/s^2 - 1/n)), n_eff = s (eq. lnL:MonteCarlo, eq. neff). */
typedef struct {
  double m, s, s2, n;
} rift_ile_lse;

/* Optional distance marginalisation: HOST node table (x_j = D_ref/D_j,
 * ln w_j) of eq. ap:dlog, built by rift_ile_dist_nodes.  When passed to the
 * lnZ calls, each draw's lnL is replaced by ln sum_j exp(K x_j - R x_j^2/2 +
 * ln w_j) with K, R the data and quadratic terms at x = 1 (eq. ap:dexp), and
 * the draw's own lnD is ignored. */
typedef struct {
  const double* x;
  const double* lnw;
  int32_t n;
} rift_ile_dist;

/* Node table of eq. ap:dlog: spacing in ln D of at most c(tol)/rho_max,
 * c(tol) = pi sqrt(2/ln(2/tol)), over [d_min, d_max], trapezoid weights in
 * ln D, prior p(D) = 3 D^2/(d_max^3 - d_min^3).  Writes up to max_nodes nodes
 * into HOST x[], lnw[]; *n_out receives the count.  Errors: INVALID_ARG,
 * SHAPE (table larger than max_nodes). */
int rift_ile_dist_nodes(double d_min, double d_max, double d_ref, double tol, double rho_max,
                        int32_t max_nodes, double* x, double* lnw, int32_t* n_out);

/* Distance-marginalised lnL per draw into DEVICE lnL_out[n] (double):
 * ln sum_j exp(K x_j - R x_j^2/2 + ln w_j), K and R the data and quadratic
 * terms of the draw at x = 1 (eq. ap:dexp); the draw's lnD is ignored.  With
 * grad_out (DEVICE [7][n], may be NULL) also its gradient, E[x] dK -
 * E[x^2] dR / 2 over the node posterior (the lnD slot is 0).  The node table
 * is copied to the device first (synchronous), then the kernel is enqueued
 * on `stream`.  Errors: INVALID_ARG (NULL, non-finite or non-decreasing
 * table), SHAPE, CUDA, ALLOC. */
int rift_ile_lnL_dist(const rift_ile_point* pt, const rift_ile_draws* draws, rift_ile_precision prec,
                      const rift_ile_dist* dist, double* lnL_out, double* grad_out, void* stream);

/* Monte Carlo lnZ of the draws (eq. lnL:MonteCarlo), fused with the lnL
 * evaluation (per-draw lnL is not stored).  out[3] (HOST) = lnZ, sigma_lnZ,
 * n_eff.  dist may be NULL.  Synchronises `stream`. */
int rift_ile_lnZ(const rift_ile_point* pt, const rift_ile_draws* draws, rift_ile_precision prec,
                 const rift_ile_dist* dist, double out[3], void* stream);

/* Same, returning the LSE state (HOST) instead, for chunked streaming and for
 * merging the partial results of several devices or processes. */
int rift_ile_lnZ_state(const rift_ile_point* pt, const rift_ile_draws* draws,
                       rift_ile_precision prec, const rift_ile_dist* dist, rift_ile_lse* state,
                       void* stream);

/* rift_ile_lnZ_state without a host round trip: enqueues the fused kernel and
 * the merge of its block partials on `stream` and writes the LSE state
 * (one rift_ile_lse, 32 bytes) to DEVICE memory state_out when they complete;
 * nothing is synchronised (except the copy of a distance table, which is
 * uploaded first as in rift_ile_lnZ_state), so many evaluations can be
 * chained on a stream and their states read once.  Uses the library's per-device workspace
 * (allocated on the first call of any lnZ entry point on the device; make
 * that first call before capturing a stream).  Calls on one device share the
 * workspace: calls that overlap on the GPU (different streams) race; calls
 * on one stream are ordered.  The out-of-table count of rift_ile_last_oob is
 * not updated.  Errors: INVALID_ARG, SHAPE, CUDA, ALLOC. */
int rift_ile_lnZ_state_async(const rift_ile_point* pt, const rift_ile_draws* draws,
                             rift_ile_precision prec, const rift_ile_dist* dist,
                             rift_ile_lse* state_out, void* stream);

/* rift_ile_lnZ_state without any allocation (the paper has no counterpart:
 * this is a deployment variant).  For callers that may not allocate device
 * memory while they run: a framework that owns the device heap through its
 * own pool and forbids other cudaMalloc/cudaFree calls, or a time-critical
 * loop where an allocation could block or fail.  Same arguments and result
 * as rift_ile_lnZ_state with dist = NULL; it never calls cudaMalloc,
 * cudaFree or an allocating library routine.  Its scratch (per-block LSE
 * partials, about 128 KB) is a fixed static device array that every GPU
 * loading the library holds until exit; a device with more than 256 SMs is
 * rejected with RIFT_ILE_ERR_UNSUPPORTED.  The first call on a device looks
 * up that array's device address (cudaGetSymbolAddress) with the device
 * current, so make it before any stream capture.  All calls on a device
 * share the array: calls whose work overlaps on the GPU race and must be
 * serialised.  rift_ile_release forgets the looked-up addresses (call it
 * after a device reset; the next call looks them up again).  Sets the count
 * of rift_ile_last_oob like rift_ile_lnZ_state.  Synchronises `stream`.
 * Errors: INVALID_ARG, SHAPE, UNSUPPORTED, CUDA. */
int rift_ile_lnZ_state_noalloc(const rift_ile_point* pt, const rift_ile_draws* draws,
                               rift_ile_precision prec, rift_ile_lse* state, void* stream);

/* rift_ile_lnZ_state for draws in HOST memory (the end-to-end path; the
 * paper's sampler produces draws on the host): the seven parameter arrays and
 * logw of host_draws are HOST pointers (page-locked memory lets the copies
 * overlap the kernels; pageable memory works but serialises).  The draws are
 * copied in chunks of `chunk` draws (0: 2^20) into two library-owned device
 * staging buffers on a library copy stream, double-buffered against the fused
 * lnL -> LSE kernel on `stream`; the per-chunk block partials are merged once
 * at the end in a fixed order.  The result agrees with rift_ile_lnZ_state on
 * the same draws to rounding (the partials group the draws differently).
 * Synchronous: returns when both streams are idle; not capturable in a graph;
 * concurrent calls on one process are serialised (they share the buffers).
 * Allocates the staging buffers and partials on first use (grown on demand,
 * freed by rift_ile_release).  The host arrays must stay valid until return.
 * Errors: INVALID_ARG, SHAPE, CUDA, ALLOC. */
int rift_ile_lnZ_state_host(const rift_ile_point* pt, const rift_ile_draws* host_draws,
                            rift_ile_precision prec, const rift_ile_dist* dist, int64_t chunk,
                            rift_ile_lse* state, void* stream);

/* Exact merge of S LSE states (HOST) into out[3] = lnZ, sigma_lnZ, n_eff;
 * merged_state (may be NULL) receives the merged state.  Host only. */
int rift_ile_lnZ_merge(const rift_ile_lse* states, int32_t S, double out[3],
                       rift_ile_lse* merged_state);

/* lnZ of P points in one launch (the ILE stage over many intrinsic points,
 * Sec. II.C): point p uses pts[p] and draws[p] (each point its own Q, U, V,
 * network and draw count).  FP32_MIXED runs one persistent kernel per group
 * of points that share a compiled kernel shape (mode-count bucket and
 * whitened width); its resident blocks take (point, tile) items (4096 draws
 * unless tuned by rift_ile_batch_tune) from the group's queue by an atomic
 * ticket, one LSE state per item, merged per point in item order (the result
 * does not depend on scheduling); FP64 runs the plain fused kernel once per
 * point.  out is DEVICE [P][3] double: lnZ, sigma_lnZ, n_eff per point.
 *
 * rift_ile_batch_create builds the work queue and the device tables once
 * (allocates, synchronous); rift_ile_batch_launch only enqueues a memset,
 * the kernel(s) and the per-point combine on `stream`, so it can be captured
 * in a CUDA graph and replayed; the draws must stay valid and unchanged in
 * place between create and the last launch.  rift_ile_lnZ_batch is
 * create + launch + synchronise + destroy.
 * Errors: INVALID_ARG, SHAPE, CUDA, ALLOC. */
typedef struct rift_ile_batch rift_ile_batch; /* opaque, library-owned */
int rift_ile_batch_create(const rift_ile_point* const* pts, const rift_ile_draws* draws, int32_t P,
                          rift_ile_precision prec, rift_ile_batch** out);
int rift_ile_batch_launch(rift_ile_batch* batch, double* out, void* stream);
int rift_ile_batch_destroy(rift_ile_batch* batch);

/* Autotuner of an FP32_MIXED batch (measurement support; the paper has no
 * counterpart).  Times rift_ile_batch_launch on `stream` (one warm-up and
 * `reps` timed launches, CUDA events) for every draw-tile size in
 * {512, 1024, 2048, 4096, 8192, 16384} and every grid of {1, 3/4, 1/2} times
 * the kernel's resident-block limit, then rebuilds the work queue for the
 * fastest pair, which later launches use.  The result of a launch depends on
 * the tile size only through the grouping of the per-item merges (lnZ
 * agrees to rounding).  Synchronous; allocates; do not call while a graph
 * holding this batch's launch may replay (the queue is reallocated: capture
 * after tuning).  tile_out, blocks_out (the chosen configuration) and ms_out
 * (its time per launch, -1 for FP64 batches, which have nothing to tune) may
 * be NULL.  Errors: INVALID_ARG (NULL batch, reps < 1), CUDA, ALLOC. */
int rift_ile_batch_tune(rift_ile_batch* batch, int32_t reps, void* stream, int32_t* tile_out,
                        int32_t* blocks_out, double* ms_out);
int rift_ile_lnZ_batch(const rift_ile_point* const* pts, const rift_ile_draws* draws, int32_t P,
                       rift_ile_precision prec, double* out, void* stream);

/* Draw count up to which rift_ile_lnL and rift_ile_lnL_grad with
 * RIFT_ILE_FP32_MIXED run the warp-pair kernel: two warps share one draw
 * (one takes the sky, the detectors and the sums, the other the harmonics,
 * the mat-vec and the adjoint's mode terms, each phase across its lanes),
 * which cuts the latency of a small batch, the regime of a gradient-based
 * extrinsic sampler (App. H of the paper: tens to thousands of draws per
 * call).  Larger batches use the one-thread-per-draw kernels, whose
 * throughput is higher.  The two agree to rounding.  The warp-pair kernel is
 * launched with programmatic stream serialisation: its prologue (the point's
 * tables into shared memory) may overlap the previous kernel in the stream,
 * and it reads the draws and writes its outputs only after that kernel has
 * completed; it lets the next kernel in the stream do the same (a kernel
 * launched after it with that attribute must itself wait before reading its
 * outputs).  Default 2048; 0 disables the warp kernel.  Process-wide; returns
 * the previous value.  Host only, no GPU call. */
int64_t rift_ile_set_small_batch(int64_t max_draws);

/* Number of Q taps that fell outside their tables in the last completed
 * lnZ call of this thread (host read; the draws get zero Q there). */
int64_t rift_ile_last_oob(void);

/* Frees the library's per-device workspace (LSE partials, batch queues). */
int rift_ile_release(void);

const char* rift_ile_last_error(void);

/* ALU issue-rate probes used as roofline denominators (measurement support;
 * the paper has no counterpart).  ops_per_second counts one FMA as one op;
 * FP32X2_FMA issues packed pair FMAs (two ops per instruction). */
enum {
  RIFT_ILE_PROBE_FP32_FMA = 0,
  RIFT_ILE_PROBE_FP64_FMA = 1,
  RIFT_ILE_PROBE_MUFU_EX2 = 2,
  RIFT_ILE_PROBE_MUFU_SIN = 3,
  RIFT_ILE_PROBE_FP32X2_FMA = 4
};
int rift_ile_probe_alu(int which, double target_seconds, double* ops_per_second, double* sm_mhz);

#ifdef __cplusplus
}
#endif
#endif
