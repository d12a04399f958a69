// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/rift_ile.h"

void rift_ile_set_error(const char* fmt, ...);

namespace rift {

constexpr int kMaxDet = RIFT_ILE_MAX_DET;
constexpr int kMaxModes = RIFT_ILE_MAX_MODES;
constexpr int kMaxDim = 2 * RIFT_ILE_MAX_MODES;  // real dimension D = 2M
constexpr int kMaxYTerms = 12;                   // terms of one Goldberg sum, l <= 8
constexpr int kMaxEll = RIFT_ILE_MAX_ELL;
constexpr int kNpar = RIFT_ILE_NPAR;

// Anchors of the double-float sine/cosine: a_j = j h, h = 2^-7, |j| <= kAnchorHalf.
constexpr int kAnchorHalf = 416;
constexpr float kAnchorStep = 0.0078125f;  // 2^-7
constexpr float kAnchorInvStep = 128.0f;
// Anchors of the double-float exponential: e^(j/128), |j| <= kExpHalf.
constexpr int kExpHalf = 46;
constexpr int kPolyDeg = 6;  // 1/2 |e(f)|^2 on one table interval is a sextic in f
// Zero rows stored before and after each detector's whitened table, so that
// any tap window whose first tap lies in [-kEhatPad, n] reads rows in memory.
constexpr int kEhatPad = 4;
// Length in float4 of a table of the intervals' cubic coefficients alone
// (3 float4 per direction pair and interval; the composite response's).
inline size_t ecub_f4(int K, int n, int R) { return (size_t)K * (n + 5) * (R / 2) * 3; }
// Float4 per interval record of PointParams::erec: the interval's cubic
// coefficients followed by its 1/2 |e|^2 sextic (7 pairs + 1).
inline int erec_rec_f4(int R) { return 3 * (R / 2) + 4; }
inline size_t erec_f4(int K, int n, int R) { return (size_t)K * (n + 5) * erec_rec_f4(R); }

// Everything a kernel needs about one intrinsic point.  Lives in device
// memory (one record per point) and is staged into shared memory by each
// block; array pointers are device pointers owned by the point.
struct PointParams {
  int K, M, D, n;   // detectors, modes, real dimension 2M, samples per table
  int q_c128;       // Q element type of the FP64 path (0 complex64, 1 complex128)
  int pad0;
  double gmst, d_ref, dt, inv_dt;
  double t0[kMaxDet];
  double pos[kMaxDet][3];
  double resp[kMaxDet][6];
  // -2Y_lm(iota, phi) = e^{i m phi} sum_r ycoef[r] c^(yk0 + 2r) s^(2l - yk0 - 2r),
  // c = cos(iota/2), s = sin(iota/2); r < ynt.
  int ell[kMaxModes], em[kMaxModes], ynt[kMaxModes], yk0[kMaxModes];
  double ycoef[kMaxModes][kMaxYTerms];
  // double-float copies for the mixed path
  float t0_hi[kMaxDet], t0_lo[kMaxDet];
  float pos_hi[kMaxDet][3], pos_lo[kMaxDet][3];
  float resp_hi[kMaxDet][6], resp_lo[kMaxDet][6];
  // antenna coefficients: F_+(0) = sum_i acoef[i] beta_i(ra, dec), i < 6
  // (Dxx, Dyy, Dxy, Dxz, Dyz, Dzz) and F_x(0) = sum_i acoef[6 + i] gamma_i,
  // i < 4 (Dxx - Dyy, Dxy, Dxz, Dyz); see antenna_basis in lnl_mixed.cu.
  float acoef_hi[kMaxDet][10], acoef_lo[kMaxDet][10];
  // the same split for the mixed path's exact products: acoef_h on the grid
  // 2^(E-9) of the detector's largest |acoef| (< 2^(E+1)), acoef_t the rest
  float acoef_h[kMaxDet][10], acoef_t[kMaxDet][10];
  int same_pos_prev[kMaxDet];  // det_order[q] sits where det_order[q - 1] does
  float gmst_hi, gmst_lo, inv_dt_hi, inv_dt_lo, ln_dref_hi, ln_dref_lo;
  float ycoef_hi[kMaxModes][kMaxYTerms], ycoef_lo[kMaxModes][kMaxYTerms];
  // the same amplitude in z = cos(iota) for the mixed path (c^2 = (1 + z)/2,
  // s^2 = (1 - z)/2, c s = sin(iota)/2): sin(iota)^ypar sum_{j <= l} yz[j] z^j
  int ypar[kMaxModes];
  int morder[kMaxModes];  // mixed path: modes by increasing |m| (stable)
  float yz_hi[kMaxModes][kMaxEll + 1], yz_lo[kMaxModes][kMaxEll + 1];
  // detector classes (identical U_k, V_k share one whitening): the detectors
  // of class c are det_order[cls_begin[c] .. cls_begin[c+1]).
  int R;            // whitened dimension (largest rank over the classes)
  int ncls;
  int cls_begin[kMaxDet + 1];
  int det_order[kMaxDet];
  int cls_of[kMaxDet];
  int has_null[kMaxDet];  // class keeps near-null directions (see point.cu)
  // FP64 path tables
  const void* Q;        // [K][n][M] complex64 or complex128
  const double2* U;     // [K][M][M]
  const double2* V;     // [K][M][M]
  // FP32-mixed path tables (whitened real form, see point.cu), (hi, lo) pairs
  const float2* A;      // [ncls][R][D]  w = A z
  const float* gm1;     // [ncls][R]     1 - lam_r/s_r^2 (0 except kept null directions)
  const float2* ehat;   // [K][n + 2 kEhatPad][R] whitened Q table, zero rows around it
  const float2* epoly;  // [K][n+3][7]   1/2|e(f)|^2 on interval j (index j+2), coefficients of f^0..f^6
  // [K][n + 5][erec_rec_f4(R)]: per interval j = -3..n+1 (index j + 3) the
  // four-tap cubic as coefficients of f, per direction pair (c0 hi, c0 lo),
  // (c1, c2), (c3, 0) with c0 the tap row j itself, then the epoly sextic
  // (zero for j = -3 and n + 1), so that one draw's reads for a detector lie
  // in one contiguous record
  const float4* erec;
  // The shared-memory image of the FP32-mixed kernels' per-point tables (the
  // split whitening, gm1 and the staged detector and mode tables, built once
  // at point creation): the warp-per-draw kernel copies it flat.
  const float4* img;
  int img_f4;           // its length in float4
  int pad1;
};

// Per-launch description of the draws.
struct DrawsParams {
  const void* p[kNpar];  // ra, dec, psi, incl, phase, lnD, t
  const void* logw;
  long long n;
  int f64;
};

// Distance marginalisation table on the device: nodes x_j = D_ref/D_j in
// decreasing order (increasing D) with ln w_j; n == 0 means no marginalisation.
struct DistParams {
  const double* x;
  const double* lnw;
  const float2* xdf;   // x_j as (hi, lo) for the FP32-mixed path
  const float* lnwf;   // ln w_j in FP32
  int n;
  double lnw_max;
  // ln x nearly uniform in j (every node within half a step of the line
  // ln x_0 - j dlnx, x > 0): the FP32-mixed kernels then start the node search
  // from the estimate j = (lnx0 - ln x) inv_dlnx, checked against the table
  int guess;
  float lnx0, inv_dlnx;
};

struct LseState {
  double m, s, s2, n;
};

// Host helpers ---------------------------------------------------------------
int check_cuda(cudaError_t e, const char* what);
// -2Y_lm(iota, phi) = e^{i m phi} sum_r coef[r] c^(k0 + 2r) s^(2l - k0 - 2r),
// c = cos(iota/2), s = sin(iota/2): fills k0 and coef, returns the term count.
int harmonic_coefficients(int l, int m, int* k0, double* coef);
int ensure_anchor_table();  // once per device (sine/cosine and exponential anchors)

}  // namespace rift

struct rift_ile_point {
  rift::PointParams host;        // host copy (pointers are device pointers)
  rift::PointParams* dev;        // device copy
  void* q_copy;                  // owned device copy of Q
  double2* uv;                   // owned U then V
  float2* A;                     // owned
  float* gm1;                    // owned
  float2* ehat;                  // owned
  float2* epoly;                 // owned
  float4* erec;                  // owned
  float4* img;                   // owned
  int device;
};
