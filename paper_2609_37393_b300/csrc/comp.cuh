// Shared declarations of the composite-index response kernels (Sec. III):
// the per-point constants, the per-draw sky geometry with its angle
// derivatives, and the library-owned point object.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/rift_ile_response.h"
#include "rift_ile_internal.h"

namespace rift {

constexpr int kMaxRespIdx = 32;  // response indices a (rotation p_max <= 3)
constexpr int kCompThreads = 128;

struct CompParams {
  int K, M, kind, p_max, na, A, n, nblk;
  int ncls;                 // detector classes: identical (U_k, V_k) share one G
  int cls_of[kMaxDet];
  double omega, gmst, d_ref, dt, inv_dt;
  double t0[kMaxDet];
  double pos[kMaxDet][3];
  double resp[kMaxDet][6];
  double armx[kMaxDet][3], army[kMaxDet][3];
  const double2* Q;  // [K][n][A]
  const double* G;   // [ncls][nblk][4][M][M]: sub-blocks (Re,Re), (Re,Im), (Im,Re), (Im,Im)
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Sky geometry of one draw: sin/cos of dec, of g = gmst - ra and of 2 psi;
// the source direction s and the transverse basis (e1, e2) of the static
// convention, and their derivatives with respect to ra and dec.
struct CompDraw {
  double sd, cd, sg, cg, s2p, c2p;
  double s[3], e1[3], e2[3];
  double ds_ra[3], ds_dec[3], de1_ra[3], de2_ra[3], de2_dec[3];
};

__device__ __forceinline__ CompDraw comp_geometry(const CompParams& C, double ra, double dec,
                                                  double psi) {
  CompDraw g;
  double sl, cl;
  sincos(ra - C.gmst, &sl, &cl);
  sincos(dec, &g.sd, &g.cd);
  g.sg = -sl;  // g = gmst - ra = -lam
  g.cg = cl;
  g.s[0] = g.cd * cl;
  g.s[1] = g.cd * sl;
  g.s[2] = g.sd;
  g.e1[0] = -sl;
  g.e1[1] = cl;
  g.e1[2] = 0.0;
  g.e2[0] = -g.sd * cl;
  g.e2[1] = -g.sd * sl;
  g.e2[2] = g.cd;
  g.ds_ra[0] = -g.cd * sl;
  g.ds_ra[1] = g.cd * cl;
  g.ds_ra[2] = 0.0;
  g.ds_dec[0] = -g.sd * cl;
  g.ds_dec[1] = -g.sd * sl;
  g.ds_dec[2] = g.cd;
  g.de1_ra[0] = -cl;
  g.de1_ra[1] = -sl;
  g.de1_ra[2] = 0.0;
  g.de2_ra[0] = g.sd * sl;
  g.de2_ra[1] = -g.sd * cl;
  g.de2_ra[2] = 0.0;
  g.de2_dec[0] = -g.cd * cl;
  g.de2_dec[1] = -g.cd * sl;
  g.de2_dec[2] = -g.sd;
  sincos(2.0 * psi, &g.s2p, &g.c2p);
  return g;
}

__device__ __forceinline__ double dot3(const double* a, const double* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// The FP32-mixed (whitened) form of a composite point, built by
// rift_ile_comp_mixed_build.  For each class of detectors the real form
// G (2A x 2A, z = (Re c, Im c) over the composite index A = a M + i) is
// diagonalised, G = sum_r lam_r v_r v_r^T, and the directions with
// lam_r > tol lam_max are kept: w_r = s_r v_r . z and e_r(t) = v_r . b(t) / s_r
// (s_r = sqrt(lam_r)), so that per detector
//   lnL_k = 1/2 |e_k(t_k)|^2 - 1/2 |e_k(t_k) - w_k|^2,
//   w_k = sum_a (Re C~^k_a a1_a + Im C~^k_a a2_a),  a1_a = B_a y,  a2_a = B_a J y,
// with B_a the columns of block a of the whitening (rows s_r v_r) and
// y = (Re Y, Im Y) as in the static mixed path.
constexpr int kCompMixedThreads = 128;
constexpr int kCompMixedKG = 4;  // detectors of a class carried together through the r loop

struct CompMixed {
  int K, M, na, A, n, R, ncls, kind, p_max, JP;  // JP: mode pairs of the kernel's bucket
  int cls_begin[kMaxDet + 1], det_order[kMaxDet];
  int pad0;
  float gmst_hi, gmst_lo, inv_dt_hi, inv_dt_lo, ln_dref_hi, ln_dref_lo, omega_hi, omega_lo;
  float4 pos_hi[kMaxDet], pos_lo[kMaxDet];  // (x, y, z, t0) as (hi, lo) vectors
  // rotation: (Dyy - Dxx, 2 Dxy, 2 Dxz, 2 Dyz, Dxx + Dyy, Dzz) of each detector;
  // finite arms: the unit arm vectors X then Y.  (hi, lo) pairs.
  float2 rc[kMaxDet][6];
  int4 mode[kMaxModes];                // visiting order j: (mode index, m, l, parity)
  float2 yz[kMaxModes][kMaxEll + 1];   // the harmonic amplitude's polynomial in cos(iota)
  float inv_fact[RIFT_ILE_MAX_ROT_PMAX + 1];
  // 1/sigma_a: powers of two that bring the coefficients of every response
  // index to a common magnitude (the whitening's columns of index a carry
  // sigma_a), so that one head grid per detector suits all of them
  float inv_sigma[kMaxRespIdx];
  const float4* Bs;    // split whitening [ncls][na][R][JP][3] (see comp_mixed.cu)
  const float* agrid;  // [ncls][R] head constants of a1_a, a2_a per direction (every a)
  const float2* ehat;  // [K][n + 2 kEhatPad][R] whitened table, direction pairs
  const float2* epoly; // [K][n + 3][7] 1/2 |e(f)|^2 per interval
  const float4* ecub;  // [K][n + 5][R/2][3] the intervals' cubic coefficients (PointParams::ecub)
};

// Dynamic shared memory of the mixed composite kernel (float4 units): the
// split whitening (when staged), the head constants, and per thread the
// coefficient slots (K na) and the table-position slots (K).
__host__ __device__ inline size_t comp_mixed_b_f4(const CompMixed& C) {
  return (size_t)C.ncls * C.na * C.R * C.JP * 3;
}
__host__ __device__ inline size_t comp_mixed_ag_f4(const CompMixed& C) {
  return ((size_t)C.ncls * C.R + 3) / 4;
}
// Per-thread float4 slots: the coefficients (K na) and one table-position slot
// per detector; the adjoint adds two per detector (arrival-time derivatives,
// post-phase step), the residual products rho (K na float2), the current
// direction pair's a1, a2 (na) and d lnL / dY of the mode pairs (JP).
__host__ __device__ inline size_t comp_mixed_thread_f4(const CompMixed& C, bool grad) {
  size_t f = (size_t)C.K * C.na + C.K;
  if (grad) f += 2 * C.K + ((size_t)C.K * C.na + 1) / 2 + C.na + C.JP;
  return f;
}
__host__ __device__ inline size_t comp_mixed_smem(const CompMixed& C, bool bsmem, int threads,
                                                  bool grad = false) {
  return ((bsmem ? comp_mixed_b_f4(C) : 0) + comp_mixed_ag_f4(C) +
          comp_mixed_thread_f4(C, grad) * threads) * 16;
}

}  // namespace rift

struct rift_ile_comp {
  rift::CompParams host;
  rift::PointParams* dev_base;  // harmonics of the modes (device)
  double2* q;                   // owned copy of Q
  double* G;                    // owned quadratic-form blocks
  int device;
  int host_ell[rift::kMaxModes], host_em[rift::kMaxModes];
  std::vector<double> Gfull;    // [ncls][2A][2A] the real form of each class (host)
  // FP32-mixed form (rift_ile_comp_mixed_build); mixed_built = 0 until then
  int mixed_built;
  int mixed_R[rift::kMaxDet];   // kept directions of each class
  int mixed_threads, mixed_bsmem;  // launch shape: block size, split whitening in shared memory
  int mixed_minb;                  // lnL kernel variant: sized for 2 or 3 resident blocks per SM
  int grad_threads, grad_bsmem;    // the same for the adjoint
  double mixed_tol;
  rift::CompMixed mixed;        // host copy (pointers are device pointers)
  rift::CompMixed* mixed_dev;   // device copy
  float4* Bs;
  float* agrid;
  float2* ehat;
  float2* epoly;
  float4* ecub;
};
