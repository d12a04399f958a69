// Shared declarations of the composite-index response kernels (Sec. III):
// the per-point constants, the per-draw sky geometry with its angle
// derivatives, and the library-owned point object.
#pragma once
#include <cuda_runtime.h>

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

}  // namespace rift

struct rift_ile_comp {
  rift::CompParams host;
  rift::PointParams* dev_base;  // harmonics of the modes (device)
  double2* q;                   // owned copy of Q
  double* G;                    // owned quadratic-form blocks
  int device;
};
