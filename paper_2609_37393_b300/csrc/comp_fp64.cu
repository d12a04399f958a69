// Composite-index response (Sec. III): Earth rotation (Paths A and B) and
// finite arms (Path D), FP64, one draw per thread.
//
// Per draw the static kernel's sky geometry and harmonics are reused; the
// antenna factor F_k is replaced by the per-draw coefficients C~^k_a:
//
// * rotation: with m = e^{i psi}(e1 - i e2) the antenna factor is
//   F = m^T D m.  In Earth-fixed axes e1 - i e2 = e^{i lam} v+ + e^{-i lam} v- + v0,
//   lam = ra - GMST = -g, v+ = (1+sin dec)/2 (i, 1, 0), v- = (1-sin dec)/2 (-i, 1, 0),
//   v0 = (0, 0, -i cos dec), so F is a trigonometric polynomial of degree 2 in g
//   whose coefficients are bilinear forms of v+, v-, v0 with D (eq.
//   slowrot:Fharm):  A_-2 = v+Dv+, A_2 = v-Dv-, A_-1 = 2 v+Dv0, A_1 = 2 v-Dv0,
//   A_0 = 2 v+Dv- + v0Dv0, each times e^{2 i psi}.  The arrival-time drift
//   -(t_k(t) - t_k(0)) = cos(dec) Re[w (e^{i Omega t} - 1)], w = (x + i y) e^{i g},
//   has harmonics cos(dec) w/2, -cos(dec) Re w, cos(dec) conj(w)/2 at
//   n = 1, 0, -1.  C_(p, n) is the n-th harmonic of F (-dt)^p / p! (eq.
//   slowrot:delay, eq. slowrot:master), a discrete convolution, and the
//   post-phase e^{i n Omega t_k} (eq. slowrot:postphase) multiplies it.
// * finite arms: b_p = 1/2 [(X.s)^p (m.X)^2 - (Y.s)^p (m.Y)^2] (eq. fsize:bp).
//
// The data term is the four-tap cubic of the widened table, and the quadratic
// term one real symmetric form per detector, z^T G z with z = (Re c, Im c) of
// c = C~ (x) Y: G is stored as blocks over pairs a <= a' of response indices
// ([2M][2M] each, off-diagonal blocks doubled), so that a thread holds the
// two M-vectors of one block pair in registers and streams G (the same
// addresses for every lane) from L1.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "comp.cuh"
#include "common.cuh"
#include "kernels.h"

namespace rift {

namespace {

constexpr int kClassCoef = 64;  // detectors x response indices kept for the class pass

// C~^k_a of one detector (composite order), out[na].
__device__ void comp_coeffs(const CompParams& C, int k, double sd, double cd, double sg,
                            double cg, double s2p, double c2p, double tk, const double s[3],
                            const double e1[3], const double e2[3], double2* out) {
  if (C.kind == RIFT_ILE_RESP_FINITE_ARM) {
    const double* X = C.armx[k];
    const double* Yv = C.army[k];
    const double ax = e1[0] * X[0] + e1[1] * X[1] + e1[2] * X[2];
    const double bx = e2[0] * X[0] + e2[1] * X[1] + e2[2] * X[2];
    const double ay = e1[0] * Yv[0] + e1[1] * Yv[1] + e1[2] * Yv[2];
    const double by = e2[0] * Yv[0] + e2[1] * Yv[1] + e2[2] * Yv[2];
    const double ux = s[0] * X[0] + s[1] * X[1] + s[2] * X[2];
    const double uy = s[0] * Yv[0] + s[1] * Yv[1] + s[2] * Yv[2];
    // (m.X)^2 = e^{2 i psi} (ax - i bx)^2
    const double2 e2p = make_double2(c2p, s2p);
    const double2 qx = cmul(e2p, make_double2(ax * ax - bx * bx, -2.0 * ax * bx));
    const double2 qy = cmul(e2p, make_double2(ay * ay - by * by, -2.0 * ay * by));
    double px = 0.5, py = 0.5;
    for (int p = 0; p <= C.p_max; ++p) {
      out[p] = make_double2(px * qx.x - py * qy.x, px * qx.y - py * qy.y);
      px *= ux;
      py *= uy;
    }
    return;
  }
  const double* D = C.resp[k];  // xx, xy, xz, yy, yz, zz
  const double al = 0.5 * (1.0 + sd), be = 0.5 * (1.0 - sd);
  double2 A[5];  // n = -2..2, before e^{2 i psi}
  A[0] = make_double2(al * al * (D[3] - D[0]), 2.0 * al * al * D[1]);
  A[4] = make_double2(be * be * (D[3] - D[0]), -2.0 * be * be * D[1]);
  A[1] = make_double2(2.0 * al * cd * D[2], -2.0 * al * cd * D[4]);
  A[3] = make_double2(-2.0 * be * cd * D[2], -2.0 * be * cd * D[4]);
  A[2] = make_double2(2.0 * al * be * (D[0] + D[3]) - cd * cd * D[5], 0.0);
  // C_(0,n) = e^{2 i psi} A_n e^{i n g}
  const double2 eg = make_double2(cg, sg), e2g = cmul(eg, eg);
  const double2 e2p = make_double2(c2p, s2p);
  double2 C0[5];
  C0[2] = cmul(e2p, A[2]);
  C0[3] = cmul(cmul(e2p, A[3]), eg);
  C0[4] = cmul(cmul(e2p, A[4]), e2g);
  C0[1] = cmul(cmul(e2p, A[1]), make_double2(cg, -sg));
  C0[0] = cmul(cmul(e2p, A[0]), make_double2(e2g.x, -e2g.y));
  // drift harmonics (m = -1, 0, 1) and the post-phase step e^{i Omega t_k}
  const double* x = C.pos[k];
  const double2 w = cmul(make_double2(x[0], x[1]), eg);
  const double2 E[3] = {make_double2(0.5 * cd * w.x, -0.5 * cd * w.y), make_double2(-cd * w.x, 0.0),
                        make_double2(0.5 * cd * w.x, 0.5 * cd * w.y)};
  double so, co;
  sincos(C.omega * tk, &so, &co);
  const double2 ep = make_double2(co, so);
  double2 P[2 * RIFT_ILE_MAX_ROT_PMAX + 1];  // harmonics of (-dt)^p, index m + p
  P[0] = make_double2(1.0, 0.0);
  int off = 0;
  double inv_fact = 1.0;
  for (int p = 0; p <= C.p_max; ++p) {
    if (p > 0) {
      inv_fact /= (double)p;
      // P <- P * E (width 2p - 1 -> 2p + 1), from the top down
      double2 Pn[2 * RIFT_ILE_MAX_ROT_PMAX + 1];
      for (int j = 0; j < 2 * p + 1; ++j) {
        double2 acc = make_double2(0.0, 0.0);
        for (int e = 0; e < 3; ++e) {
          const int src = j - e;  // P index (m' + p - 1) with m' = m - (e - 1)
          if (src >= 0 && src < 2 * p - 1) {
            const double2 t = cmul(P[src], E[e]);
            acc.x += t.x;
            acc.y += t.y;
          }
        }
        Pn[j] = acc;
      }
      for (int j = 0; j < 2 * p + 1; ++j) P[j] = Pn[j];
    }
    // C_(p, nn) = (1/p!) sum_n C0_n P_(nn - n), nn = -(2+p)..(2+p)
    const int width = 2 * (2 + p) + 1;
    // e^{i nn Omega t_k}, starting at nn = -(2 + p)
    double2 ph = make_double2(1.0, 0.0);
    for (int q = 0; q < 2 + p; ++q) ph = cmul(ph, make_double2(ep.x, -ep.y));
    for (int j = 0; j < width; ++j) {
      const int nn = j - (2 + p);
      double2 acc = make_double2(0.0, 0.0);
      for (int n = -2; n <= 2; ++n) {
        const int m = nn - n;
        if (m >= -p && m <= p) {
          const double2 t = cmul(C0[n + 2], P[m + p]);
          acc.x += t.x;
          acc.y += t.y;
        }
      }
      out[off + j] = cmul(make_double2(acc.x * inv_fact, acc.y * inv_fact), ph);
      ph = cmul(ph, ep);
    }
    off += width;
  }
}

struct CompOut {
  double lnl;
  int oob;
};

template <int MM>
__device__ CompOut comp_lnl_draw(const CompParams& C, const PointParams& P, const DrawsParams& dp,
                                 long long i) {
  const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
  const double psi = load_param_d(dp, 2, i), incl = load_param_d(dp, 3, i);
  const double phi = load_param_d(dp, 4, i), lnD = load_param_d(dp, 5, i);
  const double tc = load_param_d(dp, 6, i);
  const int M = C.M, na = C.na, A = C.A;
  const double x = C.d_ref * exp(-lnD);
  const CompDraw g = comp_geometry(C, ra, dec, psi);

  double yr[MM], yi[MM];
  {
    double sh, ch, sp, cp;
    sincos(0.5 * incl, &sh, &ch);
    sincos(phi, &sp, &cp);
#pragma unroll
    for (int m = 0; m < MM; ++m) {
      yr[m] = yi[m] = 0.0;
      if (m < M) sylm_eval<double>(P, m, ch, sh, cp, sp, P.ycoef[m], yr[m], yi[m]);
    }
  }

  double td = 0.0, tq = 0.0;
  int oob = 0;
  // the coefficients of all detectors fit a small local array: then the
  // quadratic forms are formed once per detector class (below)
  const bool by_class = C.K * na <= kClassCoef;
  double2 cfs[kClassCoef];
  for (int k = 0; k < C.K; ++k) {
    const double tk = tc - (C.pos[k][0] * g.s[0] + C.pos[k][1] * g.s[1] + C.pos[k][2] * g.s[2]);
    double2 cf[kMaxRespIdx];
    comp_coeffs(C, k, g.sd, g.cd, g.sg, g.cg, g.s2p, g.c2p, tk, g.s, g.e1, g.e2, cf);

    // data term: sum_a conj(C_a) sum_taps w sum_i conj(Y_i) Q[j][a][i]
    const double u = (tk - C.t0[k]) * C.inv_dt;
    if (!isfinite(u)) {
      td = CUDART_NAN;
    } else {
      const double jf = floor(u);
      double w[4], dw[4];
      lagrange4_d(u - jf, w, dw);
      const long long j0 = (long long)jf - 1;
      for (int a = 0; a < na; ++a) {
        double gr = 0.0, gi = 0.0;
#pragma unroll
        for (int tap = 0; tap < 4; ++tap) {
          const long long j = j0 + tap;
          if (j < 0 || j >= C.n) continue;
          const double2* row = C.Q + ((long long)k * C.n + j) * A + (long long)a * M;
          double sr = 0.0, si = 0.0;
#pragma unroll
          for (int m = 0; m < MM; ++m)
            if (m < M) {
              const double2 q = __ldg(row + m);
              sr += yr[m] * q.x + yi[m] * q.y;
              si += yr[m] * q.y - yi[m] * q.x;
            }
          gr = fma(w[tap], sr, gr);
          gi = fma(w[tap], si, gi);
        }
        td += cf[a].x * gr + cf[a].y * gi;  // Re(conj(C_a) g_a)
      }
      for (int tap = 0; tap < 4; ++tap) {
        const long long j = j0 + tap;
        if (j < 0 || j >= C.n) ++oob;
      }
    }

    if (by_class) {
      for (int a = 0; a < na; ++a) cfs[k * na + a] = cf[a];
      continue;
    }
    // quadratic term, this detector: sum over block pairs a <= b of z_a^T G_ab z_b
    const double* Gk = C.G + (size_t)C.cls_of[k] * C.nblk * 4 * M * M;
    int blk = 0;
    for (int a = 0; a < na; ++a) {
      double ar[MM], ai[MM];
#pragma unroll
      for (int m = 0; m < MM; ++m) {
        ar[m] = cf[a].x * yr[m] - cf[a].y * yi[m];
        ai[m] = cf[a].x * yi[m] + cf[a].y * yr[m];
      }
      for (int b = a; b < na; ++b, ++blk) {
        double br[MM], bi[MM];
#pragma unroll
        for (int m = 0; m < MM; ++m) {
          br[m] = cf[b].x * yr[m] - cf[b].y * yi[m];
          bi[m] = cf[b].x * yi[m] + cf[b].y * yr[m];
        }
        const double* Gb = Gk + (size_t)blk * 4 * M * M;
        double acc = 0.0;
#pragma unroll
        for (int r = 0; r < MM; ++r) {
          if (r < M) {
            double t1 = 0.0, t2 = 0.0;
#pragma unroll
            for (int c = 0; c < MM; ++c) {
              if (c < M) {
                t1 = fma(__ldg(Gb + r * M + c), br[c], t1);
                t1 = fma(__ldg(Gb + M * M + r * M + c), bi[c], t1);
                t2 = fma(__ldg(Gb + 2 * M * M + r * M + c), br[c], t2);
                t2 = fma(__ldg(Gb + 3 * M * M + r * M + c), bi[c], t2);
              }
            }
            acc = fma(ar[r], t1, acc);
            acc = fma(ai[r], t2, acc);
          }
        }
        tq += acc;
      }
    }
  }
  if (by_class) {
    // z_a = Re C_a y + Im C_a Jy with y = (Re Y, Im Y), Jy = (-Im Y, Re Y), so
    // z_a^T G_ab z_b needs only the four forms y^T G y, y^T G Jy, (Jy)^T G y,
    // (Jy)^T G Jy of each block, shared by the detectors of a class
    for (int cc = 0; cc < C.ncls; ++cc) {
      const double* Gc = C.G + (size_t)cc * C.nblk * 4 * M * M;
      int blk = 0;
      for (int a = 0; a < na; ++a) {
        for (int b = a; b < na; ++b, ++blk) {
          const double* Gb = Gc + (size_t)blk * 4 * M * M;
          double s00 = 0.0, s01 = 0.0, s10 = 0.0, s11 = 0.0;
#pragma unroll
          for (int r = 0; r < MM; ++r) {
            if (r < M) {
              double g1r = 0.0, g1i = 0.0, g2r = 0.0, g2i = 0.0;  // rows of G y and G Jy
#pragma unroll
              for (int c = 0; c < MM; ++c) {
                if (c < M) {
                  const double g00 = __ldg(Gb + r * M + c), g01 = __ldg(Gb + M * M + r * M + c);
                  const double g10 = __ldg(Gb + 2 * M * M + r * M + c);
                  const double g11 = __ldg(Gb + 3 * M * M + r * M + c);
                  g1r = fma(g00, yr[c], fma(g01, yi[c], g1r));
                  g1i = fma(g10, yr[c], fma(g11, yi[c], g1i));
                  g2r = fma(g01, yr[c], fma(-g00, yi[c], g2r));
                  g2i = fma(g11, yr[c], fma(-g10, yi[c], g2i));
                }
              }
              s00 = fma(yr[r], g1r, fma(yi[r], g1i, s00));
              s10 = fma(yr[r], g1i, fma(-yi[r], g1r, s10));
              s01 = fma(yr[r], g2r, fma(yi[r], g2i, s01));
              s11 = fma(yr[r], g2i, fma(-yi[r], g2r, s11));
            }
          }
          for (int k = 0; k < C.K; ++k) {
            if (C.cls_of[k] != cc) continue;
            const double2 ca = cfs[k * na + a], cb = cfs[k * na + b];
            tq += ca.x * (cb.x * s00 + cb.y * s01) + ca.y * (cb.x * s10 + cb.y * s11);
          }
        }
      }
    }
  }
  CompOut o;
  o.lnl = x * td - 0.25 * x * x * tq;
  o.oob = oob;
  return o;
}

template <int MM, bool LSE>
__global__ void __launch_bounds__(kCompThreads) comp_lnl_kernel(const __grid_constant__ CompParams C,
                                                                const PointParams* __restrict__ gP,
                                                                DrawsParams dp,
                                                                double* __restrict__ lnl_out,
                                                                LseState* __restrict__ partials,
                                                                unsigned long long* __restrict__ oob_count) {
  __shared__ PointParams P;
  stage_point(P, gP);
  __syncthreads();
  ThreadLse64 st = tlse64_init();
  int oob = 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    const CompOut o = comp_lnl_draw<MM>(C, P, dp, i);
    oob += o.oob;
    if (!LSE)
      lnl_out[i] = o.lnl;
    else
      tlse64_push(st, o.lnl + load_logw_d(dp, i));
  }
  if (LSE) block_lse64_write(st, partials + blockIdx.x);
  if (oob_count) {
    for (int off = 16; off > 0; off >>= 1) oob += __shfl_down_sync(0xffffffffu, oob, off);
    if ((threadIdx.x & 31) == 0 && oob) atomicAdd(oob_count, (unsigned long long)oob);
  }
}

__global__ void __launch_bounds__(kCompThreads) comp_coeffs_kernel(const __grid_constant__ CompParams C,
                                                                   DrawsParams dp,
                                                                   double2* __restrict__ out) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride) {
    const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
    const double psi = load_param_d(dp, 2, i), tc = load_param_d(dp, 6, i);
    const CompDraw g = comp_geometry(C, ra, dec, psi);
    for (int k = 0; k < C.K; ++k) {
      const double tk = tc - (C.pos[k][0] * g.s[0] + C.pos[k][1] * g.s[1] + C.pos[k][2] * g.s[2]);
      double2 cf[kMaxRespIdx];
      comp_coeffs(C, k, g.sd, g.cd, g.sg, g.cg, g.s2p, g.c2p, tk, g.s, g.e1, g.e2, cf);
      double2* o = out + (i * C.K + k) * C.na;
      for (int a = 0; a < C.na; ++a) o[a] = cf[a];
    }
  }
}

template <int MM, bool LSE>
cudaError_t launch_comp_k(const CompParams& C, const PointParams* dP, const DrawsParams& dp,
                          double* lnl_out, LseState* partials, unsigned long long* oob, int* blocks,
                          cudaStream_t st) {
  *blocks = grid_cap(grid_for(comp_lnl_kernel<MM, LSE>, kCompThreads, 0), dp.n, kCompThreads);
  comp_lnl_kernel<MM, LSE><<<*blocks, kCompThreads, 0, st>>>(C, dP, dp, lnl_out, partials, oob);
  return cudaGetLastError();
}

template <int MM>
cudaError_t launch_comp_mm(const CompParams& C, const PointParams* dP, const DrawsParams& dp,
                           double* lnl_out, LseState* partials, unsigned long long* oob, int* blocks,
                           cudaStream_t st) {
  if (partials) return launch_comp_k<MM, true>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_comp_k<MM, false>(C, dP, dp, lnl_out, partials, oob, blocks, st);
}

cudaError_t launch_comp(const CompParams& C, const PointParams* dP, const DrawsParams& dp,
                        double* lnl_out, LseState* partials, unsigned long long* oob, int* blocks,
                        cudaStream_t st) {
  const int M = C.M;
  if (M <= 2) return launch_comp_mm<2>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 4) return launch_comp_mm<4>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 6) return launch_comp_mm<6>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 8) return launch_comp_mm<8>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 10) return launch_comp_mm<10>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  if (M <= 12) return launch_comp_mm<12>(C, dP, dp, lnl_out, partials, oob, blocks, st);
  return launch_comp_mm<16>(C, dP, dp, lnl_out, partials, oob, blocks, st);
}

int n_index(int kind, int p_max) {
  if (kind == RIFT_ILE_RESP_ROTATION) {
    if (p_max < 0 || p_max > RIFT_ILE_MAX_ROT_PMAX) return RIFT_ILE_ERR_UNSUPPORTED;
    return (p_max + 1) * (p_max + 5);
  }
  if (kind == RIFT_ILE_RESP_FINITE_ARM) {
    if (p_max < 0 || p_max > RIFT_ILE_MAX_ARM_PMAX) return RIFT_ILE_ERR_UNSUPPORTED;
    return p_max + 1;
  }
  return RIFT_ILE_ERR_INVALID_ARG;
}

bool finite_all(const double* p, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(p[i])) return false;
  return true;
}

int validate_comp(const rift_ile_comp_desc* d, int* na_out) {
  if (!d) {
    rift_ile_set_error("composite description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const int na = n_index(d->kind, d->p_max);
  if (na < 0) {
    rift_ile_set_error("response kind %d with p_max %d is not supported (rotation p_max <= %d, "
                       "finite arms p_max <= %d)", d->kind, d->p_max, RIFT_ILE_MAX_ROT_PMAX,
                       RIFT_ILE_MAX_ARM_PMAX);
    return na;
  }
  if (d->n_det < 1 || d->n_det > RIFT_ILE_MAX_DET || d->n_modes < 1 ||
      d->n_modes > RIFT_ILE_MAX_MODES || na * d->n_modes > RIFT_ILE_MAX_COMP) {
    rift_ile_set_error("n_det=%d, n_modes=%d or composite dimension %d out of range", d->n_det,
                       d->n_modes, na * d->n_modes);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  if (!d->ell || !d->em || !d->Q || !d->q_t0 || !d->U || !d->V || !d->det_pos ||
      (d->kind == RIFT_ILE_RESP_ROTATION && !d->det_resp) ||
      (d->kind == RIFT_ILE_RESP_FINITE_ARM && (!d->arm_x || !d->arm_y))) {
    rift_ile_set_error("a required array of the composite description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->q_len < 4) {
    rift_ile_set_error("q_len=%d: the cubic needs at least 4 samples", d->q_len);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (!(d->q_dt > 0.0) || !std::isfinite(d->q_dt) || !std::isfinite(d->gmst) ||
      !(d->d_ref > 0.0) || !std::isfinite(d->d_ref) || !std::isfinite(d->omega)) {
    rift_ile_set_error("q_dt, gmst, d_ref or omega is not finite (q_dt, d_ref positive)");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < d->n_modes; ++i)
    if (d->ell[i] < 2 || d->ell[i] > RIFT_ILE_MAX_ELL || std::abs(d->em[i]) > d->ell[i]) {
      rift_ile_set_error("mode %d: (l=%d, m=%d) unsupported", i, d->ell[i], d->em[i]);
      return RIFT_ILE_ERR_UNSUPPORTED;
    }
  const size_t K = d->n_det, Ac = (size_t)na * d->n_modes;
  if (!finite_all(d->q_t0, K) || !finite_all(d->det_pos, 3 * K) ||
      (d->det_resp && !finite_all(d->det_resp, 6 * K)) ||
      !finite_all(d->U, 2 * K * Ac * Ac) || !finite_all(d->V, 2 * K * Ac * Ac) ||
      (d->kind == RIFT_ILE_RESP_FINITE_ARM &&
       (!finite_all(d->arm_x, 3 * K) || !finite_all(d->arm_y, 3 * K)))) {
    rift_ile_set_error("a geometry or U/V value of the composite description is not finite");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  *na_out = na;
  return RIFT_ILE_OK;
}

}  // namespace
}  // namespace rift


using namespace rift;

extern "C" int rift_ile_comp_n_index(int32_t kind, int32_t p_max) {
  const int na = n_index(kind, p_max);
  if (na < 0) rift_ile_set_error("response kind %d with p_max %d is not supported", kind, p_max);
  return na;
}

extern "C" int rift_ile_comp_create(const rift_ile_comp_desc* d, rift_ile_comp** out, void* stream) {
  if (!out) {
    rift_ile_set_error("rift_ile_comp_create: out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int na = 0;
  int rc = validate_comp(d, &na);
  if (rc) return rc;
  const int K = d->n_det, M = d->n_modes, A = na * M, n = d->q_len;
  cudaStream_t st = (cudaStream_t)stream;

  CompParams C;
  std::memset(&C, 0, sizeof(C));
  C.K = K;
  C.M = M;
  C.kind = d->kind;
  C.p_max = d->p_max;
  C.na = na;
  C.A = A;
  C.n = n;
  C.nblk = na * (na + 1) / 2;
  C.omega = d->omega;
  C.gmst = d->gmst;
  C.d_ref = d->d_ref;
  C.dt = d->q_dt;
  C.inv_dt = 1.0 / d->q_dt;
  for (int k = 0; k < K; ++k) {
    C.t0[k] = d->q_t0[k];
    for (int c = 0; c < 3; ++c) {
      C.pos[k][c] = d->det_pos[3 * k + c];
      if (d->kind == RIFT_ILE_RESP_FINITE_ARM) {
        C.armx[k][c] = d->arm_x[3 * k + c];
        C.army[k][c] = d->arm_y[3 * k + c];
      }
    }
    for (int c = 0; c < 6; ++c) C.resp[k][c] = d->det_resp ? d->det_resp[6 * k + c] : 0.0;
  }

  PointParams B;
  std::memset(&B, 0, sizeof(B));
  B.K = K;
  B.M = M;
  for (int i = 0; i < M; ++i) {
    B.ell[i] = d->ell[i];
    B.em[i] = d->em[i];
    double coef[kMaxYTerms];
    int k0 = 0;
    B.ynt[i] = harmonic_coefficients(d->ell[i], d->em[i], &k0, coef);
    B.yk0[i] = k0;
    for (int r = 0; r < B.ynt[i]; ++r) B.ycoef[i][r] = coef[r];
  }

  // real form of c^+ U c + Re(c^T V c) in z = (Re c, Im c): diagonal blocks
  // sym(Ur + Vr), sym(Ur - Vr); off-diagonal 1/2 (Ui^T - Ui - Vi - Vi^T)
  // detectors with identical U and V (the same noise curve and bank) share one form
  const size_t uv_len = 2 * (size_t)A * A;
  int rep[kMaxDet];
  C.ncls = 0;
  for (int k = 0; k < K; ++k) {
    int c = -1;
    for (int q = 0; q < C.ncls && c < 0; ++q)
      if (std::memcmp(d->U + rep[q] * uv_len, d->U + k * uv_len, uv_len * sizeof(double)) == 0 &&
          std::memcmp(d->V + rep[q] * uv_len, d->V + k * uv_len, uv_len * sizeof(double)) == 0)
        c = q;
    if (c < 0) {
      c = C.ncls++;
      rep[c] = k;
    }
    C.cls_of[k] = c;
  }
  const size_t blk_sz = 4 * (size_t)M * M;
  std::vector<double> G((size_t)C.ncls * C.nblk * blk_sz);
  auto U = [&](int k, int r, int c, int part) { return d->U[(((size_t)k * A + r) * A + c) * 2 + part]; };
  auto V = [&](int k, int r, int c, int part) { return d->V[(((size_t)k * A + r) * A + c) * 2 + part]; };
  auto Gfull = [&](int k, int pr, int r, int pc, int c) {
    if (pr == 0 && pc == 0) return 0.5 * (U(k, r, c, 0) + U(k, c, r, 0) + V(k, r, c, 0) + V(k, c, r, 0));
    if (pr == 1 && pc == 1) return 0.5 * (U(k, r, c, 0) + U(k, c, r, 0) - V(k, r, c, 0) - V(k, c, r, 0));
    if (pr == 0)  // (Re row r, Im column c)
      return 0.5 * (U(k, c, r, 1) - U(k, r, c, 1) - V(k, r, c, 1) - V(k, c, r, 1));
    return 0.5 * (U(k, r, c, 1) - U(k, c, r, 1) - V(k, c, r, 1) - V(k, r, c, 1));
  };
  for (int cc = 0; cc < C.ncls; ++cc) {
    const int k = rep[cc];
    int blk = 0;
    for (int a = 0; a < na; ++a)
      for (int b = a; b < na; ++b, ++blk) {
        const double f = (a == b) ? 1.0 : 2.0;
        double* Gb = G.data() + ((size_t)cc * C.nblk + blk) * blk_sz;
        for (int sub = 0; sub < 4; ++sub) {
          const int pr = sub >> 1, pc = sub & 1;
          for (int r = 0; r < M; ++r)
            for (int c = 0; c < M; ++c)
              Gb[(size_t)sub * M * M + r * M + c] = f * Gfull(k, pr, a * M + r, pc, b * M + c);
        }
      }
  }

  rift_ile_comp* cp = new rift_ile_comp();
  cp->dev_base = nullptr;
  cp->q = nullptr;
  cp->G = nullptr;
  cudaGetDevice(&cp->device);
  for (int i = 0; i < M; ++i) {
    cp->host_ell[i] = d->ell[i];
    cp->host_em[i] = d->em[i];
  }
  // the full real form of each class, kept for the FP32-mixed form's whitening
  {
    const size_t D = 2 * (size_t)A;
    cp->Gfull.assign((size_t)C.ncls * D * D, 0.0);
    for (int cc = 0; cc < C.ncls; ++cc) {
      double* Gc = cp->Gfull.data() + (size_t)cc * D * D;
      for (int pr = 0; pr < 2; ++pr)
        for (int r = 0; r < A; ++r)
          for (int pc = 0; pc < 2; ++pc)
            for (int c = 0; c < A; ++c)
              Gc[((size_t)pr * A + r) * D + (size_t)pc * A + c] = Gfull(rep[cc], pr, r, pc, c);
    }
  }
  const size_t qbytes = (size_t)K * n * A * sizeof(double2);
  cudaError_t e = cudaMalloc((void**)&cp->q, qbytes);
  if (e == cudaSuccess) e = cudaMalloc((void**)&cp->G, G.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&cp->dev_base, sizeof(PointParams));
  if (e != cudaSuccess) {
    cudaFree(cp->q);
    cudaFree(cp->G);
    cudaFree(cp->dev_base);
    delete cp;
    rift_ile_set_error("composite allocation failed: %s", cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  e = cudaMemcpyAsync(cp->q, d->Q, qbytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cp->G, G.data(), G.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(cp->dev_base, &B, sizeof(B), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    rift_ile_comp_destroy(cp);
    return check_cuda(e, "rift_ile_comp_create upload");
  }
  C.Q = cp->q;
  C.G = cp->G;
  cp->host = C;
  *out = cp;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_comp_destroy(rift_ile_comp* cp) {
  if (!cp) return RIFT_ILE_OK;
  cudaFree(cp->q);
  cudaFree(cp->G);
  cudaFree(cp->dev_base);
  cudaFree(cp->mixed_dev);
  cudaFree(cp->Bs);
  cudaFree(cp->agrid);
  cudaFree(cp->ehat);
  cudaFree(cp->epoly);
  delete cp;
  return RIFT_ILE_OK;
}

namespace {

int comp_args(const rift_ile_comp* cp, const rift_ile_draws* draws) {
  if (!cp) {
    rift_ile_set_error("composite point is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  return validate_draws(draws);
}

}  // namespace

extern "C" int rift_ile_comp_coeffs(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                    double* coef_out, void* stream) {
  int rc = comp_args(cp, draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!coef_out) {
    rift_ile_set_error("rift_ile_comp_coeffs: coef_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const DrawsParams dp = draws_params(draws);
  const int blocks = grid_cap(device_sms() * 8, dp.n, kCompThreads);
  comp_coeffs_kernel<<<blocks, kCompThreads, 0, (cudaStream_t)stream>>>(cp->host, dp,
                                                                       (double2*)coef_out);
  return check_cuda(cudaGetLastError(), "rift_ile_comp_coeffs launch");
}

extern "C" int rift_ile_comp_lnL(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                 double* lnL_out, void* stream) {
  int rc = comp_args(cp, draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!lnL_out) {
    rift_ile_set_error("rift_ile_comp_lnL: lnL_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int blocks = 0;
  return check_cuda(launch_comp(cp->host, cp->dev_base, draws_params(draws), lnL_out, nullptr,
                                nullptr, &blocks, (cudaStream_t)stream),
                    "rift_ile_comp_lnL launch");
}

extern "C" int rift_ile_comp_lnZ_state_async(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                             rift_ile_lse* state_out, void* stream) {
  int rc = comp_args(cp, draws);
  if (rc) return rc;
  if (!state_out) {
    rift_ile_set_error("rift_ile_comp_lnZ_state_async: state_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  LseState *partials = nullptr, *state = nullptr;
  unsigned long long* oob = nullptr;
  if ((rc = lse_workspace(&partials, &state, &oob))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  LseState* out = reinterpret_cast<LseState*>(state_out);
  if (draws->n == 0)
    return check_cuda(launch_lse_combine(partials, 0, 0.0, out, st), "lnZ combine launch");
  int blocks = 0;
  if ((rc = check_cuda(launch_comp(cp->host, cp->dev_base, draws_params(draws), nullptr, partials,
                                   nullptr, &blocks, st),
                       "composite lnZ kernel launch")))
    return rc;
  return check_cuda(launch_lse_combine(partials, blocks, (double)draws->n, out, st),
                    "lnZ combine launch");
}

extern "C" int rift_ile_comp_lnZ_state(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                       rift_ile_lse* state, void* stream) {
  int rc = comp_args(cp, draws);
  if (rc) return rc;
  if (!state) {
    rift_ile_set_error("rift_ile_comp_lnZ_state: state is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (draws->n == 0) {
    *state = rift_ile_lse{-INFINITY, 0.0, 0.0, 0.0};
    set_last_oob(0);
    return RIFT_ILE_OK;
  }
  LseState *partials = nullptr, *dstate = nullptr;
  unsigned long long* doob = nullptr;
  if ((rc = lse_workspace(&partials, &dstate, &doob))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if ((rc = check_cuda(cudaMemsetAsync(doob, 0, sizeof(unsigned long long), st), "memset")))
    return rc;
  int blocks = 0;
  if ((rc = check_cuda(launch_comp(cp->host, cp->dev_base, draws_params(draws), nullptr, partials,
                                   doob, &blocks, st),
                       "composite lnZ kernel launch")))
    return rc;
  if ((rc = check_cuda(launch_lse_combine(partials, blocks, (double)draws->n, dstate, st),
                       "lnZ combine launch")))
    return rc;
  LseState h;
  unsigned long long o = 0;
  if ((rc = check_cuda(cudaMemcpyAsync(&h, dstate, sizeof(h), cudaMemcpyDeviceToHost, st), "copy")))
    return rc;
  if ((rc = check_cuda(cudaMemcpyAsync(&o, doob, sizeof(o), cudaMemcpyDeviceToHost, st), "copy")))
    return rc;
  if ((rc = check_cuda(cudaStreamSynchronize(st), "rift_ile_comp_lnZ_state"))) return rc;
  set_last_oob((long long)o);
  *state = rift_ile_lse{h.m, h.s, h.s2, h.n};
  return RIFT_ILE_OK;
}
