// Direct marginalisation over (phi_ref, psi) and distance inside the
// likelihood (eq. direct_marginalization; ERAI of App. F.1, adaptive
// Gauss-Hermite of eq. ap:dgh), FP64, one warp per draw.
//
// Per draw (all lanes): sky basis, F_k(0), Y_lm(phi = 0); the lanes share the
// mode pairs and the (detector, mode) pairs (Q_k,lm(t_k) by the table cubic)
// and bin them by harmonic in a fixed order into the coefficients of
//   K(phi, psi) = Re[e^{-2 i psi} sum_m e^{-i m phi} c_m],
//     c_m = sum_k conj(F_k(0)) sum_{lm: m} conj(Y_lm(0)) Q_k,lm(t_k),
//   2R(phi, psi) = sum_d alpha_d e^{i d phi} + Re[e^{4 i psi} sum_s beta_s e^{i s phi}],
//     alpha_d = sum_{m_j - m_i = d} conj(Y_i) Y_j sum_k |F_k|^2 U_k,ij,
//     beta_s = sum_{m_i + m_j = s} Y_i Y_j sum_k F_k^2 V_k,ij,
// (F_k(psi) = e^{2 i psi} F_k(0), Y(phi) = e^{i m phi} Y(0)), kept in shared
// memory.  The lanes then share the n_phi phase columns: per column the three
// harmonic sums once, per polarisation node K and R in a few operations, and
// at each node the Gauss-Hermite distance integral and an online log-sum-exp.
// A first pass finds the node with the largest K^2/(2R) and evaluates it in
// full (v0); the second pass skips nodes whose upper bound
// K^2/(2R) + ln(sqrt(2 pi) sigma_x max p_x) is below v0 - T, T = 36 + ln(n_phi
// n_psi): the skipped nodes together weigh below e^-36 of v0's node.
// Geocentric time is the draw's own, or integrated over a window: by the
// fixed-spacing rule (eq. ap:tfixed, the data coefficients formed at every
// node), by the band-limited rule (eq. ap:tband, the coefficients formed at
// coarse nodes and sinc-reconstructed at the fine ones), or by the peak-local
// rule (eq. ap:tlocal) on those fine nodes: the envelope
// U(t) = 1/2 sum_k |e_k(t_k)|^2 (the network's data projected on each
// detector's template span, from the point's interval polynomials; it bounds
// the angular-and-distance integrand at t by Cauchy-Schwarz), its maxima
// within ln(1/tol) + ln(n_f) of the largest, widths from the three-point
// curvature, the fine nodes within c sigma_t of a maximum integrated and the
// others bounded by LSE(U); above the tolerance every fine node is integrated.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/rift_ile_direct.h"
#include "common.cuh"
#include "kernels.h"

namespace rift {
namespace {

#ifndef RIFT_DIRECT_MIN_BLOCKS
#define RIFT_DIRECT_MIN_BLOCKS 3  // resident blocks per SM the register budget is sized for
#endif
constexpr int kDirWarps = 4;
constexpr int kHm = 2 * kMaxEll + 1;        // data harmonics m = -8..8
constexpr int kHn = 4 * kMaxEll + 1;        // norm harmonics -16..16
constexpr int kPsiTab = 256;                // polarisation phases tabulated up to this n_psi
// Column sums (D, A, B: 5 doubles) kept between the passes in the warp's
// pair buffers (idle during the angular sweep) up to this n_phi.
constexpr int kColCache = (2 * kMaxModes * kMaxModes * 2) / 5;
static_assert(5 * kColCache <= 2 * kMaxModes * kMaxModes * 2, "column cache exceeds the pair buffers");
constexpr double kSkipNat = 36.0;  // plus ln(n_phi n_psi): the skipped mass stays below e^-36
constexpr int kMaxPeaks = 64;      // maxima the peak-local rule keeps per draw (more: the full rule)
constexpr int kMaxLocalFine = 1 << 16;  // fine nodes the peak-local rule handles

struct DirectParams {
  int n_phi, n_psi, n_gh, n_t;  // n_t = 0: the draw's own t
  int t_up;                     // > 1: fine nodes per interval (band-limited rule)
  double2* slab;                // band-limited rule: n_t * kHm coefficients per warp
  // peak-local rule (t_local): per warp, after the coefficients, U[n_f], the
  // kept flags[n_f] and the maxima (fine index, c sigma_t)[kMaxPeaks]
  int t_local;
  double t_c, ln_tol, depth;    // c, ln(tol), ln(1/tol) + ln(n_f)
  int t_mirror;                 // fine coefficients from the mirrored series
  double t_lo, t_h;             // time midpoints t_lo + (j + 1/2) t_h
  double lo, hi;          // prior range of x
  double lnnorm;          // ln of 3 d_ref^3 / (d_max^3 - d_min^3)
  double lnw;             // -ln(n_phi n_psi max(n_t, 1) max(t_up, 1))
  double ln_ub;           // ln(sqrt(2 pi) norm lo^-4), the prefactor bound over sigma_x
  double skip_nat;        // kSkipNat + ln(n_phi n_psi)
  double xi[RIFT_ILE_MAX_GH], w[RIFT_ILE_MAX_GH];
  int mixed;              // 1: the prior-weighted Gauss-Hermite sum in float
  double inv_lo;          // 1 / lo
  double hi_lo;           // hi / lo
  double lnnorm_lo;       // lnnorm - 4 ln lo (the sum taken in y = x / lo)
  float wf[RIFT_ILE_MAX_GH];
  float xif[RIFT_ILE_MAX_GH];  // the nodes in float, and hi / lo
  float hi_lof;
  double2 e2[kPsiTab];    // e^{2 i psi_b}, psi_b = pi b / n_psi (n_psi <= kPsiTab)
  double2 e4[kPsiTab];    // e^{4 i psi_b}
  float2 e2f[kPsiTab];    // the same in float, for the first pass
  float2 e4f[kPsiTab];
};

// Bytes of the band-limited (and peak-local) scratch per warp: the coarse
// coefficients, then U (padded to an even count), the kept flags (padded to a
// multiple of four) and the maxima; every part starts on 16 bytes.
__host__ __device__ inline size_t direct_slab_per_warp(const DirectParams& Q) {
  size_t b = (size_t)Q.n_t * kHm * sizeof(double2);
  if (Q.t_local) {
    const size_t nf = (size_t)Q.n_t * Q.t_up;
    b += ((nf + 1) & ~(size_t)1) * sizeof(double) + ((nf + 3) & ~(size_t)3) * sizeof(int) +
         kMaxPeaks * sizeof(double2);
  }
  return b;
}

struct DirCoef {
  double2 c[kHm];
  double2 al[kHn];
  double2 be[kHn];
};

__device__ __forceinline__ double2 cmul_d(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Per-draw values every lane keeps: Y_lm(phi = 0), F_k(psi = 0), the source direction.
template <int MM>
struct DirDraw {
  double yr[MM], yi[MM];
  double Fr[kMaxDet], Fi[kMaxDet];
  double s[3];
};

template <int MM>
__device__ void direct_setup(const PointParams& P, const DrawsParams& dp, long long i,
                             DirDraw<MM>& g) {
  const double ra = load_param_d(dp, 0, i), dec = load_param_d(dp, 1, i);
  const double incl = load_param_d(dp, 3, i);
  double sl, cl, sd, cd;
  sincos(ra - P.gmst, &sl, &cl);
  sincos(dec, &sd, &cd);
  g.s[0] = cd * cl;
  g.s[1] = cd * sl;
  g.s[2] = sd;
  const double e1[3] = {-sl, cl, 0.0};
  const double e2[3] = {-sd * cl, -sd * sl, cd};
  double sh, ch;
  sincos(0.5 * incl, &sh, &ch);
#pragma unroll
  for (int m = 0; m < MM; ++m) {
    g.yr[m] = g.yi[m] = 0.0;
    if (m < P.M) sylm_eval<double>(P, m, ch, sh, 1.0, 0.0, P.ycoef[m], g.yr[m], g.yi[m]);
  }
#pragma unroll
  for (int k = 0; k < kMaxDet; ++k) {
    g.Fr[k] = g.Fi[k] = 0.0;
    if (k < P.K) {
      const double* D = P.resp[k];
      g.Fr[k] = quad3(D, e1, e1) - quad3(D, e2, e2);
      g.Fi[k] = -2.0 * quad3(D, e1, e2);
    }
  }
}

template <int MM>
__device__ __forceinline__ double2 y_of(const DirDraw<MM>& g, int m) {
  double2 y = make_double2(0.0, 0.0);
#pragma unroll
  for (int q = 0; q < MM; ++q)
    if (q == m) y = make_double2(g.yr[q], g.yi[q]);
  return y;
}

// Norm coefficients (time independent), the lanes sharing the mode pairs:
// buf_u[p] = conj(Y_a) Y_b sum_k |F_k|^2 U_k,ab and buf_v[p] = Y_a Y_b sum_k F_k^2
// V_k,ab for p = a M + b, then lane h bins the pairs by harmonic in pair order.
template <int MM>
__device__ void direct_norm_warp(const PointParams& P, const DirDraw<MM>& g, int lane,
                                 DirCoef& C, double2* buf_u, double2* buf_v) {
  const int K = P.K, M = P.M;
  for (int p = lane; p < M * M; p += 32) {
    const int a = p / M, b = p % M;
    double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
    for (int k = 0; k < K; ++k) {
      double Fr = 0.0, Fi = 0.0;
#pragma unroll
      for (int q = 0; q < kMaxDet; ++q)
        if (q == k) {
          Fr = g.Fr[q];
          Fi = g.Fi[q];
        }
      const double F2 = Fr * Fr + Fi * Fi, FFr = Fr * Fr - Fi * Fi, FFi = 2.0 * Fr * Fi;
      const double2 uu = P.U[((size_t)k * M + a) * M + b], vv = P.V[((size_t)k * M + a) * M + b];
      ur = fma(F2, uu.x, ur);
      ui = fma(F2, uu.y, ui);
      vr += FFr * vv.x - FFi * vv.y;
      vi += FFr * vv.y + FFi * vv.x;
    }
    const double2 ya = y_of(g, a), yb = y_of(g, b);
    const double2 pu = cmul_d(make_double2(ya.x, -ya.y), yb), pv = cmul_d(ya, yb);
    buf_u[p] = cmul_d(pu, make_double2(ur, ui));
    buf_v[p] = cmul_d(pv, make_double2(vr, vi));
  }
  __syncwarp();
  for (int h = lane; h < kHn; h += 32) {
    double2 al = make_double2(0.0, 0.0), be = al;
    for (int p = 0; p < M * M; ++p) {
      const int a = p / M, b = p % M;
      if (P.em[b] - P.em[a] + 2 * kMaxEll == h) {
        al.x += buf_u[p].x;
        al.y += buf_u[p].y;
      }
      if (P.em[a] + P.em[b] + 2 * kMaxEll == h) {
        be.x += buf_v[p].x;
        be.y += buf_v[p].y;
      }
    }
    C.al[h] = al;
    C.be[h] = be;
  }
  __syncwarp();
}

// Data coefficients at geocentric time tc, the lanes sharing the (detector,
// mode) pairs: buf[p] = conj(F_k) conj(Y_m) Q_k,m(t_k), p = k M + m, binned by m.
template <int MM>
__device__ void direct_data_warp(const PointParams& P, const DirDraw<MM>& g, double tc, int lane,
                                 DirCoef& C, double2* buf) {
  const int K = P.K, M = P.M;
  for (int p = lane; p < K * M; p += 32) {
    const int k = p / M, m = p % M;
    double Fr = 0.0, Fi = 0.0;
#pragma unroll
    for (int q = 0; q < kMaxDet; ++q)
      if (q == k) {
        Fr = g.Fr[q];
        Fi = g.Fi[q];
      }
    const double tk = tc - (P.pos[k][0] * g.s[0] + P.pos[k][1] * g.s[1] + P.pos[k][2] * g.s[2]);
    const double u = (tk - P.t0[k]) * P.inv_dt;
    double gr = 0.0, gi = 0.0;
    if (!isfinite(u)) {
      gr = CUDART_NAN;
    } else {
      const double jf = floor(u);
      double w[4], dw[4];
      lagrange4_d(u - jf, w, dw);
      const long long j0 = (long long)jf - 1;
      for (int tap = 0; tap < 4; ++tap) {
        const long long j = j0 + tap;
        if (j < 0 || j >= P.n) continue;
        double qr, qi;
        if (P.q_c128) {
          const double2 q = __ldg((const double2*)P.Q + ((long long)k * P.n + j) * M + m);
          qr = q.x;
          qi = q.y;
        } else {
          const float2 q = __ldg((const float2*)P.Q + ((long long)k * P.n + j) * M + m);
          qr = q.x;
          qi = q.y;
        }
        gr = fma(w[tap], qr, gr);
        gi = fma(w[tap], qi, gi);
      }
    }
    const double2 ym = y_of(g, m);
    buf[p] = cmul_d(make_double2(Fr, -Fi), cmul_d(make_double2(ym.x, -ym.y), make_double2(gr, gi)));
  }
  __syncwarp();
  for (int h = lane; h < kHm; h += 32) {
    double2 c = make_double2(0.0, 0.0);
    for (int p = 0; p < K * M; ++p)
      if (P.em[p % M] + kMaxEll == h) {
        c.x += buf[p].x;
        c.y += buf[p].y;
      }
    C.c[h] = c;
  }
  __syncwarp();
}

// Per phase column: D = sum_m c_m e^{-i m phi}, A = Re sum_d al_d e^{i d phi},
// B = sum_s be_s e^{i s phi}.
__device__ void direct_column(const DirCoef& C, double phi_frac, double2& D, double& A,
                              double2& B) {
  double s1, c1;
  sincospi(2.0 * phi_frac, &s1, &c1);
  double2 pw[2 * kMaxEll + 1];  // e^{i k phi}, k = 0..16
  pw[0] = make_double2(1.0, 0.0);
  pw[1] = make_double2(c1, s1);
  for (int k = 2; k <= 2 * kMaxEll; ++k) pw[k] = cmul_d(pw[k - 1], pw[1]);
  D = make_double2(0.0, 0.0);
  for (int m = -kMaxEll; m <= kMaxEll; ++m) {
    const double2 e = m >= 0 ? make_double2(pw[m].x, -pw[m].y) : pw[-m];  // e^{-i m phi}
    const double2 t = cmul_d(C.c[m + kMaxEll], e);
    D.x += t.x;
    D.y += t.y;
  }
  A = 0.0;
  B = make_double2(0.0, 0.0);
  for (int d = -2 * kMaxEll; d <= 2 * kMaxEll; ++d) {
    const double2 e = d >= 0 ? pw[d] : make_double2(pw[-d].x, -pw[-d].y);  // e^{i d phi}
    const double2 a = C.al[d + 2 * kMaxEll], b = C.be[d + 2 * kMaxEll];
    A += a.x * e.x - a.y * e.y;
    const double2 t = cmul_d(b, e);
    B.x += t.x;
    B.y += t.y;
  }
}

// K, R at one polarisation node from the column sums; e2 = e^{2 i psi}, e4 = e2^2.
__device__ __forceinline__ void direct_node(const double2& D, double A, const double2& B,
                                            double2 e2, double2 e4, double& K, double& R) {
  K = e2.x * D.x + e2.y * D.y;  // Re(e^{-2 i psi} D)
  R = 0.5 * (A + (e4.x * B.x - e4.y * B.y));
}

// ln of the Gauss-Hermite distance integral at one node (eq. ap:dgh).
__device__ double direct_distance(const DirectParams& Q, double K, double R) {
  if (!(R > 0.0)) return -CUDART_INF;
  const double sig = rsqrt(R);
  const double h = 1.4142135623730951 * sig;
  if (Q.mixed) {
    // y = x / lo in [1, hi / lo] inside the prior, so y^-4 lies in [(lo/hi)^4, 1];
    // x* = K / R as K sig^2.  The nodes y in float (error ~1e-6, far below
    // the integrand's needs); a node within 1e-5 of either edge of the prior
    // is placed in double, so that every in/out decision is the double one
    const double ys = K * (sig * sig) * Q.inv_lo, hy = h * Q.inv_lo;
    const float ysf = (float)ys, hyf = (float)hy, hlf = Q.hi_lof;
    float sf = 0.0f;
    for (int j = 0; j < Q.n_gh; ++j) {
      float y = fmaf(hyf, Q.xif[j], ysf);
      bool in = y >= 1.0f && y <= hlf;
      if (fabsf(y - 1.0f) < 1e-5f || fabsf(y - hlf) < 1e-5f * hlf) {
        const double yd = fma(hy, Q.xi[j], ys);
        in = yd >= 1.0 && yd <= Q.hi_lo;
        y = (float)yd;
      }
      if (in) {
        const float r = __frcp_rn(y), r2 = r * r;
        sf = fmaf(Q.wf[j], r2 * r2, sf);
      }
    }
    if (!(sf > 0.0f)) return -CUDART_INF;
    // K^2/(2R) = (K sig)^2 / 2 in double; the logarithm of the O(1) factor
    // h sf in float (absolute error ~1e-7 nat)
    const double ks = K * sig;
    return 0.5 * ks * ks + (double)__logf((float)h * sf) + Q.lnnorm_lo;
  }
  const double xs = K / R;
  double s = 0.0;
  for (int j = 0; j < Q.n_gh; ++j) {
    const double x = fma(h, Q.xi[j], xs);
    if (x >= Q.lo && x <= Q.hi) {
      const double r = 1.0 / x, r2 = r * r;
      s = fma(Q.w[j], r2 * r2, s);
    }
  }
  if (!(s > 0.0)) return -CUDART_INF;
  return K * K / (2.0 * R) + log(h * s) + Q.lnnorm;
}

// The peak-local rule's envelope at geocentric time t: 1/2 sum_k |e_k(t_k)|^2
// from the interval polynomials of the point (zero where no tap is in a
// detector's table).
template <int MM>
__device__ double envelope_at(const PointParams& P, const DirDraw<MM>& g, double t) {
  double u_sum = 0.0;
  for (int k = 0; k < P.K; ++k) {
    const double tk = t - (P.pos[k][0] * g.s[0] + P.pos[k][1] * g.s[1] + P.pos[k][2] * g.s[2]);
    const double u = (tk - P.t0[k]) * P.inv_dt;
    const double jf = floor(u);
    if (!(jf >= -2.0 && jf <= (double)P.n)) continue;
    const double f = u - jf;
    const float2* pc = P.epoly + ((size_t)k * (P.n + 3) + (size_t)((long long)jf + 2)) * (kPolyDeg + 1);
    double acc = 0.0;
    for (int p = kPolyDeg; p >= 0; --p) {
      const float2 c = __ldg(pc + p);
      acc = fma(acc, f, (double)c.x + (double)c.y);
    }
    u_sum += acc;
  }
  return u_sum;
}

// The same with the exponential of the (non-positive) offset in float, for the
// mixed form: the running maximum and sum stay double; every term the sum
// takes lies within the skip depth (~45 nat) of the maximum, where a float
// exponential errs by ~1e-7 relative.
__device__ __forceinline__ void lse_add_f(double& m, double& s, double v) {
  if (!(v > -CUDART_INF)) return;
  if (v > m) {
    s = fma(s, (double)__expf((float)(m - v)), 1.0);
    m = v;
  } else {
    s += (double)__expf((float)(v - m));
  }
}

__device__ __forceinline__ void lse_add(double& m, double& s, double v) {
  if (!(v > -CUDART_INF)) return;
  if (v > m) {
    s = fma(s, exp(m - v), 1.0);
    m = v;
  } else {
    s += exp(v - m);
  }
}

// K, R at polarisation node b: e^{2 i psi_b}, e^{4 i psi_b} from the launch's
// tables (uniform across the warp: one constant-cache access), else computed.
__device__ __forceinline__ void direct_node_b(const DirectParams& Q, int b, const double2& D,
                                              double A, const double2& B, double& K, double& R) {
  if (Q.n_psi <= kPsiTab) {
    direct_node(D, A, B, Q.e2[b], Q.e4[b], K, R);
    return;
  }
  double s2, c2;
  sincospi(2.0 * (double)b / Q.n_psi, &s2, &c2);
  const double2 e2 = make_double2(c2, s2);
  direct_node(D, A, B, e2, cmul_d(e2, e2), K, R);
}

// The angular and distance integral at one time node (coefficients in C),
// accumulated into the lane's log-sum-exp (m, s).  Pass 1 picks a node of
// largest K^2/(2R), in float and by cross-multiplication; any evaluated node
// makes a valid skip reference (its value v0 is then taken in double), the
// largest skips the most.  Pass 2 skips
// nodes whose bound K^2/(2R) - ln(R)/2 + ln_ub is below v0 - T, tested in
// float with a margin of 1e-3 nat + 2e-6 of the magnitudes (above the float
// error), or in double where R is outside the normal float range: a skipped
// node adds below e^-T of v0, all of them below e^-36 (T = skip_nat).
__device__ __forceinline__ void column_store(double* col, int a, const double2& D, double A,
                                             const double2& B) {
  col[a] = D.x;
  col[kColCache + a] = D.y;
  col[2 * kColCache + a] = A;
  col[3 * kColCache + a] = B.x;
  col[4 * kColCache + a] = B.y;
}

__device__ __forceinline__ void column_load(const double* col, int a, double2& D, double& A,
                                            double2& B) {
  D = make_double2(col[a], col[kColCache + a]);
  A = col[2 * kColCache + a];
  B = make_double2(col[3 * kColCache + a], col[4 * kColCache + a]);
}

__device__ __noinline__ void direct_time_node(const DirCoef& C, const DirectParams& Q, int lane,
                                              double& m, double& s, bool& nan_seen, double* col) {
  const bool cached = Q.n_phi <= kColCache;
  // pass 1 in float (first in node order on ties): it only chooses the
  // reference node, and any node is a valid one
  float bk = 0.0f, br = 0.0f;  // K^2 and R of the best node; br = 0: none yet
  long long best_idx = (long long)Q.n_phi * Q.n_psi;
  for (int a = lane; a < Q.n_phi; a += 32) {
    double2 D, B;
    double A;
    direct_column(C, (double)a / Q.n_phi, D, A, B);
    if (cached) column_store(col, a, D, A, B);
    const float dx = (float)D.x, dy = (float)D.y, af = (float)A, bx = (float)B.x,
                by = (float)B.y;
    for (int b = 0; b < Q.n_psi; ++b) {
      float2 e2, e4;
      if (Q.n_psi <= kPsiTab) {
        e2 = Q.e2f[b];
        e4 = Q.e4f[b];
      } else {
        sincospif(2.0f * (float)b / (float)Q.n_psi, &e2.y, &e2.x);
        e4 = make_float2(e2.x * e2.x - e2.y * e2.y, 2.0f * e2.x * e2.y);
      }
      const float K = e2.x * dx + e2.y * dy;
      const float R = 0.5f * (af + (e4.x * bx - e4.y * by));
      if (!(R > 0.0f) || isnan(K)) continue;
      const float kk = K * K;
      if (br == 0.0f || kk * br > bk * R) {
        bk = kk;
        br = R;
        best_idx = (long long)a * Q.n_psi + b;
      }
    }
  }
  __syncwarp();  // the cached columns are read by other lanes below
  for (int off = 16; off > 0; off >>= 1) {
    const float ok = __shfl_xor_sync(0xffffffffu, bk, off);
    const float orr = __shfl_xor_sync(0xffffffffu, br, off);
    const long long oi = __shfl_xor_sync(0xffffffffu, best_idx, off);
    if (orr > 0.0f) {
      const float l = ok * br, r = bk * orr;
      if (br == 0.0f || l > r || (l == r && oi < best_idx)) {
        bk = ok;
        br = orr;
        best_idx = oi;
      }
    }
  }
  double v0 = -CUDART_INF;
  if (best_idx < (long long)Q.n_phi * Q.n_psi) {
    const int a = (int)(best_idx / Q.n_psi), b = (int)(best_idx % Q.n_psi);
    double2 D, B;
    double A;
    if (cached)
      column_load(col, a, D, A, B);
    else
      direct_column(C, (double)a / Q.n_phi, D, A, B);
    double K, R;
    direct_node_b(Q, b, D, A, B, K, R);
    v0 = direct_distance(Q, K, R);
  }
  const double c0 = v0 - Q.skip_nat - Q.ln_ub - 1e-3;
  const float c0f = (float)c0;
  // pass 2: the log-sum-exp over the nodes that can matter.  A float screen
  // first: |K| <= |K_f| + eK and R >= R_f - eR bound the double values (eK,
  // eR cover the conversions and the float products, 8 units of 2^-24 of the
  // summed magnitudes), so the bound K^2/(2R) - ln(R)/2 taken at those ends
  // is an upper bound; only nodes it cannot exclude are formed in double.
  for (int a = lane; a < Q.n_phi; a += 32) {
    double2 D, B;
    double A;
    if (cached)
      column_load(col, a, D, A, B);
    else
      direct_column(C, (double)a / Q.n_phi, D, A, B);
    const float dx = (float)D.x, dy = (float)D.y, af = (float)A, bx = (float)B.x,
                by = (float)B.y;
    const float eK = 4.8e-7f * (fabsf(dx) + fabsf(dy));
    const float eR = 2.4e-7f * (fabsf(af) + fabsf(bx) + fabsf(by));
    for (int b = 0; b < Q.n_psi; ++b) {
      if (Q.n_psi <= kPsiTab) {
        const float2 e2 = Q.e2f[b], e4 = Q.e4f[b];
        const float Ka = fabsf(e2.x * dx + e2.y * dy) + eK;
        const float Rl = 0.5f * (af + (e4.x * bx - e4.y * by)) - eR;
        if (Rl > 1e-30f && Rl < 1e30f && Ka < 1e18f) {
          const float hu = __fdividef(Ka * Ka, 2.0f * Rl);
          const float lg = __logf(Rl);
          if (hu - 0.5f * lg < c0f - (1e-3f + 2e-6f * (hu + fabsf(lg) + fabsf(c0f)))) continue;
        }
      }
      double K, R;
      direct_node_b(Q, b, D, A, B, K, R);
      if (isnan(K + R)) {  // either is NaN (or they are opposite infinities)
        nan_seen = true;
        continue;
      }
      if (!(R > 0.0)) continue;
      const float rf = (float)R;
      if (rf > 1e-30f && rf < 1e30f) {
        // in float: K^2/(2R) - ln(R)/2 errs by < 1e-6 (|K^2/(2R)| + 1)
        const float kf = (float)K;
        const float hf = __fdividef(kf * kf, 2.0f * rf);
        const float lhs = hf - 0.5f * __logf(rf);
        if (lhs < c0f - (1e-3f + 2e-6f * (hf + fabsf(c0f)))) continue;
      } else if (K * K < 2.0 * R * (c0 + 0.5 * log(R))) {
        continue;
      }
      if (Q.mixed)
        lse_add_f(m, s, direct_distance(Q, K, R));
      else
        lse_add(m, s, direct_distance(Q, K, R));
    }
  }
}

template <int MM>
__global__ void __launch_bounds__(32 * kDirWarps, RIFT_DIRECT_MIN_BLOCKS) direct_kernel(const PointParams* __restrict__ gP,
                                                                DrawsParams dp,
                                                                const __grid_constant__ DirectParams Q,
                                                                double* __restrict__ out) {
  __shared__ PointParams P;
  __shared__ DirCoef coef[kDirWarps];
  __shared__ double2 pairbuf[kDirWarps][2][kMaxModes * kMaxModes];
  stage_point(P, gP);
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  DirCoef& C = coef[wid];
  const long long stride = (long long)gridDim.x * kDirWarps;
  for (long long i = blockIdx.x * (long long)kDirWarps + wid; i < dp.n; i += stride) {
    DirDraw<MM> g;
    direct_setup<MM>(P, dp, i, g);
    direct_norm_warp<MM>(P, g, lane, C, pairbuf[wid][0], pairbuf[wid][1]);
    double m = -CUDART_INF, s = 0.0;
    bool nan_seen = false;
    if (Q.t_up > 1) {
      // band-limited rule: the data coefficients at the coarse midpoints
      // (lane h keeps harmonic h), then their sinc sum at each fine midpoint,
      // (t_f - t_j) / h = (2 f + 1 - t_up (2 j + 1)) / (2 t_up)
      double2* my = reinterpret_cast<double2*>(reinterpret_cast<char*>(Q.slab) +
                                               (size_t)(blockIdx.x * kDirWarps + wid) *
                                                   direct_slab_per_warp(Q));
      for (int jt = 0; jt < Q.n_t; ++jt) {
        direct_data_warp<MM>(P, g, Q.t_lo + (jt + 0.5) * Q.t_h, lane, C, pairbuf[wid][0]);
        if (lane < kHm) my[jt * kHm + lane] = C.c[lane];
        __syncwarp();
      }
      const int nf = Q.n_t * Q.t_up;
      const double inv2u = 1.0 / (2.0 * Q.t_up);
      // the data coefficients at fine node f by the sinc sum, then the angular
      // and distance integral there into (m, s)
      auto fine_node = [&](int f) {
        if (lane < kHm) {
          double2 c = make_double2(0.0, 0.0);
          for (int j = 0; j < Q.n_t; ++j) {
            const long long num = 2LL * f + 1 - (long long)Q.t_up * (2 * j + 1);
            double w;
            if (Q.t_mirror) {
              // the mirrored series: D(t_f - t_j) + D(t_f + t_j) in units of
              // h, D the interpolant kernel of period 2 n_t with |k| < n_t
              const long long nump = 2LL * f + 1 + (long long)Q.t_up * (2 * j + 1);
              const double inv2n = 1.0 / (2.0 * Q.n_t), k2n = 2.0 * Q.n_t - 1.0;
              double d1 = k2n * inv2n;
              if (num != 0) {
                const double z = (double)num * inv2u;
                d1 = sinpi(k2n * z * inv2n) / (2.0 * Q.n_t * sinpi(z * inv2n));
              }
              const double zp = (double)nump * inv2u;
              const double d2 = sinpi(k2n * zp * inv2n) / (2.0 * Q.n_t * sinpi(zp * inv2n));
              w = d1 + d2;
            } else {
              w = 1.0;
              if (num != 0) {
                const double z = (double)num * inv2u;
                w = sinpi(z) / (CUDART_PI * z);
              }
            }
            const double2 v = my[j * kHm + lane];
            c.x = fma(w, v.x, c.x);
            c.y = fma(w, v.y, c.y);
          }
          C.c[lane] = c;
        }
        __syncwarp();
        direct_time_node(C, Q, lane, m, s, nan_seen, reinterpret_cast<double*>(pairbuf[wid]));
        __syncwarp();  // C is rewritten for the next fine node
      };
      bool local = Q.t_local != 0;
      double* U = reinterpret_cast<double*>(my + Q.n_t * kHm);
      int* kept = reinterpret_cast<int*>(U + ((nf + 1) & ~1));
      double2* peaks = reinterpret_cast<double2*>(kept + ((nf + 3) & ~3));
      const double hf = Q.t_h / Q.t_up;
      if (local) {
        // eq. ap:tlocal: the envelope, its maxima and their neighbourhoods
        double top = -CUDART_INF;
        for (int f = lane; f < nf; f += 32) {
          const double u = envelope_at<MM>(P, g, Q.t_lo + (f + 0.5) * hf);
          U[f] = u;
          top = fmax(top, u);
        }
        for (int off = 16; off > 0; off >>= 1) top = fmax(top, __shfl_xor_sync(0xffffffffu, top, off));
        __syncwarp();
        int npk = 0;
        bool flat = false;
        for (int base = 0; base < nf; base += 32) {
          const int f = base + lane;
          bool is_max = false;
          double csig = 0.0;
          if (f < nf && nf > 1) {
            const double um = U[f];
            const double ul = f > 0 ? U[f - 1] : U[1];
            const double ur = f < nf - 1 ? U[f + 1] : U[nf - 2];
            if (um >= ul && um > ur && um >= top - Q.depth) {
              is_max = true;
              const double curv = 2.0 * um - ul - ur;
              if (curv > 0.0) csig = Q.t_c * hf / sqrt(curv);
              else flat = true;
            }
          } else if (f < nf) {  // a single node
            is_max = true;
            csig = CUDART_INF;
          }
          const unsigned bal = __ballot_sync(0xffffffffu, is_max);
          const int rank = __popc(bal & ((1u << lane) - 1u));
          if (is_max && npk + rank < kMaxPeaks) peaks[npk + rank] = make_double2((double)f, csig);
          npk += __popc(bal);
        }
        flat = __any_sync(0xffffffffu, flat);
        if (flat || npk > kMaxPeaks) local = false;  // no justified width, or too many maxima
        __syncwarp();
        if (local) {
          int nkept = 0;
          for (int f = lane; f < nf; f += 32) {
            int k = 0;
            for (int q = 0; q < npk && !k; ++q) {
              const double2 pk = peaks[q];
              k = fabs(((double)f - pk.x) * hf) <= pk.y;
            }
            kept[f] = k;
            nkept += k;
          }
          for (int off = 16; off > 0; off >>= 1) nkept += __shfl_xor_sync(0xffffffffu, nkept, off);
          if (nkept == nf) local = false;  // nothing to skip: the full rule
          __syncwarp();
        }
      }
      if (!local) {
        for (int f = 0; f < nf; ++f) fine_node(f);
      } else {
        // the kept neighbourhoods, and the bound of the rest (lane-uniform)
        double mb = -CUDART_INF, sb = 0.0;
        for (int f = 0; f < nf; ++f) {
          if (kept[f]) fine_node(f);
          else lse_add(mb, sb, U[f]);
        }
        // the kept value (a merged copy of the lanes' sums) against the bound
        double mk = m, sk = s;
        for (int off = 16; off > 0; off >>= 1) {
          const double om = __shfl_xor_sync(0xffffffffu, mk, off);
          const double os = __shfl_xor_sync(0xffffffffu, sk, off);
          if (om > mk) {
            sk = fma(sk, exp(mk - om), os);
            mk = om;
          } else if (om > -CUDART_INF) {
            sk = fma(os, exp(om - mk), sk);
          }
        }
        const double vk = mk > -CUDART_INF ? mk + log(sk) + Q.lnw : -CUDART_INF;
        const double vb = mb + log(sb) - log((double)nf);
        if (!(vb - vk <= Q.ln_tol)) {  // the remainder may matter: every fine node
          for (int f = 0; f < nf; ++f)
            if (!kept[f]) fine_node(f);
        }
      }
    } else {
      const int nt = Q.n_t > 0 ? Q.n_t : 1;
      for (int jt = 0; jt < nt; ++jt) {
        const double tc = Q.n_t > 0 ? Q.t_lo + (jt + 0.5) * Q.t_h : load_param_d(dp, 6, i);
        direct_data_warp<MM>(P, g, tc, lane, C, pairbuf[wid][0]);
        direct_time_node(C, Q, lane, m, s, nan_seen, reinterpret_cast<double*>(pairbuf[wid]));
        __syncwarp();  // C is rewritten for the next time node
      }
    }
    nan_seen = __any_sync(0xffffffffu, nan_seen);
    for (int off = 16; off > 0; off >>= 1) {
      const double om = __shfl_xor_sync(0xffffffffu, m, off);
      const double os = __shfl_xor_sync(0xffffffffu, s, off);
      if (om > m) {
        s = fma(s, exp(m - om), os);
        m = om;
      } else if (om > -CUDART_INF) {
        s = fma(os, exp(om - m), s);
      }
    }
    if (lane == 0) out[i] = nan_seen ? CUDART_NAN : (m > -CUDART_INF ? m + log(s) + Q.lnw : -CUDART_INF);
    __syncwarp();
  }
}

template <int MM>
cudaError_t launch_direct_mm(const PointParams* dP, const DrawsParams& dp, const DirectParams& Q,
                             double* out, cudaStream_t st) {
  const int threads = 32 * kDirWarps;
  const long long need = (dp.n + kDirWarps - 1) / kDirWarps;
  int blocks = grid_for(direct_kernel<MM>, threads, 0);
  if (need < blocks) blocks = (int)(need > 0 ? need : 1);
  if (Q.t_up <= 1) {
    direct_kernel<MM><<<blocks, threads, 0, st>>>(dP, dp, Q, out);
    return cudaGetLastError();
  }
  DirectParams Qb = Q;
  const size_t bytes = (size_t)blocks * kDirWarps * direct_slab_per_warp(Q);
  cudaError_t e = cudaMallocAsync((void**)&Qb.slab, bytes, st);
  if (e != cudaSuccess) return e;
  direct_kernel<MM><<<blocks, threads, 0, st>>>(dP, dp, Qb, out);
  e = cudaGetLastError();
  const cudaError_t f = cudaFreeAsync(Qb.slab, st);
  return e != cudaSuccess ? e : f;
}

cudaError_t launch_direct(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                          const DirectParams& Q, double* out, cudaStream_t st) {
  const int M = hp.M;
  if (M <= 2) return launch_direct_mm<2>(dP, dp, Q, out, st);
  if (M <= 4) return launch_direct_mm<4>(dP, dp, Q, out, st);
  if (M <= 6) return launch_direct_mm<6>(dP, dp, Q, out, st);
  if (M <= 8) return launch_direct_mm<8>(dP, dp, Q, out, st);
  if (M <= 10) return launch_direct_mm<10>(dP, dp, Q, out, st);
  if (M <= 12) return launch_direct_mm<12>(dP, dp, Q, out, st);
  return launch_direct_mm<16>(dP, dp, Q, out, st);
}

// Orthonormal Hermite polynomials p_0..p_n at x (weight e^{-x^2}):
// p_0 = pi^(-1/4), p_(k+1) = sqrt(2/(k+1)) x p_k - sqrt(k/(k+1)) p_(k-1).
void hermite_orthonormal(int n, double x, double* p) {
  p[0] = std::pow(M_PI, -0.25);
  if (n >= 1) p[1] = std::sqrt(2.0) * x * p[0];
  for (int k = 1; k < n; ++k)
    p[k + 1] = std::sqrt(2.0 / (k + 1)) * x * p[k] - std::sqrt((double)k / (k + 1)) * p[k - 1];
}

// Gauss-Hermite nodes as the zeros of p_n (bracketed by a scan of
// (-sqrt(2n+1)-1, sqrt(2n+1)+1), refined by bisection) and the Christoffel
// weights w_i = 1 / sum_{k<n} p_k(x_i)^2.
int gauss_hermite(int n, double* x, double* w) {
  std::vector<double> p(n + 1);
  const double lim = std::sqrt(2.0 * n + 1.0) + 1.0;
  const int steps = 400 * n + 400;
  int found = 0;
  double xa = -lim;
  hermite_orthonormal(n, xa, p.data());
  double fa = p[n];
  for (int s = 1; s <= steps && found < n; ++s) {
    const double xb = -lim + 2.0 * lim * s / steps;
    hermite_orthonormal(n, xb, p.data());
    const double fb = p[n];
    if (fb == 0.0 || (fa < 0.0) != (fb < 0.0)) {
      double lo = xa, hi = xb, flo = fa;
      for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        hermite_orthonormal(n, mid, p.data());
        if ((p[n] < 0.0) == (flo < 0.0)) {
          lo = mid;
          flo = p[n];
        } else {
          hi = mid;
        }
      }
      x[found++] = 0.5 * (lo + hi);
    }
    xa = xb;
    fa = fb;
  }
  if (found != n) return RIFT_ILE_ERR_INVALID_ARG;
  for (int i = 0; i < n; ++i) {
    hermite_orthonormal(n, x[i], p.data());
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += p[k] * p[k];
    w[i] = 1.0 / s;
  }
  return RIFT_ILE_OK;
}

}  // namespace
}  // namespace rift

using namespace rift;

extern "C" int rift_ile_gauss_hermite(int32_t n, double* x, double* w) {
  if (n < 1 || n > RIFT_ILE_MAX_GH || !x || !w) {
    rift_ile_set_error("rift_ile_gauss_hermite: n=%d outside 1..%d or NULL output", n, RIFT_ILE_MAX_GH);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const int rc = gauss_hermite(n, x, w);
  if (rc) rift_ile_set_error("rift_ile_gauss_hermite: root bracketing failed for n=%d", n);
  return rc;
}

extern "C" int rift_ile_lnL_direct(const rift_ile_point* pt, const rift_ile_draws* draws,
                                   const rift_ile_direct_rule* rule, double* out, void* stream) {
  if (!pt || !rule) {
    rift_ile_set_error("rift_ile_lnL_direct: point or rule is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int rc = validate_draws(draws);
  if (rc) return rc;
  if (rule->n_phi < 1 || rule->n_psi < 1 || (long long)rule->n_phi * rule->n_psi > (1LL << 26) ||
      rule->n_gh < 1 || rule->n_gh > RIFT_ILE_MAX_GH) {
    rift_ile_set_error("rift_ile_lnL_direct: grid %d x %d or n_gh=%d out of range", rule->n_phi,
                       rule->n_psi, rule->n_gh);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (rule->n_t < 0 || rule->n_t > (1 << 20) ||
      (rule->n_t > 0 && !(rule->t_hi > rule->t_lo && std::isfinite(rule->t_lo) &&
                          std::isfinite(rule->t_hi)))) {
    rift_ile_set_error("rift_ile_lnL_direct: n_t=%d needs 0 <= n_t <= 2^20 and t_lo < t_hi finite",
                       rule->n_t);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (rule->t_up < 0 ||
      (rule->t_up > 1 && (rule->n_t < 1 || rule->n_t > 1024 ||
                          (long long)rule->n_t * rule->t_up > (1LL << 20)))) {
    rift_ile_set_error("rift_ile_lnL_direct: t_up=%d needs n_t in 1..1024 and n_t t_up <= 2^20",
                       rule->t_up);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (!(rule->d_min > 0.0) || !(rule->d_max > rule->d_min) || !std::isfinite(rule->d_max)) {
    rift_ile_set_error("rift_ile_lnL_direct: need 0 < d_min < d_max finite");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (rule->t_mirror && rule->t_up < 2) {
    rift_ile_set_error("rift_ile_lnL_direct: the mirrored reconstruction needs t_up >= 2");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (rule->t_local &&
      (rule->t_up < 2 || (long long)rule->n_t * rule->t_up > kMaxLocalFine ||
       !(rule->t_c > 0.0) || !std::isfinite(rule->t_c) || !(rule->t_tol > 0.0) ||
       !(rule->t_tol < 1.0))) {
    rift_ile_set_error("rift_ile_lnL_direct: the peak-local rule needs t_up >= 2, n_t t_up <= "
                       "%d, t_c > 0 finite and 0 < t_tol < 1", kMaxLocalFine);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (rule->precision != RIFT_ILE_FP64 && rule->precision != RIFT_ILE_FP32_MIXED) {
    rift_ile_set_error("rift_ile_lnL_direct: precision %d unknown", rule->precision);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (rule->precision == RIFT_ILE_FP32_MIXED && rule->d_max > 1e9 * rule->d_min) {
    rift_ile_set_error("rift_ile_lnL_direct: the mixed rule needs d_max / d_min <= 1e9");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!out) {
    rift_ile_set_error("rift_ile_lnL_direct: out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const PointParams& hp = pt->host;
  DirectParams Q;
  std::memset(&Q, 0, sizeof(Q));
  Q.n_phi = rule->n_phi;
  Q.n_psi = rule->n_psi;
  Q.n_gh = rule->n_gh;
  const double dref = hp.d_ref;
  Q.lo = dref / rule->d_max;
  Q.hi = dref / rule->d_min;
  const double norm = 3.0 * dref * dref * dref /
                      (rule->d_max * rule->d_max * rule->d_max - rule->d_min * rule->d_min * rule->d_min);
  Q.lnnorm = std::log(norm);
  Q.n_t = rule->n_t;
  Q.t_lo = rule->t_lo;
  Q.t_h = rule->n_t > 0 ? (rule->t_hi - rule->t_lo) / rule->n_t : 0.0;
  Q.t_up = rule->t_up > 1 ? rule->t_up : 1;
  Q.slab = nullptr;
  Q.t_local = rule->t_local ? 1 : 0;
  Q.t_mirror = rule->t_mirror ? 1 : 0;
  if (Q.t_local) {
    Q.t_c = rule->t_c;
    Q.ln_tol = std::log(rule->t_tol);
    Q.depth = -std::log(rule->t_tol) + std::log((double)Q.n_t * Q.t_up);
  }
  Q.lnw = -std::log((double)rule->n_phi * rule->n_psi * (rule->n_t > 0 ? rule->n_t : 1) * Q.t_up);
  Q.ln_ub = std::log(std::sqrt(2.0 * M_PI) * norm) - 4.0 * std::log(Q.lo);
  Q.skip_nat = kSkipNat + std::log((double)rule->n_phi * rule->n_psi);
  if ((rc = gauss_hermite(Q.n_gh, Q.xi, Q.w))) {
    rift_ile_set_error("rift_ile_lnL_direct: Gauss-Hermite rule failed for n=%d", Q.n_gh);
    return rc;
  }
  Q.mixed = rule->precision == RIFT_ILE_FP32_MIXED ? 1 : 0;
  Q.inv_lo = 1.0 / Q.lo;
  Q.hi_lo = Q.hi / Q.lo;
  Q.lnnorm_lo = Q.lnnorm - 4.0 * std::log(Q.lo);
  for (int j = 0; j < Q.n_gh; ++j) {
    Q.wf[j] = (float)Q.w[j];
    Q.xif[j] = (float)Q.xi[j];
  }
  Q.hi_lof = (float)Q.hi_lo;
  if (Q.n_psi <= kPsiTab)
    for (int b = 0; b < Q.n_psi; ++b) {
      const double ang = 2.0 * M_PI * b / Q.n_psi;
      Q.e2[b] = make_double2(std::cos(ang), std::sin(ang));
      Q.e4[b] = make_double2(std::cos(2.0 * ang), std::sin(2.0 * ang));
      Q.e2f[b] = make_float2((float)Q.e2[b].x, (float)Q.e2[b].y);
      Q.e4f[b] = make_float2((float)Q.e4[b].x, (float)Q.e4[b].y);
    }
  return check_cuda(launch_direct(hp, pt->dev, draws_params(draws), Q, out, (cudaStream_t)stream),
                    "rift_ile_lnL_direct launch");
}

namespace rift {
namespace {

// LSE partials of values[i] + logw[i], one per block (fixed reduction order).
__global__ void __launch_bounds__(256) lse_array_kernel(const double* __restrict__ v, DrawsParams dp,
                                                        LseState* __restrict__ partials) {
  ThreadLse64 st = tlse64_init();
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < dp.n; i += stride)
    tlse64_push(st, v[i] + load_logw_d(dp, i));
  block_lse64_write(st, partials + blockIdx.x);
}

}  // namespace
}  // namespace rift

extern "C" int rift_ile_lnZ_direct_state(const rift_ile_point* pt, const rift_ile_draws* draws,
                                         const rift_ile_direct_rule* rule, double* scratch,
                                         rift_ile_lse* state_out, void* stream) {
  using namespace rift;
  if (!state_out || (!scratch && draws && draws->n > 0)) {
    rift_ile_set_error("rift_ile_lnZ_direct_state: state_out or scratch is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int rc = rift_ile_lnL_direct(pt, draws, rule, scratch, stream);
  if (rc) return rc;
  LseState *partials = nullptr, *state = nullptr;
  unsigned long long* oob = nullptr;
  if ((rc = lse_workspace(&partials, &state, &oob))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  LseState* out = reinterpret_cast<LseState*>(state_out);
  if (draws->n == 0)
    return check_cuda(launch_lse_combine(partials, 0, 0.0, out, st), "lnZ combine launch");
  const int blocks = grid_cap(device_sms() * 4, draws->n, 256);
  lse_array_kernel<<<blocks, 256, 0, st>>>(scratch, draws_params(draws), partials);
  if ((rc = check_cuda(cudaGetLastError(), "lse_array_kernel launch"))) return rc;
  return check_cuda(launch_lse_combine(partials, blocks, (double)draws->n, out, st),
                    "lnZ combine launch");
}
