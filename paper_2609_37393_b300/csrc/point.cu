// Construction of an intrinsic point: validation, constant tables, and the
// whitened form of each detector's quadratic term used by the FP32-mixed path.
//
// The factored likelihood of one detector (eq. def:lnL:Decomposed), written in
// the real 2M-vector z = (Re c, Im c) of the template coefficients
// c_lm = x F_k Y_lm and the real 2M-vector b(t) = (Re Q_lm(t), Im Q_lm(t)), is
//     lnL_k = z.b - z^T G z / 2,
//     G = 1/2 [[Ur + Vr, -Ui - Vi], [Ui - Vi, Ur - Vr]]
// (U = Ur + i Ui, V = Vr + i Vi; this block form equals Re(c^+ U c) + Re(c^T V c)
// for any U, V).  With the eigen-decomposition G = sum_r lam_r v_r v_r^T and
// scales s_r = sqrt|lam_r|,
//     w_r = s_r v_r.z,   e_r(t) = v_r.b(t) / s_r,
//     lnL_k = sum_r w_r e_r - 1/2 |w|^2 = 1/2 |e|^2 - 1/2 |e - w|^2.
// Because the cubic is linear in the table, e(t) is the cubic interpolant of
// the whitened table e[j], built here once per point in FP64 and stored as
// double-float pairs; on each table interval 1/2 |e(f)|^2 is a sextic in the
// cubic's offset f, whose coefficients are tabulated too.  The kernel then
// needs the large term 1/2|e|^2 only through that polynomial (double-float
// Horner) and forms the residual e - w, which is small where the likelihood
// matters, in FP32.
//
// Directions with lam_r ~ 0 (for aligned-spin mode pairs (l, +-m), half of
// them: the template depends on c_lm + (-1)^l conj(c_l,-m) only) are dropped
// when the data has no component along them beyond FP64 rounding, so the
// whitened dimension R is the rank of G.  Detectors with identical U and V
// (a shared noise curve) form a class and share one whitening.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return RIFT_ILE_OK;
  rift_ile_set_error("%s: %s", what, cudaGetErrorString(e));
  return RIFT_ILE_ERR_CUDA;
}

namespace {

double fact(int n) {
  double f = 1.0;
  for (int i = 2; i <= n; ++i) f *= i;
  return f;
}

// -2Y_lm(iota, phi) = sqrt((2l+1)/(4 pi)) d^l_{m,2}(iota) e^{i m phi}, with the
// Wigner small-d explicit sum
//   d^l_{m'm}(b) = sum_k (-1)^(m'-m+k) sqrt((l+m')!(l-m')!(l+m)!(l-m)!)
//                  / ((l+m-k)! k! (m'-m+k)! (l-m'-k)!)
//                  cos(b/2)^(2l+m-m'-2k) sin(b/2)^(m'-m+2k).
// Returns the terms as coefficients of c^p s^(2l-p), p = k0 + 2r, r < nt.
int harmonic_terms(int l, int mp, int* k0, double* coef) {
  const int m = 2;
  struct Term {
    int p;
    double a;
  } terms[2 * RIFT_ILE_MAX_ELL + 4];
  int nt = 0;
  const double norm = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) *
                      std::sqrt(fact(l + mp) * fact(l - mp) * fact(l + m) * fact(l - m));
  for (int k = 0; k <= 2 * l; ++k) {
    int a = l + m - k, b = k, c = mp - m + k, d = l - mp - k;
    if (a < 0 || b < 0 || c < 0 || d < 0) continue;
    double sign = ((mp - m + k) & 1) ? -1.0 : 1.0;
    terms[nt].p = 2 * l + m - mp - 2 * k;
    terms[nt].a = sign * norm / (fact(a) * fact(b) * fact(c) * fact(d));
    ++nt;
  }
  if (nt == 0) return 0;
  // ascending cosine power, spaced by two
  for (int i = 0; i < nt; ++i)
    for (int j = i + 1; j < nt; ++j)
      if (terms[j].p < terms[i].p) std::swap(terms[i], terms[j]);
  *k0 = terms[0].p;
  for (int i = 0; i < nt; ++i) coef[i] = terms[i].a;
  return nt;
}

}  // namespace

// The Goldberg sum of harmonic_terms rewritten in z = cos(iota): every term
// c^p s^q (p + q = 2l, p of one parity) is ((1+z)/2)^(p/2) ((1-z)/2)^(q/2)
// for even p, and sin(iota)/2 times ((1+z)/2)^((p-1)/2) ((1-z)/2)^((q-1)/2)
// for odd p.  Writes the coefficients of z^0..z^l and returns the parity.
int harmonic_zpoly(int l, int nt, int k0, const double* coef, double* out) {
  const int par = k0 & 1;
  for (int j = 0; j <= l; ++j) out[j] = 0.0;
  for (int r = 0; r < nt; ++r) {
    const int p = k0 + 2 * r, q = 2 * l - p;
    const int a = (p - par) / 2, b = (q - par) / 2;
    double poly[RIFT_ILE_MAX_ELL + 1] = {1.0};
    int deg = 0;
    for (int u = 0; u < a + b; ++u) {  // times (1 + z)/2 a times, then (1 - z)/2 b times
      const double sgn = u < a ? 1.0 : -1.0;
      for (int j = deg + 1; j >= 1; --j) poly[j] = 0.5 * (poly[j] + sgn * poly[j - 1]);
      poly[0] *= 0.5;
      ++deg;
    }
    const double w = par ? 0.5 * coef[r] : coef[r];
    for (int j = 0; j <= deg; ++j) out[j] += w * poly[j];
  }
  return par;
}

// Cyclic Jacobi eigenvalue iteration for a symmetric n x n matrix (row-major,
// destroyed).  Eigenvalues to lam[], eigenvectors to the columns of V.
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& lam, std::vector<double>& V) {
  V.assign(n * n, 0.0);
  for (int i = 0; i < n; ++i) V[i * n + i] = 1.0;
  double total = 0.0;
  for (int i = 0; i < n * n; ++i) total += a[i] * a[i];
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += a[p * n + q] * a[p * n + q];
    if (off <= 1e-32 * total || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        double apq = a[p * n + q];
        if (apq == 0.0) continue;
        double theta = (a[q * n + q] - a[p * n + p]) / (2.0 * apq);
        double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          double akp = a[k * n + p], akq = a[k * n + q];
          a[k * n + p] = c * akp - s * akq;
          a[k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          double apk = a[p * n + k], aqk = a[q * n + k];
          a[p * n + k] = c * apk - s * aqk;
          a[q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          double vkp = V[k * n + p], vkq = V[k * n + q];
          V[k * n + p] = c * vkp - s * vkq;
          V[k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
  lam.resize(n);
  for (int i = 0; i < n; ++i) lam[i] = a[i * n + i];
}

void split_df(double x, float* hi, float* lo) {
  float h = (float)x;
  *hi = h;
  *lo = (float)(x - (double)h);
}

namespace {

// proj[k][j][r] = v_r . b_k[j] for every eigen-direction r of detector k's
// class (FP64), with b = (Re Q[k][j][:], Im Q[k][j][:]).
template <typename QT>
__global__ void project_kernel(const QT* __restrict__ Q, const double* __restrict__ Vt,
                               const int* __restrict__ cls_of, int K, int n, int M,
                               double* __restrict__ proj) {
  const int D = 2 * M;
  long long total = (long long)K * n * D;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int r = (int)(idx % D);
    long long kj = idx / D;
    int k = (int)(kj / n);
    const QT* row = Q + kj * M;
    const double* v = Vt + ((long long)cls_of[k] * D + r) * D;
    double acc = 0.0;
    for (int a = 0; a < M; ++a) {
      acc = fma(v[a], (double)row[a].x, acc);
      acc = fma(v[M + a], (double)row[a].y, acc);
    }
    proj[idx] = acc;
  }
}

// colmax[k][r] = max_j |proj[k][j][r]| (one block per (k, r)).
__global__ void colmax_kernel(const double* __restrict__ proj, int n, int D,
                              double* __restrict__ colmax) {
  const int k = blockIdx.x / D, r = blockIdx.x % D;
  double m = 0.0;
  for (int j = threadIdx.x; j < n; j += blockDim.x)
    m = fmax(m, fabs(proj[((long long)k * n + j) * D + r]));
  __shared__ double red[256];
  red[threadIdx.x] = m;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) colmax[blockIdx.x] = red[0];
}

__device__ __forceinline__ float2 split2(double x) {
  float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}

// ehat[k][kEhatPad + j] = proj[k][j][r] * inv_s[k][r], r < R, as (hi, lo)
// pairs laid out by direction pairs: floats (hi_r, hi_r+1, lo_r, lo_r+1) for
// even r, so that one 16-byte load gives the packed operands of two directions.
__global__ void whiten_kernel(const double* __restrict__ proj, const double* __restrict__ inv_s,
                              int K, int n, int D, int R, float2* __restrict__ ehat) {
  // rows are stored with kEhatPad zero rows before and after (already zeroed)
  long long total = (long long)K * n * R;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int r = (int)(idx % R);
    long long kj = idx / R;
    int k = (int)(kj / n);
    int j = (int)(kj % n);
    // directions r >= D exist only as zero padding (inv_s = 0 there)
    const double v = r < D ? proj[kj * D + r] * inv_s[k * R + r] : 0.0;
    const float2 hl = split2(v);
    float* row = reinterpret_cast<float*>(ehat + ((long long)k * (n + 2 * kEhatPad) + kEhatPad + j) * R);
    row[4 * (r / 2) + (r & 1)] = hl.x;
    row[4 * (r / 2) + 2 + (r & 1)] = hl.y;
  }
}

// The interpolating cubic of each interval j = -3..n+1 (taps j-1..j+2 of the
// zero-padded table; the four-point cubic C_3 of eq. q-time-pregrid):
// e(f) = c0 + c1 f + c2 f^2 + c3 f^3 with, for the tap
// values e_{-1}, e_0, e_1, e_2 (nodes -1, 0, 1, 2),
//   c0 = e_0,  c1 = -e_{-1}/3 - e_0/2 + e_1 - e_2/6,  c2 = e_{-1}/2 - e_0 + e_1/2,
//   c3 = -e_{-1}/6 + e_0/2 - e_1/2 + e_2/6
// (the monomial coefficients of the four Lagrange cubics), formed in FP64 from
// the (hi, lo) rows; c0 is copied as its (hi, lo) pair, c1..c3 rounded to FP32
// (their rounding is of the order of the FP32 tap weights' in the four-tap
// sum they replace).  Interval records of rec_f4 float4 (3 R/2, or more where
// the record carries more after the cubic), entry (k (n + 5) + j + 3) rec_f4 +
// 3 p + {0, 1, 2} for direction pair p: (c0 hi r, c0 hi r+1, c0 lo r,
// c0 lo r+1), (c1 r, c1 r+1, c2 r, c2 r+1), (c3 r, c3 r+1, 0, 0).
__global__ void cubic_table_kernel(const float2* __restrict__ ehat, int K, int n, int R,
                                   int rec_f4, float4* __restrict__ ecub) {
  const int NP = R / 2, per = n + 5;
  const long long total = (long long)K * per * NP;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(idx % NP);
    const long long kq = idx / NP;
    const int k = (int)(kq / per), j = (int)(kq % per) - 3;
    // rows j - 1 .. j + 2 lie in [-4, n + 3], inside the padded table
    const float* rows = reinterpret_cast<const float*>(
        ehat + ((long long)k * (n + 2 * kEhatPad) + kEhatPad + (j - 1)) * R);
    double c[4][2];
    float4 a0;
    for (int h = 0; h < 2; ++h) {
      double e[4];
      for (int i = 0; i < 4; ++i) {
        const float* row = rows + (long long)i * 2 * R;
        e[i] = (double)row[4 * p + h] + (double)row[4 * p + 2 + h];
      }
      c[1][h] = -e[0] / 3.0 - 0.5 * e[1] + e[2] - e[3] / 6.0;
      c[2][h] = 0.5 * e[0] - e[1] + 0.5 * e[2];
      c[3][h] = (e[3] - e[0]) / 6.0 + 0.5 * (e[1] - e[2]);
    }
    const float* r0 = rows + 2 * R;  // row j
    a0 = make_float4(r0[4 * p], r0[4 * p + 1], r0[4 * p + 2], r0[4 * p + 3]);
    float4* o = ecub + kq * rec_f4 + 3 * p;
    o[0] = a0;
    o[1] = make_float4((float)c[1][0], (float)c[1][1], (float)c[2][0], (float)c[2][1]);
    o[2] = make_float4((float)c[3][0], (float)c[3][1], 0.f, 0.f);
  }
}

// The sextic tails of the interval records of PointParams::erec (after the
// cubic): the epoly coefficients of interval j = -2..n as pairs (c0, c1),
// (c2, c3), (c4, c5), (c6, 0); zero for j = -3 and n + 1.
__global__ void interval_sextic_kernel(const float2* __restrict__ epoly, int K, int n, int R,
                                       float4* __restrict__ erec) {
  const int NP = R / 2, rec = 3 * NP + 4, per = n + 5;
  const long long total = (long long)K * per * 4;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(idx % 4);
    const long long kq = idx / 4;
    const int k = (int)(kq / per), j = (int)(kq % per) - 3;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j >= -2 && j <= n) {
      const float2* pc = epoly + ((size_t)k * (n + 3) + (size_t)(j + 2)) * (kPolyDeg + 1);
      const float2 a = pc[2 * w];
      const float2 b = 2 * w + 1 <= kPolyDeg ? pc[2 * w + 1] : make_float2(0.f, 0.f);
      v = make_float4(a.x, a.y, b.x, b.y);
    }
    erec[kq * rec + 3 * NP + w] = v;
  }
}

// Coefficients of 1/2 |e(f)|^2 on interval j (taps j-1..j+2, zero outside
// the table): with e(f) = sum_i L_i(f) e_{j-1+i} and the Lagrange cubics
// L_i(f) on nodes -1, 0, 1, 2, it is 1/2 sum_{i,i'} G_ii' L_i(f) L_i'(f), a
// sextic in f (G the Gram matrix of the four taps).  Entry j + 2, j = -2..n.
__global__ void halfnorm_poly_kernel(const double* __restrict__ proj,
                                     const double* __restrict__ inv_s, int K, int n, int D,
                                     int R, float2* __restrict__ poly) {
  const double L[4][4] = {{0.0, -1.0 / 3.0, 0.5, -1.0 / 6.0},
                          {1.0, -0.5, -1.0, 0.5},
                          {0.0, 1.0, 0.5, -0.5},
                          {0.0, -1.0 / 6.0, 0.0, 1.0 / 6.0}};
  const int per = n + 3;
  long long total = (long long)K * per;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    int k = (int)(idx / per);
    int j = (int)(idx % per) - 2;
    double G[4][4];
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) G[a][b] = 0.0;
    for (int a = 0; a < 4; ++a) {
      int ja = j - 1 + a;
      if (ja < 0 || ja >= n) continue;
      for (int b = a; b < 4; ++b) {
        int jb = j - 1 + b;
        if (jb < 0 || jb >= n) continue;
        double acc = 0.0;
        for (int r = 0; r < R && r < D; ++r) {  // directions r >= D are zero padding
          double ea = proj[((long long)k * n + ja) * D + r] * inv_s[k * R + r];
          double eb = proj[((long long)k * n + jb) * D + r] * inv_s[k * R + r];
          acc = fma(ea, eb, acc);
        }
        G[a][b] = G[b][a] = acc;
      }
    }
    double c[7] = {0, 0, 0, 0, 0, 0, 0};
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b)
        for (int p = 0; p < 4; ++p)
          for (int q = 0; q < 4; ++q) c[p + q] += 0.5 * G[a][b] * L[a][p] * L[b][q];
    for (int p = 0; p < 7; ++p) poly[idx * 7 + p] = split2(c[p]);
  }
}

template <typename T>
int dev_alloc(T** p, size_t count) {
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    rift_ile_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  return RIFT_ILE_OK;
}

int validate(const rift_ile_point_desc* d) {
  if (!d) {
    rift_ile_set_error("point description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->n_det < 1 || d->n_det > RIFT_ILE_MAX_DET || d->n_modes < 1 ||
      d->n_modes > RIFT_ILE_MAX_MODES) {
    rift_ile_set_error("n_det=%d (1..%d) or n_modes=%d (1..%d) out of range", d->n_det,
                       RIFT_ILE_MAX_DET, d->n_modes, RIFT_ILE_MAX_MODES);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  if (!d->ell || !d->em || !d->Q || !d->q_t0 || !d->U || !d->V || !d->det_pos || !d->det_resp) {
    rift_ile_set_error("a required array of the point description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->q_len < 4) {
    rift_ile_set_error("q_len=%d: the cubic needs at least 4 samples", d->q_len);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (d->q_dtype != RIFT_ILE_C64 && d->q_dtype != RIFT_ILE_C128) {
    rift_ile_set_error("q_dtype=%d is neither RIFT_ILE_C64 nor RIFT_ILE_C128", d->q_dtype);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!(d->q_dt > 0.0) || !std::isfinite(d->q_dt) || !std::isfinite(d->gmst) ||
      !(d->d_ref > 0.0) || !std::isfinite(d->d_ref)) {
    rift_ile_set_error("q_dt, gmst or d_ref is not finite and positive");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  for (int i = 0; i < d->n_modes; ++i) {
    if (d->ell[i] < 2 || d->ell[i] > RIFT_ILE_MAX_ELL || std::abs(d->em[i]) > d->ell[i]) {
      rift_ile_set_error("mode %d: (l=%d, m=%d) unsupported (2 <= l <= %d, |m| <= l)", i,
                         d->ell[i], d->em[i], RIFT_ILE_MAX_ELL);
      return RIFT_ILE_ERR_UNSUPPORTED;
    }
  }
  for (int k = 0; k < d->n_det; ++k) {
    if (!std::isfinite(d->q_t0[k])) {
      rift_ile_set_error("q_t0[%d] is not finite", k);
      return RIFT_ILE_ERR_INVALID_ARG;
    }
    for (int c = 0; c < 3; ++c)
      if (!std::isfinite(d->det_pos[3 * k + c])) {
        rift_ile_set_error("det_pos[%d] is not finite", k);
        return RIFT_ILE_ERR_INVALID_ARG;
      }
    for (int c = 0; c < 6; ++c)
      if (!std::isfinite(d->det_resp[6 * k + c])) {
        rift_ile_set_error("det_resp[%d] is not finite", k);
        return RIFT_ILE_ERR_INVALID_ARG;
      }
  }
  const int M = d->n_modes;
  for (long i = 0; i < (long)d->n_det * M * M * 2; ++i)
    if (!std::isfinite(d->U[i]) || !std::isfinite(d->V[i])) {
      rift_ile_set_error("U or V holds a non-finite value");
      return RIFT_ILE_ERR_INVALID_ARG;
    }
  return RIFT_ILE_OK;
}

}  // namespace

int harmonic_coefficients(int l, int m, int* k0, double* coef) {
  return harmonic_terms(l, m, k0, coef);
}

int whitened_tables(const void* Q, int q_c128, int K, int n, int Mq, int ncls, const int* cls_of,
                    const double* Vt, const double* inv_s, int R, float2* ehat, float2* epoly,
                    float4* ecub, cudaStream_t st) {
  const int D = 2 * Mq;
  double *dVt = nullptr, *dproj = nullptr, *dinv_s = nullptr;
  int* dcls = nullptr;
  int rc = RIFT_ILE_OK;
  do {
    if ((rc = dev_alloc(&dVt, (size_t)ncls * D * D))) break;
    if ((rc = dev_alloc(&dproj, (size_t)K * n * D))) break;
    if ((rc = dev_alloc(&dinv_s, (size_t)K * R))) break;
    if ((rc = dev_alloc(&dcls, (size_t)K))) break;
    if ((rc = check_cuda(cudaMemcpyAsync(dVt, Vt, (size_t)ncls * D * D * sizeof(double),
                                         cudaMemcpyHostToDevice, st), "copy of eigenvectors")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(dinv_s, inv_s, (size_t)K * R * sizeof(double),
                                         cudaMemcpyHostToDevice, st), "copy of scales")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(dcls, cls_of, K * sizeof(int), cudaMemcpyHostToDevice, st),
                         "copy of classes")))
      break;
    if ((rc = check_cuda(cudaMemsetAsync(ehat, 0, (size_t)K * (n + 2 * kEhatPad) * R * sizeof(float2),
                                         st), "table padding")))
      break;
    const long long total = (long long)K * n * D;
    const int blocks = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
    if (q_c128)
      project_kernel<double2><<<blocks, 256, 0, st>>>((const double2*)Q, dVt, dcls, K, n, Mq, dproj);
    else
      project_kernel<float2><<<blocks, 256, 0, st>>>((const float2*)Q, dVt, dcls, K, n, Mq, dproj);
    const long long tw = (long long)K * n * R;
    whiten_kernel<<<(int)std::min<long long>((tw + 255) / 256, 148LL * 16), 256, 0, st>>>(
        dproj, dinv_s, K, n, D, R, ehat);
    const long long tp = (long long)K * (n + 3);
    halfnorm_poly_kernel<<<(int)std::min<long long>((tp + 127) / 128, 148LL * 16), 128, 0, st>>>(
        dproj, dinv_s, K, n, D, R, epoly);
    const long long tc3 = (long long)K * (n + 5) * (R / 2);
    cubic_table_kernel<<<(int)std::min<long long>((tc3 + 127) / 128, 148LL * 16), 128, 0, st>>>(
        ehat, K, n, R, 3 * (R / 2), ecub);
    if ((rc = check_cuda(cudaGetLastError(), "whitened table kernels"))) break;
    rc = check_cuda(cudaStreamSynchronize(st), "whitened tables");
  } while (0);
  cudaFree(dVt);
  cudaFree(dproj);
  cudaFree(dinv_s);
  cudaFree(dcls);
  return rc;
}

}  // namespace rift

using namespace rift;

extern "C" int rift_ile_point_destroy(rift_ile_point* pt) {
  if (!pt) return RIFT_ILE_OK;
  cudaFree(pt->dev);
  cudaFree(pt->q_copy);
  cudaFree(pt->uv);
  cudaFree(pt->A);
  cudaFree(pt->gm1);
  cudaFree(pt->ehat);
  cudaFree(pt->epoly);
  cudaFree(pt->erec);
  cudaFree(pt->img);
  delete pt;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_point_info(const rift_ile_point* pt, int32_t out[6]) {
  if (!pt || !out) {
    rift_ile_set_error("rift_ile_point_info: NULL argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const PointParams& P = pt->host;
  int any_null = 0;
  for (int c = 0; c < P.ncls; ++c) any_null |= P.has_null[c];
  out[0] = P.K;
  out[1] = P.M;
  out[2] = P.n;
  out[3] = P.R;
  out[4] = P.ncls;
  out[5] = any_null;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_point_create(const rift_ile_point_desc* d, rift_ile_point** out,
                                     void* stream_ptr) {
  if (!out) {
    rift_ile_set_error("rift_ile_point_create: out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int rc = validate(d);
  if (rc) return rc;
  cudaStream_t stream = (cudaStream_t)stream_ptr;
  if ((rc = ensure_anchor_table())) return rc;

  const int K = d->n_det, M = d->n_modes, D = 2 * M, n = d->q_len;
  rift_ile_point* pt = new rift_ile_point();
  std::memset(&pt->host, 0, sizeof(PointParams));
  cudaGetDevice(&pt->device);
  PointParams& P = pt->host;
  P.K = K;
  P.M = M;
  P.D = D;
  P.n = n;
  P.q_c128 = (d->q_dtype == RIFT_ILE_C128);
  P.gmst = d->gmst;
  P.d_ref = d->d_ref;
  P.dt = d->q_dt;
  P.inv_dt = 1.0 / d->q_dt;
  split_df(d->gmst, &P.gmst_hi, &P.gmst_lo);
  split_df(P.inv_dt, &P.inv_dt_hi, &P.inv_dt_lo);
  for (int k = 0; k < K; ++k) {
    P.t0[k] = d->q_t0[k];
    split_df(d->q_t0[k], &P.t0_hi[k], &P.t0_lo[k]);
    for (int c = 0; c < 3; ++c) {
      P.pos[k][c] = d->det_pos[3 * k + c];
      split_df(P.pos[k][c], &P.pos_hi[k][c], &P.pos_lo[k][c]);
    }
    for (int c = 0; c < 6; ++c) P.resp[k][c] = d->det_resp[6 * k + c];
  }
  for (int i = 0; i < M; ++i) {
    P.ell[i] = d->ell[i];
    P.em[i] = d->em[i];
    double coef[kMaxYTerms];
    int k0 = 0;
    int nt = harmonic_terms(d->ell[i], d->em[i], &k0, coef);
    P.ynt[i] = nt;
    P.yk0[i] = k0;
    for (int r = 0; r < nt; ++r) P.ycoef[i][r] = coef[r];
  }

  {  // the FP32-mixed kernels visit the modes by increasing |m| (stable)
    int j = 0;
    for (int am = 0; am <= RIFT_ILE_MAX_ELL; ++am)
      for (int i = 0; i < M; ++i)
        if (std::abs(P.em[i]) == am) P.morder[j++] = i;
  }
  split_df(std::log(d->d_ref), &P.ln_dref_hi, &P.ln_dref_lo);
  for (int k = 0; k < K; ++k) {
    for (int c = 0; c < 6; ++c) split_df(P.resp[k][c], &P.resp_hi[k][c], &P.resp_lo[k][c]);
    const double* D = P.resp[k];  // xx, xy, xz, yy, yz, zz
    const double coef[10] = {D[0], D[3], D[1], D[2], D[4], D[5], D[0] - D[3], D[1], D[2], D[4]};
    for (int c = 0; c < 10; ++c) split_df(coef[c], &P.acoef_hi[k][c], &P.acoef_lo[k][c]);
    double amax = 0.0;
    for (int c = 0; c < 10; ++c) amax = std::fmax(amax, std::fabs(coef[c]));
    int e = 0;
    std::frexp(amax, &e);  // amax < 2^e
    const double q = std::ldexp(1.0, e - 10);  // head grid 2^(E-9) with E = e - 1
    for (int c = 0; c < 10; ++c) {
      const double h = amax > 0.0 ? std::nearbyint(coef[c] / q) * q : 0.0;
      P.acoef_h[k][c] = (float)h;
      P.acoef_t[k][c] = (float)(coef[c] - h);
    }
  }
  for (int i = 0; i < M; ++i) {
    for (int r = 0; r < P.ynt[i]; ++r) split_df(P.ycoef[i][r], &P.ycoef_hi[i][r], &P.ycoef_lo[i][r]);
    double yz[RIFT_ILE_MAX_ELL + 1];
    P.ypar[i] = harmonic_zpoly(P.ell[i], P.ynt[i], P.yk0[i], P.ycoef[i], yz);
    for (int j = 0; j <= P.ell[i]; ++j) split_df(yz[j], &P.yz_hi[i][j], &P.yz_lo[i][j]);
  }

  // ---- detector classes: detectors with identical U_k and V_k.
  int ncls = 0;
  int rep[kMaxDet];
  for (int k = 0; k < K; ++k) {
    const size_t bytes = (size_t)M * M * 2 * sizeof(double);
    int c = 0;
    for (; c < ncls; ++c) {
      const int r0 = rep[c];
      if (!std::memcmp(d->U + (size_t)k * M * M * 2, d->U + (size_t)r0 * M * M * 2, bytes) &&
          !std::memcmp(d->V + (size_t)k * M * M * 2, d->V + (size_t)r0 * M * M * 2, bytes))
        break;
    }
    if (c == ncls) rep[ncls++] = k;
    P.cls_of[k] = c;
  }
  P.ncls = ncls;
  {
    int pos = 0;
    for (int c = 0; c < ncls; ++c) {
      P.cls_begin[c] = pos;
      for (int k = 0; k < K; ++k)
        if (P.cls_of[k] == c) P.det_order[pos++] = k;
    }
    P.cls_begin[ncls] = pos;
    for (int q = 0; q < K; ++q) {
      const int k = P.det_order[q], kp = q ? P.det_order[q - 1] : -1;
      P.same_pos_prev[q] = q > 0 && P.pos[k][0] == P.pos[kp][0] && P.pos[k][1] == P.pos[kp][1] &&
                           P.pos[k][2] == P.pos[kp][2];
    }
  }

  // ---- eigen-decomposition of each class's real quadratic form (descending).
  std::vector<double> Vt((size_t)ncls * D * D), lamv((size_t)ncls * D);
  for (int c = 0; c < ncls; ++c) {
    const int k = rep[c];
    std::vector<double> G((size_t)D * D);
    const double* U = d->U + (size_t)k * M * M * 2;
    const double* V = d->V + (size_t)k * M * M * 2;
    for (int i = 0; i < M; ++i) {
      for (int j = 0; j < M; ++j) {
        double ur = U[(i * M + j) * 2], ui = U[(i * M + j) * 2 + 1];
        double vr = V[(i * M + j) * 2], vi = V[(i * M + j) * 2 + 1];
        G[i * D + j] = 0.5 * (ur + vr);
        G[i * D + (M + j)] = 0.5 * (-ui - vi);
        G[(M + i) * D + j] = 0.5 * (ui - vi);
        G[(M + i) * D + (M + j)] = 0.5 * (ur - vr);
      }
    }
    for (int i = 0; i < D; ++i)  // the quadratic form only sees the symmetric part
      for (int j = i + 1; j < D; ++j) {
        double sym = 0.5 * (G[i * D + j] + G[j * D + i]);
        G[i * D + j] = G[j * D + i] = sym;
      }
    std::vector<double> lam, Vec;
    jacobi_eigen(D, G, lam, Vec);
    std::vector<int> order(D);
    for (int r = 0; r < D; ++r) order[r] = r;
    for (int a2 = 0; a2 < D; ++a2)
      for (int b2 = a2 + 1; b2 < D; ++b2)
        if (lam[order[b2]] > lam[order[a2]]) std::swap(order[a2], order[b2]);
    for (int rr = 0; rr < D; ++rr) {
      lamv[(size_t)c * D + rr] = lam[order[rr]];
      for (int a2 = 0; a2 < D; ++a2) Vt[((size_t)c * D + rr) * D + a2] = Vec[a2 * D + order[rr]];
    }
  }

  size_t qbytes = (size_t)K * n * M * (P.q_c128 ? 16 : 8);
  std::vector<double2> uvh((size_t)2 * K * M * M);
  for (size_t i = 0; i < (size_t)K * M * M; ++i) {
    uvh[i] = make_double2(d->U[2 * i], d->U[2 * i + 1]);
    uvh[(size_t)K * M * M + i] = make_double2(d->V[2 * i], d->V[2 * i + 1]);
  }
  double *dVt = nullptr, *dproj = nullptr, *dcolmax = nullptr, *dinv_s = nullptr;
  int* dcls = nullptr;
  do {
    if ((rc = dev_alloc((char**)&pt->q_copy, qbytes))) break;
    if ((rc = dev_alloc(&pt->uv, uvh.size()))) break;
    if ((rc = dev_alloc(&dVt, Vt.size()))) break;
    if ((rc = dev_alloc(&dproj, (size_t)K * n * D))) break;
    if ((rc = dev_alloc(&dcolmax, (size_t)K * D))) break;
    if ((rc = dev_alloc(&dcls, (size_t)K))) break;
    if ((rc = dev_alloc(&pt->dev, 1))) break;
    if ((rc = check_cuda(cudaMemcpyAsync(pt->q_copy, d->Q, qbytes, cudaMemcpyDeviceToDevice, stream),
                         "copy of Q")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(pt->uv, uvh.data(), uvh.size() * sizeof(double2),
                                         cudaMemcpyHostToDevice, stream), "copy of U, V")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(dVt, Vt.data(), Vt.size() * sizeof(double),
                                         cudaMemcpyHostToDevice, stream), "copy of eigenvectors")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(dcls, P.cls_of, K * sizeof(int), cudaMemcpyHostToDevice,
                                         stream), "copy of classes")))
      break;
    const long long total = (long long)K * n * D;
    const int threads = 256;
    const int blocks = (int)std::min<long long>((total + threads - 1) / threads, 148LL * 16);
    if (P.q_c128)
      project_kernel<double2><<<blocks, threads, 0, stream>>>((const double2*)pt->q_copy, dVt,
                                                              dcls, K, n, M, dproj);
    else
      project_kernel<float2><<<blocks, threads, 0, stream>>>((const float2*)pt->q_copy, dVt, dcls,
                                                             K, n, M, dproj);
    colmax_kernel<<<K * D, 256, 0, stream>>>(dproj, n, D, dcolmax);
    if ((rc = check_cuda(cudaGetLastError(), "projection kernels"))) break;
    std::vector<double> colmax((size_t)K * D);
    if ((rc = check_cuda(cudaMemcpyAsync(colmax.data(), dcolmax, colmax.size() * sizeof(double),
                                         cudaMemcpyDeviceToHost, stream), "copy of column maxima")))
      break;
    if ((rc = check_cuda(cudaStreamSynchronize(stream), "projection"))) break;

    // Rank of each class: directions with |lam| <= 1e-10 max|lam| are dropped
    // when the data of every detector of the class has no component along
    // them beyond FP64 rounding (1e-12 of its largest component); otherwise
    // all directions are kept, with s^2 floored at 1e-8 max|lam| and the
    // quadratic weight carried by gm1.
    std::vector<int> Rc(ncls);
    std::vector<double> sc((size_t)ncls * D), gm1v((size_t)ncls * D);
    int R = 1;
    for (int c = 0; c < ncls; ++c) {
      double lmax = 0.0;
      for (int r = 0; r < D; ++r) lmax = std::fmax(lmax, std::fabs(lamv[(size_t)c * D + r]));
      if (!(lmax > 0.0)) lmax = 1.0;
      int nnorm = 0;
      for (int r = 0; r < D; ++r)
        if (std::fabs(lamv[(size_t)c * D + r]) > 1e-10 * lmax) ++nnorm;
      bool null_clean = true;
      for (int k = 0; k < K; ++k) {
        if (P.cls_of[k] != c) continue;
        double big = 0.0;
        for (int r = 0; r < D; ++r) big = std::fmax(big, colmax[(size_t)k * D + r]);
        for (int r = 0; r < D; ++r)
          if (std::fabs(lamv[(size_t)c * D + r]) <= 1e-10 * lmax &&
              colmax[(size_t)k * D + r] > 1e-12 * big)
            null_clean = false;
      }
      // keep the normal directions first: they lead the descending order
      // unless some eigenvalues are negative (indefinite input)
      bool normal_first = true;
      for (int r = 0; r < D; ++r) {
        bool normal = std::fabs(lamv[(size_t)c * D + r]) > 1e-10 * lmax;
        if (r >= nnorm && normal) normal_first = false;
      }
      const bool drop = null_clean && normal_first && nnorm >= 1;
      Rc[c] = drop ? nnorm : D;
      P.has_null[c] = drop ? 0 : 1;
      for (int r = 0; r < D; ++r) {
        double lam = lamv[(size_t)c * D + r];
        double s2 = std::fabs(lam);
        if (std::fabs(lam) <= 1e-10 * lmax) s2 = std::fmax(s2, 1e-8 * lmax);
        sc[(size_t)c * D + r] = std::sqrt(s2);
        gm1v[(size_t)c * D + r] = 1.0 - lam / s2;
      }
      R = std::max(R, Rc[c]);
    }
    // rows are padded with zero directions to the width the FP32-mixed kernels
    // are compiled for (the mode-count bucket MM >= M, or 2 MM), so that their
    // per-direction loops need no bounds tests; the width is even, so two
    // table entries fit one 16-byte load.  Zero rows add exact zeros.
    {
      const int mm = M <= 2 ? 2 : M <= 4 ? 4 : M <= 6 ? 6 : M <= 8 ? 8 : M <= 10 ? 10 : M <= 12 ? 12 : 16;
      R = R <= mm ? mm : 2 * mm;
    }
    P.R = R;
    std::vector<float2> A((size_t)ncls * R * D, make_float2(0.f, 0.f));
    std::vector<float> gm1((size_t)ncls * R, 0.f);
    std::vector<double> inv_s((size_t)K * R, 0.0);
    for (int c = 0; c < ncls; ++c) {
      for (int r = 0; r < Rc[c]; ++r) {
        const double s = sc[(size_t)c * D + r];
        gm1[(size_t)c * R + r] = (float)gm1v[(size_t)c * D + r];
        for (int a2 = 0; a2 < D; ++a2) {
          double v = s * Vt[((size_t)c * D + r) * D + a2];
          float hi = (float)v;
          A[((size_t)c * R + r) * D + a2] = make_float2(hi, (float)(v - (double)hi));
        }
      }
    }
    for (int k = 0; k < K; ++k)
      for (int r = 0; r < Rc[P.cls_of[k]]; ++r)
        inv_s[(size_t)k * R + r] = 1.0 / sc[(size_t)P.cls_of[k] * D + r];
    if ((rc = dev_alloc(&pt->A, A.size()))) break;
    if ((rc = dev_alloc(&pt->gm1, gm1.size()))) break;
    if ((rc = dev_alloc(&pt->ehat, (size_t)K * (n + 2 * kEhatPad) * R))) break;
    if ((rc = check_cuda(cudaMemsetAsync(pt->ehat, 0, (size_t)K * (n + 2 * kEhatPad) * R * sizeof(float2),
                                         stream), "table padding")))
      break;
    if ((rc = dev_alloc(&pt->epoly, (size_t)K * (n + 3) * (kPolyDeg + 1)))) break;
    if ((rc = dev_alloc(&pt->erec, erec_f4(K, n, R)))) break;
    if ((rc = dev_alloc(&dinv_s, inv_s.size()))) break;
    if ((rc = check_cuda(cudaMemcpyAsync(pt->A, A.data(), A.size() * sizeof(float2),
                                         cudaMemcpyHostToDevice, stream), "copy of A")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(pt->gm1, gm1.data(), gm1.size() * sizeof(float),
                                         cudaMemcpyHostToDevice, stream), "copy of gm1")))
      break;
    if ((rc = check_cuda(cudaMemcpyAsync(dinv_s, inv_s.data(), inv_s.size() * sizeof(double),
                                         cudaMemcpyHostToDevice, stream), "copy of scales")))
      break;
    const long long tw = (long long)K * n * R;
    whiten_kernel<<<(int)std::min<long long>((tw + 255) / 256, 148LL * 16), 256, 0, stream>>>(
        dproj, dinv_s, K, n, D, R, pt->ehat);
    const long long tp = (long long)K * (n + 3);
    halfnorm_poly_kernel<<<(int)std::min<long long>((tp + 127) / 128, 148LL * 16), 128, 0, stream>>>(
        dproj, dinv_s, K, n, D, R, pt->epoly);
    const long long tc3 = (long long)K * (n + 5) * (R / 2);
    cubic_table_kernel<<<(int)std::min<long long>((tc3 + 127) / 128, 148LL * 16), 128, 0, stream>>>(
        pt->ehat, K, n, R, erec_rec_f4(R), pt->erec);
    const long long tr = (long long)K * (n + 5) * 4;
    interval_sextic_kernel<<<(int)std::min<long long>((tr + 255) / 256, 148LL * 16), 256, 0, stream>>>(
        pt->epoly, K, n, R, pt->erec);
    if ((rc = check_cuda(cudaGetLastError(), "table kernels"))) break;
    P.Q = pt->q_copy;
    P.U = pt->uv;
    P.V = pt->uv + (size_t)K * M * M;
    P.A = pt->A;
    P.gm1 = pt->gm1;
    P.ehat = pt->ehat;
    P.epoly = pt->epoly;
    P.erec = pt->erec;
    if ((rc = build_mixed_image(P, &pt->img, &P.img_f4, stream))) break;
    P.img = pt->img;
    if ((rc = check_cuda(cudaMemcpyAsync(pt->dev, &P, sizeof(PointParams), cudaMemcpyHostToDevice,
                                         stream), "copy of point parameters")))
      break;
    rc = check_cuda(cudaStreamSynchronize(stream), "rift_ile_point_create");
  } while (0);
  cudaFree(dVt);
  cudaFree(dproj);
  cudaFree(dcolmax);
  cudaFree(dinv_s);
  cudaFree(dcls);
  if (rc) {
    rift_ile_point_destroy(pt);
    return rc;
  }
  *out = pt;
  return RIFT_ILE_OK;
}
