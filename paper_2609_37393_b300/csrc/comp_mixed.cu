// FP32-mixed form of the composite-index response (Sec. III): construction of
// the whitened tables and the C entry points.  The kernels are in
// comp_mixed_impl.cuh, instantiated per mode-count bucket by lnl_mixed_m4,
// lnl_mixed_m10 and lnl_mixed_m16.cu.
//
// Whitening.  The quadratic term of detector k is 1/2 x^2 z^T G z with
// z = (Re c, Im c) over the composite index (G = 1/2 of the stored real form of
// c^+ U c + Re(c^T V c)), and the data term x z . b(t), b = (Re Q, Im Q).  With
// G = sum_r lam_r v_r v_r^T (cyclic Jacobi), the directions with
// lam_r > tol lam_max are kept (s_r = sqrt(lam_r)); the rest carry, per draw,
// sum_r (b_r zeta_r - lam_r zeta_r^2 / 2) with zeta_r = x v_r . z, which the
// mixed form leaves out: with G's spectrum falling continuously (nearly
// degenerate elementary templates) those directions hold the part of the
// interpolated data outside the bank's numerical span.  An eigenvalue below
// -max(tol, 1e-10) lam_max (an indefinite form, beyond rounding) is an error.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>

#include "comp.cuh"
#include "kernels.h"

namespace rift {

template <int MM>
cudaError_t comp_mixed_lnl(const CompMixed& C, bool bsmem, int threads, int minb,
                           const DrawsParams& dp, double* lnl_out, LseState* partials,
                           unsigned long long* oob, int* blocks, cudaStream_t st);
template <int MM>
cudaError_t comp_mixed_grad(const CompMixed& C, bool bsmem, int threads, const DrawsParams& dp,
                            double* lnl_out, double* grad_out, cudaStream_t st);
template <int MM>
int comp_mixed_regs(bool grad, int minb);

namespace {

int mm_bucket(int M) { return M <= 4 ? 4 : (M <= 10 ? 10 : 16); }

cudaError_t launch_comp_mixed(const rift_ile_comp* cp, const DrawsParams& dp, double* lnl_out,
                              LseState* partials, unsigned long long* oob, int* blocks,
                              cudaStream_t st) {
  const CompMixed& C = cp->mixed;
  const bool bs = cp->mixed_bsmem != 0;
  const int th = cp->mixed_threads, mb = cp->mixed_minb;
  switch (mm_bucket(C.M)) {
    case 4: return comp_mixed_lnl<4>(C, bs, th, mb, dp, lnl_out, partials, oob, blocks, st);
    case 10: return comp_mixed_lnl<10>(C, bs, th, mb, dp, lnl_out, partials, oob, blocks, st);
    default: return comp_mixed_lnl<16>(C, bs, th, mb, dp, lnl_out, partials, oob, blocks, st);
  }
}

cudaError_t launch_comp_mixed_grad(const rift_ile_comp* cp, const DrawsParams& dp,
                                   double* lnl_out, double* grad_out, cudaStream_t st) {
  const CompMixed& C = cp->mixed;
  const bool bs = cp->grad_bsmem != 0;
  const int th = cp->grad_threads;
  switch (mm_bucket(C.M)) {
    case 4: return comp_mixed_grad<4>(C, bs, th, dp, lnl_out, grad_out, st);
    case 10: return comp_mixed_grad<10>(C, bs, th, dp, lnl_out, grad_out, st);
    default: return comp_mixed_grad<16>(C, bs, th, dp, lnl_out, grad_out, st);
  }
}

// Head constant of a value bound m (see head_constant in lnl_mixed_impl.cuh):
// 1.5 2^(E + 15) with 2^E <= m < 2^(E + 1), so that (v + C) - C rounds |v| <= m
// to a multiple of 2^(E - 8).
float head_constant_host(double m) {
  if (!(m > 0.0)) return std::ldexp(1.5f, -100);
  int e = 0;
  std::frexp(m, &e);  // m = f 2^e, f in [0.5, 1): E = e - 1
  return (float)std::ldexp(1.5, e - 1 + 15);
}

void free_mixed(rift_ile_comp* cp) {
  cudaFree(cp->Bs);
  cudaFree(cp->agrid);
  cudaFree(cp->ehat);
  cudaFree(cp->epoly);
  cudaFree(cp->ecub);
  cp->Bs = nullptr;
  cp->agrid = nullptr;
  cp->ehat = nullptr;
  cp->epoly = nullptr;
  cp->ecub = nullptr;
  cp->mixed_built = 0;
}

// sigma_a = the smallest power of two >= max |C~^k_a| over 24 x 13 x 4 sky
// positions (ra, dec, psi) and the detectors, at x = 1 and t_c = 0 (1 for an
// index that vanishes there).  Only the balance of the magnitudes matters:
// the kernel's head grids follow the actual values.
int coefficient_scales(const rift_ile_comp* cp, int na, double* sigma, cudaStream_t st) {
  const int nra = 24, ndec = 13, npsi = 4, ns = nra * ndec * npsi, K = cp->host.K;
  std::vector<double> h(7 * (size_t)ns, 0.0);
  for (int i = 0, q = 0; i < nra; ++i)
    for (int j = 0; j < ndec; ++j)
      for (int l = 0; l < npsi; ++l, ++q) {
        h[q] = 2.0 * M_PI * (i + 0.5) / nra;                    // ra
        h[(size_t)ns + q] = M_PI * (j / (ndec - 1.0) - 0.5);     // dec
        h[2 * (size_t)ns + q] = M_PI * (l + 0.25) / npsi;        // psi
      }
  double* dbuf = nullptr;
  double2* dcoef = nullptr;
  cudaError_t e = cudaMalloc((void**)&dbuf, h.size() * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&dcoef, (size_t)ns * K * na * sizeof(double2));
  std::vector<double2> coef((size_t)ns * K * na);
  int rc = RIFT_ILE_OK;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dbuf, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    rift_ile_draws d;
    std::memset(&d, 0, sizeof(d));
    d.n = ns;
    d.dtype = RIFT_ILE_F64;
    d.ra = dbuf;
    d.dec = dbuf + ns;
    d.psi = dbuf + 2 * (size_t)ns;
    d.incl = d.phase = d.lnD = d.t = dbuf + 3 * (size_t)ns;  // zeros
    rc = rift_ile_comp_coeffs(cp, &d, (double*)dcoef, st);
    if (!rc)
      e = cudaMemcpyAsync(coef.data(), dcoef, coef.size() * sizeof(double2), cudaMemcpyDeviceToHost, st);
    if (!rc && e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  cudaFree(dbuf);
  cudaFree(dcoef);
  if (rc) return rc;
  if (e != cudaSuccess) return check_cuda(e, "rift_ile_comp_mixed_build coefficient scales");
  for (int a = 0; a < na; ++a) {
    double m = 0.0;
    for (size_t q = 0; q < (size_t)ns * K; ++q)
      m = std::fmax(m, std::hypot(coef[q * na + a].x, coef[q * na + a].y));
    int ex = 0;
    std::frexp(m, &ex);  // m < 2^ex
    sigma[a] = m > 0.0 && std::isfinite(m) ? std::ldexp(1.0, ex) : 1.0;
  }
  return RIFT_ILE_OK;
}

int mixed_args(const rift_ile_comp* cp, const rift_ile_draws* draws) {
  if (!cp) {
    rift_ile_set_error("composite point is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!cp->mixed_built) {
    rift_ile_set_error("the FP32-mixed form of this composite point is not built "
                       "(rift_ile_comp_mixed_build)");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  return validate_draws(draws);
}

}  // namespace
}  // namespace rift

using namespace rift;

extern "C" int rift_ile_comp_mixed_build(rift_ile_comp* cp, double tol, void* stream) {
  if (!cp) {
    rift_ile_set_error("rift_ile_comp_mixed_build: composite point is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!(tol > 0.0 && tol < 1.0)) {
    rift_ile_set_error("rift_ile_comp_mixed_build: tol=%g must lie in (0, 1)", tol);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int rc = ensure_anchor_table();
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  free_mixed(cp);
  const CompParams& P = cp->host;
  const int K = P.K, M = P.M, na = P.na, A = P.A, n = P.n, ncls = P.ncls, D = 2 * A;
  const int MMb = M <= 4 ? 4 : (M <= 10 ? 10 : 16), JP = MMb / 2;

  // ---- eigen-decomposition of each class's form, descending
  std::vector<double> Vt((size_t)ncls * D * D, 0.0), sc((size_t)ncls * D, 0.0);
  int Rc[kMaxDet] = {0};
  int R = 2;
  for (int c = 0; c < ncls; ++c) {
    std::vector<double> G(cp->Gfull.begin() + (size_t)c * D * D,
                          cp->Gfull.begin() + (size_t)(c + 1) * D * D);
    for (double& g : G) g *= 0.5;
    std::vector<double> lam, Vec;
    jacobi_eigen(D, G, lam, Vec);
    std::vector<int> order(D);
    for (int r = 0; r < D; ++r) order[r] = r;
    for (int a = 0; a < D; ++a)
      for (int b = a + 1; b < D; ++b)
        if (lam[order[b]] > lam[order[a]]) std::swap(order[a], order[b]);
    const double lmax = lam[order[0]];
    if (!(lmax > 0.0)) {
      rift_ile_set_error("rift_ile_comp_mixed_build: the quadratic form of class %d is not "
                         "positive (largest eigenvalue %g)", c, lmax);
      return RIFT_ILE_ERR_UNSUPPORTED;
    }
    if (lam[order[D - 1]] < -std::fmax(tol, 1e-10) * lmax) {
      rift_ile_set_error("rift_ile_comp_mixed_build: the quadratic form of class %d is "
                         "indefinite (eigenvalue %g against %g)", c, lam[order[D - 1]], lmax);
      return RIFT_ILE_ERR_UNSUPPORTED;
    }
    int kept = 0;
    for (int r = 0; r < D; ++r) {
      const double l = lam[order[r]];
      for (int a = 0; a < D; ++a) Vt[((size_t)c * D + r) * D + a] = Vec[(size_t)a * D + order[r]];
      if (l > tol * lmax) {
        sc[(size_t)c * D + r] = std::sqrt(l);
        ++kept;
      }
    }
    Rc[c] = kept;
    R = std::max(R, (kept + 1) & ~1);
  }
  for (int c = 0; c < ncls; ++c) cp->mixed_R[c] = Rc[c];

  // ---- the scales sigma_a: the largest |C~^k_a| (at x = 1) over a grid of sky
  // positions and polarisations and every detector, by the FP64 coefficient
  // kernel, rounded up to a power of two
  double sigma[kMaxRespIdx];
  if ((rc = coefficient_scales(cp, na, sigma, st))) return rc;

  // ---- the split whitening, in the kernel's layout [c][a][r][jp][3] with the
  // modes in visiting order (increasing |m|), each index's columns times
  // sigma_a, and the head constants of a1, a2
  int morder[kMaxModes];
  {
    int j = 0;
    for (int am = 0; am <= RIFT_ILE_MAX_ELL; ++am)
      for (int i = 0; i < M; ++i)
        if (std::abs(cp->host_em[i]) == am) morder[j++] = i;
  }
  std::vector<float4> Bs((size_t)ncls * na * R * JP * 3, make_float4(0.f, 0.f, 0.f, 0.f));
  std::vector<float> ag((size_t)ncls * R, 0.f);
  for (int c = 0; c < ncls; ++c) {
    for (int r = 0; r < Rc[c]; ++r) {
      const double s = sc[(size_t)c * D + r];
      const double* v = Vt.data() + ((size_t)c * D + r) * D;
      double bound = 0.0;
      for (int a = 0; a < na; ++a) {
        double th[kMaxModes] = {0}, tt[kMaxModes] = {0}, bh[kMaxModes] = {0}, bt[kMaxModes] = {0};
        double amax = 0.0, sum = 0.0;
        for (int j = 0; j < M; ++j) {
          const int i = morder[j];
          const double t = sigma[a] * s * v[a * M + i], b = sigma[a] * s * v[A + a * M + i];
          amax = std::fmax(amax, std::fmax(std::fabs(t), std::fabs(b)));
          const int l = cp->host_ell[i];
          sum += (std::fabs(t) + std::fabs(b)) * std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI)) * 1.01;
        }
        bound = std::fmax(bound, sum);
        int e = 0;
        std::frexp(amax, &e);
        const double q = std::ldexp(1.0, e - 10);  // heads on 2^(E - 9), E = e - 1
        for (int j = 0; j < M; ++j) {
          const int i = morder[j];
          const double t = sigma[a] * s * v[a * M + i], b = sigma[a] * s * v[A + a * M + i];
          th[j] = amax > 0.0 ? std::nearbyint(t / q) * q : 0.0;
          bh[j] = amax > 0.0 ? std::nearbyint(b / q) * q : 0.0;
          tt[j] = t - th[j];
          bt[j] = b - bh[j];
        }
        for (int jp = 0; jp < JP; ++jp) {
          const int j0 = 2 * jp, j1 = 2 * jp + 1;
          float4* o = Bs.data() + ((((size_t)c * na + a) * R + r) * JP + jp) * 3;
          o[0] = make_float4((float)th[j0], (float)th[j1], (float)bh[j0], (float)bh[j1]);
          o[1] = make_float4((float)-th[j0], (float)-th[j1], (float)tt[j0], (float)tt[j1]);
          o[2] = make_float4((float)bt[j0], (float)bt[j1], (float)-tt[j0], (float)-tt[j1]);
        }
      }
      ag[(size_t)c * R + r] = head_constant_host(bound);
    }
    for (int r = Rc[c]; r < R; ++r) ag[(size_t)c * R + r] = head_constant_host(0.0);
  }
  std::vector<double> inv_s((size_t)K * R, 0.0);
  for (int k = 0; k < K; ++k)
    for (int r = 0; r < Rc[P.cls_of[k]]; ++r)
      inv_s[(size_t)k * R + r] = 1.0 / sc[(size_t)P.cls_of[k] * D + r];

  // ---- the kernel's constants
  CompMixed& C = cp->mixed;
  std::memset(&C, 0, sizeof(C));
  C.K = K;
  C.M = M;
  C.na = na;
  C.A = A;
  C.n = n;
  C.R = R;
  C.ncls = ncls;
  C.kind = P.kind;
  C.p_max = P.p_max;
  C.JP = JP;
  {
    int pos = 0;
    for (int c = 0; c < ncls; ++c) {
      C.cls_begin[c] = pos;
      for (int k = 0; k < K; ++k)
        if (P.cls_of[k] == c) C.det_order[pos++] = k;
    }
    C.cls_begin[ncls] = pos;
  }
  split_df(P.gmst, &C.gmst_hi, &C.gmst_lo);
  split_df(P.inv_dt, &C.inv_dt_hi, &C.inv_dt_lo);
  split_df(std::log(P.d_ref), &C.ln_dref_hi, &C.ln_dref_lo);
  split_df(P.omega, &C.omega_hi, &C.omega_lo);
  for (int k = 0; k < K; ++k) {
    float h[4], l[4];
    for (int q = 0; q < 3; ++q) split_df(P.pos[k][q], &h[q], &l[q]);
    split_df(P.t0[k], &h[3], &l[3]);
    C.pos_hi[k] = make_float4(h[0], h[1], h[2], h[3]);
    C.pos_lo[k] = make_float4(l[0], l[1], l[2], l[3]);
    double v[6];
    if (P.kind == RIFT_ILE_RESP_ROTATION) {
      const double* Dk = P.resp[k];  // xx, xy, xz, yy, yz, zz
      v[0] = Dk[3] - Dk[0];
      v[1] = 2.0 * Dk[1];
      v[2] = 2.0 * Dk[2];
      v[3] = 2.0 * Dk[4];
      v[4] = Dk[0] + Dk[3];
      v[5] = Dk[5];
    } else {
      for (int q = 0; q < 3; ++q) {
        v[q] = P.armx[k][q];
        v[3 + q] = P.army[k][q];
      }
    }
    for (int q = 0; q < 6; ++q) {
      float hi, lo;
      split_df(v[q], &hi, &lo);
      C.rc[k][q] = make_float2(hi, lo);
    }
  }
  for (int j = 0; j < M; ++j) {
    const int i = morder[j];
    const int l = cp->host_ell[i];
    double coef[kMaxYTerms];
    int k0 = 0;
    const int nt = harmonic_coefficients(l, cp->host_em[i], &k0, coef);
    double yz[RIFT_ILE_MAX_ELL + 1];
    const int par = harmonic_zpoly(l, nt, k0, coef, yz);
    C.mode[j] = make_int4(i, cp->host_em[i], l, par);
    for (int q = 0; q <= l; ++q) {
      float hi, lo;
      split_df(yz[q], &hi, &lo);
      C.yz[j][q] = make_float2(hi, lo);
    }
  }
  for (int a = 0; a < na; ++a) C.inv_sigma[a] = (float)(1.0 / sigma[a]);
  {
    double f = 1.0;
    for (int p = 0; p <= RIFT_ILE_MAX_ROT_PMAX; ++p) {
      if (p > 0) f *= p;
      C.inv_fact[p] = (float)(1.0 / f);
    }
  }

  // ---- device tables
  cudaError_t e = cudaMalloc((void**)&cp->Bs, Bs.size() * sizeof(float4));
  if (e == cudaSuccess) e = cudaMalloc((void**)&cp->agrid, ag.size() * sizeof(float));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&cp->ehat, (size_t)K * (n + 2 * kEhatPad) * R * sizeof(float2));
  if (e == cudaSuccess)
    e = cudaMalloc((void**)&cp->epoly, (size_t)K * (n + 3) * (kPolyDeg + 1) * sizeof(float2));
  if (e == cudaSuccess) e = cudaMalloc((void**)&cp->ecub, ecub_f4(K, n, R) * sizeof(float4));
  if (e != cudaSuccess) {
    free_mixed(cp);
    rift_ile_set_error("rift_ile_comp_mixed_build: allocation failed: %s", cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  e = cudaMemcpyAsync(cp->Bs, Bs.data(), Bs.size() * sizeof(float4), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cp->agrid, ag.data(), ag.size() * sizeof(float), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) {
    free_mixed(cp);
    return check_cuda(e, "rift_ile_comp_mixed_build upload");
  }
  if ((rc = whitened_tables(cp->q, 1, K, n, A, ncls, P.cls_of, Vt.data(), inv_s.data(), R, cp->ehat,
                            cp->epoly, cp->ecub, st))) {
    free_mixed(cp);
    return rc;
  }
  C.Bs = cp->Bs;
  C.agrid = cp->agrid;
  C.ehat = cp->ehat;
  C.epoly = cp->epoly;
  C.ecub = cp->ecub;

  // ---- launch shapes (block size, split whitening in shared memory or read
  // through L1)
  int optin = 0;
  if ((rc = check_cuda(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                                              cp->device), "device attribute"))) {
    free_mixed(cp);
    return rc;
  }
  cp->mixed_threads = cp->grad_threads = 0;
  const size_t static_smem = 2048;  // the LSE kernels' static shared memory, with margin
  const int shapes[6][2] = {{128, 1}, {128, 0}, {64, 1}, {64, 0}, {32, 1}, {32, 0}};
  // for the lnL kernels and for the adjoint, the shape with the most resident
  // warps per SM given the kernel's registers and shared memory (ties: the
  // whitening staged, then the larger block; for the lnL kernels also the
  // variant sized for two or three blocks per SM, ties to two, whose larger
  // register budget costs fewer instructions).  Without a fitting shape for
  // the adjoint only the gradient entry point reports UNSUPPORTED.
  {
    int smem_sm = 0;
    if ((rc = check_cuda(cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                                cp->device), "device attribute"))) {
      free_mixed(cp);
      return rc;
    }
    for (int grad = 0; grad < 2; ++grad) {
      int best = 0;
      for (int minb = 2; minb <= (grad ? 2 : 3); ++minb) {
        int regs = 0;
        switch (mm_bucket(C.M)) {
          case 4: regs = comp_mixed_regs<4>(grad != 0, minb); break;
          case 10: regs = comp_mixed_regs<10>(grad != 0, minb); break;
          default: regs = comp_mixed_regs<16>(grad != 0, minb); break;
        }
        if (regs <= 0) {
          if (minb > 2) continue;  // no such variant for this bucket
          regs = 255;
        }
        const int regs_r = (regs + 7) & ~7;  // allocation granularity
        for (const auto& sh : shapes) {
          const size_t sm = comp_mixed_smem(C, sh[1] != 0, sh[0], grad != 0) + static_smem;
          if (sm > (size_t)optin) continue;
          const int by_smem = (int)((size_t)smem_sm / (sm + 1024));  // 1 KB reserved per block
          const int by_regs = 65536 / (regs_r * sh[0]);
          const int warps = std::min(by_smem, by_regs) * (sh[0] / 32);
          if (warps > best) {
            best = warps;
            if (grad) {
              cp->grad_threads = sh[0];
              cp->grad_bsmem = sh[1];
            } else {
              cp->mixed_threads = sh[0];
              cp->mixed_bsmem = sh[1];
              cp->mixed_minb = minb;
            }
          }
        }
      }
    }
  }
  if (!cp->mixed_threads) {
    free_mixed(cp);
    rift_ile_set_error("rift_ile_comp_mixed_build: %d detectors x %d response indices need more "
                       "shared memory per thread than the device has", K, na);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  cp->mixed_tol = tol;
  cp->mixed_built = 1;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_comp_mixed_info(const rift_ile_comp* cp, int32_t out[4]) {
  if (!cp || !out) {
    rift_ile_set_error("rift_ile_comp_mixed_info: NULL argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!cp->mixed_built) {
    out[0] = out[1] = out[2] = out[3] = 0;
    return RIFT_ILE_OK;
  }
  int kept = 0;
  for (int c = 0; c < cp->mixed.ncls; ++c) kept = std::max(kept, cp->mixed_R[c]);
  out[0] = cp->mixed.R;
  out[1] = kept;
  out[2] = cp->mixed.ncls;
  out[3] = cp->mixed_threads;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_comp_lnL_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                       double* lnL_out, void* stream) {
  int rc = mixed_args(cp, draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!lnL_out) {
    rift_ile_set_error("rift_ile_comp_lnL_mixed: lnL_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int blocks = 0;
  return check_cuda(launch_comp_mixed(cp, draws_params(draws), lnL_out, nullptr, nullptr, &blocks,
                                      (cudaStream_t)stream),
                    "rift_ile_comp_lnL_mixed launch");
}

extern "C" int rift_ile_comp_lnL_grad_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                            double* lnL_out, double* grad_out, void* stream) {
  int rc = mixed_args(cp, draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!grad_out) {
    rift_ile_set_error("rift_ile_comp_lnL_grad_mixed: grad_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!cp->grad_threads) {
    rift_ile_set_error("rift_ile_comp_lnL_grad_mixed: %d detectors x %d response indices need "
                       "more shared memory per thread than the device has",
                       cp->mixed.K, cp->mixed.na);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  return check_cuda(launch_comp_mixed_grad(cp, draws_params(draws), lnL_out, grad_out,
                                           (cudaStream_t)stream),
                    "rift_ile_comp_lnL_grad_mixed launch");
}

extern "C" int rift_ile_comp_lnZ_state_mixed_async(const rift_ile_comp* cp,
                                                   const rift_ile_draws* draws,
                                                   rift_ile_lse* state_out, void* stream) {
  int rc = mixed_args(cp, draws);
  if (rc) return rc;
  if (!state_out) {
    rift_ile_set_error("rift_ile_comp_lnZ_state_mixed_async: state_out is NULL");
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
  if ((rc = check_cuda(launch_comp_mixed(cp, draws_params(draws), nullptr, partials, nullptr,
                                         &blocks, st),
                       "composite mixed lnZ kernel launch")))
    return rc;
  return check_cuda(launch_lse_combine(partials, blocks, (double)draws->n, out, st),
                    "lnZ combine launch");
}

extern "C" int rift_ile_comp_lnZ_state_mixed(const rift_ile_comp* cp, const rift_ile_draws* draws,
                                             rift_ile_lse* state, void* stream) {
  int rc = mixed_args(cp, draws);
  if (rc) return rc;
  if (!state) {
    rift_ile_set_error("rift_ile_comp_lnZ_state_mixed: state is NULL");
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
  if ((rc = check_cuda(launch_comp_mixed(cp, draws_params(draws), nullptr, partials, doob, &blocks,
                                         st),
                       "composite mixed lnZ kernel launch")))
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
  if ((rc = check_cuda(cudaStreamSynchronize(st), "rift_ile_comp_lnZ_state_mixed"))) return rc;
  set_last_oob((long long)o);
  *state = rift_ile_lse{h.m, h.s, h.s2, h.n};
  return RIFT_ILE_OK;
}
