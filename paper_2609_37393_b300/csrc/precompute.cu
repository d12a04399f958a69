// GPU precompute of Q, U, V (eq. QUV) for one intrinsic point, FP64.
//
// Q: the weighted cross spectrum X_{k,i}(f) = w_k(f) conj(h_i(f)) d_k(f)
// e^{2 pi i f t0_k} is scattered into a zero-padded FFT frame of length
// nfft = 1/(df dt) at bin (f/df) mod nfft (the pregrid of eq. q-time-pregrid),
// one frame per (detector, mode); one batched inverse Z2Z transform (cuFFT,
// unnormalised, e^{+2 pi i b j / nfft}) turns bin b = f/df into
// e^{2 pi i f j dt}, so output j is Q_{k,i}(t0_k + j dt) exactly as the sum of
// eq. QUV; a gather kernel transposes the first q_len samples to [K][n][M].
// U, V: one block per (k, i <= j) (U Hermitian, V symmetric), each thread a
// fixed strided subset of the frequencies, a fixed shared-memory tree:
// reproducible bit for bit.
#include <cuda_runtime.h>
#include <cufft.h>
#include <math_constants.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/rift_ile_precompute.h"
#include "../../include/rift_ile_response.h"
#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {
namespace {

constexpr int kUvThreads = 256;

__device__ __forceinline__ double2 cmul_pc(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

struct Times {
  double t0[kMaxDet];
};

__global__ void q_scatter_kernel(const double2* __restrict__ hlm, const double2* __restrict__ dk,
                                 const double* __restrict__ wgt, Times T, int K, int M, int nf,
                                 double df, long long nfft, double2* __restrict__ Y) {
  const long long total = (long long)K * M * nf;
  const long long nh = (nf - 1) / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % nf);
    const long long ki = idx / nf;
    const int i = (int)(ki % M);
    const int k = (int)(ki / M);
    const double w = wgt[(long long)k * nf + q];
    if (w == 0.0) continue;  // the frame is zeroed; out-of-band bins stay 0
    const long long qs = q - nh;
    const double f = (double)qs * df;
    double s, c;
    sincospi(2.0 * f * T.t0[k], &s, &c);
    const double2 h = hlm[(long long)i * nf + q];
    const double2 d = dk[(long long)k * nf + q];
    // conj(h) d
    const double xr = h.x * d.x + h.y * d.y, xi = h.x * d.y - h.y * d.x;
    const long long bin = (qs % nfft + nfft) % nfft;
    Y[ki * nfft + bin] = make_double2(w * (xr * c - xi * s), w * (xr * s + xi * c));
  }
}

__device__ __forceinline__ void store_q(double2* p, double2 v) { *p = v; }
__device__ __forceinline__ void store_q(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}

template <typename T>
__global__ void q_gather_kernel(const double2* __restrict__ Y, int K, int M, int n, long long nfft,
                                T* __restrict__ Q) {
  const long long total = (long long)K * n * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % M);
    const long long kj = idx / M;
    const int j = (int)(kj % n);
    const int k = (int)(kj / n);
    const double2 v = Y[((long long)k * M + i) * nfft + j];
    store_q(Q + idx, v);
  }
}

__global__ void __launch_bounds__(kUvThreads) uv_kernel(const double2* __restrict__ hlm,
                                                        const double* __restrict__ wgt, int M,
                                                        int nf, double2* __restrict__ U,
                                                        double2* __restrict__ V) {
  // one block per (k, i <= j): U is Hermitian and V symmetric by construction
  const int npair = M * (M + 1) / 2;
  const int k = blockIdx.x / npair;
  int r = blockIdx.x % npair, i = 0;
  while (r >= M - i) {
    r -= M - i;
    ++i;
  }
  const int j = i + r;
  const double2* hi = hlm + (long long)i * nf;
  const double2* hj = hlm + (long long)j * nf;
  const double* w = wgt + (long long)k * nf;
  double ur = 0.0, ui = 0.0, vr = 0.0, vi = 0.0;
  for (int q = threadIdx.x; q < nf; q += kUvThreads) {
    const double wq = w[q];
    const double2 a = hi[q], b = hj[q], m = hi[nf - 1 - q];
    // conj(a) b and m b, m = h_i(-f)
    ur = fma(wq, a.x * b.x + a.y * b.y, ur);
    ui = fma(wq, a.x * b.y - a.y * b.x, ui);
    vr = fma(wq, m.x * b.x - m.y * b.y, vr);
    vi = fma(wq, m.x * b.y + m.y * b.x, vi);
  }
  __shared__ double red[4][kUvThreads];
  red[0][threadIdx.x] = ur;
  red[1][threadIdx.x] = ui;
  red[2][threadIdx.x] = vr;
  red[3][threadIdx.x] = vi;
  __syncthreads();
  for (int s = kUvThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int c = 0; c < 4; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const long long o = ((long long)k * M + i) * M + j, ot = ((long long)k * M + j) * M + i;
    if (U) {
      U[o] = make_double2(red[0][0], red[1][0]);
      U[ot] = make_double2(red[0][0], -red[1][0]);
    }
    if (V) {
      V[o] = make_double2(red[2][0], red[3][0]);
      V[ot] = V[o];
    }
  }
}

struct Plan {
  int device;
  long long nfft;
  int batch;
  cufftHandle h;
};
std::mutex g_plan_mu;
std::vector<Plan> g_plans;

int get_plan(long long nfft, int batch, cufftHandle* out) {
  int dev = 0;
  cudaGetDevice(&dev);
  for (const Plan& p : g_plans)
    if (p.device == dev && p.nfft == nfft && p.batch == batch) {
      *out = p.h;
      return RIFT_ILE_OK;
    }
  cufftHandle h;
  int n = (int)nfft;
  const cufftResult r = cufftPlanMany(&h, 1, &n, nullptr, 1, n, nullptr, 1, n, CUFFT_Z2Z, batch);
  if (r != CUFFT_SUCCESS) {
    rift_ile_set_error("cufftPlanMany(nfft=%lld, batch=%d) failed: cufftResult %d", nfft, batch,
                       (int)r);
    return RIFT_ILE_ERR_CUDA;
  }
  g_plans.push_back(Plan{dev, nfft, batch, h});
  *out = h;
  return RIFT_ILE_OK;
}

int validate(const rift_ile_precompute_desc* d, long long* nfft) {
  if (!d) {
    rift_ile_set_error("precompute description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->n_det < 1 || d->n_det > RIFT_ILE_MAX_DET || d->n_modes < 1 ||
      d->n_modes > RIFT_ILE_MAX_MODES) {
    rift_ile_set_error("n_det=%d or n_modes=%d out of range", d->n_det, d->n_modes);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  if (d->nf < 1 || (d->nf % 2) == 0) {
    rift_ile_set_error("nf=%d: the two-sided grid needs an odd, positive length", d->nf);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (!d->hlm || !d->dk || !d->wgt || !d->q_t0) {
    rift_ile_set_error("a required array of the precompute description is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (!(d->df > 0.0) || !std::isfinite(d->df) || !(d->q_dt > 0.0) || !std::isfinite(d->q_dt)) {
    rift_ile_set_error("df and q_dt must be finite and positive");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->q_dtype != RIFT_ILE_C64 && d->q_dtype != RIFT_ILE_C128) {
    rift_ile_set_error("q_dtype=%d is neither RIFT_ILE_C64 nor RIFT_ILE_C128", d->q_dtype);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const double r = 1.0 / (d->df * d->q_dt);
  const long long n = std::llround(r);
  if (!(std::fabs(n * d->df * d->q_dt - 1.0) < 1e-9) || n < d->nf || n < d->q_len || d->q_len < 1 ||
      n > (1LL << 28)) {
    rift_ile_set_error("1/(df q_dt) = %.9g must be an integer >= nf=%d and >= q_len=%d", r, d->nf,
                       d->q_len);
    return RIFT_ILE_ERR_SHAPE;
  }
  for (int k = 0; k < d->n_det; ++k)
    if (!std::isfinite(d->q_t0[k])) {
      rift_ile_set_error("q_t0[%d] is not finite", k);
      return RIFT_ILE_ERR_INVALID_ARG;
    }
  *nfft = n;
  return RIFT_ILE_OK;
}

int blocks_for(long long total) {
  const long long b = (total + 255) / 256;
  const long long cap = (long long)device_sms() * 16;
  return (int)(b < cap ? (b > 0 ? b : 1) : cap);
}

}  // namespace

int fft_z2z_inplace(double2* data, long long nfft, int batch, int direction, cudaStream_t st) {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  cufftHandle plan;
  int rc = get_plan(nfft, batch, &plan);
  if (rc) return rc;
  cufftResult r = cufftSetStream(plan, st);
  if (r == CUFFT_SUCCESS)
    r = cufftExecZ2Z(plan, (cufftDoubleComplex*)data, (cufftDoubleComplex*)data,
                     direction < 0 ? CUFFT_FORWARD : CUFFT_INVERSE);
  if (r != CUFFT_SUCCESS) {
    rift_ile_set_error("cuFFT transform of length %lld (batch %d) failed: cufftResult %d", nfft,
                       batch, (int)r);
    return RIFT_ILE_ERR_CUDA;
  }
  return RIFT_ILE_OK;
}

void release_fft_plans() {
  std::lock_guard<std::mutex> lock(g_plan_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (const Plan& p : g_plans) {
    cudaSetDevice(p.device);
    cufftDestroy(p.h);
  }
  g_plans.clear();
  cudaSetDevice(cur);
}

}  // namespace rift

using namespace rift;

extern "C" int rift_ile_precompute(const rift_ile_precompute_desc* d, void* Q_out, double* U_out,
                                   double* V_out, void* stream) {
  long long nfft = 0;
  int rc = validate(d, &nfft);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const int K = d->n_det, M = d->n_modes, nf = d->nf;
  if (U_out || V_out) {
    uv_kernel<<<K * M * (M + 1) / 2, kUvThreads, 0, st>>>((const double2*)d->hlm, d->wgt, M, nf,
                                                 (double2*)U_out, (double2*)V_out);
    if ((rc = check_cuda(cudaGetLastError(), "uv_kernel launch"))) return rc;
  }
  if (!Q_out) return RIFT_ILE_OK;
  const int batch = K * M;
  const size_t bytes = (size_t)batch * nfft * sizeof(double2);
  double2* Y = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&Y, bytes, st);
  if (e != cudaSuccess) {
    rift_ile_set_error("precompute work buffer of %zu bytes: %s", bytes, cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  Times T{};
  for (int k = 0; k < K; ++k) T.t0[k] = d->q_t0[k];
  e = cudaMemsetAsync(Y, 0, bytes, st);
  if (e == cudaSuccess) {
    q_scatter_kernel<<<blocks_for((long long)batch * nf), 256, 0, st>>>(
        (const double2*)d->hlm, (const double2*)d->dk, d->wgt, T, K, M, nf, d->df, nfft, Y);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    cufftHandle plan;
    rc = get_plan(nfft, batch, &plan);
    if (!rc) {
      cufftResult r = cufftSetStream(plan, st);
      if (r == CUFFT_SUCCESS) r = cufftExecZ2Z(plan, (cufftDoubleComplex*)Y, (cufftDoubleComplex*)Y,
                                               CUFFT_INVERSE);
      if (r != CUFFT_SUCCESS) {
        rift_ile_set_error("cuFFT transform failed: cufftResult %d", (int)r);
        rc = RIFT_ILE_ERR_CUDA;
      }
    }
  }
  if (e == cudaSuccess && !rc) {
    const long long total = (long long)K * d->q_len * M;
    if (d->q_dtype == RIFT_ILE_C128)
      q_gather_kernel<double2><<<blocks_for(total), 256, 0, st>>>(Y, K, M, d->q_len, nfft,
                                                                  (double2*)Q_out);
    else
      q_gather_kernel<float2><<<blocks_for(total), 256, 0, st>>>(Y, K, M, d->q_len, nfft,
                                                                 (float2*)Q_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(Y, st);
  if (rc) return rc;
  return check_cuda(e, "rift_ile_precompute");
}

// ----------------------------------------------- widened rotation bank

namespace rift {
namespace {

// X[(p M + i)][(q - nh) mod nf] = h_i(f_q) (2 pi i f_q)^p
__global__ void bank_weight_kernel(const double2* __restrict__ hlm, int M, int nf, double df,
                                   int np, double2* __restrict__ X) {
  const long long total = (long long)np * M * nf;
  const int nh = (nf - 1) / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % nf);
    const long long row = idx / nf;
    const int i = (int)(row % M), p = (int)(row / M);
    const double w = 2.0 * CUDART_PI * (double)(q - nh) * df;  // 2 pi f
    double2 v = hlm[(long long)i * nf + q];
    for (int k = 0; k < p; ++k) v = make_double2(-w * v.y, w * v.x);  // times i 2 pi f
    const int qs = ((q - nh) % nf + nf) % nf;
    X[row * nf + qs] = v;
  }
}

// Z[(a M + i)][j] = x[(p(a) M + i)][j] e^{i n(a) Omega t_j}, t_j centred
__global__ void bank_modulate_kernel(const double2* __restrict__ x, int M, int nf, double df,
                                     double omega, int p_max, double2* __restrict__ Z) {
  const int na = (p_max + 1) * (p_max + 5);
  const long long total = (long long)na * M * nf;
  const int nh = (nf - 1) / 2;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(idx % nf);
    const long long row = idx / nf;
    const int i = (int)(row % M), a = (int)(row / M);
    int p = 0, off = 0;
    while (off + 5 + 2 * p <= a) {
      off += 5 + 2 * p;
      ++p;
    }
    const int n = a - off - (2 + p);
    const double t = (double)(j <= nh ? j : j - nf) / ((double)nf * df);
    double s, c;
    sincos((double)n * omega * t, &s, &c);
    const double2 v = x[((long long)p * M + i) * nf + j];
    Z[idx] = make_double2(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// bank[(row)][q] = Z[row][(q - nh) mod nf] / nf
__global__ void bank_gather_kernel(const double2* __restrict__ Z, long long rows, int nf,
                                   double2* __restrict__ bank) {
  const long long total = rows * nf;
  const int nh = (nf - 1) / 2;
  const double inv = 1.0 / (double)nf;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(idx % nf);
    const long long row = idx / nf;
    const int qs = ((q - nh) % nf + nf) % nf;
    const double2 v = Z[row * nf + qs];
    bank[idx] = make_double2(v.x * inv, v.y * inv);
  }
}

}  // namespace
}  // namespace rift

extern "C" int rift_ile_rotation_bank(const double* hlm, int32_t n_modes, int32_t nf, double df,
                                      double omega, int32_t p_max, double* bank_out,
                                      void* stream) {
  using namespace rift;
  if (!hlm || !bank_out) {
    rift_ile_set_error("rift_ile_rotation_bank: hlm or bank_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (n_modes < 1 || n_modes > RIFT_ILE_MAX_MODES || p_max < 0 || p_max > 3) {
    rift_ile_set_error("rift_ile_rotation_bank: n_modes=%d or p_max=%d unsupported", n_modes, p_max);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  if (nf < 1 || nf % 2 == 0 || nf > (1 << 26)) {
    rift_ile_set_error("rift_ile_rotation_bank: nf=%d must be odd and positive", nf);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (!(df > 0.0) || !std::isfinite(df) || !std::isfinite(omega)) {
    rift_ile_set_error("rift_ile_rotation_bank: df must be positive and omega finite");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const int M = n_modes, np = p_max + 1, na = (p_max + 1) * (p_max + 5);
  cudaStream_t st = (cudaStream_t)stream;
  double2 *X = nullptr, *Z = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&X, (size_t)np * M * nf * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&Z, (size_t)na * M * nf * sizeof(double2), st);
  if (e != cudaSuccess) {
    if (X) cudaFreeAsync(X, st);
    rift_ile_set_error("rift_ile_rotation_bank work buffers: %s", cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  int rc = RIFT_ILE_OK;
  bank_weight_kernel<<<blocks_for((long long)np * M * nf), 256, 0, st>>>((const double2*)hlm, M, nf,
                                                                         df, np, X);
  e = cudaGetLastError();
  if (e == cudaSuccess) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    cufftHandle plan;
    rc = get_plan(nf, np * M, &plan);
    cufftResult r = CUFFT_SUCCESS;
    if (!rc) r = cufftSetStream(plan, st);
    if (!rc && r == CUFFT_SUCCESS)
      r = cufftExecZ2Z(plan, (cufftDoubleComplex*)X, (cufftDoubleComplex*)X, CUFFT_INVERSE);
    if (!rc && r != CUFFT_SUCCESS) {
      rift_ile_set_error("cuFFT inverse transform failed: cufftResult %d", (int)r);
      rc = RIFT_ILE_ERR_CUDA;
    }
  }
  if (e == cudaSuccess && !rc) {
    bank_modulate_kernel<<<blocks_for((long long)na * M * nf), 256, 0, st>>>(X, M, nf, df, omega,
                                                                             p_max, Z);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && !rc) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    cufftHandle plan;
    rc = get_plan(nf, na * M, &plan);
    cufftResult r = CUFFT_SUCCESS;
    if (!rc) r = cufftSetStream(plan, st);
    if (!rc && r == CUFFT_SUCCESS)
      r = cufftExecZ2Z(plan, (cufftDoubleComplex*)Z, (cufftDoubleComplex*)Z, CUFFT_FORWARD);
    if (!rc && r != CUFFT_SUCCESS) {
      rift_ile_set_error("cuFFT forward transform failed: cufftResult %d", (int)r);
      rc = RIFT_ILE_ERR_CUDA;
    }
  }
  if (e == cudaSuccess && !rc) {
    bank_gather_kernel<<<blocks_for((long long)na * M * nf), 256, 0, st>>>(Z, (long long)na * M, nf,
                                                                           (double2*)bank_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(X, st);
  cudaFreeAsync(Z, st);
  if (rc) return rc;
  return check_cuda(e, "rift_ile_rotation_bank");
}

// ------------------------------------------------------- finite-arm bank

namespace rift {
namespace {

constexpr int kCauchyNodes = 64;

__device__ __forceinline__ double2 csin_d(double2 z) {  // sin(a + i b)
  double sa, ca;
  sincos(z.x, &sa, &ca);
  return make_double2(sa * cosh(z.y), ca * sinh(z.y));
}

__device__ __forceinline__ double2 cdiv_d(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

__device__ __forceinline__ double2 csinc_d(double2 z) {
  if (z.x * z.x + z.y * z.y < 1e-16) {  // 1 - z^2/6, error ~ |z|^4/120
    return make_double2(1.0 - (z.x * z.x - z.y * z.y) / 6.0, -(2.0 * z.x * z.y) / 6.0);
  }
  return cdiv_d(csin_d(z), z);
}

// e^{a + i b}
__device__ __forceinline__ double2 cexp_d(double a, double b) {
  double s, c;
  sincos(b, &s, &c);
  const double e = exp(a);
  return make_double2(e * c, e * s);
}

__global__ void arm_bank_kernel(const double2* __restrict__ hlm, int M, int nf, double df, double T,
                                int p_max, double2* __restrict__ bank) {
  const int nh = (nf - 1) / 2;
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nf; q += gridDim.x * blockDim.x) {
    const double f = (double)(q - nh) * df;
    const double x = CUDART_PI * f * T;
    double2 W[RIFT_ILE_MAX_ARM_PMAX + 1];
    for (int p = 0; p <= p_max; ++p) W[p] = make_double2(0.0, 0.0);
    for (int j = 0; j < kCauchyNodes; ++j) {
      double s, c;
      sincospi(2.0 * j / kCauchyNodes, &s, &c);  // u = c + i s on the unit circle
      // D^ = 1/2 [e^{i x (1-u)} sinc(x (1+u)) + e^{-i x (1+u)} sinc(x (1-u))]
      const double2 t1 = cmul_pc(cexp_d(x * s, x * (1.0 - c)), csinc_d(make_double2(x * (1.0 + c), x * s)));
      const double2 t2 = cmul_pc(cexp_d(x * s, -x * (1.0 + c)), csinc_d(make_double2(x * (1.0 - c), -x * s)));
      const double2 D = make_double2(0.5 * (t1.x + t2.x), 0.5 * (t1.y + t2.y));
      // W_p += D e^{-i p phi_j} / N
      double2 e = make_double2(1.0, 0.0);
      for (int p = 0; p <= p_max; ++p) {
        const double2 t = cmul_pc(D, e);
        W[p].x += t.x / kCauchyNodes;
        W[p].y += t.y / kCauchyNodes;
        e = cmul_pc(e, make_double2(c, -s));
      }
    }
    double sd, cd;
    sincospi(-2.0 * f * T, &sd, &cd);
    const double2 delay = make_double2(cd, sd);
    for (int p = 0; p <= p_max; ++p) {
      const double2 wp = cmul_pc(W[p], delay);
      for (int i = 0; i < M; ++i)
        bank[((long long)p * M + i) * nf + q] = cmul_pc(wp, hlm[(long long)i * nf + q]);
    }
  }
}

}  // namespace
}  // namespace rift

extern "C" int rift_ile_arm_bank(const double* hlm, int32_t n_modes, int32_t nf, double df, double T,
                                 int32_t p_max, double* bank_out, void* stream) {
  using namespace rift;
  if (!hlm || !bank_out) {
    rift_ile_set_error("rift_ile_arm_bank: hlm or bank_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (n_modes < 1 || n_modes > RIFT_ILE_MAX_MODES || p_max < 0 || p_max > RIFT_ILE_MAX_ARM_PMAX) {
    rift_ile_set_error("rift_ile_arm_bank: n_modes=%d or p_max=%d unsupported", n_modes, p_max);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  if (nf < 1 || nf % 2 == 0) {
    rift_ile_set_error("rift_ile_arm_bank: nf=%d must be odd and positive", nf);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (!(df > 0.0) || !std::isfinite(df) || !(T >= 0.0) || !std::isfinite(T)) {
    rift_ile_set_error("rift_ile_arm_bank: df must be positive and T finite, non-negative");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  arm_bank_kernel<<<blocks_for(nf), 256, 0, (cudaStream_t)stream>>>((const double2*)hlm, n_modes, nf, df,
                                                                    T, p_max, (double2*)bank_out);
  return check_cuda(cudaGetLastError(), "rift_ile_arm_bank launch");
}
