// Fine table of eq. q-time-pregrid from a native-rate table (rift_ile_pregrid).
//
// Per (detector, mode) series: reflect (q_0 .. q_{n-1}, q_{n-1} .. q_0),
// forward DFT of length 2n, zero-pad the coefficients to length 2rn
// (frequencies 0 .. n-1 at the start, -(n-1) .. -1 at the end; the reflected
// series has no Nyquist component), inverse DFT scaled by 1/(2n), keep the
// native window's r (n - 1) + 1 samples.  Both transforms are batched over the
// K M series with cached cuFFT plans; three small kernels move the data in
// and out of the [K][n][M] table layout.
#include <cuda_runtime.h>

#include "../../include/rift_ile_precompute.h"
#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {
namespace {

__device__ __forceinline__ double2 load_c(const float2* p) {
  const float2 v = *p;
  return make_double2((double)v.x, (double)v.y);
}
__device__ __forceinline__ double2 load_c(const double2* p) { return *p; }
__device__ __forceinline__ void store_c(float2* p, double2 v) {
  *p = make_float2((float)v.x, (float)v.y);
}
__device__ __forceinline__ void store_c(double2* p, double2 v) { *p = v; }

// X[k M + i][j] = q[k][j][i] for j < n and q[k][2n - 1 - j][i] for n <= j < 2n
template <typename T>
__global__ void reflect_kernel(const T* __restrict__ q, int K, int n, int M,
                               double2* __restrict__ X) {
  const long long len = 2LL * n;
  const long long total = (long long)K * M * len;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long j = idx % len;
    const long long row = idx / len;
    const int i = (int)(row % M);
    const long long k = row / M;
    const long long src = j < n ? j : len - 1 - j;
    X[idx] = load_c(q + (k * n + src) * M + i);
  }
}

// Y[row][m], m < 2rn: X[row][m] / (2n) for m < n, X[row][m - 2rn + 2n] / (2n)
// for m > 2rn - n, zero between
__global__ void pad_kernel(const double2* __restrict__ X, int n, int r, long long rows,
                           double2* __restrict__ Y) {
  const long long len = 2LL * n, L = len * r;
  const long long total = rows * L;
  const double s = 1.0 / (double)len;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const long long m = idx % L;
    const long long row = idx / L;
    double2 v = make_double2(0.0, 0.0);
    if (m < n) {
      v = X[row * len + m];
    } else if (m > L - n) {
      v = X[row * len + (m - L + len)];
    }
    Y[idx] = make_double2(v.x * s, v.y * s);
  }
}

// out[k][m][i] = Y[k M + i][m], m < nfine
template <typename T>
__global__ void fine_gather_kernel(const double2* __restrict__ Y, int K, int M, long long L,
                                   long long nfine, T* __restrict__ out) {
  const long long total = (long long)K * nfine * M;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(idx % M);
    const long long km = idx / M;
    const long long m = km % nfine;
    const long long k = km / nfine;
    store_c(out + idx, Y[(k * M + i) * L + m]);
  }
}

int grid_for_total(long long total) {
  const long long b = (total + 255) / 256;
  const long long cap = (long long)device_sms() * 16;
  return (int)(b < 1 ? 1 : (b < cap ? b : cap));
}

}  // namespace
}  // namespace rift

using namespace rift;

extern "C" int rift_ile_pregrid(const void* Q_native, int32_t n_det, int32_t n_modes, int32_t n,
                                int32_t q_dtype_in, int32_t r, void* Q_fine, int32_t q_dtype_out,
                                void* stream) {
  if (!Q_native || !Q_fine) {
    rift_ile_set_error("rift_ile_pregrid: NULL table");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if ((q_dtype_in != RIFT_ILE_C64 && q_dtype_in != RIFT_ILE_C128) ||
      (q_dtype_out != RIFT_ILE_C64 && q_dtype_out != RIFT_ILE_C128)) {
    rift_ile_set_error("rift_ile_pregrid: q_dtype_in=%d, q_dtype_out=%d must be RIFT_ILE_C64 or "
                       "RIFT_ILE_C128", q_dtype_in, q_dtype_out);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (n_det < 1 || n_modes < 1 || n < 1 || (long long)n_det * n_modes > 4096) {
    rift_ile_set_error("rift_ile_pregrid: n_det=%d, n_modes=%d, n=%d out of range", n_det,
                       n_modes, n);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (r < 1 || r > 64 || 2LL * r * n > (1LL << 27)) {
    rift_ile_set_error("rift_ile_pregrid: r=%d with n=%d gives a fine series beyond 2^27 (r must "
                       "be in [1, 64])", r, n);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int K = n_det, M = n_modes, batch = K * M;
  const long long len = 2LL * n, L = len * r, nfine = (long long)r * (n - 1) + 1;
  double2 *X = nullptr, *Y = nullptr;
  cudaError_t e = cudaMallocAsync((void**)&X, (size_t)batch * len * sizeof(double2), st);
  if (e == cudaSuccess) e = cudaMallocAsync((void**)&Y, (size_t)batch * L * sizeof(double2), st);
  if (e != cudaSuccess) {
    if (X) cudaFreeAsync(X, st);
    rift_ile_set_error("rift_ile_pregrid: work buffers of %lld complex doubles: %s",
                       (long long)batch * (len + L), cudaGetErrorString(e));
    return RIFT_ILE_ERR_ALLOC;
  }
  int rc = RIFT_ILE_OK;
  if (q_dtype_in == RIFT_ILE_C128)
    reflect_kernel<double2><<<grid_for_total(batch * len), 256, 0, st>>>(
        (const double2*)Q_native, K, n, M, X);
  else
    reflect_kernel<float2><<<grid_for_total(batch * len), 256, 0, st>>>(
        (const float2*)Q_native, K, n, M, X);
  rc = check_cuda(cudaGetLastError(), "rift_ile_pregrid: reflect launch");
  if (!rc) rc = fft_z2z_inplace(X, len, batch, -1, st);
  if (!rc) {
    pad_kernel<<<grid_for_total(batch * L), 256, 0, st>>>(X, n, r, batch, Y);
    rc = check_cuda(cudaGetLastError(), "rift_ile_pregrid: pad launch");
  }
  if (!rc) rc = fft_z2z_inplace(Y, L, batch, +1, st);
  if (!rc) {
    if (q_dtype_out == RIFT_ILE_C128)
      fine_gather_kernel<double2><<<grid_for_total(K * nfine * M), 256, 0, st>>>(
          Y, K, M, L, nfine, (double2*)Q_fine);
    else
      fine_gather_kernel<float2><<<grid_for_total(K * nfine * M), 256, 0, st>>>(
          Y, K, M, L, nfine, (float2*)Q_fine);
    rc = check_cuda(cudaGetLastError(), "rift_ile_pregrid: gather launch");
  }
  cudaFreeAsync(X, st);
  cudaFreeAsync(Y, st);
  return rc;
}
