// Host side of the FP32-mixed path: the anchor tables of the double-float
// sine/cosine and exponential, and the dispatch of a point's mode count M to
// the kernels instantiated for MM >= M (one translation unit per MM,
// lnl_mixed_m*.cu, so that the compiler front end runs on them in parallel).
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <mutex>

#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {

template <int MM>
cudaError_t mixed_lnl(const PointParams&, const PointParams*, const DrawsParams&, double*,
                      LseState*, unsigned long long*, int*, cudaStream_t);
template <int MM>
cudaError_t mixed_lnl_sms(const PointParams&, const PointParams*, const DrawsParams&, double*,
                          LseState*, unsigned long long*, int, int*, cudaStream_t);
template <int MM>
cudaError_t mixed_dist(const PointParams&, const PointParams*, const DrawsParams&,
                       const DistParams&, double*, LseState*, unsigned long long*, int*,
                       cudaStream_t);
template <int MM>
cudaError_t mixed_grad(const PointParams&, const PointParams*, const DrawsParams&, double*,
                       double*, cudaStream_t);
template <int MM>
cudaError_t mixed_grad_dist(const PointParams&, const PointParams*, const DrawsParams&,
                            const DistParams&, double*, double*, cudaStream_t);
template <int MM>
BatchKernelFn mixed_batch_kernel(int R);
template <int MM>
size_t mixed_batch_smem(int R, int ncls, int Rp, int Mp, int Kp);
template <int MM>
int mixed_upload_anchors(const float4* sincos_tab, const float2* exp_tab);
template <int MM>
int mixed_image(const PointParams& hp, float4** img, int* nf4, cudaStream_t st);

namespace {
std::atomic<long long> g_small_batch_max{2048};
}

long long small_batch_max() { return g_small_batch_max.load(std::memory_order_relaxed); }

// Sine/cosine of a_j = j 2^-7 and e^(j/128) as (hi, lo) float pairs, copied
// into every mode-count unit's tables once per device.
int ensure_anchor_table() {
  static std::mutex mu;
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    rift_ile_set_error("ensure_anchor_table: no current CUDA device");
    return RIFT_ILE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(mu);
  if (done[dev]) return RIFT_ILE_OK;
  static float4 h[2 * kAnchorHalf + 1];
  for (int j = -kAnchorHalf; j <= kAnchorHalf; ++j) {
    double a = j * (double)kAnchorStep;
    double s = std::sin(a), c = std::cos(a);
    float sh = (float)s, ch = (float)c;
    h[j + kAnchorHalf] = make_float4(sh, (float)(s - sh), ch, (float)(c - ch));
  }
  static float2 e[2 * kExpHalf + 1];
  for (int j = -kExpHalf; j <= kExpHalf; ++j) {
    double v = std::exp(j / 128.0);
    float hi = (float)v;
    e[j + kExpHalf] = make_float2(hi, (float)(v - hi));
  }
  int rc = mixed_upload_anchors<2>(h, e);
  if (!rc) rc = mixed_upload_anchors<4>(h, e);
  if (!rc) rc = mixed_upload_anchors<6>(h, e);
  if (!rc) rc = mixed_upload_anchors<8>(h, e);
  if (!rc) rc = mixed_upload_anchors<10>(h, e);
  if (!rc) rc = mixed_upload_anchors<12>(h, e);
  if (!rc) rc = mixed_upload_anchors<16>(h, e);
  if (!rc) done[dev] = true;
  return rc;
}

// Calls F<MM>(args...) for the smallest instantiated MM >= M.
#define RIFT_DISPATCH_M(M, F, ...)                  \
  ((M) <= 2    ? F<2>(__VA_ARGS__)                  \
   : (M) <= 4  ? F<4>(__VA_ARGS__)                  \
   : (M) <= 6  ? F<6>(__VA_ARGS__)                  \
   : (M) <= 8  ? F<8>(__VA_ARGS__)                  \
   : (M) <= 10 ? F<10>(__VA_ARGS__)                 \
   : (M) <= 12 ? F<12>(__VA_ARGS__)                 \
               : F<16>(__VA_ARGS__))

cudaError_t launch_lnl_mixed(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                             double* lnl_out, LseState* partials, unsigned long long* oob,
                             int* blocks, cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_lnl, hp, dP, dp, lnl_out, partials, oob, blocks, st);
}

cudaError_t launch_lnl_mixed_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                 double* lnl_out, LseState* partials, unsigned long long* oob,
                                 int sms, int* blocks, cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_lnl_sms, hp, dP, dp, lnl_out, partials, oob, sms, blocks, st);
}

cudaError_t launch_lnl_mixed_dist(const PointParams& hp, const PointParams* dP,
                                  const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                  LseState* partials, unsigned long long* oob, int* blocks,
                                  cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_dist, hp, dP, dp, dist, lnl_out, partials, oob, blocks, st);
}

cudaError_t launch_grad_mixed(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                              double* lnl_out, double* grad_out, cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_grad, hp, dP, dp, lnl_out, grad_out, st);
}

cudaError_t launch_grad_mixed_dist(const PointParams& hp, const PointParams* dP,
                                   const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                   double* grad_out, cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_grad_dist, hp, dP, dp, dist, lnl_out, grad_out, st);
}

int build_mixed_image(const PointParams& hp, float4** img, int* nf4, cudaStream_t st) {
  return RIFT_DISPATCH_M(hp.M, mixed_image, hp, img, nf4, st);
}

BatchKernelFn batch_kernel_for(int M, int R) { return RIFT_DISPATCH_M(M, mixed_batch_kernel, R); }

size_t batch_smem_for(int M, int R, int ncls, int Rp, int Mp, int Kp) {
  return RIFT_DISPATCH_M(M, mixed_batch_smem, R, ncls, Rp, Mp, Kp);
}

}  // namespace rift

extern "C" int64_t rift_ile_set_small_batch(int64_t max_draws) {
  if (max_draws < 0) max_draws = 0;
  return (int64_t)rift::g_small_batch_max.exchange((long long)max_draws);
}
