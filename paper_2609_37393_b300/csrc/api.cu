// C-ABI entry points: argument checks, the per-device workspace, launches,
// and the deterministic combination of per-block log-sum-exp states.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {
namespace {

thread_local long long t_last_oob = 0;

// Library-owned scratch per device: per-block LSE partials, the combined
// state and the out-of-table tap counter.  Allocated on first use.
struct Workspace {
  LseState* partials = nullptr;
  int capacity = 0;
  LseState* state = nullptr;
  unsigned long long* oob = nullptr;
  int sms = 0;
  // distance node table (grown on demand)
  double* dist_x = nullptr;
  double* dist_lnw = nullptr;
  float2* dist_xdf = nullptr;
  float* dist_lnwf = nullptr;
  int dist_cap = 0;
};

std::mutex g_ws_mu;
Workspace g_ws[64];

int get_workspace(Workspace** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    rift_ile_set_error("no current CUDA device");
    return RIFT_ILE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_ws_mu);
  Workspace& w = g_ws[dev];
  if (!w.partials) {
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
      rift_ile_set_error("cannot query the SM count");
      return RIFT_ILE_ERR_CUDA;
    }
    const int cap = sms * kMaxPartialsPerSM;
    if (cudaMalloc((void**)&w.partials, cap * sizeof(LseState)) != cudaSuccess ||
        cudaMalloc((void**)&w.state, sizeof(LseState)) != cudaSuccess ||
        cudaMalloc((void**)&w.oob, sizeof(unsigned long long)) != cudaSuccess) {
      cudaFree(w.partials);
      cudaFree(w.state);
      w = Workspace();
      rift_ile_set_error("workspace allocation failed");
      return RIFT_ILE_ERR_ALLOC;
    }
    w.capacity = cap;
    w.sms = sms;
  }
  *out = &w;
  return RIFT_ILE_OK;
}

// Merges the per-block states in two passes over them: the largest maximum
// M (a max is order-free), then the sums of s_i e^(m_i - M) and
// s2_i e^(2(m_i - M)), each thread over a fixed strided subset and then a
// fixed tree.  The exponentials are independent of one another, so they
// pipeline instead of forming a chain of dependent merges (FP64 issues at
// 2 per clock per SM on this part).  The result is reproducible bit for bit.
__global__ void __launch_bounds__(256) lse_combine_kernel(const LseState* __restrict__ partials,
                                                          int nparts, double n_total,
                                                          LseState* __restrict__ out) {
  __shared__ double red[256];
  __shared__ double red2[256];
  const int t = threadIdx.x;
  double mx = -CUDART_INF;
  int bad = 0;
  for (int i = t; i < nparts; i += blockDim.x) {
    const double m = partials[i].m;
    if (isnan(m)) bad = 1;
    else mx = fmax(mx, m);
  }
  bad = __syncthreads_or(bad);
  red[t] = mx;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) red[t] = fmax(red[t], red[t + w]);
    __syncthreads();
  }
  const double M = red[0];
  __syncthreads();
  double s = 0.0, s2 = 0.0;
  if (M > -CUDART_INF) {
    for (int i = t; i < nparts; i += blockDim.x) {
      const LseState p = partials[i];
      if (!(p.m > -CUDART_INF)) continue;
      const double e = lse_exp(p.m - M);
      s = fma(p.s, e, s);
      s2 = fma(p.s2, e * e, s2);
    }
  }
  red[t] = s;
  red2[t] = s2;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (t < w) {
      red[t] += red[t + w];
      red2[t] += red2[t + w];
    }
    __syncthreads();
  }
  if (t == 0) {
    LseState acc{M, red[0], red2[0], n_total};
    if (!(M > -CUDART_INF)) acc = LseState{-CUDART_INF, 0.0, 0.0, n_total};
    if (bad) acc.m = acc.s = acc.s2 = CUDART_NAN;
    *out = acc;
  }
}

// Copies a host node table into the workspace and describes it for the
// kernels.  The nodes must be finite with x strictly decreasing (increasing D).
int upload_dist(Workspace* ws, const rift_ile_dist* dist, cudaStream_t st, DistParams* out) {
  if (!dist->x || !dist->lnw || dist->n < 1) {
    rift_ile_set_error("distance table: NULL arrays or n < 1");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const int n = dist->n;
  double lnw_max = -INFINITY;
  for (int j = 0; j < n; ++j) {
    if (!std::isfinite(dist->x[j]) || std::isnan(dist->lnw[j]) || dist->lnw[j] == INFINITY ||
        (j > 0 && !(dist->x[j] < dist->x[j - 1]))) {
      rift_ile_set_error("distance table: node %d is not finite or x is not strictly decreasing", j);
      return RIFT_ILE_ERR_INVALID_ARG;
    }
    lnw_max = std::fmax(lnw_max, dist->lnw[j]);
  }
  std::lock_guard<std::mutex> lock(g_ws_mu);
  if (ws->dist_cap < n) {
    cudaFree(ws->dist_x);
    cudaFree(ws->dist_lnw);
    cudaFree(ws->dist_xdf);
    cudaFree(ws->dist_lnwf);
    ws->dist_x = ws->dist_lnw = nullptr;
    ws->dist_xdf = nullptr;
    ws->dist_lnwf = nullptr;
    ws->dist_cap = 0;
    if (cudaMalloc((void**)&ws->dist_x, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&ws->dist_lnw, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void**)&ws->dist_xdf, n * sizeof(float2)) != cudaSuccess ||
        cudaMalloc((void**)&ws->dist_lnwf, n * sizeof(float)) != cudaSuccess) {
      rift_ile_set_error("distance table allocation failed");
      return RIFT_ILE_ERR_ALLOC;
    }
    ws->dist_cap = n;
  }
  std::vector<float2> xdf(n);
  std::vector<float> lnwf(n);
  for (int j = 0; j < n; ++j) {
    const float hi = (float)dist->x[j];
    xdf[j] = make_float2(hi, (float)(dist->x[j] - (double)hi));
    lnwf[j] = (float)dist->lnw[j];
  }
  int rc;
  if ((rc = check_cuda(cudaMemcpyAsync(ws->dist_x, dist->x, n * sizeof(double), cudaMemcpyHostToDevice, st), "table copy")) ||
      (rc = check_cuda(cudaMemcpyAsync(ws->dist_lnw, dist->lnw, n * sizeof(double), cudaMemcpyHostToDevice, st), "table copy")) ||
      (rc = check_cuda(cudaMemcpyAsync(ws->dist_xdf, xdf.data(), n * sizeof(float2), cudaMemcpyHostToDevice, st), "table copy")) ||
      (rc = check_cuda(cudaMemcpyAsync(ws->dist_lnwf, lnwf.data(), n * sizeof(float), cudaMemcpyHostToDevice, st), "table copy")))
    return rc;
  // the host staging vectors die here: finish the copies first
  if ((rc = check_cuda(cudaStreamSynchronize(st), "table copy"))) return rc;
  out->x = ws->dist_x;
  out->lnw = ws->dist_lnw;
  out->xdf = ws->dist_xdf;
  out->lnwf = ws->dist_lnwf;
  out->n = n;
  out->lnw_max = lnw_max;
  out->guess = 0;
  out->lnx0 = 0.f;
  out->inv_dlnx = 0.f;
  if (n >= 3 && dist->x[n - 1] > 0.0) {
    const double l0 = std::log(dist->x[0]);
    const double d = (l0 - std::log(dist->x[n - 1])) / (n - 1);
    bool ok = d > 0.0;
    for (int j = 1; ok && j < n - 1; ++j)
      ok = std::fabs(std::log(dist->x[j]) - (l0 - j * d)) <= 0.5 * d;
    if (ok) {
      out->guess = 1;
      out->lnx0 = (float)l0;
      out->inv_dlnx = (float)(1.0 / d);
    }
  }
  return RIFT_ILE_OK;
}

int check_draws(const rift_ile_draws* d) {
  if (!d) {
    rift_ile_set_error("draws is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->n < 0) {
    rift_ile_set_error("draws->n = %lld is negative", (long long)d->n);
    return RIFT_ILE_ERR_SHAPE;
  }
  if (d->dtype != RIFT_ILE_F32 && d->dtype != RIFT_ILE_F64) {
    rift_ile_set_error("draws->dtype = %d is neither RIFT_ILE_F32 nor RIFT_ILE_F64", d->dtype);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (d->n > 0 && (!d->ra || !d->dec || !d->psi || !d->incl || !d->phase || !d->lnD || !d->t)) {
    rift_ile_set_error("a draw parameter array is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  return RIFT_ILE_OK;
}

DrawsParams to_params(const rift_ile_draws* d) {
  DrawsParams p;
  p.p[0] = d->ra;
  p.p[1] = d->dec;
  p.p[2] = d->psi;
  p.p[3] = d->incl;
  p.p[4] = d->phase;
  p.p[5] = d->lnD;
  p.p[6] = d->t;
  p.logw = d->logw;
  p.n = d->n;
  p.f64 = (d->dtype == RIFT_ILE_F64);
  return p;
}

int check_point(const rift_ile_point* pt, rift_ile_precision prec) {
  if (!pt) {
    rift_ile_set_error("point is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (prec != RIFT_ILE_FP64 && prec != RIFT_ILE_FP32_MIXED) {
    rift_ile_set_error("precision %d is neither RIFT_ILE_FP64 nor RIFT_ILE_FP32_MIXED", (int)prec);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  return RIFT_ILE_OK;
}

cudaError_t launch_lnl(const rift_ile_point* pt, const DrawsParams& dp, rift_ile_precision prec,
                       double* lnl_out, LseState* partials, unsigned long long* oob, int* blocks,
                       cudaStream_t st) {
  if (prec == RIFT_ILE_FP64)
    return launch_lnl_fp64(pt->host, pt->dev, dp, lnl_out, partials, oob, blocks, st);
  return launch_lnl_mixed(pt->host, pt->dev, dp, lnl_out, partials, oob, blocks, st);
}

}  // namespace

int device_sms() {
  Workspace* ws = nullptr;
  if (get_workspace(&ws)) return 1;
  return ws->sms;
}

cudaError_t launch_lse_combine(const LseState* partials, int nparts, double n_total,
                               LseState* state_out, cudaStream_t st) {
  lse_combine_kernel<<<1, 256, 0, st>>>(partials, nparts, n_total, state_out);
  return cudaGetLastError();
}

int lse_workspace(LseState** partials, LseState** state, unsigned long long** oob) {
  Workspace* ws = nullptr;
  int rc = get_workspace(&ws);
  if (rc) return rc;
  *partials = ws->partials;
  *state = ws->state;
  *oob = ws->oob;
  return RIFT_ILE_OK;
}

int validate_draws(const rift_ile_draws* d) { return check_draws(d); }

DrawsParams draws_params(const rift_ile_draws* d) { return to_params(d); }

void set_last_oob(long long v) { t_last_oob = v; }

}  // namespace rift

using namespace rift;

extern "C" int rift_ile_lnL(const rift_ile_point* pt, const rift_ile_draws* draws,
                            rift_ile_precision prec, double* lnL_out, void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!lnL_out) {
    rift_ile_set_error("rift_ile_lnL: lnL_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int blocks = 0;
  return check_cuda(launch_lnl(pt, to_params(draws), prec, lnL_out, nullptr, nullptr, &blocks,
                               (cudaStream_t)stream),
                    "rift_ile_lnL launch");
}

extern "C" int rift_ile_lnZ_state(const rift_ile_point* pt, const rift_ile_draws* draws,
                                  rift_ile_precision prec, const rift_ile_dist* dist,
                                  rift_ile_lse* state, void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(draws);
  if (rc) return rc;
  if (!state) {
    rift_ile_set_error("rift_ile_lnZ_state: state is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (draws->n == 0) {
    *state = rift_ile_lse{-INFINITY, 0.0, 0.0, 0.0};
    t_last_oob = 0;
    return RIFT_ILE_OK;
  }
  Workspace* ws = nullptr;
  if ((rc = get_workspace(&ws))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  int blocks = 0;
  DistParams dd{};
  if (dist && (rc = upload_dist(ws, dist, st, &dd))) return rc;
  if ((rc = check_cuda(cudaMemsetAsync(ws->oob, 0, sizeof(unsigned long long), st), "memset")))
    return rc;
  cudaError_t le;
  if (!dist)
    le = launch_lnl(pt, to_params(draws), prec, nullptr, ws->partials, ws->oob, &blocks, st);
  else if (prec == RIFT_ILE_FP64)
    le = launch_lnl_fp64_dist(pt->host, pt->dev, to_params(draws), dd, nullptr, ws->partials, ws->oob, &blocks, st);
  else
    le = launch_lnl_mixed_dist(pt->host, pt->dev, to_params(draws), dd, nullptr, ws->partials, ws->oob, &blocks, st);
  if ((rc = check_cuda(le, "lnZ kernel launch"))) return rc;
  if ((rc = check_cuda(launch_lse_combine(ws->partials, blocks, (double)draws->n, ws->state, st),
                       "lnZ combine launch")))
    return rc;
  LseState h;
  unsigned long long oob = 0;
  if ((rc = check_cuda(cudaMemcpyAsync(&h, ws->state, sizeof(h), cudaMemcpyDeviceToHost, st),
                       "lnZ copy")))
    return rc;
  if ((rc = check_cuda(cudaMemcpyAsync(&oob, ws->oob, sizeof(oob), cudaMemcpyDeviceToHost, st),
                       "lnZ copy")))
    return rc;
  if ((rc = check_cuda(cudaStreamSynchronize(st), "rift_ile_lnZ"))) return rc;
  t_last_oob = (long long)oob;
  *state = rift_ile_lse{h.m, h.s, h.s2, h.n};
  return RIFT_ILE_OK;
}

namespace rift {
namespace {

// Per-device state of the host-streaming lnZ: two staging buffer sets, a copy
// stream, the events that order copies and kernels, and the partials of all
// chunks of one call.  Allocated on first use, grown on demand.
struct HostStream {
  char* buf[2] = {nullptr, nullptr};
  size_t buf_bytes = 0;
  cudaStream_t copy = nullptr;
  cudaEvent_t copied[2] = {nullptr, nullptr}, consumed[2] = {nullptr, nullptr};
  LseState* partials = nullptr;
  size_t cap = 0;
};

HostStream g_hs[64];
std::mutex g_hs_mu;

int get_host_stream(size_t bytes_per_buf, size_t nparts, HostStream** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    rift_ile_set_error("no current CUDA device");
    return RIFT_ILE_ERR_CUDA;
  }
  HostStream& h = g_hs[dev];
  int rc = RIFT_ILE_OK;
  if (!h.copy) {
    if ((rc = check_cuda(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking), "copy stream")))
      return rc;
    for (int b = 0; b < 2 && !rc; ++b) {
      rc = check_cuda(cudaEventCreateWithFlags(&h.copied[b], cudaEventDisableTiming), "event");
      if (!rc) rc = check_cuda(cudaEventCreateWithFlags(&h.consumed[b], cudaEventDisableTiming), "event");
    }
    if (rc) return rc;
  }
  if (h.buf_bytes < bytes_per_buf) {
    cudaFree(h.buf[0]);
    cudaFree(h.buf[1]);
    h.buf[0] = h.buf[1] = nullptr;
    h.buf_bytes = 0;
    if (cudaMalloc((void**)&h.buf[0], bytes_per_buf) != cudaSuccess ||
        cudaMalloc((void**)&h.buf[1], bytes_per_buf) != cudaSuccess) {
      rift_ile_set_error("host-stream staging allocation failed");
      return RIFT_ILE_ERR_ALLOC;
    }
    h.buf_bytes = bytes_per_buf;
  }
  if (h.cap < nparts) {
    cudaFree(h.partials);
    h.partials = nullptr;
    h.cap = 0;
    if (cudaMalloc((void**)&h.partials, nparts * sizeof(LseState)) != cudaSuccess) {
      rift_ile_set_error("host-stream partials allocation failed");
      return RIFT_ILE_ERR_ALLOC;
    }
    h.cap = nparts;
  }
  *out = &h;
  return RIFT_ILE_OK;
}

}  // namespace
}  // namespace rift

extern "C" int rift_ile_lnZ_state_host(const rift_ile_point* pt, const rift_ile_draws* host_draws,
                                       rift_ile_precision prec, const rift_ile_dist* dist,
                                       int64_t chunk, rift_ile_lse* state, void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(host_draws);
  if (rc) return rc;
  if (!state || chunk < 0) {
    rift_ile_set_error("rift_ile_lnZ_state_host: state is NULL or chunk < 0");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const long long n = host_draws->n;
  if (n == 0) {
    *state = rift_ile_lse{-INFINITY, 0.0, 0.0, 0.0};
    t_last_oob = 0;
    return RIFT_ILE_OK;
  }
  if (chunk == 0) chunk = 1 << 20;
  chunk = std::min<long long>(chunk, n);
  const size_t esz = host_draws->dtype == RIFT_ILE_F64 ? 8 : 4;
  const int narr = host_draws->logw ? 8 : 7;
  const long long nchunks = (n + chunk - 1) / chunk;
  Workspace* ws = nullptr;
  if ((rc = get_workspace(&ws))) return rc;
  const size_t per_chunk_parts = (size_t)ws->sms * kMaxPartialsPerSM;
  HostStream* hs = nullptr;
  // one call at a time uses the staging buffers (concurrent callers queue here)
  std::lock_guard<std::mutex> lock(g_hs_mu);
  if ((rc = get_host_stream((size_t)narr * chunk * esz, per_chunk_parts * nchunks, &hs))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DistParams dd{};
  if (dist && (rc = upload_dist(ws, dist, st, &dd))) return rc;
  if ((rc = check_cuda(cudaMemsetAsync(ws->oob, 0, sizeof(unsigned long long), st), "memset")))
    return rc;
  // the copy stream starts after what the caller queued before this call
  cudaEvent_t start = hs->consumed[1];
  if ((rc = check_cuda(cudaEventRecord(start, st), "event"))) return rc;
  if ((rc = check_cuda(cudaStreamWaitEvent(hs->copy, start, 0), "stream wait"))) return rc;
  const void* src[8] = {host_draws->ra, host_draws->dec, host_draws->psi, host_draws->incl,
                        host_draws->phase, host_draws->lnD, host_draws->t, host_draws->logw};
  size_t off_parts = 0;
  for (long long c = 0; c < nchunks && !rc; ++c) {
    const int b = (int)(c & 1);
    const long long a0 = c * chunk, cnt = std::min<long long>(chunk, n - a0);
    // copies of chunk c into buffer b once the kernel of chunk c - 2 is done with it
    if (c >= 2) rc = check_cuda(cudaStreamWaitEvent(hs->copy, hs->consumed[b], 0), "stream wait");
    DrawsParams dp{};
    for (int q = 0; q < narr && !rc; ++q) {
      char* dst = hs->buf[b] + (size_t)q * chunk * esz;
      rc = check_cuda(cudaMemcpyAsync(dst, (const char*)src[q] + (size_t)a0 * esz, (size_t)cnt * esz,
                                      cudaMemcpyHostToDevice, hs->copy),
                      "host-to-device copy");
      if (q < 7) dp.p[q] = dst;
      else dp.logw = dst;
    }
    if (!rc) rc = check_cuda(cudaEventRecord(hs->copied[b], hs->copy), "event");
    if (!rc) rc = check_cuda(cudaStreamWaitEvent(st, hs->copied[b], 0), "stream wait");
    if (rc) break;
    dp.n = cnt;
    dp.f64 = (host_draws->dtype == RIFT_ILE_F64);
    int blocks = 0;
    cudaError_t le;
    if (!dist)
      le = launch_lnl(pt, dp, prec, nullptr, hs->partials + off_parts, ws->oob, &blocks, st);
    else if (prec == RIFT_ILE_FP64)
      le = launch_lnl_fp64_dist(pt->host, pt->dev, dp, dd, nullptr, hs->partials + off_parts, ws->oob,
                                &blocks, st);
    else
      le = launch_lnl_mixed_dist(pt->host, pt->dev, dp, dd, nullptr, hs->partials + off_parts, ws->oob,
                                 &blocks, st);
    if ((rc = check_cuda(le, "lnZ kernel launch"))) break;
    off_parts += blocks;
    rc = check_cuda(cudaEventRecord(hs->consumed[b], st), "event");
  }
  if (!rc)
    rc = check_cuda(launch_lse_combine(hs->partials, (int)off_parts, (double)n, ws->state, st),
                    "lnZ combine launch");
  LseState h{};
  unsigned long long oob = 0;
  if (!rc) rc = check_cuda(cudaMemcpyAsync(&h, ws->state, sizeof(h), cudaMemcpyDeviceToHost, st), "copy");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(&oob, ws->oob, sizeof(oob), cudaMemcpyDeviceToHost, st), "copy");
  // both streams are idle when this returns (also after an error)
  cudaError_t e1 = cudaStreamSynchronize(hs->copy), e2 = cudaStreamSynchronize(st);
  if (!rc) rc = check_cuda(e1 != cudaSuccess ? e1 : e2, "rift_ile_lnZ_state_host");
  if (rc) return rc;
  t_last_oob = (long long)oob;
  *state = rift_ile_lse{h.m, h.s, h.s2, h.n};
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_lnZ_state_async(const rift_ile_point* pt, const rift_ile_draws* draws,
                                        rift_ile_precision prec, const rift_ile_dist* dist,
                                        rift_ile_lse* state_out, void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(draws);
  if (rc) return rc;
  if (!state_out) {
    rift_ile_set_error("rift_ile_lnZ_state_async: state_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  static_assert(sizeof(rift_ile_lse) == sizeof(LseState), "state layouts differ");
  LseState* out = reinterpret_cast<LseState*>(state_out);
  Workspace* ws = nullptr;
  if ((rc = get_workspace(&ws))) return rc;
  if (draws->n == 0)  // the merge of no partials is the empty state
    return check_cuda(launch_lse_combine(ws->partials, 0, 0.0, out, st), "lnZ combine launch");
  DistParams dd{};
  if (dist && (rc = upload_dist(ws, dist, st, &dd))) return rc;
  int blocks = 0;
  cudaError_t le;
  if (!dist)
    le = launch_lnl(pt, to_params(draws), prec, nullptr, ws->partials, nullptr, &blocks, st);
  else if (prec == RIFT_ILE_FP64)
    le = launch_lnl_fp64_dist(pt->host, pt->dev, to_params(draws), dd, nullptr, ws->partials, nullptr, &blocks, st);
  else
    le = launch_lnl_mixed_dist(pt->host, pt->dev, to_params(draws), dd, nullptr, ws->partials, nullptr, &blocks, st);
  if ((rc = check_cuda(le, "lnZ kernel launch"))) return rc;
  return check_cuda(launch_lse_combine(ws->partials, blocks, (double)draws->n, out, st),
                    "lnZ combine launch");
}

extern "C" int rift_ile_lnZ_merge(const rift_ile_lse* states, int32_t S, double out[3],
                                  rift_ile_lse* merged) {
  if ((!states && S > 0) || S < 0) {
    rift_ile_set_error("rift_ile_lnZ_merge: bad states/S");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  double m = -INFINITY, n = 0.0;
  bool bad = false;
  for (int i = 0; i < S; ++i) {
    if (std::isnan(states[i].m)) bad = true;
    if (states[i].m > m) m = states[i].m;
    n += states[i].n;
  }
  double s = 0.0, s2 = 0.0;
  if (std::isfinite(m)) {
    for (int i = 0; i < S; ++i) {
      if (!(states[i].m > -INFINITY)) continue;
      double e = std::exp(states[i].m - m);
      s += states[i].s * e;
      s2 += states[i].s2 * e * e;
    }
  }
  if (bad) m = s = s2 = NAN;
  if (merged) *merged = rift_ile_lse{m, s, s2, n};
  if (out) {
    if (n <= 0) {
      out[0] = -INFINITY;
      out[1] = NAN;
      out[2] = 0.0;
    } else {
      out[0] = m + std::log(s) - std::log(n);
      double var = s2 / (s * s) - 1.0 / n;
      out[1] = std::sqrt(var > 0 ? var : 0.0);
      out[2] = s;
    }
  }
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_lnZ(const rift_ile_point* pt, const rift_ile_draws* draws,
                            rift_ile_precision prec, const rift_ile_dist* dist, double out[3],
                            void* stream) {
  if (!out) {
    rift_ile_set_error("rift_ile_lnZ: out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  rift_ile_lse st;
  int rc = rift_ile_lnZ_state(pt, draws, prec, dist, &st, stream);
  if (rc) return rc;
  return rift_ile_lnZ_merge(&st, 1, out, nullptr);
}

extern "C" int64_t rift_ile_last_oob(void) { return t_last_oob; }

extern "C" int rift_ile_lnL_grad(const rift_ile_point* pt, const rift_ile_draws* draws,
                                 rift_ile_precision prec, double* lnL_out, double* grad_out,
                                 void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(draws);
  if (rc) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  if (!grad_out) {
    rift_ile_set_error("rift_ile_lnL_grad: grad_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const DrawsParams dp = to_params(draws);
  cudaError_t e = (prec == RIFT_ILE_FP64)
                      ? launch_grad_fp64(pt->host, pt->dev, dp, lnL_out, grad_out, (cudaStream_t)stream)
                      : launch_grad_mixed(pt->host, pt->dev, dp, lnL_out, grad_out, (cudaStream_t)stream);
  return check_cuda(e, "rift_ile_lnL_grad launch");
}

extern "C" int rift_ile_lnL_dist(const rift_ile_point* pt, const rift_ile_draws* draws,
                                 rift_ile_precision prec, const rift_ile_dist* dist, double* lnL_out,
                                 double* grad_out, void* stream) {
  int rc = check_point(pt, prec);
  if (!rc) rc = check_draws(draws);
  if (rc) return rc;
  if (!dist || !lnL_out) {
    rift_ile_set_error("rift_ile_lnL_dist: dist or lnL_out is NULL");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  Workspace* ws = nullptr;
  if ((rc = get_workspace(&ws))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  DistParams dd{};
  if ((rc = upload_dist(ws, dist, st, &dd))) return rc;
  if (draws->n == 0) return RIFT_ILE_OK;
  int blocks = 0;
  cudaError_t le;
  if (grad_out)
    le = (prec == RIFT_ILE_FP64)
             ? launch_grad_fp64_dist(pt->host, pt->dev, to_params(draws), dd, lnL_out, grad_out, st)
             : launch_grad_mixed_dist(pt->host, pt->dev, to_params(draws), dd, lnL_out, grad_out, st);
  else
    le = (prec == RIFT_ILE_FP64)
             ? launch_lnl_fp64_dist(pt->host, pt->dev, to_params(draws), dd, lnL_out, nullptr, nullptr, &blocks, st)
             : launch_lnl_mixed_dist(pt->host, pt->dev, to_params(draws), dd, lnL_out, nullptr, nullptr, &blocks, st);
  return check_cuda(le, "rift_ile_lnL_dist launch");
}

// Log-uniform node table in ln D (eq. ap:dlog): the spacing in ln D is the
// largest h <= c(tol)/rho_max, c(tol) = pi sqrt(2/ln(2/tol)), that divides
// [ln d_min, ln d_max] into whole steps; trapezoid weights in ln D; the prior
// p(D) = 3 D^2/(d_max^3 - d_min^3) (uniform in Euclidean volume) enters with
// the Jacobian D of D -> ln D: ln w_j = ln(h_j) + ln p(D_j) + ln D_j.
extern "C" int rift_ile_dist_nodes(double d_min, double d_max, double d_ref, double tol,
                                   double rho_max, int32_t max_nodes, double* x, double* lnw,
                                   int32_t* n_out) {
  if (!x || !lnw || !n_out || !(d_min > 0) || !(d_max > d_min) || !(d_ref > 0) || !(tol > 0) ||
      !(tol < 2) || !(rho_max > 0) || max_nodes < 2) {
    rift_ile_set_error("rift_ile_dist_nodes: invalid argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  const double c = M_PI * std::sqrt(2.0 / std::log(2.0 / tol));
  const double span = std::log(d_max / d_min);
  const double steps = std::ceil(span * rho_max / c);
  if (steps + 1 > max_nodes) {
    rift_ile_set_error("rift_ile_dist_nodes: %.0f nodes exceed max_nodes = %d", steps + 1, max_nodes);
    return RIFT_ILE_ERR_SHAPE;
  }
  const int n = (int)steps + 1;
  const double h = span / steps;
  const double ln_norm = std::log(3.0 / (d_max * d_max * d_max - d_min * d_min * d_min));
  for (int j = 0; j < n; ++j) {
    const double lnd = std::log(d_min) + j * h;
    const double wt = (j == 0 || j == n - 1) ? 0.5 * h : h;
    x[j] = d_ref * std::exp(-lnd);
    lnw[j] = std::log(wt) + ln_norm + 3.0 * lnd;
  }
  *n_out = n;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_release(void) {
  release_fft_plans();
  forget_noalloc_scratch();
  std::lock_guard<std::mutex> lock(g_ws_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < 64; ++d) {
    Workspace& w = g_ws[d];
    if (!w.partials) continue;
    cudaSetDevice(d);
    cudaFree(w.partials);
    cudaFree(w.state);
    cudaFree(w.oob);
    cudaFree(w.dist_x);
    cudaFree(w.dist_lnw);
    cudaFree(w.dist_xdf);
    cudaFree(w.dist_lnwf);
    w = Workspace();
  }
  {
    std::lock_guard<std::mutex> lock2(g_hs_mu);
    for (int d = 0; d < 64; ++d) {
      HostStream& h = g_hs[d];
      if (!h.copy) continue;
      cudaSetDevice(d);
      cudaFree(h.buf[0]);
      cudaFree(h.buf[1]);
      cudaFree(h.partials);
      for (int b = 0; b < 2; ++b) {
        cudaEventDestroy(h.copied[b]);
        cudaEventDestroy(h.consumed[b]);
      }
      cudaStreamDestroy(h.copy);
      h = HostStream();
    }
  }
  cudaSetDevice(cur);
  return RIFT_ILE_OK;
}
