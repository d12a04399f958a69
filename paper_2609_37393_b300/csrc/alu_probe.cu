// Measured ALU issue rates on the current GPU: FP32 FMA, FP64 FMA, MUFU ex2
// and MUFU sin.  The likelihood kernels are bound by these pipes (not by HBM
// and not by tensor cores), so their roofline denominators are measured here,
// at the clock the probe itself observes, instead of being taken from a data
// sheet.  Each probe runs CHAINS independent dependency chains per thread so
// that pipe latency is hidden; throughput is counted as operations per second
// (one FMA = one operation = two flops).
#include <cuda_runtime.h>
#include <stdint.h>

#include "rift_ile_internal.h"

namespace {

constexpr int kChains = 8;

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Block 0 / thread 0 records (sm cycles, ns) over its own run: the ratio is
// the SM clock seen by the probe.
template <typename T>
__global__ void probe_fma(T* sink, long long* clk, T b, T c, int iters) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = T(threadIdx.x) * T(1e-3) + T(i);
  long long c0 = clock64();
  uint64_t t0 = global_ns();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == T(12345.678)) sink[0] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = (long long)(global_ns() - t0);
  }
}

// Packed pairs: each __ffma2_rn is one instruction carrying two FP32 FMAs
// (sm_100 and later); counted as two operations.
__global__ void probe_fma2(float* sink, long long* clk, float b, float c, int iters) {
  float2 a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i)
    a[i] = make_float2(threadIdx.x * 1e-3f + (float)i, threadIdx.x * 2e-3f - (float)i);
  const float2 b2 = make_float2(b, b), c2 = make_float2(c, c);
  long long c0 = clock64();
  uint64_t t0 = global_ns();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = __ffma2_rn(a[i], b2, c2);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i].x + a[i].y;
  if (s == 12345.678f) sink[0] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = (long long)(global_ns() - t0);
  }
}

__global__ void probe_ex2(float* sink, long long* clk, float b, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 0.1f + 1e-4f * (threadIdx.x + i);
  long long c0 = clock64();
  uint64_t t0 = global_ns();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      float y;
      asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
      a[i] = y * b;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) sink[0] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = (long long)(global_ns() - t0);
  }
}

__global__ void probe_sin(float* sink, long long* clk, float b, int iters) {
  float a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = 0.1f + 1e-4f * (threadIdx.x + i);
  long long c0 = clock64();
  uint64_t t0 = global_ns();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) {
      float y;
      asm volatile("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(a[i]));
      a[i] = y + b;
    }
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == 12345.678f) sink[0] = s;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    clk[0] = clock64() - c0;
    clk[1] = (long long)(global_ns() - t0);
  }
}

// One timed launch of probe `which` with `iters` loop trips; returns seconds.
int run_probe(int which, int blocks, int threads, int iters, void* sink,
              long long* d_clk, float* ms_out) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1;
  if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return -1; }
  cudaEventRecord(e0, 0);
  switch (which) {
    case RIFT_ILE_PROBE_FP32_FMA:
      probe_fma<float><<<blocks, threads>>>((float*)sink, d_clk, 0.9999999f, 1e-7f, iters);
      break;
    case RIFT_ILE_PROBE_FP64_FMA:
      probe_fma<double><<<blocks, threads>>>((double*)sink, d_clk, 0.9999999, 1e-7, iters);
      break;
    case RIFT_ILE_PROBE_MUFU_EX2:
      probe_ex2<<<blocks, threads>>>((float*)sink, d_clk, 0.5f, iters);
      break;
    case RIFT_ILE_PROBE_FP32X2_FMA:
      probe_fma2<<<blocks, threads>>>((float*)sink, d_clk, 0.9999999f, 1e-7f, iters);
      break;
    case RIFT_ILE_PROBE_MUFU_SIN:
      probe_sin<<<blocks, threads>>>((float*)sink, d_clk, 0.25f, iters);
      break;
    default:
      break;
  }
  cudaEventRecord(e1, 0);
  cudaError_t err = cudaEventSynchronize(e1);
  float ms = 0.f;
  if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err != cudaSuccess) return -1;
  *ms_out = ms;
  return 0;
}

}  // namespace

extern "C" int rift_ile_probe_alu(int which, double target_seconds, double* ops_per_second,
                                  double* sm_mhz) {
  if (!ops_per_second || which < 0 || which > RIFT_ILE_PROBE_FP32X2_FMA || !(target_seconds > 0)) {
    rift_ile_set_error("rift_ile_probe_alu: invalid argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    rift_ile_set_error("rift_ile_probe_alu: no CUDA device");
    return RIFT_ILE_ERR_CUDA;
  }
  const int threads = 256;
  const int blocks = sms * 8;
  void* sink = nullptr;
  long long* d_clk = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess || cudaMalloc((void**)&d_clk, 2 * sizeof(long long)) != cudaSuccess) {
    cudaFree(sink);
    rift_ile_set_error("rift_ile_probe_alu: cudaMalloc failed");
    return RIFT_ILE_ERR_CUDA;
  }
  // Warm up and calibrate on a short run, then scale the trip count so that
  // the measured launch lasts about target_seconds.
  int iters = (which == RIFT_ILE_PROBE_FP64_FMA) ? 16 : 256;
  float ms = 0.f;
  int rc = run_probe(which, blocks, threads, iters, sink, d_clk, &ms);
  for (int rep = 0; rc == 0 && rep < 6 && ms < 0.25f * 1e3f * (float)target_seconds; ++rep) {
    double scale = (ms > 0.05f) ? (1e3 * target_seconds / ms) : 8.0;
    if (scale > 64.0) scale = 64.0;
    if (scale < 1.0) break;
    double next = iters * scale;
    if (next > 1.0e8) next = 1.0e8;
    iters = (int)next;
    rc = run_probe(which, blocks, threads, iters, sink, d_clk, &ms);
  }
  if (rc == 0) rc = run_probe(which, blocks, threads, iters, sink, d_clk, &ms);
  long long h_clk[2] = {0, 0};
  if (rc == 0 && cudaMemcpy(h_clk, d_clk, sizeof(h_clk), cudaMemcpyDeviceToHost) != cudaSuccess) rc = -1;
  cudaFree(sink);
  cudaFree(d_clk);
  if (rc != 0) {
    rift_ile_set_error("rift_ile_probe_alu: probe launch failed");
    return RIFT_ILE_ERR_CUDA;
  }
  const double ops = (double)blocks * threads * (double)iters * kChains *
                     (which == RIFT_ILE_PROBE_FP32X2_FMA ? 2.0 : 1.0);
  *ops_per_second = ops / (1e-3 * ms);
  if (sm_mhz) *sm_mhz = (h_clk[1] > 0) ? (double)h_clk[0] / (double)h_clk[1] * 1e3 : 0.0;
  return RIFT_ILE_OK;
}
