// Allocation-free form of the Monte Carlo lnZ state (rift_ile_lnZ_state_noalloc).
//
// Who needs it: callers that may not allocate device memory while they run --
// for example a host framework that owns the whole device heap through its own
// pool allocator and forbids other code to call cudaMalloc/cudaFree, or code
// running where an allocation could block or fail (a latency-critical sampler
// loop, a process sharing the GPU under a fixed memory quota).  The regular
// rift_ile_lnZ_state allocates the library's per-device workspace on its
// first call; this variant never allocates.
//
// Its scratch is one file-scope __device__ array of fixed size,
// kScratchPartials + 2 LSE states (about 128 KB): per-block partials in
// [0, kScratchPartials), the combined state in [kScratchPartials], and the
// out-of-table tap counter in the first 8 bytes of [kScratchPartials + 1].
// Every GPU that loads the library holds this array until the process exits.
// The kernels need its device address, which host code must not take from the
// symbol itself (in host code the name is only a host-side stand-in); it is
// obtained once per device, with that device current, by cudaGetSymbolAddress
// on the first call of the entry point on that device, so that first call
// should be made before any stream capture.
//
// All calls on one device share the array, and it keeps the last call's
// contents: the counter is cleared on every call, and the partials and the
// combined state are overwritten before they are read.  Calls whose work
// overlaps on the GPU (different streams, or different host threads) race on
// the array; serialise them.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "kernels.h"
#include "rift_ile_internal.h"

namespace rift {
namespace {

constexpr int kScratchPartials = 4096;  // per-block partials the scratch can hold

static __device__ __align__(256) LseState g_noalloc_scratch[kScratchPartials + 2];

std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

// Device address of the scratch array on the current device (set up once per device).
int scratch_address(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    rift_ile_set_error("rift_ile_lnZ_state_noalloc: no current CUDA device");
    return RIFT_ILE_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      rift_ile_set_error("rift_ile_lnZ_state_noalloc: cudaGetSymbolAddress failed: %s",
                         cudaGetErrorString(e));
      return RIFT_ILE_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return RIFT_ILE_OK;
}

}  // namespace

// Forgets the cached device addresses (rift_ile_release): after a device
// reset the module is loaded again and the array may sit elsewhere, so the
// next call looks the address up afresh (cudaGetSymbolAddress allocates nothing).
void forget_noalloc_scratch() {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  for (auto& a : g_scratch_addr) a = nullptr;
}

}  // namespace rift

using namespace rift;

extern "C" int rift_ile_lnZ_state_noalloc(const rift_ile_point* pt, const rift_ile_draws* draws,
                                          rift_ile_precision prec, rift_ile_lse* state,
                                          void* stream) {
  if (!pt || !state) {
    rift_ile_set_error("rift_ile_lnZ_state_noalloc: NULL argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  if (prec != RIFT_ILE_FP64 && prec != RIFT_ILE_FP32_MIXED) {
    rift_ile_set_error("rift_ile_lnZ_state_noalloc: precision %d is neither RIFT_ILE_FP64 nor "
                       "RIFT_ILE_FP32_MIXED", (int)prec);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  // the same draw rules (and error codes) as every other entry point
  int rc = validate_draws(draws);
  if (rc) return rc;
  if (draws->n == 0) {
    *state = rift_ile_lse{-INFINITY, 0.0, 0.0, 0.0};
    return RIFT_ILE_OK;
  }
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    rift_ile_set_error("rift_ile_lnZ_state_noalloc: cannot query the device");
    return RIFT_ILE_ERR_CUDA;
  }
  // The grid is at most kMaxPartialsPerSM blocks per SM, one partial each.
  if ((long long)sms * kMaxPartialsPerSM > kScratchPartials) {
    rift_ile_set_error("rift_ile_lnZ_state_noalloc: %d SMs x %d blocks need more than the %d "
                       "partials of the static scratch", sms, kMaxPartialsPerSM, kScratchPartials);
    return RIFT_ILE_ERR_UNSUPPORTED;
  }
  void* base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  LseState* partials = static_cast<LseState*>(base);
  LseState* combined = partials + kScratchPartials;
  unsigned long long* oob = reinterpret_cast<unsigned long long*>(partials + kScratchPartials + 1);
  cudaStream_t st = (cudaStream_t)stream;

  const DrawsParams dp = draws_params(draws);

  if ((rc = check_cuda(cudaMemsetAsync(oob, 0, sizeof(unsigned long long), st),
                       "rift_ile_lnZ_state_noalloc: clear")))
    return rc;
  int blocks = 0;
  cudaError_t e = (prec == RIFT_ILE_FP64)
                      ? launch_lnl_fp64_sms(pt->host, pt->dev, dp, nullptr, partials, oob, sms, &blocks, st)
                      : launch_lnl_mixed_sms(pt->host, pt->dev, dp, nullptr, partials, oob, sms, &blocks, st);
  if ((rc = check_cuda(e, "rift_ile_lnZ_state_noalloc: kernel launch"))) return rc;
  if ((rc = check_cuda(launch_lse_combine(partials, blocks, (double)draws->n, combined, st),
                       "rift_ile_lnZ_state_noalloc: combine launch")))
    return rc;
  // the combined state and the tap counter are adjacent: one copy brings both
  LseState h[2];
  if ((rc = check_cuda(cudaMemcpyAsync(h, combined, sizeof(h), cudaMemcpyDeviceToHost, st),
                       "rift_ile_lnZ_state_noalloc: copy")))
    return rc;
  if ((rc = check_cuda(cudaStreamSynchronize(st), "rift_ile_lnZ_state_noalloc"))) return rc;
  unsigned long long taps = 0;
  memcpy(&taps, &h[1], sizeof(taps));
  set_last_oob((long long)taps);
  *state = rift_ile_lse{h[0].m, h[0].s, h[0].s2, h[0].n};
  return RIFT_ILE_OK;
}
