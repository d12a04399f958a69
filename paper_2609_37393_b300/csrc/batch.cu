// lnZ of many intrinsic points in persistent launches (rift_ile_lnZ_batch,
// rift_ile_batch_*).  The paper's ILE stage evaluates the marginal likelihood
// of many intrinsic points (Sec. II.C: each worker handles a set of points);
// here their draws are cut into tiles and the (point, tile) items form work
// queues, one per group of points that share a compiled kernel shape (the
// mode-count bucket and the padded whitened width), so that every launch runs
// the exact-width kernel.  Resident blocks take items from their group's queue
// with an atomic ticket until it is empty; each item leaves one LSE state and
// a final kernel merges the states of each point in item order, so the
// result does not depend on which block took which item.  No block waits on
// another.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace rift {
namespace {

constexpr int kDefaultTile = 4096;  // draws per queue item unless tuned

// Marks LSE states as empty (m = -inf).
__global__ void fill_empty_kernel(LseState* __restrict__ st, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    st[i] = LseState{-CUDART_INF, 0.0, 0.0, 0.0};
}

// out[p] = (lnZ, sigma_lnZ, n_eff) from the states of point p's items
// [first[2p], first[2p+1]): one warp per point, two passes (the largest
// maximum, then the rescaled sums), each lane over a fixed strided subset and
// a fixed shuffle tree, so the exponentials pipeline and the result is
// reproducible.
__global__ void batch_combine_kernel(const LseState* __restrict__ partials,
                                     const int* __restrict__ first, const double* __restrict__ ndraws,
                                     int P, double* __restrict__ out) {
  const int p = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (p >= P) return;  // whole warps leave together
  const int i0 = first[2 * p], i1 = first[2 * p + 1];
  double M = -CUDART_INF;
  int bad = 0;
  for (int i = i0 + lane; i < i1; i += 32) {
    const double m = partials[i].m;
    if (isnan(m)) bad = 1;
    else M = fmax(M, m);
  }
  for (int off = 16; off > 0; off >>= 1) {
    M = fmax(M, __shfl_xor_sync(0xffffffffu, M, off));
    bad |= __shfl_xor_sync(0xffffffffu, bad, off);
  }
  double s = 0.0, s2 = 0.0;
  if (M > -CUDART_INF) {
    for (int i = i0 + lane; i < i1; i += 32) {
      const LseState q = partials[i];
      if (!(q.m > -CUDART_INF)) continue;
      const double e = lse_exp(q.m - M);
      s = fma(q.s, e, s);
      s2 = fma(q.s2, e * e, s2);
    }
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_down_sync(0xffffffffu, s, off);
    s2 += __shfl_down_sync(0xffffffffu, s2, off);
  }
  if (lane != 0) return;
  const double n = ndraws[p];
  double lnz, sig, neff;
  if (bad) {
    lnz = sig = neff = CUDART_NAN;
  } else if (n <= 0.0 || !(M > -CUDART_INF)) {
    lnz = -CUDART_INF;
    sig = CUDART_NAN;
    neff = 0.0;
  } else {
    lnz = M + log(s) - log(n);
    const double var = s2 / (s * s) - 1.0 / n;
    sig = sqrt(var > 0.0 ? var : 0.0);
    neff = s;
  }
  out[3 * p] = lnz;
  out[3 * p + 1] = sig;
  out[3 * p + 2] = neff;
}

template <typename T>
int alloc_copy(T** dst, const T* src, size_t count, const char* what) {
  if (cudaMalloc((void**)dst, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
    *dst = nullptr;
    rift_ile_set_error("rift_ile_batch_create: allocation of %s failed", what);
    return RIFT_ILE_ERR_ALLOC;
  }
  if (count && src) return check_cuda(cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice), what);
  return RIFT_ILE_OK;
}

}  // namespace
}  // namespace rift

using namespace rift;

struct rift_ile_batch {
  int P = 0;
  int prec = 0;
  // FP32-mixed persistent form
  const PointParams** d_pts = nullptr;
  DrawsParams* d_dps = nullptr;
  BatchItem* d_items = nullptr;
  int n_items = 0;
  int* d_first = nullptr;
  double* d_ndraws = nullptr;
  unsigned int* d_head = nullptr;  // one ticket counter per group
  LseState* d_partials = nullptr;
  unsigned long long* d_oob = nullptr;
  struct Group {
    BatchKernelFn kernel = nullptr;
    size_t smem = 0;
    int max_blocks = 0;  // resident-block limit of the kernel (SMs x occupancy)
    int item0 = 0, n_items = 0;
    std::vector<int> points;  // in queue order
  };
  std::vector<Group> groups;
  int quarters = 4;  // grid = quarters/4 of each group's resident-block limit
  int tile = 0;      // draws per queue item
  std::vector<long long> n_host;  // draw count of each point
  // FP64 per-point form
  std::vector<const rift_ile_point*> pts;
  std::vector<DrawsParams> dps;
  int parts_per_point = 0;
};

// (Re)builds the FP32-mixed work queues for items of `tile` draws: group by
// group, point by point, in draw order; the items of point p are
// [ranges[2p], ranges[2p+1]), one partial each.
static int build_queue(rift_ile_batch* b, int tile) {
  std::vector<BatchItem> items;
  std::vector<int> ranges(2 * b->P, 0);  // [first item, end) of each point
  for (auto& g : b->groups) {
    g.item0 = (int)items.size();
    for (int p : g.points) {
      ranges[2 * p] = (int)items.size();
      for (long long a = 0; a < b->n_host[p]; a += tile)
        items.push_back(BatchItem{a, (int)std::min<long long>(tile, b->n_host[p] - a), p});
      ranges[2 * p + 1] = (int)items.size();
    }
    g.n_items = (int)items.size() - g.item0;
  }
  cudaFree(b->d_items);
  cudaFree(b->d_first);
  cudaFree(b->d_partials);
  b->d_items = nullptr;
  b->d_first = nullptr;
  b->d_partials = nullptr;
  int rc = alloc_copy(&b->d_items, items.data(), items.size(), "work queue");
  if (!rc) rc = alloc_copy(&b->d_first, ranges.data(), ranges.size(), "item ranges");
  if (!rc) rc = alloc_copy(&b->d_partials, (LseState*)nullptr, items.size(), "partials");
  b->n_items = (int)items.size();
  b->tile = tile;
  return rc;
}

extern "C" int rift_ile_batch_destroy(rift_ile_batch* b) {
  if (!b) return RIFT_ILE_OK;
  cudaFree(b->d_pts);
  cudaFree(b->d_dps);
  cudaFree(b->d_items);
  cudaFree(b->d_first);
  cudaFree(b->d_ndraws);
  cudaFree(b->d_head);
  cudaFree(b->d_partials);
  cudaFree(b->d_oob);
  delete b;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_batch_create(const rift_ile_point* const* pts, const rift_ile_draws* draws,
                                     int32_t P, rift_ile_precision prec, rift_ile_batch** out) {
  if (!out || !pts || !draws || P < 1) {
    rift_ile_set_error("rift_ile_batch_create: bad arguments (P = %d)", P);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  *out = nullptr;
  if (prec != RIFT_ILE_FP64 && prec != RIFT_ILE_FP32_MIXED) {
    rift_ile_set_error("rift_ile_batch_create: bad precision %d", (int)prec);
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  rift_ile_batch* b = new rift_ile_batch();
  b->P = P;
  b->prec = prec;
  std::vector<const PointParams*> hp(P);
  std::vector<DrawsParams> hd(P);
  std::vector<double> nd(P);
  int rc = RIFT_ILE_OK;
  for (int p = 0; p < P && !rc; ++p) {
    const rift_ile_point* pt = pts[p];
    const rift_ile_draws* d = draws + p;
    if (!pt || d->n < 0 || (d->dtype != RIFT_ILE_F32 && d->dtype != RIFT_ILE_F64) ||
        (d->n > 0 && (!d->ra || !d->dec || !d->psi || !d->incl || !d->phase || !d->lnD || !d->t))) {
      rift_ile_set_error("rift_ile_batch_create: point or draws %d invalid", p);
      rc = RIFT_ILE_ERR_INVALID_ARG;
      break;
    }
    hp[p] = pt->dev;
    DrawsParams& dp = hd[p];
    dp.p[0] = d->ra;
    dp.p[1] = d->dec;
    dp.p[2] = d->psi;
    dp.p[3] = d->incl;
    dp.p[4] = d->phase;
    dp.p[5] = d->lnD;
    dp.p[6] = d->t;
    dp.logw = d->logw;
    dp.n = d->n;
    dp.f64 = (d->dtype == RIFT_ILE_F64);
    nd[p] = (double)d->n;
    b->pts.push_back(pt);
  }
  b->dps = hd;
  if (!rc && prec == RIFT_ILE_FP32_MIXED) {
    // one group per compiled kernel shape, in order of first appearance
    for (int p = 0; p < P && !rc; ++p) {
      const BatchKernelFn k = batch_kernel_for(pts[p]->host.M, pts[p]->host.R);
      if (!k) {
        rift_ile_set_error("rift_ile_batch_create: point %d has no kernel of width %d", p,
                           pts[p]->host.R);
        rc = RIFT_ILE_ERR_UNSUPPORTED;
        break;
      }
      size_t gi = 0;
      while (gi < b->groups.size() && b->groups[gi].kernel != k) ++gi;
      if (gi == b->groups.size()) {
        b->groups.emplace_back();
        b->groups.back().kernel = k;
      }
      auto& g = b->groups[gi];
      g.points.push_back(p);
      g.smem = std::max(g.smem, batch_smem_for(pts[p]->host.M, pts[p]->host.R, pts[p]->host.ncls,
                                               pts[p]->host.R, pts[p]->host.M, pts[p]->host.K));
    }
    for (auto& g : b->groups) {
      cudaFuncSetAttribute(g.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      g.max_blocks = grid_for(g.kernel, 128, g.smem);
    }
    b->n_host.resize(P);
    for (int p = 0; p < P; ++p) b->n_host[p] = hd[p].n;
    if (!rc) rc = alloc_copy(&b->d_pts, hp.data(), P, "point table");
    if (!rc) rc = alloc_copy(&b->d_dps, hd.data(), P, "draw table");
    if (!rc) rc = build_queue(b, kDefaultTile);
    if (!rc) rc = alloc_copy(&b->d_ndraws, nd.data(), P, "draw counts");
    if (!rc) rc = alloc_copy(&b->d_head, (unsigned int*)nullptr, b->groups.size(), "queue heads");
    if (!rc) rc = alloc_copy(&b->d_oob, (unsigned long long*)nullptr, 1, "counter");
  } else if (!rc) {
    // FP64: one fused lnL -> LSE launch per point into its own slice of partials
    b->parts_per_point = device_sms() * kMaxPartialsPerSM;
    std::vector<int> f2(2 * P);
    for (int p = 0; p < P; ++p) {
      f2[2 * p] = p * b->parts_per_point;
      f2[2 * p + 1] = (p + 1) * b->parts_per_point;
    }
    if (!rc) rc = alloc_copy(&b->d_first, f2.data(), 2 * P, "item ranges");
    if (!rc) rc = alloc_copy(&b->d_ndraws, nd.data(), P, "draw counts");
    if (!rc) rc = alloc_copy(&b->d_partials, (LseState*)nullptr, (size_t)P * b->parts_per_point, "partials");
    if (!rc) rc = alloc_copy(&b->d_oob, (unsigned long long*)nullptr, 1, "counter");
  }
  if (rc) {
    rift_ile_batch_destroy(b);
    return rc;
  }
  *out = b;
  return RIFT_ILE_OK;
}

extern "C" int rift_ile_batch_launch(rift_ile_batch* b, double* out, void* stream) {
  if (!b || !out) {
    rift_ile_set_error("rift_ile_batch_launch: NULL argument");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc;
  if ((rc = check_cuda(cudaMemsetAsync(b->d_oob, 0, sizeof(unsigned long long), st), "batch clear")))
    return rc;
  if (b->prec == RIFT_ILE_FP32_MIXED) {
    if ((rc = check_cuda(cudaMemsetAsync(b->d_head, 0, b->groups.size() * sizeof(unsigned int), st),
                         "batch clear")))
      return rc;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
      const auto& g = b->groups[gi];
      if (g.n_items == 0) continue;
      const int blocks = std::max(1, g.max_blocks * b->quarters / 4);
      g.kernel<<<blocks, 128, g.smem, st>>>(b->d_pts, b->d_dps, b->d_items + g.item0, g.n_items,
                                            b->d_head + gi, b->d_partials + g.item0, b->d_oob);
      if ((rc = check_cuda(cudaGetLastError(), "batch kernel launch"))) return rc;
    }
  } else {
    // FP64: the plain path, one launch per point; unused partial slots are
    // empty states
    const long long np = (long long)b->P * b->parts_per_point;
    fill_empty_kernel<<<(int)std::min<long long>((np + 255) / 256, 4096), 256, 0, st>>>(b->d_partials, np);
    if ((rc = check_cuda(cudaGetLastError(), "batch clear"))) return rc;
    for (int p = 0; p < b->P; ++p) {
      if (b->dps[p].n == 0) continue;
      int blocks = 0;
      cudaError_t e = launch_lnl_fp64(b->pts[p]->host, b->pts[p]->dev, b->dps[p], nullptr,
                                      b->d_partials + (size_t)p * b->parts_per_point, b->d_oob,
                                      &blocks, st);
      if ((rc = check_cuda(e, "batch FP64 launch"))) return rc;
    }
  }
  batch_combine_kernel<<<(b->P + 3) / 4, 128, 0, st>>>(b->d_partials, b->d_first, b->d_ndraws,
                                                       b->P, out);
  return check_cuda(cudaGetLastError(), "batch combine launch");
}

extern "C" int rift_ile_batch_tune(rift_ile_batch* b, int32_t reps, void* stream,
                                   int32_t* tile_out, int32_t* blocks_out, double* ms_out) {
  if (!b || reps < 1) {
    rift_ile_set_error("rift_ile_batch_tune: NULL batch or reps < 1");
    return RIFT_ILE_ERR_INVALID_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  int rc = RIFT_ILE_OK;
  double best_ms = -1.0;
  int best_tile = b->tile, best_quarters = b->quarters;
  if (b->prec == RIFT_ILE_FP32_MIXED && b->n_items > 0) {
    double* out = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaMalloc((void**)&out, (size_t)3 * b->P * sizeof(double)) != cudaSuccess) {
      rift_ile_set_error("rift_ile_batch_tune: allocation failed");
      return RIFT_ILE_ERR_ALLOC;
    }
    rc = check_cuda(cudaEventCreate(&e0), "tune events");
    if (!rc) rc = check_cuda(cudaEventCreate(&e1), "tune events");
    static const int kTiles[] = {512, 1024, 2048, 4096, 8192, 16384};
    static const int kQuarters[] = {4, 3, 2};
    for (int ti = 0; ti < 6 && !rc; ++ti) {
      rc = build_queue(b, kTiles[ti]);
      for (int qi = 0; qi < 3 && !rc; ++qi) {
        b->quarters = kQuarters[qi];
        rc = rift_ile_batch_launch(b, out, stream);  // warm-up
        if (!rc) rc = check_cuda(cudaEventRecord(e0, st), "tune timing");
        for (int r = 0; r < reps && !rc; ++r) rc = rift_ile_batch_launch(b, out, stream);
        if (!rc) rc = check_cuda(cudaEventRecord(e1, st), "tune timing");
        if (!rc) rc = check_cuda(cudaEventSynchronize(e1), "tune timing");
        float ms = 0.f;
        if (!rc) rc = check_cuda(cudaEventElapsedTime(&ms, e0, e1), "tune timing");
        if (!rc && (best_ms < 0.0 || ms / reps < best_ms)) {
          best_ms = ms / reps;
          best_tile = kTiles[ti];
          best_quarters = b->quarters;
        }
      }
    }
    if (!rc) rc = build_queue(b, best_tile);
    b->quarters = best_quarters;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(out);
  }
  if (tile_out) *tile_out = b->tile;
  if (blocks_out) {  // blocks of the largest group's launch
    int bl = 0;
    size_t big = 0;
    for (const auto& g : b->groups)
      if ((size_t)g.n_items >= big) {
        big = g.n_items;
        bl = std::max(1, g.max_blocks * b->quarters / 4);
      }
    *blocks_out = bl;
  }
  if (ms_out) *ms_out = best_ms;
  return rc;
}

extern "C" int rift_ile_lnZ_batch(const rift_ile_point* const* pts, const rift_ile_draws* draws,
                                  int32_t P, rift_ile_precision prec, double* out, void* stream) {
  rift_ile_batch* b = nullptr;
  int rc = rift_ile_batch_create(pts, draws, P, prec, &b);
  if (rc) return rc;
  rc = rift_ile_batch_launch(b, out, stream);
  if (!rc) rc = check_cuda(cudaStreamSynchronize((cudaStream_t)stream), "rift_ile_lnZ_batch");
  rift_ile_batch_destroy(b);
  return rc;
}
