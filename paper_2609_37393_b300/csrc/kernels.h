// Kernel launchers of the library (each returns the launch status).  The grid
// is a fixed number of resident blocks per SM for the kernel (occupancy API),
// written to *blocks; partials, when non-NULL, receives one LSE state per
// block (at most kMaxPartialsPerSM per SM) and switches the kernel to the
// fused lnZ form.
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "rift_ile_internal.h"

namespace rift {

constexpr int kMaxPartialsPerSM = 16;

cudaError_t launch_lnl_fp64(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                            double* lnl_out, LseState* partials, unsigned long long* oob,
                            int* blocks, cudaStream_t st);
cudaError_t launch_lnl_mixed(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                             double* lnl_out, LseState* partials, unsigned long long* oob,
                             int* blocks, cudaStream_t st);
// One work item of the batched lnZ: draws [begin, begin + count) of a point.
struct BatchItem {
  long long begin;
  int count;
  int point;
};
typedef void (*BatchKernelFn)(const PointParams* const*, const DrawsParams*, const BatchItem*, int,
                              unsigned int*, LseState*, unsigned long long*);
// The persistent FP32-mixed batch kernel for points of M modes and padded
// whitened width R (nullptr if no kernel has exactly that width); launched
// with 128 threads.
BatchKernelFn batch_kernel_for(int M, int R);
// Its dynamic shared memory for one point (ncls classes, width Rp, Mp modes,
// Kp detectors).
size_t batch_smem_for(int M, int R, int ncls, int Rp, int Mp, int Kp);

// lnL (lnl_out may be NULL) and its gradient, grad_out[7][n].
cudaError_t launch_grad_mixed(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                              double* lnl_out, double* grad_out, cudaStream_t st);
cudaError_t launch_grad_fp64(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                             double* lnl_out, double* grad_out, cudaStream_t st);
// Distance-marginalised lnL (per draw into lnl_out, or fused into partials).
cudaError_t launch_lnl_fp64_dist(const PointParams& hp, const PointParams* dP,
                                 const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                 LseState* partials, unsigned long long* oob, int* blocks,
                                 cudaStream_t st);
cudaError_t launch_lnl_mixed_dist(const PointParams& hp, const PointParams* dP,
                                  const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                  LseState* partials, unsigned long long* oob, int* blocks,
                                  cudaStream_t st);
cudaError_t launch_grad_fp64_dist(const PointParams& hp, const PointParams* dP,
                                  const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                  double* grad_out, cudaStream_t st);
cudaError_t launch_grad_mixed_dist(const PointParams& hp, const PointParams* dP,
                                   const DrawsParams& dp, const DistParams& dist, double* lnl_out,
                                   double* grad_out, cudaStream_t st);
cudaError_t launch_lse_combine(const LseState* partials, int nparts, double n_total,
                               LseState* state_out, cudaStream_t st);

// Builds the shared-memory image of the FP32-mixed tables of a point (hp
// complete apart from img); *img is a new device buffer of *nf4 float4.
int build_mixed_image(const PointParams& hp, float4** img, int* nf4, cudaStream_t st);
// Host helpers of point.cu shared with the composite response: the cyclic
// Jacobi eigen-decomposition of a symmetric n x n matrix (row-major, destroyed;
// eigenvectors in the columns of V), the harmonic's polynomial in cos(iota)
// (returns its parity), and the (hi, lo) float split of a double.
void jacobi_eigen(int n, std::vector<double>& a, std::vector<double>& lam, std::vector<double>& V);
int harmonic_zpoly(int l, int nt, int k0, const double* coef, double* out);
void split_df(double x, float* hi, float* lo);
// The whitened tables of K detectors from a complex table Q [K][n][Mq]
// (complex128 if q_c128, else complex64; device): with the eigenvectors Vt
// [ncls][2 Mq][2 Mq] (rows, host) and the scales inv_s [K][R] (host; zero for
// dropped or padding directions), writes ehat [K][n + 2 kEhatPad][R], the
// interval polynomials epoly [K][n + 3][7] and the intervals' cubic
// coefficients ecub [ecub_f4(K, n, R)] (device, caller-allocated; R even) and
// synchronises st.
int whitened_tables(const void* Q, int q_c128, int K, int n, int Mq, int ncls, const int* cls_of,
                    const double* Vt, const double* inv_s, int R, float2* ehat, float2* epoly,
                    float4* ecub, cudaStream_t st);
// SM count of the current device (cached).
int device_sms();
// Draw count up to which FP32-mixed lnL and lnL + gradient calls (no
// distance table) run the warp-per-draw kernel (rift_ile_set_small_batch).
long long small_batch_max();

// The library's per-device scratch (LSE partials, combined state, tap
// counter), allocated on first use; draw validation and marshalling; the
// thread-local out-of-table tap count reported by rift_ile_last_oob.
int lse_workspace(LseState** partials, LseState** state, unsigned long long** oob);
int validate_draws(const rift_ile_draws* d);
DrawsParams draws_params(const rift_ile_draws* d);
void set_last_oob(long long v);
// Drops the cached device addresses of the allocation-free entry point's scratch (rift_ile_release).
void forget_noalloc_scratch();
// One batched in-place double-complex transform with the cached cuFFT plan of
// (device, nfft, batch): direction < 0 forward (e^{-2 pi i}), else inverse
// (e^{+2 pi i}, unnormalised).  Thread-safe; asynchronous on st.
int fft_z2z_inplace(double2* data, long long nfft, int batch, int direction, cudaStream_t st);
// Destroys the cuFFT plans the precompute keeps (rift_ile_release).
void release_fft_plans();

// Grid of a per-draw kernel: SMs x resident blocks per SM, capped so that the
// per-block partials fit the workspace.  Fixed for a given device and build,
// so results do not depend on the launch history.
template <typename KernelT>
int grid_for(KernelT kernel, int threads, size_t smem) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1)
    nb = 1;
  if (nb > kMaxPartialsPerSM) nb = kMaxPartialsPerSM;
  return device_sms() * nb;
}

// A grid-stride launch needs no more blocks than there are draws to cover
// (small batches: fewer idle blocks and fewer partials to merge).
inline int grid_cap(int blocks, long long n, int threads) {
  const long long need = (n + threads - 1) / threads;
  return (int)(need < blocks ? (need > 0 ? need : 1) : blocks);
}

// The same launches with the SM count given by the caller, for code that must
// not touch the library's workspace (grid = sms x resident blocks per SM, at
// most kMaxPartialsPerSM per SM).
template <typename KernelT>
int grid_for_sms(KernelT kernel, int threads, size_t smem, int sms) {
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, threads, smem) != cudaSuccess || nb < 1)
    nb = 1;
  if (nb > kMaxPartialsPerSM) nb = kMaxPartialsPerSM;
  return sms * nb;
}
cudaError_t launch_lnl_fp64_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                double* lnl_out, LseState* partials, unsigned long long* oob,
                                int sms, int* blocks, cudaStream_t st);
cudaError_t launch_lnl_mixed_sms(const PointParams& hp, const PointParams* dP, const DrawsParams& dp,
                                 double* lnl_out, LseState* partials, unsigned long long* oob,
                                 int sms, int* blocks, cudaStream_t st);

}  // namespace rift
