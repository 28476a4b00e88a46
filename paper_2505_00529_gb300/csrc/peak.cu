// Binary64 FMA rate of the device: the denominator of the roofline of the
// binary64-bound kernels (eigendecomposition refinement, derivative
// preparation), measured rather than taken from unit counts.
//
// Every thread runs kChains independent FMA chains of kIters steps on values
// that stay finite (x <- x * a + b with |a| < 1), so the issue rate, not the
// latency of one chain, bounds the kernel; the sum of the chains is written
// out so that nothing is eliminated.  One launch covers `ctas_per_sm` CTAs of
// 256 threads per SM.
//
// Also the failure-detection self-test: the bounded mbarrier wait of the
// sweeps, run on a barrier that nothing completes.
#include <cuda_runtime.h>

#include "common.cuh"
#include "kernels.hpp"
#include "qoc.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) k_fp64_fma_rate(double a, double b, double* out) {
  double x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = 1.0 + 1e-3 * (threadIdx.x + c);
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
  }
  double s = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// One warp: thread 0 initialises an mbarrier expecting one arrival that never
// comes (no copy is issued), every thread waits on it with the sweeps' bounded
// wait, and the first to give up raises DEV_TIMEOUT.
__global__ void k_wait_selftest(int* status, unsigned long long limit_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    qoc::mbar_init(&bar, 1);
    qoc::mbar_fence_init();
  }
  __syncthreads();
  const bool ok = qoc::mbar_wait_bounded(&bar, 0, limit_ns);
  if (!__all_sync(0xffffffffu, ok) && threadIdx.x == 0) qoc::raise_status(status, qoc::DEV_TIMEOUT);
}

}  // namespace

namespace qoc {
cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(status, limit_ns);
  return cudaGetLastError();
}
}  // namespace qoc

extern "C" qoc_status qoc_measure_fp64_rate(int ctas_per_sm, int repeats, double* tflops, double* ms) {
  if (!tflops || ctas_per_sm < 1 || ctas_per_sm > 64 || repeats < 1) return QOC_EINVAL;
  const int grid = qoc::num_sms() * ctas_per_sm, threads = 256;
  double* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(double) * (size_t)grid * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best = 0.f;
  if (e == cudaSuccess) {
    k_fp64_fma_rate<<<grid, threads>>>(0.999, 1e-3, out);   // warm-up
    for (int r = 0; r < repeats && e == cudaSuccess; ++r) {
      cudaEventRecord(e0);
      k_fp64_fma_rate<<<grid, threads>>>(0.999, 1e-3, out);
      cudaEventRecord(e1);
      e = cudaEventSynchronize(e1);
      float t = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
      if (e == cudaSuccess && (best == 0.f || t < best)) best = t;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    qoc::note_error(cudaGetErrorString(e));
    return QOC_ECUDA;
  }
  const double flops = 2.0 * kChains * kIters * (double)grid * threads;
  *tflops = flops / (best * 1e-3) / 1e12;
  if (ms) *ms = best;
  return QOC_OK;
}
