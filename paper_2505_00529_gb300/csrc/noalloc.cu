// Gradient and Hessian assembly with no device allocation.
//
// Some callers cannot call cudaMalloc at the moment they need the result:
// code that runs while a stream is being captured into a CUDA graph in a
// mode that forbids allocation, code whose framework hands every byte of
// device memory to its own pool (so a raw allocation fails or fragments it),
// and latency-bound loops that must not take the implicit device
// synchronisation an allocation can cause.  They pass inputs and outputs
// they already own; the Hessian assembly's partial sums over chunks of
// steps then go to the fixed array below instead of a buffer of a
// qoc_problem.
//
// The array lives in this library's device image: every GPU on which the
// library is loaded holds it (QOC_NOALLOC_SCRATCH_DOUBLES doubles) until the
// process exits.  All calls share it and it keeps the last call's contents;
// every element a call reads is written earlier by the same call, so nothing
// is cleared.  Calls whose kernels overlap on a GPU (different streams, no
// ordering between them) race on the array.
#include <cuda_runtime.h>

#include <cstdio>
#include <mutex>

#include "kernels.hpp"
#include "qoc.h"

namespace {

static __device__ __align__(256) double noalloc_scratch[QOC_NOALLOC_SCRATCH_DOUBLES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {};

// Device address of the array on the current device.  Outside a stream
// capture the address is looked up again on every call and the per-device
// copy refreshed: the library's device image is reloaded, possibly at another
// address, when the device's primary context is destroyed and recreated (for
// example after cudaDeviceReset), so a copy kept from before would be stale.
// While `st` is being captured the copy from the last uncaptured call is
// used, because the lookup may load the module, which a capture does not
// allow; a first call on a device that comes during a capture is refused.
cudaError_t scratch_address(cudaStream_t st, double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_mu);
  if (cap == cudaStreamCaptureStatusNone) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<double*>(ptr);
  }
  if (!g_scratch[dev]) return cudaErrorStreamCaptureUnsupported;
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" size_t qoc_assemble_noalloc_scratch_doubles(int steps, int K) {
  if (steps < 1 || K < 1) return 0;
  return qoc::assemble_work_doubles(steps, K) + (size_t)K * K + 1;
}

extern "C" qoc_status qoc_assemble_grad_hess_noalloc(int steps, int K, const double* basis_dev,
                                                      const double* f_dev, const double* g_dev,
                                                      const double* c_dev, const double* U_dev,
                                                      const double* V_dev, double w_ctrl,
                                                      double* out_dev, void* cuda_stream) {
  if (steps < 1 || K < 1 || !basis_dev || !f_dev || !g_dev || !c_dev || !U_dev || !V_dev || !out_dev)
    return QOC_EINVAL;
  const size_t need = qoc_assemble_noalloc_scratch_doubles(steps, K);
  if (need > (size_t)QOC_NOALLOC_SCRATCH_DOUBLES) {
    char msg[200];
    std::snprintf(msg, sizeof(msg),
                  "qoc_assemble_grad_hess_noalloc: steps=%d, K=%d need %zu scratch doubles, the "
                  "maximum is %d",
                  steps, K, need, (int)QOC_NOALLOC_SCRATCH_DOUBLES);
    qoc::note_error(msg);
    return QOC_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_address(static_cast<cudaStream_t>(cuda_stream), &scratch);
  if (e == cudaSuccess) {
    const size_t nwork = qoc::assemble_work_doubles(steps, K);
    double* hess_raw = scratch + nwork;
    double* asym = hess_raw + (size_t)K * K;
    e = qoc::launch_assemble(basis_dev, K, f_dev, g_dev, c_dev, V_dev, U_dev, 0, nullptr, 0, steps, K,
                             w_ctrl, 0.0, 0, 1, scratch, out_dev, hess_raw, asym,
                             static_cast<cudaStream_t>(cuda_stream));
  }
  if (e == cudaSuccess) return QOC_OK;
  char msg[200];
  std::snprintf(msg, sizeof(msg), "%s: %s (noalloc.cu)", cudaGetErrorName(e), cudaGetErrorString(e));
  qoc::note_error(msg);
  return QOC_ECUDA;
}
