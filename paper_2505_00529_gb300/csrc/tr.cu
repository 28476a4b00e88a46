// Trust-region subproblem on the device (Sec. IV-B: exact gradient and
// Hessian from Alg. 2 fed to a trust-region Newton method; the paper uses a
// library trust-region solver without giving its internals, so this is the
// textbook exact subproblem).
//
// Given the eigendecomposition Hess = Q diag(d) Q^T (computed by the same
// Jacobi kernel as the step Hamiltonians) and g = grad J:
//   minimise g^T s + s^T Hess s / 2 subject to |s| <= radius
// s(sigma) = -Q (Q^T g) / (d + sigma) with sigma >= max(0, -d_min) solving
// |s(sigma)| = radius (Newton on 1/|s| - 1/radius, safeguarded by a
// bracket), sigma = 0 when Hess is positive definite and the Newton step
// fits, and the "hard case" (g orthogonal to the lowest eigenspace) closed
// with a multiple of the lowest eigenvector.  One CTA, binary64.
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

__device__ double block_sum(double v, double* red) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  double s = 0;
  const int nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nw; ++k) s += red[k];
  return s;
}

// work layout: [0..K) gt, [K..2K) st
// info: [0] predicted decrease, [1] |s|, [2] sigma, [3] |g|
__global__ void k_tr_subproblem(const double* __restrict__ gh, const double* __restrict__ Q,
                                const double* __restrict__ d, int K, double radius,
                                double* __restrict__ work, double* __restrict__ step,
                                double* __restrict__ info, int* status) {
  __shared__ double red[32];
  double* gt = work;
  double* st = work + K;
  const double* g = gh + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  double gn = 0;
  for (int q = tid; q < K; q += nt) {
    double acc = 0;
    for (int p = 0; p < K; ++p) acc = fma(Q[(size_t)p * K + q], g[p], acc);
    gt[q] = acc;
    gn = fma(g[q], g[q], gn);
  }
  gn = sqrt(block_sum(gn, red));
  __syncthreads();
  const double dmin = d[0];
  double sigma = 0.0;
  bool done = false;
  if (dmin > 0) {
    double ns = 0;
    for (int q = tid; q < K; q += nt) {
      double v = -gt[q] / d[q];
      st[q] = v;
      ns = fma(v, v, ns);
    }
    ns = sqrt(block_sum(ns, red));
    if (ns <= radius) done = true;
  }
  const double lo = fmax(0.0, -dmin);
  if (!done) {
    // hard case?
    const double tol = 1e-12 * fmax(1.0, fabs(dmin));
    double gm = 0, gall = 0;
    int first = K;
    for (int q = 0; q < K; ++q) {   // small K: every thread scans (no divergence in results)
      if (fabs(d[q] - dmin) <= tol) { gm = fma(gt[q], gt[q], gm); if (first == K) first = q; }
      gall = fma(gt[q], gt[q], gall);
    }
    if (sqrt(gm) <= 1e-14 * fmax(1.0, sqrt(gall))) {
      double ns = 0;
      for (int q = tid; q < K; q += nt) {
        double v = (fabs(d[q] - dmin) <= tol) ? 0.0 : -gt[q] / (d[q] + lo);
        st[q] = v;
        ns = fma(v, v, ns);
      }
      ns = block_sum(ns, red);
      if (sqrt(ns) <= radius) {
        __syncthreads();
        if (tid == 0) st[first] += sqrt(fmax(radius * radius - ns, 0.0));
        sigma = lo;
        done = true;
      }
    }
  }
  if (!done) {
    auto snorm = [&](double sig) {
      double ns = 0;
      for (int q = tid; q < K; q += nt) {
        double v = gt[q] / (d[q] + sig);
        ns = fma(v, v, ns);
      }
      return sqrt(block_sum(ns, red));
    };
    double hi = lo + gn / radius + 1.0;
    for (int k = 0; k < 200 && snorm(hi) > radius; ++k) hi *= 2.0;
    double sig = hi, slo = lo;
    for (int itn = 0; itn < 200; ++itn) {
      double ns = 0, dd = 0;
      for (int q = tid; q < K; q += nt) {
        double den = d[q] + sig;
        double v = gt[q] / den;
        ns = fma(v, v, ns);
        dd += gt[q] * gt[q] / (den * den * den);
      }
      ns = sqrt(block_sum(ns, red));
      dd = block_sum(dd, red);
      if (fabs(ns - radius) <= 1e-13 * radius) break;
      double phi = 1.0 / ns - 1.0 / radius;
      if (phi < 0) slo = sig; else hi = sig;
      double dns = -dd / ns;
      double dphi = -dns / (ns * ns);
      double nw = sig - phi / dphi;
      if (!(nw > slo && nw < hi)) nw = 0.5 * (slo + hi);
      sig = nw;
    }
    for (int q = tid; q < K; q += nt) st[q] = -gt[q] / (d[q] + sig);
    sigma = sig;
  }
  __syncthreads();
  // predicted decrease in eigen-coordinates, |s|, and s = Q st
  double pr = 0, ns = 0;
  for (int q = tid; q < K; q += nt) {
    pr += gt[q] * st[q] + 0.5 * d[q] * st[q] * st[q];
    ns = fma(st[q], st[q], ns);
  }
  pr = block_sum(pr, red);
  ns = block_sum(ns, red);
  for (int p = tid; p < K; p += nt) {
    double acc = 0;
    for (int q = 0; q < K; ++q) acc = fma(Q[(size_t)p * K + q], st[q], acc);
    step[p] = acc;
    if (!isfinite(acc)) raise_status(status, DEV_NONFINITE);
  }
  if (tid == 0) {
    info[0] = -pr;
    info[1] = sqrt(ns);
    info[2] = sigma;
    info[3] = gn;
  }
}

__global__ void k_axpy(const double* __restrict__ x, const double* __restrict__ s, int K,
                       double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) y[i] = x[i] + s[i];
}

size_t tr_work_doubles(int K) { return 3 * (size_t)K + (size_t)K * K; }

cudaError_t launch_tr_subproblem(const double* out_gh, int K, double radius, double* work,
                                 double* step, double* info, int* status, cudaStream_t st) {
  // eigendecomposition of the Hessian is expected in work + 2K (d) and work + 3K (Q)
  const double* d = work + 2 * K;
  const double* Q = work + 3 * K;
  k_tr_subproblem<<<1, 128, 0, st>>>(out_gh, Q, d, K, radius, work, step, info, status);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double* x, const double* s, int K, double* y, cudaStream_t st) {
  k_axpy<<<(K + 127) / 128, 128, 0, st>>>(x, s, K, y);
  return cudaGetLastError();
}

}  // namespace qoc
