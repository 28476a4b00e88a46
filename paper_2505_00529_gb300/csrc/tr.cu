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
#include "qoc.h"

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
// (the body of one CTA; `red` is 32 doubles of shared memory)
__device__ void tr_subproblem_body(const double* __restrict__ gh, const double* __restrict__ Q,
                                   const double* __restrict__ d, int K, double radius,
                                   double* __restrict__ work, double* __restrict__ step,
                                   double* __restrict__ info, int* status, double* red) {
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
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The same subproblem without the eigendecomposition (K >= kTriMin): the
// Hessian is reduced to tridiagonal form T = Q^T Hess Q by Householder
// reflections (Golub & Van Loan, Sec. 8.3.1), the secular equation is solved
// on T with tridiagonal LDL^T solves of (T + sigma I) x = -Q^T g, and the step
// is mapped back with Q.  The lowest eigenvalue of T (the bracket of sigma)
// comes from bisection on Sturm sequence counts; in the hard case its
// eigenvector comes from inverse iteration.  The reduction costs 4K^3/3
// flops where the binary64 Jacobi costs about ten sweeps of 3K^3.
// work: [gt K | st K | a K | b K | beta K | u K | w K | z K | A K*K] (8K + K*K)
// ---------------------------------------------------------------------------

// (T + sigma I) x = r by LDL^T without pivoting (T + sigma I positive
// definite); l, dd: K scratch each.  One thread.
__device__ void tri_solve(const double* a, const double* b, int K, double sigma, const double* r,
                          double* x, double* l, double* dd) {
  dd[0] = a[0] + sigma;
  x[0] = r[0];
  for (int i = 1; i < K; ++i) {
    l[i] = b[i - 1] / dd[i - 1];
    dd[i] = (a[i] + sigma) - l[i] * b[i - 1];
    x[i] = r[i] - l[i] * x[i - 1];
  }
  x[K - 1] = x[K - 1] / dd[K - 1];
  for (int i = K - 2; i >= 0; --i) x[i] = x[i] / dd[i] - l[i + 1] * x[i + 1];
}

// Binary32 version of tri_solve for the secular equation's starting point;
// l is recomputed from dd in the backward pass, so only dd is stored.
__device__ void tri_solve_f(const float* a, const float* b, int K, float sigma, const float* r, float* x,
                            float* dd) {
  dd[0] = a[0] + sigma;
  x[0] = r[0];
  for (int i = 1; i < K; ++i) {
    const float l = __fdividef(b[i - 1], dd[i - 1]);
    dd[i] = (a[i] + sigma) - l * b[i - 1];
    x[i] = r[i] - l * x[i - 1];
  }
  x[K - 1] = __fdividef(x[K - 1], dd[K - 1]);
  for (int i = K - 2; i >= 0; --i) x[i] = __fdividef(x[i], dd[i]) - __fdividef(b[i], dd[i]) * x[i + 1];
}

// number of eigenvalues of T below x (Sturm sequence of the LDL^T pivots);
// b2[i] = b[i]^2
__device__ int sturm_count(const double* a, const double* b2, int K, double x) {
  int cnt = 0;
  double q = a[0] - x;
  if (q < 0) ++cnt;
  for (int i = 1; i < K; ++i) {
    if (q == 0) q = 1e-300;
    q = (a[i] - x) - b2[i - 1] / q;
    if (q < 0) ++cnt;
  }
  return cnt;
}

__device__ double dot_norm(const double* x, int K) {
  double s = 0;
  for (int i = 0; i < K; ++i) s = fma(x[i], x[i], s);
  return sqrt(s);
}

// sw: the same work area in this CTA's shared memory (rows of A padded to
// K + 1 doubles, so that the threads' row-wise matrix-vector reads fall in
// different banks) when it fits, else nullptr and `work` is used
__device__ void tr_subproblem_tri_body(const double* __restrict__ gh, int K, double radius,
                                       double* __restrict__ work, double* __restrict__ step,
                                       double* __restrict__ info, int* status, double* red,
                                       double* sw = nullptr) {
  if (sw) work = sw;
  const int lda = sw ? K + 1 : K;
  double* gt = work;
  double* st = gt + K;
  double* a = st + K;
  double* b = a + K;
  double* bet = b + K;
  double* u = bet + K;
  double* w = u + K;
  double* z = w + K;
  double* A = z + K;
  const double* H = gh + 1 + K;
  const double* g = gh + 1;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < K * K; e += nt) A[(size_t)(e / K) * lda + e % K] = H[e];
  for (int l = tid; l < K; l += nt) gt[l] = g[l];
  __syncthreads();
  // ---- Householder reduction: column k below the diagonal -> b_k e_1 ----
  for (int k = 0; k + 2 < K; ++k) {
    const int n = K - k - 1;
    double xs = 0;
    for (int i = tid; i < n; i += nt) {
      const double x = A[(size_t)(k + 1 + i) * lda + k];
      xs = fma(x, x, xs);
    }
    xs = block_sum(xs, red);
    const double x0 = A[(size_t)(k + 1) * lda + k];
    const double nrm = sqrt(xs);
    const double alpha = x0 >= 0 ? -nrm : nrm;
    const double vtv = xs - 2.0 * alpha * x0 + alpha * alpha;
    const double beta = (nrm > 0 && vtv > 0) ? 2.0 / vtv : 0.0;
    for (int i = tid; i < n; i += nt) u[i] = i == 0 ? x0 - alpha : A[(size_t)(k + 1 + i) * lda + k];
    if (tid == 0) {
      a[k] = A[(size_t)k * lda + k];
      b[k] = beta != 0.0 ? alpha : x0;
      bet[k] = beta;
    }
    __syncthreads();
    if (beta != 0.0) {
      // p = beta A22 u, then w = p - (beta/2)(p^T u) u, A22 -= u w^T + w u^T
      double pu = 0;
      for (int i = tid; i < n; i += nt) {
        const double* row = A + (size_t)(k + 1 + i) * lda + (k + 1);
        double acc = 0;
        for (int j = 0; j < n; ++j) acc = fma(row[j], u[j], acc);
        w[i] = beta * acc;
        pu = fma(w[i], u[i], pu);
      }
      pu = block_sum(pu, red);
      const double c = 0.5 * beta * pu;
      for (int i = tid; i < n; i += nt) w[i] -= c * u[i];
      __syncthreads();
      for (int e = tid; e < n * n; e += nt) {
        const int i = e / n, j = e % n;
        A[(size_t)(k + 1 + i) * lda + (k + 1 + j)] -= u[i] * w[j] + w[i] * u[j];
      }
    }
    // the reflector's vector replaces column k below the diagonal
    for (int i = tid; i < n; i += nt) A[(size_t)(k + 1 + i) * lda + k] = u[i];
    __syncthreads();
  }
  if (tid == 0) {
    if (K >= 2) {
      a[K - 2] = A[(size_t)(K - 2) * lda + (K - 2)];
      b[K - 2] = A[(size_t)(K - 1) * lda + (K - 2)];
    }
    a[K - 1] = A[(size_t)(K - 1) * lda + (K - 1)];
  }
  __syncthreads();
  // ---- gt = Q^T g: reflectors 0 .. K-3 in order, by one warp (a chain of
  // short dot products: warp shuffles instead of a block barrier each) ----
  if (tid < 32) {
    for (int k = 0; k + 2 < K; ++k) {
      const int n = K - k - 1;
      const double beta = bet[k];
      if (beta == 0.0) continue;   // uniform
      double vg = 0;
      for (int i = tid; i < n; i += 32) vg = fma(A[(size_t)(k + 1 + i) * lda + k], gt[k + 1 + i], vg);
      vg = warp_sum(vg);
      for (int i = tid; i < n; i += 32) gt[k + 1 + i] -= beta * vg * A[(size_t)(k + 1 + i) * lda + k];
      __syncwarp();
    }
  }
  __syncthreads();
  // ---- lowest eigenvalue of T: multisection of the Gershgorin bracket, mp
  // threads taking one Sturm count each per round (the interval shrinks
  // mp + 1 fold).  At most 128 points: every warp issuing a binary64 Sturm
  // chain occupies its sub-partition's pipe, so a second warp per
  // sub-partition costs as much as it gains.  Down to 1e-13 of the values
  // (the hard case shifts by 1e-12 of |lambda_min|).  b^2 in w (free until
  // the secular equation). ----
  __shared__ double ms_lo, ms_hi;
  __shared__ int ms_first;
  const int mp = nt < 128 ? nt : 128;
  for (int i = tid; i + 1 < K; i += nt) w[i] = b[i] * b[i];
  if (tid == 0) {
    double glo = a[0], ghi = a[0];
    for (int i = 0; i < K; ++i) {
      const double r = (i > 0 ? fabs(b[i - 1]) : 0.0) + (i + 1 < K ? fabs(b[i]) : 0.0);
      glo = fmin(glo, a[i] - r);
      ghi = fmax(ghi, a[i] + r);
    }
    ms_lo = glo;
    ms_hi = ghi;
  }
  __syncthreads();
  for (int round = 0; round < 64; ++round) {
    const double lo = ms_lo, hi = ms_hi;
    if (!(hi - lo > 1e-13 * fmax(fabs(lo), fabs(hi)) + 1e-300)) break;   // uniform
    if (tid == 0) ms_first = mp;
    __syncthreads();
    if (tid < mp) {
      const double x = lo + (hi - lo) * ((double)(tid + 1) / (double)(mp + 1));
      if (x > lo && x < hi && sturm_count(a, w, K, x) >= 1) atomicMin(&ms_first, tid);
    }
    __syncthreads();
    if (tid == 0) {
      const int t = ms_first;   // smallest point with an eigenvalue below it
      const double nlo = t == 0 ? lo : lo + (hi - lo) * ((double)t / (double)(mp + 1));
      const double nhi = t == mp ? hi : lo + (hi - lo) * ((double)(t + 1) / (double)(mp + 1));
      ms_lo = nlo;
      ms_hi = nhi;
    }
    __syncthreads();
  }
  const double dmin = 0.5 * (ms_lo + ms_hi);
  // ---- secular equation on T (one thread) ----
  if (tid == 0) {
    const double gn = dot_norm(gt, K);
    double sigma = 0.0;
    bool done = false;
    for (int i = 0; i < K; ++i) z[i] = -gt[i];
    if (dmin > 0) {
      tri_solve(a, b, K, 0.0, z, st, u, w);
      if (dot_norm(st, K) <= radius) done = true;
    }
    const double slo0 = fmax(0.0, -dmin);
    if (!done) {
      // hard case: g (nearly) orthogonal to the lowest eigenvector, so that the
      // step stays inside the region as sigma approaches its lower limit
      const double sh = slo0 + 1e-12 * fmax(1.0, fabs(dmin));
      tri_solve(a, b, K, sh, z, st, u, w);
      const double nh = dot_norm(st, K);
      if (nh <= radius) {
        // eigenvector of the lowest eigenvalue by inverse iteration on T + sh I
        // (tri_solve may run in place: x[i] reads r[i] before writing it)
        double* v = z;
        for (int i = 0; i < K; ++i) v[i] = 1.0 / sqrt((double)K);
        for (int itr = 0; itr < 3; ++itr) {
          tri_solve(a, b, K, sh, v, v, u, w);
          const double nv = dot_norm(v, K);
          for (int i = 0; i < K; ++i) v[i] /= nv;
        }
        double xz = 0;
        for (int i = 0; i < K; ++i) xz = fma(st[i], v[i], xz);
        const double tau = -xz + sqrt(fmax(xz * xz + radius * radius - nh * nh, 0.0));
        for (int i = 0; i < K; ++i) st[i] = fma(tau, v[i], st[i]);
        sigma = slo0;
        done = true;
      }
    }
    if (!done) {
      for (int i = 0; i < K; ++i) z[i] = -gt[i];
      double shi = slo0 + gn / radius + 1.0;
      for (int k = 0; k < 200; ++k) {
        tri_solve(a, b, K, shi, z, st, u, w);
        if (dot_norm(st, K) <= radius) break;
        shi *= 2.0;
      }
      double sig = shi, slo = slo0;
      {
        // Starting point: the same safeguarded Newton iteration in binary32
        // (a binary64 instruction occupies its pipe for every lane, and this
        // runs on one thread), to about 1e-5; the binary64 iteration below
        // then converges from it in two or three steps.  u and w hold the
        // binary32 T, right-hand side, solution and pivots, step the
        // derivative solve.
        float* af = reinterpret_cast<float*>(u);
        float* bf = af + K;
        float* zf = reinterpret_cast<float*>(w);
        float* xf = zf + K;
        float* df = reinterpret_cast<float*>(step);
        float* yf = df + K;
        for (int i = 0; i < K; ++i) {
          af[i] = (float)a[i];
          bf[i] = (float)b[i];
          zf[i] = (float)z[i];
        }
        float fs = (float)shi, flo = (float)slo, fhi = (float)shi;
        const float fr = (float)radius;
        for (int itn = 0; itn < 60; ++itn) {
          tri_solve_f(af, bf, K, fs, zf, xf, df);
          float n2 = 0.f;
          for (int i = 0; i < K; ++i) n2 = fmaf(xf[i], xf[i], n2);
          const float ns = sqrtf(n2);
          if (!(ns > 0.f) || fabsf(ns - fr) <= 1e-5f * fr) break;
          const float phi = 1.f / ns - 1.f / fr;
          if (phi < 0.f) flo = fs; else fhi = fs;
          tri_solve_f(af, bf, K, fs, xf, yf, df);
          float d2 = 0.f;
          for (int i = 0; i < K; ++i) d2 = fmaf(xf[i], yf[i], d2);
          const float dphi = d2 / (ns * ns * ns);
          float nw = fs - phi / dphi;
          if (!(nw > flo && nw < fhi)) nw = 0.5f * (flo + fhi);
          fs = nw;
        }
        if (isfinite(fs) && (double)fs > slo && (double)fs < shi) sig = (double)fs;
      }
      for (int itn = 0; itn < 200; ++itn) {
        tri_solve(a, b, K, sig, z, st, u, w);
        const double ns = dot_norm(st, K);
        if (fabs(ns - radius) <= 1e-13 * radius) break;
        const double phi = 1.0 / ns - 1.0 / radius;
        if (phi < 0) slo = sig; else shi = sig;
        // d|s|/dsigma = -s^T (T + sigma I)^-1 s / |s| (the step buffer as scratch)
        tri_solve(a, b, K, sig, st, step, u, w);
        double dd = 0;
        for (int i = 0; i < K; ++i) dd = fma(st[i], step[i], dd);
        const double dns = -dd / ns;
        const double dphi = -dns / (ns * ns);
        double nw = sig - phi / dphi;
        if (!(nw > slo && nw < shi)) nw = 0.5 * (slo + shi);
        sig = nw;
      }
      tri_solve(a, b, K, sig, z, st, u, w);
      sigma = sig;
    }
    // predicted decrease from T directly, |s|
    double pr = 0, ns2 = 0;
    for (int i = 0; i < K; ++i) {
      double ts = a[i] * st[i];
      if (i > 0) ts = fma(b[i - 1], st[i - 1], ts);
      if (i + 1 < K) ts = fma(b[i], st[i + 1], ts);
      pr += gt[i] * st[i] + 0.5 * st[i] * ts;
      ns2 = fma(st[i], st[i], ns2);
    }
    info[0] = -pr;
    info[1] = sqrt(ns2);
    info[2] = sigma;
    info[3] = gn;
  }
  __syncthreads();
  // ---- s = Q st: reflectors K-3 .. 0 ----
  for (int l = tid; l < K; l += nt) step[l] = st[l];
  __syncthreads();
  if (tid < 32) {   // one warp, as for Q^T g
    for (int k = K - 3; k >= 0; --k) {
      const int n = K - k - 1;
      const double beta = bet[k];
      if (beta == 0.0) continue;
      double vs = 0;
      for (int i = tid; i < n; i += 32) vs = fma(A[(size_t)(k + 1 + i) * lda + k], step[k + 1 + i], vs);
      vs = warp_sum(vs);
      for (int i = tid; i < n; i += 32) step[k + 1 + i] -= beta * vs * A[(size_t)(k + 1 + i) * lda + k];
      __syncwarp();
    }
  }
  __syncthreads();
  for (int l = tid; l < K; l += nt)
    if (!isfinite(step[l])) raise_status(status, DEV_NONFINITE);
  __syncthreads();
}

// shared memory of the tridiagonal subproblem's work area (A padded to K + 1)
constexpr size_t kTriSmemMax = 200 * 1024;
static inline size_t tri_smem_bytes(int K) {
  return (8 * (size_t)K + (size_t)K * (K + 1)) * sizeof(double);
}

// method: 0 by K (eigendecomposition below kTriMin), 1 eigendecomposition, 2 tridiagonal
__global__ void k_tr_subproblem(const double* __restrict__ gh, const double* __restrict__ Q,
                                const double* __restrict__ d, int K, double radius,
                                double* __restrict__ work, double* __restrict__ step,
                                double* __restrict__ info, int* status, int method, int use_sw) {
  __shared__ double red[32];
  extern __shared__ __align__(16) double dsm[];
  const bool tri = method == 2 || (method == 0 && !tr_needs_eig(K));
  if (tri) tr_subproblem_tri_body(gh, K, radius, work, step, info, status, red, use_sw ? dsm : nullptr);
  else tr_subproblem_body(gh, Q, d, K, radius, work, step, info, status, red);
}

// ---------------------------------------------------------------------------
// Batched trust region (one CTA per problem, problems in a TrSlot array).
// The iteration is the same basic trust region as the single-problem solve
// (gtol test on the current gradient, exact subproblem, ratio test, radius
// update, acceptance, xtol test), except that the trial point is evaluated
// with its gradient and Hessian (by the batched evaluation between the two
// kernels below), so that an accepted step needs no further evaluation.
// ---------------------------------------------------------------------------

// first half of iteration `it`: gtol test, subproblem, trial point
__global__ void k_tr_batch_propose(TrSlot* slots, int n, int it, double gtol, int use_sw) {
  __shared__ double red[32];
  extern __shared__ __align__(16) double dsm[];
  const int i = blockIdx.x;
  if (i >= n) return;
  TrSlot& t = slots[i];
  if (!t.active) return;
  const int K = t.K;
  if (threadIdx.x == 0) {
    double gn = 0;
    for (int l = 0; l < K; ++l) gn = fma(t.gh[1 + l], t.gh[1 + l], gn);
    red[31] = sqrt(gn);
  }
  __syncthreads();
  if (red[31] < gtol) {
    __syncthreads();
    if (threadIdx.x == 0) { t.stop = 0; t.iters = it - 1; t.active = 0; }
    return;
  }
  __syncthreads();
  if (tr_needs_eig(K))
    tr_subproblem_body(t.gh, t.work + 3 * K, t.work + 2 * K, K, t.radius, t.work, t.step, t.info,
                       t.status, red);
  else
    tr_subproblem_tri_body(t.gh, K, t.radius, t.work, t.step, t.info, t.status, red,
                           use_sw ? dsm : nullptr);
  const double pred = t.info[0];
  if (!(pred > 0) || !isfinite(pred)) {
    if (threadIdx.x == 0) { t.stop = 3; t.iters = it; t.active = 0; }
    return;
  }
  for (int l = threadIdx.x; l < K; l += blockDim.x) t.theta_trial[l] = t.theta[l] + t.step[l];
}

// second half: ratio test on the evaluated trial, radius update, acceptance
// (theta, [J, grad, Hess] and the Hessian's eigendecomposition taken from the
// trial), xtol and iteration-cap tests.  Device status bits of the trial
// evaluation: a non-finite value or an unconverged eigensolver rejects the
// step; a timeout or an unsupported shape ends the problem's solve with
// stop = 4 and the bits kept in `fail`.
__global__ void k_tr_batch_update(TrSlot* slots, int n, int it, int max_iter, double xtol,
                                  double radius_max, double eta) {
  __shared__ int acc;
  const int i = blockIdx.x;
  if (i >= n) return;
  TrSlot& t = slots[i];
  if (!t.active) return;
  const int K = t.K;
  if (threadIdx.x == 0) {
    const int st = *t.status;
    *t.status = 0;
    acc = 0;
    t.n_eval_J += 1;
    if (st & (DEV_TIMEOUT | DEV_BADSHAPE)) {
      t.fail = st;
      t.stop = 4;
      t.iters = it;
      t.active = 0;
    } else {
      const double pred = t.info[0], snorm = t.info[1];
      const double Jc = t.gh[0], Jt = t.gh_trial[0];
      const bool ok = st == 0 && isfinite(Jt);
      const double rho = ok ? (Jc - Jt) / pred : -1.0;
      double r = t.radius;
      if (rho < 0.25) r *= 0.25;
      else if (rho > 0.75 && fabs(snorm - r) <= 1e-8 * r) r = fmin(2.0 * r, radius_max);
      t.radius = r;
      if (rho > eta) {
        acc = 1;
        t.n_eval_gh += 1;
      }
    }
  }
  __syncthreads();
  if (!t.active) return;
  if (acc) {
    for (int l = threadIdx.x; l < K; l += blockDim.x) t.theta[l] = t.theta_trial[l];
    const size_t ngh = 1 + (size_t)K + (size_t)K * K;
    for (size_t e = threadIdx.x; e < ngh; e += blockDim.x) t.gh[e] = t.gh_trial[e];
    if (tr_needs_eig(K)) {
      const size_t neig = (size_t)K + (size_t)K * K;   // eigenvalues d, eigenvectors Q
      for (size_t e = threadIdx.x; e < neig; e += blockDim.x) t.work[2 * K + e] = t.eig_trial[e];
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (t.radius < xtol) { t.stop = 1; t.iters = it; t.active = 0; }
    else if (it >= max_iter) { t.stop = 2; t.iters = max_iter; t.active = 0; }
  }
}

// the initial point: [J, grad, Hess] and eigendecomposition taken as current
__global__ void k_tr_batch_init(TrSlot* slots, int n, double radius0) {
  const int i = blockIdx.x;
  if (i >= n) return;
  TrSlot& t = slots[i];
  const int K = t.K;
  const size_t ngh = 1 + (size_t)K + (size_t)K * K;
  for (size_t e = threadIdx.x; e < ngh; e += blockDim.x) t.gh[e] = t.gh_trial[e];
  if (tr_needs_eig(K)) {
    const size_t neig = (size_t)K + (size_t)K * K;
    for (size_t e = threadIdx.x; e < neig; e += blockDim.x) t.work[2 * K + e] = t.eig_trial[e];
  }
  for (int l = threadIdx.x; l < K; l += blockDim.x) t.theta[l] = t.theta_trial[l];
  if (threadIdx.x == 0) {
    const int st = *t.status;
    *t.status = 0;
    t.radius = radius0;
    t.iters = 0; t.n_eval_J = 0; t.n_eval_gh = 1;
    t.stop = 2;
    t.fail = st;
    t.active = st == 0 && isfinite(t.gh[0]) ? 1 : 0;
    if (!t.active) t.stop = 4;
  }
}

// ---------------------------------------------------------------------------
// BFGS update of the Hessian approximation of the gradient-only trust region
// (Alg. 1 with the quasi-Newton model; Nocedal & Wright, Eq. 6.19), one CTA:
//   y = g_new - g_old, s = the trial step;
//   first update with y^T s > 0: B <- (y^T y / y^T s) I (state[0] = 1 after);
//   y^T s > min_curv |s| |y|:   B <- B - (B s)(B s)^T / (s^T B s) + y y^T / (y^T s),
// otherwise B is kept.  B is K x K row-major, symmetric.
// ---------------------------------------------------------------------------
__global__ void k_bfgs_update(double* __restrict__ B, const double* __restrict__ s,
                              const double* __restrict__ g_old, const double* __restrict__ g_new,
                              int K, double* __restrict__ state, double min_curv,
                              double* __restrict__ Bs) {
  __shared__ double red[32];
  __shared__ double sc[4];
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) sc[2] = state[0];
  double sy = 0, yy = 0, ss = 0;
  for (int l = tid; l < K; l += nt) {
    const double y = g_new[l] - g_old[l];
    sy = fma(y, s[l], sy);
    yy = fma(y, y, yy);
    ss = fma(s[l], s[l], ss);
  }
  sy = block_sum(sy, red);
  yy = block_sum(yy, red);
  ss = block_sum(ss, red);
  __syncthreads();
  if (sc[2] == 0.0 && sy > 0) {   // sc[2] read before block_sum's barriers
    const double scale = yy / sy;
    for (int e = tid; e < K * K; e += nt) B[e] = (e / K == e % K) ? scale : 0.0;
    __syncthreads();
    if (tid == 0) state[0] = 1.0;
  }
  if (!(sy > min_curv * sqrt(ss) * sqrt(yy))) return;   // uniform across the CTA
  double sbs = 0;
  for (int i = tid; i < K; i += nt) {
    double acc = 0;
    for (int k = 0; k < K; ++k) acc = fma(B[(size_t)i * K + k], s[k], acc);
    Bs[i] = acc;
    sbs = fma(s[i], acc, sbs);
  }
  sbs = block_sum(sbs, red);
  __syncthreads();
  if (tid == 0) { sc[0] = sbs; sc[1] = sy; }
  __syncthreads();
  for (int e = tid; e < K * K; e += nt) {
    const int i = e / K, k = e % K;
    const double yi = g_new[i] - g_old[i], yk = g_new[k] - g_old[k];
    B[e] = B[e] - (Bs[i] * Bs[k]) / sc[0] + (yi * yk) / sc[1];
  }
}

__global__ void k_set_identity(double* __restrict__ B, int K) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < K * K; e += gridDim.x * blockDim.x)
    B[e] = (e / K == e % K) ? 1.0 : 0.0;
}

cudaError_t launch_bfgs_update(double* B, const double* s, const double* g_old, const double* g_new, int K,
                               double* state, double min_curv, double* scratch, cudaStream_t st) {
  k_bfgs_update<<<1, 256, 0, st>>>(B, s, g_old, g_new, K, state, min_curv, scratch);
  return cudaGetLastError();
}

cudaError_t launch_set_identity(double* B, int K, cudaStream_t st) {
  k_set_identity<<<(K * K + 255) / 256, 256, 0, st>>>(B, K);
  return cudaGetLastError();
}

cudaError_t launch_tr_batch(int phase, TrSlot* slots, int n, int it, const TrBatchOptions& o,
                            cudaStream_t st) {
  if (n < 1) return cudaSuccess;
  if (phase == 0) k_tr_batch_init<<<n, 128, 0, st>>>(slots, n, o.radius0);
  else if (phase == 1) {
    const size_t sw = tri_smem_bytes(o.kmax);
    set_max_smem((const void*)k_tr_batch_propose);
    const bool fits = o.kmax >= kTriMin && sw <= kTriSmemMax;
    k_tr_batch_propose<<<n, 128, fits ? sw : 0, st>>>(slots, n, it, o.gtol, fits ? 1 : 0);
  }
  else k_tr_batch_update<<<n, 128, 0, st>>>(slots, n, it, o.max_iter, o.xtol, o.radius_max, o.eta);
  return cudaGetLastError();
}

__global__ void k_axpy(const double* __restrict__ x, const double* __restrict__ s, int K,
                       double* __restrict__ y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < K) y[i] = x[i] + s[i];
}

size_t tr_work_doubles(int K) { return 8 * (size_t)K + (size_t)K * K; }

cudaError_t launch_tr_subproblem(const double* out_gh, int K, double radius, double* work,
                                 double* step, double* info, int* status, cudaStream_t st, int method) {
  // eigendecomposition of the Hessian (eigendecomposition method) expected in
  // work + 2K (d) and work + 3K (Q)
  const double* d = work + 2 * K;
  const double* Q = work + 3 * K;
  const bool tri = method == 2 || (method == 0 && !tr_needs_eig(K));
  const size_t sw = tri_smem_bytes(K);
  const bool fits = tri && sw <= kTriSmemMax;
  if (fits) set_max_smem((const void*)k_tr_subproblem);
  k_tr_subproblem<<<1, K >= kTriMin ? 256 : 128, fits ? sw : 0, st>>>(out_gh, Q, d, K, radius, work, step,
                                                                     info, status, method, fits ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_axpy(const double* x, const double* s, int K, double* y, cudaStream_t st) {
  k_axpy<<<(K + 127) / 128, 128, 0, st>>>(x, s, K, y);
  return cudaGetLastError();
}

}  // namespace qoc

// ---------------------------------------------------------------------------
// C ABI: one subproblem from host data (see include/qoc.h)
// ---------------------------------------------------------------------------
extern "C" qoc_status qoc_tr_subproblem(int K, const double* g, const double* H, double radius,
                                        int method, double* s, double* info) {
  using namespace qoc;
  if (K < 1 || K > 4096 || !g || !H || !s || !info || !(radius > 0) || method < 0 || method > 2)
    return QOC_EINVAL;
  const bool eig = method == 1 || (method == 0 && tr_needs_eig(K));
  const size_t ngh = 1 + (size_t)K + (size_t)K * K;
  double *dgh = nullptr, *work = nullptr, *step = nullptr, *dinfo = nullptr, *zero = nullptr;
  int* status = nullptr;
  StepSpace ws;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMalloc(&dgh, 8 * ngh);
  if (e == cudaSuccess) e = cudaMalloc(&work, 8 * tr_work_doubles(K));
  if (e == cudaSuccess) e = cudaMalloc(&step, 8 * (size_t)K);
  if (e == cudaSuccess) e = cudaMalloc(&dinfo, 8 * 8);
  if (e == cudaSuccess) e = cudaMalloc(&zero, 8 * ((size_t)K * K + 1));
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess && eig) {
    ws.bytes = (eig_step_bytes(K) + 255) & ~size_t(255);
    e = cudaMalloc(&ws.base, ws.bytes);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(zero, 0, 8 * ((size_t)K * K + 1), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dgh, 0, 8, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dgh + 1, g, 8 * (size_t)K, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dgh + 1 + K, H, 8 * (size_t)K * K, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && eig)
    e = launch_eig(dgh + 1 + K, zero, zero, K, 1, work + 3 * K, work + 2 * K, status, EIG_JACOBI_FP64, 0,
                   0.0, st, ws);
  if (e == cudaSuccess) e = launch_tr_subproblem(dgh, K, radius, work, step, dinfo, status, st, eig ? 1 : 2);
  int hst = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(s, step, 8 * (size_t)K, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(info, dinfo, 4 * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hst, status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dgh); cudaFree(work); cudaFree(step); cudaFree(dinfo); cudaFree(zero); cudaFree(status);
  cudaFree(ws.base);
  if (st) cudaStreamDestroy(st);
  if (e != cudaSuccess) {
    note_error(cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? QOC_ENOMEM : QOC_ECUDA;
  }
  if (hst & DEV_TIMEOUT) return QOC_ETIMEOUT;
  if (hst) return QOC_ENUMERIC;
  return QOC_OK;
}
