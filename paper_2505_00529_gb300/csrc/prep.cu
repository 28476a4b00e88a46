// Per-step spectral preparation, parallel over the steps j (Alg. 2, third
// loop: "use the eigendecomposition of Z_j to compute ... dexp . M and
// d^2exp . (M x M)"; Sec. III-A: once V, D are known these are cheap).
//
// With phi(x) = exp(-i dt x) and H_j = W diag(lambda) W^T (W real orthogonal):
//   U_j          = W diag(phi(lambda)) W^T
//   dU_j/df_j    = W (Gamma1 o M~) W^T,      Gamma1_pq = phi[lambda_p, lambda_q]
//   d2U_j/df_j^2 = W X' W^T,  X'_pq = 2 sum_r M~_pr M~_rq phi[lambda_p, lambda_r, lambda_q]
// with M~ = W^T M W (Daleckii-Krein formulas; the paper omits these
// derivations).  This kernel stores, per step:
//   D_j  = exp(i dt m) U_j - I = W diag(phi(lambda - m) - 1) W^T  (the increment
//          the sweeps apply; m is a fixed spectral shift, so |D_j| ~ dt |lambda - m|),
//   P~_j = Gamma1 o M~                                     (binary64, complex),
//   X'_j                                                   (binary64, complex).
// X' is formed from the commutator identity
//   sum_r M~_pr M~_rq phi[l_p, l_r, l_q] = ((P~ M~)_pq - (P~ M~)_qp) / (l_p - l_q)
// (the recurrence phi[p,r,q] = (phi[p,r] - phi[r,q]) / (l_p - l_q) summed over
// r), which costs one complex-by-real N^3 product, and from the direct
// N-term sum with a stable second divided difference for the pairs with
// dt |l_p - l_q| <= TAU_DD2 (always including p == q).
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

// sin(x)/x: Taylor polynomial for |x| < 1/4 (next term < 3e-21), else sin/x.
__device__ __forceinline__ double sinc_d(double x) {
  double ax = fabs(x);
  if (ax < 0.25) {
    double x2 = x * x;
    double p = 1.0 / 6227020800.0;            // 1/13!
    p = fma(p, x2, -1.0 / 39916800.0);        // 1/11!
    p = fma(p, x2, 1.0 / 362880.0);           // 1/9!
    p = fma(p, x2, -1.0 / 5040.0);            // 1/7!
    p = fma(p, x2, 1.0 / 120.0);              // 1/5!
    p = fma(p, x2, -1.0 / 6.0);               // 1/3!
    return fma(p, x2, 1.0);
  }
  return sin(x) / x;
}

// phi[l_a, l_b] = -i dt exp(-i dt (l_a + l_b)/2) sinc(dt (l_a - l_b)/2),
// with eh[a] = exp(-i dt l_a / 2).
__device__ __forceinline__ double2 gamma1(int a, int b, const double* lam, const double2* eh, double dt) {
  double2 e = cmul(eh[a], eh[b]);
  double s = dt * sinc_d(0.5 * dt * (lam[a] - lam[b]));
  return make_double2(e.y * s, -e.x * s);   // -i * s * e
}

// phi[l_a, l_b, l_c]: symmetric; extremes lo, hi.  Far: recurrence on the
// extremes; near (dt (hi - lo) <= TAU_DD2): exp(-i dt c) sum_{n=2}^{10}
// (-i dt)^n / n! h_{n-2}(lo - c, mid - c, hi - c), c the mean.
__device__ double2 dd2_dev(int a, int b, int c, const double* lam, const double2* eh, double dt) {
  int lo = a, mid = b, hi = c;
  if (lam[lo] > lam[mid]) { int t = lo; lo = mid; mid = t; }
  if (lam[mid] > lam[hi]) { int t = mid; mid = hi; hi = t; }
  if (lam[lo] > lam[mid]) { int t = lo; lo = mid; mid = t; }
  double xl = lam[lo], xm = lam[mid], xh = lam[hi];
  if (dt * (xh - xl) > TAU_DD2) {
    double2 g1 = gamma1(lo, mid, lam, eh, dt);
    double2 g2 = gamma1(mid, hi, lam, eh, dt);
    return cscale(csub(g1, g2), 1.0 / (xl - xh));
  }
  double cm = (xl + xm + xh) * (1.0 / 3.0);
  double u = xl - cm, v = xm - cm, w = xh - cm;
  double h2 = 1.0, h3 = 1.0, uk = 1.0;   // h_k(u,v), h_k(u,v,w), u^k at k = 0
  double re = 0, im = 0;
  double dtn = dt * dt, fact = 2.0;
  for (int n = 2; n <= 10; ++n) {
    int k = n - 2;
    if (k > 0) {
      uk *= u;
      h2 = fma(v, h2, uk);
      h3 = fma(w, h3, h2);
    }
    double t = dtn / fact * h3;
    switch (n & 3) {                       // (-i)^n
      case 0: re += t; break;
      case 1: im -= t; break;
      case 2: re -= t; break;
      default: im += t; break;
    }
    dtn *= dt;
    fact *= (double)(n + 1);
  }
  double2 e = cexpi(-dt * cm);
  return cmul(e, make_double2(re, im));
}

__global__ void k_prep(const double* __restrict__ Wg, const double* __restrict__ eig,
                       const double* __restrict__ Mg, int N, int J, double dt, double mshift,
                       void* __restrict__ Dout, size_t dstride, int d_fp64, int derivs,
                       double2* __restrict__ Ptil, double2* __restrict__ Xp, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.x;
  if (j >= J) return;
  const int ld = N + 1;
  double* W = reinterpret_cast<double*>(smem_raw);      // [N][ld]
  double* T = W + N * ld;                               // [N][ld]
  double* Mt = T + N * ld;                              // [N][ld]
  double2* P = reinterpret_cast<double2*>(Mt + N * ld); // [N][ld]
  double* lam = reinterpret_cast<double*>(P + N * ld);  // [N]
  double2* eh = reinterpret_cast<double2*>(lam + N + (N & 1));  // [N]
  double2* pm1 = eh + N;                                // [N] phi(lambda - m) - 1
  double2* Y = reinterpret_cast<double2*>(W);           // [N][ld] overlays W and T

  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Wj = Wg + (size_t)j * N * N;
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    W[p * ld + q] = Wj[e];
    Mt[p * ld + q] = Mg[e];
  }
  for (int p = tid; p < N; p += nt) {
    double l = eig[(size_t)j * N + p];
    lam[p] = l;
    double x = dt * (l - mshift);
    double s, c, sh;
    sincos(x, &s, &c);
    sh = sin(0.5 * x);
    pm1[p] = make_double2(-2.0 * sh * sh, -s);   // exp(-i x) - 1 without cancellation
    eh[p] = cexpi(-0.5 * dt * l);
  }
  __syncthreads();

  // D = W diag(pm1) W^T (complex symmetric)
  if (d_fp64) {
    double2* D = reinterpret_cast<double2*>(reinterpret_cast<unsigned char*>(Dout) + (size_t)j * dstride);
    for (int e = tid; e < N * N; e += nt) {
      int p = e / N, q = e % N;
      if (q < p) continue;
      double re = 0, im = 0;
      for (int r = 0; r < N; ++r) {
        double w = W[p * ld + r] * W[q * ld + r];
        re = fma(w, pm1[r].x, re);
        im = fma(w, pm1[r].y, im);
      }
      D[p * N + q] = make_double2(re, im);
      D[q * N + p] = make_double2(re, im);
    }
  } else {
    float2* D = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(Dout) + (size_t)j * dstride);
    for (int e = tid; e < N * N; e += nt) {
      int p = e / N, q = e % N;
      if (q < p) continue;
      float re = 0, im = 0;
      for (int r = 0; r < N; ++r) {
        float w = (float)W[p * ld + r] * (float)W[q * ld + r];
        re = fmaf(w, (float)pm1[r].x, re);
        im = fmaf(w, (float)pm1[r].y, im);
      }
      D[p * N + q] = make_float2(re, im);
      D[q * N + p] = make_float2(re, im);
    }
  }
  if (!derivs) return;

  // T = M W ; M~ = W^T T
  for (int e = tid; e < N * N; e += nt) {
    int i = e / N, k = e % N;
    double acc = 0;
    for (int r = 0; r < N; ++r) acc = fma(Mt[i * ld + r], W[r * ld + k], acc);
    T[i * ld + k] = acc;
  }
  __syncthreads();
  for (int e = tid; e < N * N; e += nt) {
    int i = e / N, k = e % N;
    double acc = 0;
    for (int r = 0; r < N; ++r) acc = fma(W[r * ld + i], T[r * ld + k], acc);
    Mt[i * ld + k] = acc;   // M no longer needed
  }
  __syncthreads();
  for (int e = tid; e < N * N; e += nt) {   // exact symmetry
    int i = e / N, k = e % N;
    if (k > i) {
      double s = 0.5 * (Mt[i * ld + k] + Mt[k * ld + i]);
      Mt[i * ld + k] = s;
      Mt[k * ld + i] = s;
    }
  }
  __syncthreads();
  // P~ = Gamma1 o M~
  double2* Pg = Ptil + (size_t)j * N * N;
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    double2 g = gamma1(p, q, lam, eh, dt);
    double2 v = cscale(g, Mt[p * ld + q]);
    P[p * ld + q] = v;
    Pg[e] = v;
  }
  __syncthreads();
  // Y = P~ M~  (W, T are dead: Y overlays them)
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    double re = 0, im = 0;
    for (int r = 0; r < N; ++r) {
      double m = Mt[r * ld + q];
      re = fma(P[p * ld + r].x, m, re);
      im = fma(P[p * ld + r].y, m, im);
    }
    Y[p * ld + q] = make_double2(re, im);
  }
  __syncthreads();
  double2* Xg = Xp + (size_t)j * N * N;
  bool bad = false;
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    double2 x;
    if (dt * fabs(lam[p] - lam[q]) > TAU_DD2) {
      double2 d = csub(Y[p * ld + q], Y[q * ld + p]);
      x = cscale(d, 2.0 / (lam[p] - lam[q]));
    } else {
      double re = 0, im = 0;
      for (int r = 0; r < N; ++r) {
        double m2 = Mt[p * ld + r] * Mt[r * ld + q];
        double2 g2 = dd2_dev(p, r, q, lam, eh, dt);
        re = fma(m2, g2.x, re);
        im = fma(m2, g2.y, im);
      }
      x = make_double2(2.0 * re, 2.0 * im);
    }
    bad |= !(isfinite(x.x) && isfinite(x.y));
    Xg[e] = x;
  }
  if (bad) raise_status(status, DEV_NONFINITE);
}

size_t prep_smem_bytes(int N) {
  return (5 * (size_t)N * (N + 1) + (N + (N & 1)) + 4 * (size_t)N) * sizeof(double);
}

cudaError_t launch_prep(const double* W, const double* eig, const double* M, int N, int J,
                        double dt, double mshift, void* D, size_t dstride, int d_fp64,
                        int derivs, double2* Ptil, double2* Xp, int* status, cudaStream_t st) {
  size_t sm = prep_smem_bytes(N);
  cudaFuncSetAttribute(k_prep, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  int threads = N <= 8 ? 64 : (N <= 16 ? 128 : 256);
  k_prep<<<J, threads, sm, st>>>(W, eig, M, N, J, dt, mshift, D, dstride, d_fp64, derivs, Ptil,
                                 Xp, status);
  return cudaGetLastError();
}

}  // namespace qoc
