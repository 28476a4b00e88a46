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
// r), which costs one complex-by-real N^3 product, for the pairs with
// dt |l_p - l_q| > TAU_DD2; on the diagonal from the same recurrence term by
// term (phi[p,r,p] = (Gamma1_pp - Gamma1_pr) / (l_p - l_r) for far r, the stable
// series for near r); and for the remaining near pairs from the direct N-term
// sum with a stable second divided difference.
#include <type_traits>

#include "common.cuh"
#include "kernels.hpp"
#include "ozaki.cuh"

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

// Integer tests and keys, so that bookkeeping stays off the binary64 pipe.
__device__ __forceinline__ bool finite_bits(double x) {
  return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool nonzero_bits(double x) {
  return (__double_as_longlong(x) << 1) != 0;
}
// order-preserving integer key of a binary64 value (not NaN)
__device__ __forceinline__ long long value_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}

// Coefficients dt^n / n!, n = 0 .. kSeriesTerms, of the near-triple series below
constexpr int kSeriesTerms = 10;

// phi[l_a, l_b, l_c] (symmetric in its arguments) with extremes lo, hi.
// rinv(x, y) = 1 / (l_x - l_y) for every far pair (dt |l_x - l_y| > TAU_DD2)
// and 0 for near pairs, as left in the real parts of Y by the far-pair pass.
// Far extremes: the recurrence phi[lo, mid, hi] = (Gamma1[lo, mid] - Gamma1[mid, hi])
// / (l_lo - l_hi).  Near: the Taylor series of phi about l_lo,
//   phi[lo, mid, hi] = exp(-i dt l_lo) sum_{n=2}^{10} (-i dt)^n / n! h_{n-2}(0, v, w),
// v = l_mid - l_lo, w = l_hi - l_lo >= 0, h_k the complete homogeneous
// polynomial (the divided difference of (x - l_lo)^n).  The series runs only
// when the extremes are a near pair, dt (l_hi - l_lo) <= TAU_DD2, so the first
// dropped term is below 20 TAU_DD2^9 / 11! of the leading one.
__device__ __noinline__ double2 dd2_dev(int a, int b, int c, const double* lam, const double2* eh,
                           const double2* Y, int ld, const double* cser, double dt) {
  const long long ka = value_key(lam[a]), kb = value_key(lam[b]), kc = value_key(lam[c]);
  // sort (a, b, c) by (value, index) with integer compares
  int lo = a, mid = b, hi = c;
  long long klo = ka, kmid = kb, khi = kc;
  if (klo > kmid || (klo == kmid && lo > mid)) { int t = lo; lo = mid; mid = t; long long u = klo; klo = kmid; kmid = u; }
  if (kmid > khi || (kmid == khi && mid > hi)) { int t = mid; mid = hi; hi = t; long long u = kmid; kmid = khi; khi = u; }
  if (klo > kmid || (klo == kmid && lo > mid)) { int t = lo; lo = mid; mid = t; }
  const double r = lo != hi ? Y[lo * ld + hi].x : 0.0;
  if (nonzero_bits(r)) {
    const double2 g1 = gamma1(lo, mid, lam, eh, dt);
    const double2 g2 = gamma1(mid, hi, lam, eh, dt);
    return cscale(csub(g1, g2), r);
  }
  const double v = lam[mid] - lam[lo], w = lam[hi] - lam[lo];
  double vk = 1.0, h3 = 1.0;   // v^k, h_k(0, v, w) at k = 0
  double re = -cser[2], im = 0.0;   // n = 2: (-i)^2 = -1
#pragma unroll
  for (int n = 3; n <= kSeriesTerms; ++n) {
    vk *= v;
    h3 = fma(w, h3, vk);
    const double t = cser[n] * h3;
    switch (n & 3) {   // (-i)^n
      case 0: re += t; break;
      case 1: im -= t; break;
      case 2: re -= t; break;
      default: im += t; break;
    }
  }
  const double2 e = cmul(eh[lo], eh[lo]);   // exp(-i dt l_lo)
  return cmul(e, make_double2(re, im));
}

// row-major upper-triangle index t (0 <= t < N(N+1)/2) -> (i, k), k >= i
__device__ __forceinline__ void tri_index(int t, int N, int& i, int& k) {
  const float b = 2.0f * N + 1.0f;
  int r = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * t, 0.0f))));
  r = max(0, min(r, N - 1));
  while (r > 0 && r * N - r * (r - 1) / 2 > t) --r;
  while (r + 1 < N && (r + 1) * N - (r + 1) * r / 2 <= t) ++r;
  i = r;
  k = t - (r * N - r * (r - 1) / 2) + r;
}

// OZ (binary32-sweep problems, N <= 32, 256 threads): the N^3 products
// M W, W^T (M W) and the two real factors of P~ M~ on the tensor cores by
// error-free splitting (ozaki.cuh), binary64-accurate to about 2^-43 of the
// factors' scales.
constexpr int kOzPrepSlices = 6;
__host__ __device__ inline size_t oz_prep_bytes() {
  return 3 * (size_t)kOzPrepSlices * 32 * oz::LD * 2 + 3 * 32 * 4 + 16;
}

template <bool OZ>
__device__ __forceinline__ void prep_step(const double* __restrict__ Wg,
                                          const double* __restrict__ eig,
                                          const double* __restrict__ Mg, int N, int j, double dt,
                                          int derivs, double2* __restrict__ Ptil,
                                          double2* __restrict__ Xp, double* __restrict__ Mtil,
                                          int* status, unsigned char* smem_raw) {
  const int ld = N + 1;
  const int NT = N * (N + 1) / 2;
  double* W = reinterpret_cast<double*>(smem_raw);      // [N][ld]
  double* T = W + N * ld;                               // [N][ld]
  double* Mt = T + N * ld;                              // [N][ld]
  double2* P = reinterpret_cast<double2*>(Mt + N * ld); // [N][ld]: P~, later Gamma1
  double* lam = reinterpret_cast<double*>(P + N * ld);  // [N]
  double2* eh = reinterpret_cast<double2*>(lam + N + (N & 1));  // [N]
  int* near = reinterpret_cast<int*>(eh + N);           // [NT] packed near pairs
  double2* Y = reinterpret_cast<double2*>(W);           // [N][ld] overlays W and T
  __shared__ int n_near;
  __shared__ double cser[kSeriesTerms + 1];   // dt^n / n!
  __nv_bfloat16 *s0 = nullptr, *s1 = nullptr, *s2 = nullptr;   // slice sets (OZ)
  int *e0 = nullptr, *e1 = nullptr, *e2 = nullptr;
  if (OZ) {
    unsigned char* ob = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(near + N * (N + 1) / 2) + 15) & ~uintptr_t(15));
    const size_t sl = (size_t)kOzPrepSlices * 32 * oz::LD;
    s0 = reinterpret_cast<__nv_bfloat16*>(ob);
    s1 = s0 + sl;
    s2 = s1 + sl;
    e0 = reinterpret_cast<int*>(s2 + sl);
    e1 = e0 + 32;
    e2 = e1 + 32;
  }

  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Wj = Wg + (size_t)j * N * N;
  // parts: PREP_P (M~ and P~; M~ also stored when Mtil is given), PREP_X (X';
  // from this launch's M~, P~ or, alone, from the stored ones).  The
  // increments D_j (PREP_D) are k_increments' work.
  const bool doP = derivs & PREP_P, doX = derivs & PREP_X;
  const bool loadMP = doX && !doP;
  if (tid == 0) n_near = 0;
  for (int e = tid; e < N * N; e += nt) {
    const int p = e / N, q = e % N;
    if (doP) {
      W[p * ld + q] = Wj[e];
      Mt[p * ld + q] = Mg[e];
    }
    if (loadMP) {
      Mt[p * ld + q] = Mtil[(size_t)j * N * N + e];
      P[p * ld + q] = Ptil[(size_t)j * N * N + e];
    }
  }
  for (int p = tid; p < N; p += nt) {
    const double l = eig[(size_t)j * N + p];
    lam[p] = l;
    eh[p] = cexpi(-0.5 * dt * l);
  }
  if (tid <= kSeriesTerms) {
    double c = 1.0;
    for (int n = 1; n <= tid; ++n) c = c * dt / n;
    cser[tid] = c;
  }
  __syncthreads();

  if (!doP && !doX) return;
  double2* Pg = Ptil + (size_t)j * N * N;
  if (doP) {
  // T = M W ; M~ = W^T T (upper triangle, mirrored: exactly symmetric)
  if (OZ) {
    oz::split32<kOzPrepSlices>(Mt, ld, N, true, s0, e0);    // M by rows
    oz::split32<kOzPrepSlices>(W, ld, N, false, s1, e1);    // W by columns (= W^T by rows)
    oz::mm32<kOzPrepSlices>(s0, e0, s1, e1, T, ld, N);
    __syncthreads();
    oz::split32<kOzPrepSlices>(T, ld, N, false, s2, e2);    // T by columns
    oz::mm32<kOzPrepSlices>(s1, e1, s2, e2, Mt, ld, N);     // M~ = W^T T (M already split)
    __syncthreads();
    for (int t = tid; t < NT; t += nt) {
      int i, k;
      tri_index(t, N, i, k);
      Mt[k * ld + i] = Mt[i * ld + k];
    }
    __syncthreads();
  } else {
  for (int e = tid; e < N * N; e += nt) {
    const int i = e / N, k = e % N;
    double acc = 0;
    for (int r = 0; r < N; ++r) acc = fma(Mt[i * ld + r], W[r * ld + k], acc);
    T[i * ld + k] = acc;
  }
  __syncthreads();
  for (int t = tid; t < NT; t += nt) {
    int i, k;
    tri_index(t, N, i, k);
    double acc = 0;
    for (int r = 0; r < N; ++r) acc = fma(W[r * ld + i], T[r * ld + k], acc);
    Mt[i * ld + k] = acc;   // M no longer needed; rows i < k only read by this thread's pair
    Mt[k * ld + i] = acc;
  }
  __syncthreads();
  }
  // P~ = Gamma1 o M~: complex symmetric (Gamma1 and M~ are), so over the
  // upper triangle, mirrored
  for (int t = tid; t < NT; t += nt) {
    int p, q;
    tri_index(t, N, p, q);
    const double2 v = cscale(gamma1(p, q, lam, eh, dt), Mt[p * ld + q]);
    P[p * ld + q] = v;
    P[q * ld + p] = v;
    Pg[p * N + q] = v;
    Pg[q * N + p] = v;
    if (Mtil) {
      Mtil[(size_t)j * N * N + p * N + q] = Mt[p * ld + q];
      Mtil[(size_t)j * N * N + q * N + p] = Mt[p * ld + q];
    }
  }
  }
  if (!doX) return;
  __syncthreads();
  // Y = P~ M~  (W, T are dead: Y overlays them)
  if (OZ) {
    const double* Pd = reinterpret_cast<const double*>(P);
    oz::split32<kOzPrepSlices>(Pd, ld, N, true, s0, e0, 2);       // Re P~ by rows
    oz::split32<kOzPrepSlices>(Pd + 1, ld, N, true, s1, e1, 2);   // Im P~ by rows
    oz::split32<kOzPrepSlices>(Mt, ld, N, false, s2, e2);         // M~ by columns
    double* Yd = reinterpret_cast<double*>(Y);
    oz::mm32<kOzPrepSlices>(s0, e0, s2, e2, Yd, ld, N, 2);
    oz::mm32<kOzPrepSlices>(s1, e1, s2, e2, Yd + 1, ld, N, 2);
  } else {
  for (int e = tid; e < N * N; e += nt) {
    const int p = e / N, q = e % N;
    double re = 0, im = 0;
    for (int r = 0; r < N; ++r) {
      const double m = Mt[r * ld + q];
      re = fma(P[p * ld + r].x, m, re);
      im = fma(P[p * ld + r].y, m, im);
    }
    Y[p * ld + q] = make_double2(re, im);
  }
  }
  __syncthreads();
  double2* Xg = Xp + (size_t)j * N * N;
  bool bad = false;
  // Pairs p < q.  Far (dt |l_p - l_q| > TAU_DD2): X' is symmetric, so one
  // thread forms X'_pq = X'_qp = 2 (Y_pq - Y_qp) / (l_p - l_q) and leaves the
  // reciprocal of l_p - l_q (and of l_q - l_p) in the real part of its two
  // (now dead) Y entries for the near-triple recurrences below.  Near: listed
  // for the direct sum, their Y entries zeroed as the mark.
  //
  // The same thread also forms the pair's two terms of the diagonal sums
  // X'_pp = 2 sum_r M~_pr^2 phi[l_p, l_r, l_p] and leaves them in P (whose
  // P~ it reads once, and which nothing reads afterwards): for far r the
  // recurrence on the extremes gives phi[l_p, l_r, l_p] = (Gamma1_pp -
  // Gamma1_pr) / (l_p - l_r), so the term of row p is
  // M~_pr (Gamma1_pp M~_pr - P~_pr) / (l_p - l_r) (P~ = Gamma1 o M~, symmetric).
  // At r = p, phi[l_p, l_p, l_p] = phi''(l_p) / 2 = -dt^2 / 2 exp(-i dt l_p);
  // the near r != p terms follow (series), then each row is summed in order.
  for (int t = tid; t < NT; t += nt) {
    int p, q;
    tri_index(t, N, p, q);
    const double m = Mt[p * ld + q];
    if (p == q) {
      const double2 ep = cmul(eh[p], eh[p]);                 // exp(-i dt l_p)
      P[p * ld + p] = cscale(ep, -cser[2] * (m * m));
      continue;
    }
    const double dl = lam[p] - lam[q];
    if (!(dt * fabs(dl) > TAU_DD2)) {
      near[atomicAdd(&n_near, 1)] = p * N + q;
      Y[p * ld + q].x = 0.0;
      Y[q * ld + p].x = 0.0;
      continue;
    }
    const double rec = 1.0 / dl;
    const double2 x = cscale(csub(Y[p * ld + q], Y[q * ld + p]), 2.0 * rec);
    bad |= !(finite_bits(x.x) && finite_bits(x.y));
    Xg[(size_t)p * N + q] = x;
    Xg[(size_t)q * N + p] = x;
    Y[p * ld + q].x = rec;
    Y[q * ld + p].x = -rec;
    const double2 pv = P[p * ld + q];
    const double2 ep = cmul(eh[p], eh[p]), eq = cmul(eh[q], eh[q]);
    const double2 gp = make_double2(ep.y * dt, -ep.x * dt);   // Gamma1_pp = -i dt exp(-i dt l_p)
    const double2 gq = make_double2(eq.y * dt, -eq.x * dt);
    const double mr = m * rec;
    P[p * ld + q] = cscale(csub(cscale(gp, m), pv), mr);
    P[q * ld + p] = cscale(csub(cscale(gq, m), pv), -mr);
  }
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31, nwarp = (nt + 31) >> 5;
  // near r != p terms of the diagonal sums, one series per thread: entry
  // 2k + s is pair k's term in row p (s = 0) or q (s = 1)
  for (int e = tid; e < 2 * n_near; e += nt) {
    const int pq = near[e >> 1];
    const int a = (e & 1) ? pq % N : pq / N, b = (e & 1) ? pq / N : pq % N;
    const double m = Mt[a * ld + b];
    P[a * ld + b] = cscale(dd2_dev(a, b, a, lam, eh, Y, ld, cser, dt), m * m);
  }
  __syncthreads();
  for (int p = tid; p < N; p += nt) {   // X'_pp, each row summed in order
    double re = 0, im = 0;
    for (int r = 0; r < N; ++r) {
      re += P[p * ld + r].x;
      im += P[p * ld + r].y;
    }
    const double2 x = make_double2(2.0 * re, 2.0 * im);
    bad |= !(finite_bits(x.x) && finite_bits(x.y));
    Xg[(size_t)p * N + p] = x;
  }
  // near pairs p < q: the direct N-term sum, one warp per pair, lanes over r
  for (int k = warp; k < n_near; k += nwarp) {
    const int p = near[k] / N, q = near[k] % N;
    double re = 0, im = 0;
    for (int r = lane; r < N; r += 32) {
      const double m2 = Mt[p * ld + r] * Mt[r * ld + q];
      const double2 g2 = dd2_dev(p, r, q, lam, eh, Y, ld, cser, dt);
      re = fma(m2, g2.x, re);
      im = fma(m2, g2.y, im);
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) {
      const double2 x = make_double2(2.0 * re, 2.0 * im);
      bad |= !(finite_bits(x.x) && finite_bits(x.y));
      Xg[(size_t)p * N + q] = x;
      Xg[(size_t)q * N + p] = x;
    }
  }
  if (bad) raise_status(status, DEV_NONFINITE);
}

// One step per CTA in shared memory, or (gws != nullptr, large N) a persistent
// grid whose CTAs each own a slice of a global workspace.
// MAXT: the launch's thread count bound (256: at least 3 CTAs of registers
// per SM; 512: the large-N launch).  GWS: storage in the global workspace (a
// compile-time choice, so that the shared-memory instantiation keeps
// shared-memory loads).
template <int MAXT, bool GWS, bool OZ = false>
__global__ void __launch_bounds__(MAXT, OZ ? 2 : (MAXT <= 256 ? 3 : 1))
k_prep(const double* __restrict__ Wg, const double* __restrict__ eig,
                       const double* __restrict__ Mg, int N, int J, double dt, int derivs,
                       double2* __restrict__ Ptil, double2* __restrict__ Xp,
                       double* __restrict__ Mtil, int* status, unsigned char* gws,
                       size_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int j = blockIdx.x; j < J; j += gridDim.x) {
    prep_step<OZ>(Wg, eig, Mg, N, j, dt, derivs, Ptil, Xp, Mtil, status, base);
    __syncthreads();
  }
}

size_t prep_smem_bytes(int N) {
  const size_t NT = (size_t)N * (N + 1) / 2;
  return (5 * (size_t)N * (N + 1) + (N + (N & 1)) + 2 * (size_t)N) * sizeof(double) +
         NT * sizeof(int) + 16;
}

// ---------------------------------------------------------------------------
// Increments D_j = W diag(phi(lambda - m) - 1) W^T (complex symmetric; upper
// triangle computed, mirrored), one step per CTA: binary64 for the binary64
// sweeps, binary32 from a binary32 copy of W for the mixed ones.  With
// phi(x) - 1 = (-2 sin^2(x/2), -sin x) there is no cancellation.
// ---------------------------------------------------------------------------
template <typename R, bool GWS>
__global__ void __launch_bounds__(256) k_increments(const double* __restrict__ Wg,
                                                    const double* __restrict__ eig, int N, int J,
                                                    double dt, double mshift,
                                                    void* __restrict__ Dout, size_t dstride,
                                                    unsigned char* gws, size_t per_cta) {
  using C = typename std::conditional<sizeof(R) == 8, double2, float2>::type;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  const int ld = N + 1, NT = N * (N + 1) / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  C* pm = reinterpret_cast<C*>(base);                 // [N]
  R* Ws = reinterpret_cast<R*>(pm + N);               // [N][ld]
  for (int j = blockIdx.x; j < J; j += gridDim.x) {
    const double* Wj = Wg + (size_t)j * N * N;
    for (int e = tid; e < N * N; e += nt) Ws[(e / N) * ld + (e % N)] = (R)Wj[e];
    for (int p = tid; p < N; p += nt) {
      const double x = dt * (eig[(size_t)j * N + p] - mshift);
      const double sh = sin(0.5 * x);
      C v;
      v.x = (R)(-2.0 * sh * sh);
      v.y = (R)(-sin(x));
      pm[p] = v;
    }
    __syncthreads();
    C* D = reinterpret_cast<C*>(reinterpret_cast<unsigned char*>(Dout) + (size_t)j * dstride);
    for (int t = tid; t < NT; t += nt) {
      int p, q;
      tri_index(t, N, p, q);
      R re = 0, im = 0;
      for (int r = 0; r < N; ++r) {
        const R w = Ws[p * ld + r] * Ws[q * ld + r];
        re = fma(w, pm[r].x, re);
        im = fma(w, pm[r].y, im);
      }
      C v;
      v.x = re;
      v.y = im;
      D[p * N + q] = v;
      D[q * N + p] = v;
    }
    __syncthreads();
  }
}

static size_t increments_bytes(int N, int d_fp64) {
  return (size_t)N * (d_fp64 ? 16 : 8) + (size_t)N * (N + 1) * (d_fp64 ? 8 : 4) + 16;
}

template <typename R>
static cudaError_t launch_inc(const double* W, const double* eig, int N, int J, double dt,
                              double mshift, void* D, size_t dstride, cudaStream_t st,
                              const StepSpace& ws) {
  StepGrid g;
  if (!step_grid(increments_bytes(N, sizeof(R) == 8), J, ws, (const void*)k_increments<R, false>, g))
    return cudaErrorInvalidConfiguration;
  const int threads = N <= 16 ? 128 : 256;
  if (g.gws)
    k_increments<R, true><<<g.grid, threads, g.smem, st>>>(W, eig, N, J, dt, mshift, D, dstride, g.gws,
                                                           g.per_cta);
  else
    k_increments<R, false><<<g.grid, threads, g.smem, st>>>(W, eig, N, J, dt, mshift, D, dstride, g.gws,
                                                            g.per_cta);
  return cudaGetLastError();
}

cudaError_t launch_prep(const double* W, const double* eig, const double* M, int N, int J,
                        double dt, double mshift, void* D, size_t dstride, int d_fp64,
                        int parts, double2* Ptil, double2* Xp, double* Mtil, int* status,
                        cudaStream_t st, const StepSpace& ws) {
  if (parts & PREP_D) {
    cudaError_t e = d_fp64 ? launch_inc<double>(W, eig, N, J, dt, mshift, D, dstride, st, ws)
                           : launch_inc<float>(W, eig, N, J, dt, mshift, D, dstride, st, ws);
    if (e != cudaSuccess) return e;
    parts &= ~PREP_D;
    if (!parts) return cudaSuccess;
  }
  StepGrid g;
  if (!d_fp64 && N <= 32) {
    // binary32-sweep problems: the products on the tensor cores
    const size_t sm = prep_smem_bytes(N) + oz_prep_bytes();
    if (sm <= max_dyn_smem((const void*)k_prep<256, false, true>)) {
      k_prep<256, false, true><<<J, 256, sm, st>>>(W, eig, M, N, J, dt, parts, Ptil, Xp, Mtil, status,
                                                   nullptr, 0);
      return cudaGetLastError();
    }
  }
  const int threads = N <= 8 ? 64 : (N <= 16 ? 128 : (N <= 128 ? 256 : 512));
  if (threads <= 256) {
    if (!step_grid(prep_smem_bytes(N), J, ws, (const void*)k_prep<256, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_prep<256, true><<<g.grid, threads, g.smem, st>>>(W, eig, M, N, J, dt, parts, Ptil, Xp, Mtil,
                                                         status, g.gws, g.per_cta);
    else
      k_prep<256, false><<<g.grid, threads, g.smem, st>>>(W, eig, M, N, J, dt, parts, Ptil, Xp, Mtil,
                                                          status, g.gws, g.per_cta);
  } else {
    if (!step_grid(prep_smem_bytes(N), J, ws, (const void*)k_prep<512, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_prep<512, true><<<g.grid, threads, g.smem, st>>>(W, eig, M, N, J, dt, parts, Ptil, Xp, Mtil,
                                                         status, g.gws, g.per_cta);
    else
      k_prep<512, false><<<g.grid, threads, g.smem, st>>>(W, eig, M, N, J, dt, parts, Ptil, Xp, Mtil,
                                                          status, g.gws, g.per_cta);
  }
  return cudaGetLastError();
}

}  // namespace qoc
