// Per-step eigendecompositions H_j = H0 + f_j M = W_j diag(lambda_j) W_j^T
// (Alg. 2, first loop: "compute and store the decomposition"; Sec. III-A
// takes exp(Z_j) through it).  All J decompositions are independent, so the
// grid runs one CTA per step.
//
//  * k_eig_jacobi<T>: parallel cyclic Jacobi in shared memory, round-robin
//    pair ordering (N/2 disjoint rotations per round), T = float or double.
//  * k_eig_refine: binary64 refinement of approximate eigenvectors by the
//    Ogita-Aishima iteration (Japan J. Indust. Appl. Math. 35, 2018,
//    "Iterative refinement for symmetric eigenvalue decomposition"): with
//    R = I - W^T W, S = W^T H W it sets lambda_i = S_ii / (1 - R_ii),
//    E_ik = (S_ik + lambda_k R_ik) / (lambda_k - lambda_i) for separated
//    pairs and R_ik / 2 inside clusters, and W <- W + W E.  Each sweep
//    squares the eigenvector error, so a binary32 Jacobi result reaches
//    binary64 accuracy in one or two sweeps at a fraction of the binary64
//    work of a full binary64 Jacobi (binary64 runs at 1/58 of the binary32
//    rate on GB300).
#include "common.cuh"
#include "kernels.hpp"
#include "ozaki.cuh"

namespace qoc {

template <typename T> struct JacobiEps;
template <> struct JacobiEps<float> { static constexpr double eps = 5.96e-8; static constexpr int max_sweeps = 24; };
template <> struct JacobiEps<double> { static constexpr double eps = 1.12e-16; static constexpr int max_sweeps = 40; };

// element at position `pos` of the round-robin schedule in round r (NP players)
__device__ __forceinline__ int rr_elem(int pos, int r, int NP) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (NP - 1)) + 1;
}

// Parallel cyclic Jacobi sweeps on the symmetric A (N x N, leading dimension
// ld, shared memory), accumulating the rotations into V (V <- V R).  In each
// round the N/2 disjoint pairs of the round-robin schedule are rotated at
// once: A <- R^T A R on 2 x 2 blocks (upper triangle, mirrored), V <- V R.
// A pair (p, q) is rotated when |a_pq| exceeds both the classical threshold
// (0.01 eps sqrt|a_pp a_qq|) and angle_tol |a_qq - a_pp| (a rotation smaller
// than angle_tol is not worth applying).  Stops when a sweep rotates nothing
// or off(A)^2 <= off_tol^2 * |A|_F^2.  Returns 1 when converged.
// Scratch: cs [NP], pr [NP] ints, red [>= 2*nwarps + 2] doubles (16-aligned).
template <typename T>
__device__ int jacobi_sweeps(T* A, T* V, int N, int ld, int max_sweeps, T angle_tol,
                             double off_tol, T* cs, int* pr, double* red) {
  const int NP = N + (N & 1);
  const int NH = NP / 2;
  const int tid = threadIdx.x, nt = blockDim.x;
  const T eps = (T)JacobiEps<T>::eps;
  __shared__ int nrot;
  int converged = 0;
  for (int sweep = 0; sweep < max_sweeps && !converged; ++sweep) {
    if (tid == 0) nrot = 0;
    __syncthreads();
    for (int r = 0; r < NP - 1; ++r) {
      if (tid < NH) {
        int p = rr_elem(tid, r, NP), q = rr_elem(NP - 1 - tid, r, NP);
        if (p > q) { int t = p; p = q; q = t; }
        T c = 1, s = 0;
        if (q < N) {
          T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          T thr = eps * (T)0.01 * sqrt(fabs(app) * fabs(aqq));
          T athr = angle_tol * fabs(aqq - app);
          if (fabs(apq) > thr && fabs(apq) > athr && apq != (T)0) {
            T th = (aqq - app) / (2 * apq);
            T t = (th >= 0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + 1));
            c = 1 / sqrt(t * t + 1);
            s = t * c;
            atomicAdd(&nrot, 1);
          }
        }
        pr[2 * tid] = p;
        pr[2 * tid + 1] = q;
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
      }
      __syncthreads();
      const int nblk = NH * (NH + 1) / 2;
      for (int b = tid; b < nblk + N * NH; b += nt) {
        if (b < nblk) {
          int k = 0, rem = b;
          while (rem >= NH - k) { rem -= NH - k; ++k; }
          const int l = k + rem;
          const T sk = cs[2 * k + 1], sl = cs[2 * l + 1];
          if (sk == (T)0 && sl == (T)0) continue;   // both identity: block unchanged
          const T ck = cs[2 * k], cl = cs[2 * l];
          const int p0 = pr[2 * k], p1 = pr[2 * k + 1], q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (p1 >= N || q1 >= N) {
            // blocks touching the dummy index of odd N: only real rows/cols move
            if (p1 < N && q1 >= N) {  // rows p0,p1 x column q0 (q0 unpaired)
              T x0 = A[p0 * ld + q0], x1 = A[p1 * ld + q0];
              T y0 = ck * x0 - sk * x1, y1 = sk * x0 + ck * x1;
              A[p0 * ld + q0] = y0; A[p1 * ld + q0] = y1;
              A[q0 * ld + p0] = y0; A[q0 * ld + p1] = y1;
            } else if (p1 >= N && q1 < N) {  // row p0 (unpaired) x columns q0,q1
              T x0 = A[p0 * ld + q0], x1 = A[p0 * ld + q1];
              T y0 = cl * x0 - sl * x1, y1 = sl * x0 + cl * x1;
              A[p0 * ld + q0] = y0; A[p0 * ld + q1] = y1;
              A[q0 * ld + p0] = y0; A[q1 * ld + p0] = y1;
            }
            continue;
          }
          T a00 = A[p0 * ld + q0], a01 = A[p0 * ld + q1], a10 = A[p1 * ld + q0], a11 = A[p1 * ld + q1];
          // left: R_k^T X, R = [[c s][-s c]];  right: (...) R_l
          T b00 = ck * a00 - sk * a10, b01 = ck * a01 - sk * a11;
          T b10 = sk * a00 + ck * a10, b11 = sk * a01 + ck * a11;
          T c00 = cl * b00 - sl * b01, c01 = sl * b00 + cl * b01;
          T c10 = cl * b10 - sl * b11, c11 = sl * b10 + cl * b11;
          if (k == l) {  // the rotated pair: its off-diagonal is zero by construction
            c01 = (T)0;
            c10 = (T)0;
          }
          A[p0 * ld + q0] = c00; A[p0 * ld + q1] = c01; A[p1 * ld + q0] = c10; A[p1 * ld + q1] = c11;
          if (k != l) {
            A[q0 * ld + p0] = c00; A[q1 * ld + p0] = c01; A[q0 * ld + p1] = c10; A[q1 * ld + p1] = c11;
          }
        } else {
          const int e = b - nblk;
          const int i = e / NH, l = e % NH;
          const T sl = cs[2 * l + 1];
          const int q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (q1 >= N || sl == (T)0) continue;
          const T cl = cs[2 * l];
          T v0 = V[i * ld + q0], v1 = V[i * ld + q1];
          V[i * ld + q0] = cl * v0 - sl * v1;
          V[i * ld + q1] = sl * v0 + cl * v1;
        }
      }
      __syncthreads();
    }
    // convergence: no rotation in the sweep, or off-diagonal small
    double off = 0, tot = 0;
    for (int e = tid; e < N * N; e += nt) {
      const int p = e / N, q = e % N;
      const double v = (double)A[p * ld + q];
      tot += v * v;
      if (p != q) off += v * v;
    }
    off = warp_sum(off);
    tot = warp_sum(tot);
    if ((tid & 31) == 0) { red[2 * (tid >> 5)] = off; red[2 * (tid >> 5) + 1] = tot; }
    __syncthreads();
    if (tid == 0) {
      double o = 0, t = 0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { o += red[2 * w]; t += red[2 * w + 1]; }
      red[63] = (nrot == 0 || o <= off_tol * off_tol * t || o == 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    converged = red[63] != 0.0;
    __syncthreads();
  }
  return converged;
}

// row-major upper-triangle index t -> (i, k), k >= i
__device__ __forceinline__ void tri_index_e(int t, int N, int& i, int& k) {
  const float b = 2.0f * N + 1.0f;
  int r = (int)floorf(0.5f * (b - sqrtf(fmaxf(b * b - 8.0f * t, 0.0f))));
  r = max(0, min(r, N - 1));
  while (r > 0 && r * N - r * (r - 1) / 2 > t) --r;
  while (r + 1 < N && (r + 1) * N - (r + 1) * r / 2 <= t) ++r;
  i = r;
  k = t - (r * N - r * (r - 1) / 2) + r;
}

// order-preserving integer key of a binary64 value (not NaN): comparing keys
// compares the values, without binary64 comparison instructions
__device__ __forceinline__ long long order_key(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ long long order_key(float x) { return order_key((double)x); }

// rank-sort the diagonal of A ascending (ties by index) and write W = V(:, order), lambda
template <typename T>
__device__ void sort_write(const T* A, const T* V, int N, int ld, double* Wj, double* ej) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const T di = A[i * ld + i];
    const long long ki = order_key(di);
    int rank = 0;
    for (int k = 0; k < N; ++k) {
      const long long kk = order_key(A[k * ld + k]);
      rank += (kk < ki) || (kk == ki && k < i);
    }
    ej[rank] = (double)di;
    for (int row = 0; row < N; ++row) Wj[row * N + rank] = (double)V[row * ld + i];
  }
}

template <typename T>
__device__ __forceinline__ void eig_jacobi_step(const double* __restrict__ H0,
                                                const double* __restrict__ M,
                                                const double* __restrict__ f, int N, int j,
                                                double* __restrict__ W_out,
                                                double* __restrict__ eig_out, int* status,
                                                unsigned char* smem_raw) {
  const int ld = N + 1;
  const int NP = N + (N & 1);
  T* A = reinterpret_cast<T*>(smem_raw);
  T* V = A + N * ld;
  T* cs = V + N * ld;
  int* pr = reinterpret_cast<int*>(cs + NP);
  double* red = reinterpret_cast<double*>(pr + NP + 2);
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 15) & ~uintptr_t(15));
  const int tid = threadIdx.x, nt = blockDim.x;
  const double fj = f[j];
  for (int e = tid; e < N * N; e += nt) {
    const int p = e / N, q = e % N;
    A[p * ld + q] = (T)(H0[e] + fj * M[e]);
    V[p * ld + q] = (T)(p == q ? 1.0 : 0.0);
  }
  __syncthreads();
  // The rounding floor of off(A) grows with N (about sqrt(N) eps |A|_F), so the
  // stopping tolerance does too: 4 eps for N <= 16, 4 eps sqrt(N / 16) above.
  // A binary32 result only seeds the binary64 refinement, which checks the
  // outcome itself; only the binary64 method reports non-convergence here.
  const double off_tol = 4.0 * JacobiEps<T>::eps * sqrt(fmax(1.0, N / 16.0));
  const int ok = jacobi_sweeps<T>(A, V, N, ld, JacobiEps<T>::max_sweeps, (T)0, off_tol, cs, pr, red);
  if (!ok && sizeof(T) == sizeof(double) && tid == 0) raise_status(status, DEV_EIG_NOCONV);
  sort_write<T>(A, V, N, ld, W_out + (size_t)j * N * N, eig_out + (size_t)j * N);
}

// One matrix per CTA in shared memory, or (gws != nullptr, large N) a
// persistent grid whose CTAs each own a slice of a global workspace.
// GWS: storage in the global workspace (compile-time, see k_eig_refine)
template <typename T, bool GWS>
__global__ void k_eig_jacobi(const double* __restrict__ H0, const double* __restrict__ M,
                             const double* __restrict__ f, int N, int J,
                             double* __restrict__ W_out, double* __restrict__ eig_out,
                             int* status, unsigned char* gws, size_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int j = blockIdx.x; j < J; j += gridDim.x) {
    eig_jacobi_step<T>(H0, M, f, N, j, W_out, eig_out, status, base);
    __syncthreads();
  }
}

// Ogita-Aishima refinement sweeps in binary64 (at most `sweeps` updates,
// stopping once |I - W^T W|_F reaches the binary64 floor), then a binary64
// Jacobi clean-up of S = W^T H W that resolves what the refinement leaves
// alone (pairs closer than its cluster threshold), then W <- W V.
// OZ: the binary64 products H W, W^T (H W) and W^T W on the tensor cores by
// error-free splitting (ozaki.cuh; N <= 32, 256 threads); used for the
// relaxed refinement of problems on binary32 sweeps.
constexpr int kOzSlices = 6;
struct OzSpace {
  __nv_bfloat16 *Hs, *Ws, *Ts;   // [kOzSlices][32][oz::LD] each
  int *eH, *eW, *eT;             // [32] each
};
__host__ __device__ inline size_t oz_smem_bytes() {
  return 3 * (size_t)kOzSlices * 32 * oz::LD * 2 + 3 * 32 * 4 + 16;
}

template <bool OZ>
__device__ __forceinline__ void eig_refine_step(const double* __restrict__ H0,
                                                const double* __restrict__ M,
                                                const double* __restrict__ f, int N, int j,
                                                int sweeps, double angle_tol,
                                                double* __restrict__ W_io,
                                                double* __restrict__ eig_out, int* status,
                                                unsigned int* stats, double finish_tol,
                                                unsigned char* smem_raw) {
  const int ld = N + 1;
  const int NP = N + (N & 1);
  double *H, *W, *T, *S, *R, *lam, *red, *cs;
  int* pr;
  float *Wf, *Ef;
  double* Tc;                        // scratch of the clean-up's W V product
  OzSpace oz{};
  if (OZ) {
    // Three binary64 matrices instead of five, so that three CTAs fit an SM:
    // H lives in T until it is split (its slices are all the products use),
    // S overwrites T once T is split, and the binary32 W and E of the update
    // (and the clean-up's scratch) use the slice buffers of W and T, which
    // are dead from the S and R products to the next update's split of W.
    W = reinterpret_cast<double*>(smem_raw);
    T = W + N * ld;
    R = T + N * ld;
    H = T;
    S = T;
    lam = R + N * ld;
    red = lam + N + 1;
    cs = red + 64;
    pr = reinterpret_cast<int*>(cs + NP);
    unsigned char* ob = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(pr + NP + 2) + 15) & ~uintptr_t(15));
    const size_t sl = (size_t)kOzSlices * 32 * oz::LD;
    oz.Hs = reinterpret_cast<__nv_bfloat16*>(ob);
    oz.Ws = oz.Hs + sl;
    oz.Ts = oz.Ws + sl;
    oz.eH = reinterpret_cast<int*>(oz.Ts + sl);
    oz.eW = oz.eH + 32;
    oz.eT = oz.eW + 32;
    Wf = reinterpret_cast<float*>(oz.Ws);
    Ef = reinterpret_cast<float*>(oz.Ts);
    Tc = reinterpret_cast<double*>(oz.Ws);
  } else {
    H = reinterpret_cast<double*>(smem_raw);
    W = H + N * ld;
    T = W + N * ld;
    S = T + N * ld;
    R = S + N * ld;
    lam = R + N * ld;                // [N + 1]
    red = lam + N + 1;               // [64]
    cs = red + 64;                   // [NP]
    pr = reinterpret_cast<int*>(cs + NP);  // [NP + 2]
    Wf = reinterpret_cast<float*>(
        (reinterpret_cast<uintptr_t>(pr + NP + 2) + 15) & ~uintptr_t(15));   // [N][ld] binary32 W
    Ef = Wf + N * ld;                                                        // [N][ld] binary32 E
    Tc = T;
  }
  const int tid = threadIdx.x, nt = blockDim.x;
  const double fj = f[j];
  double* Wg = W_io + (size_t)j * N * N;
  double hn = 0;
  for (int e = tid; e < N * N; e += nt) {
    const int p = e / N, q = e % N;
    const double h = H0[e] + fj * M[e];
    H[p * ld + q] = h;
    W[p * ld + q] = Wg[e];
    hn += h * h;
  }
  hn = warp_sum(hn);
  if ((tid & 31) == 0) red[tid >> 5] = hn;
  __syncthreads();
  if (tid == 0) {
    double s = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) s += red[w];
    red[40] = sqrt(s);
  }
  __syncthreads();
  const double Hnorm = red[40];
  if (OZ) oz::split32<kOzSlices>(H, ld, N, true, oz.Hs, oz.eH);

  // Refinement sweeps until W is orthonormal to the binary64 floor: each sweep
  // computes S = W^T H W and R = I - W^T W; when |R|_F <= orth_tol, S is the
  // matrix the clean-up diagonalises, otherwise W <- W (I + E).
  // rounding floor of |I - W^T W|_F for an orthonormal W: ~ eps N^1.5
  const double orth_tol = 8.0 * 1.12e-16 * (double)N * sqrt((double)N);
  // Early finish: when an update has no cluster pairs and both |R|_F and the
  // largest |E_ik| are below kDone = sqrt(orth_tol) / 10, the updated W is
  // orthonormal and accurate to the binary64 floor (the next residual is
  // O(|E|^2 + |R| |E|) <= orth_tol / 50), and the Rayleigh quotients lambda of
  // this pass are exact to O(|E|^2 |H|): the final residual pass and the
  // clean-up are skipped.
  // finish_tol > 0 (relaxed finish, for callers whose results need only the
  // residual H W - W Lambda, relative to |H|, at about 1e-9): an update with
  // no cluster pairs, |R|_F <= finish_tol and |E|_F |off(S)|_F <= kRes |H|_F
  // ends the refinement.  The update cancels the residual to first order, so
  // what it leaves is O(|E| |off(S)| + |R|^2) -- a pair of close eigenvalues
  // may keep a sizeable rotation between its two eigenvectors, which moves
  // smooth functions of H (the propagator and its Frechet derivatives) only
  // through that residual.  Its W E is formed in binary32 like every
  // non-final update.
  const bool relaxed = finish_tol > 0;
  constexpr double kRes = 1e-9;
  const double kDone = relaxed ? finish_tol : 0.1 * sqrt(orth_tol);
  __shared__ int not_done;
  bool finished = false;
  for (int it = 0;; ++it) {
    double rn = 0;
    if (OZ) {
      // T = H W, S = W^T T, R <- W^T W on the tensor cores; then the upper
      // triangles mirrored (exactly symmetric S, R) and R = I - W^T W
      oz::split32<kOzSlices>(W, ld, N, false, oz.Ws, oz.eW);
      oz::mm32<kOzSlices>(oz.Hs, oz.eH, oz.Ws, oz.eW, T, ld, N);
      __syncthreads();
      oz::split32<kOzSlices>(T, ld, N, false, oz.Ts, oz.eT);
      oz::mm32<kOzSlices>(oz.Ws, oz.eW, oz.Ts, oz.eT, S, ld, N);
      oz::mm32<kOzSlices>(oz.Ws, oz.eW, oz.Ws, oz.eW, R, ld, N);
      __syncthreads();
      for (int t = tid; t < N * (N + 1) / 2; t += nt) {
        int i, k;
        tri_index_e(t, N, i, k);
        S[k * ld + i] = S[i * ld + k];
        const double rr = (i == k ? 1.0 : 0.0) - R[i * ld + k];
        R[i * ld + k] = rr;
        R[k * ld + i] = rr;
        rn += (i == k ? 1.0 : 2.0) * rr * rr;
      }
      __syncthreads();
    } else {
    // T = H W
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, k = e % N;
      double acc = 0;
      for (int r = 0; r < N; ++r) acc = fma(H[i * ld + r], W[r * ld + k], acc);
      T[i * ld + k] = acc;
    }
    __syncthreads();
    // S = W^T T, R = I - W^T W (both symmetric: upper triangle, mirrored)
    for (int t = tid; t < N * (N + 1) / 2; t += nt) {
      int i, k;
      tri_index_e(t, N, i, k);
      double sa = 0, w = 0;
      for (int r = 0; r < N; ++r) {
        const double wri = W[r * ld + i];
        sa = fma(wri, T[r * ld + k], sa);
        w = fma(wri, W[r * ld + k], w);
      }
      S[i * ld + k] = sa;
      S[k * ld + i] = sa;
      const double rr = (i == k ? 1.0 : 0.0) - w;
      R[i * ld + k] = rr;
      R[k * ld + i] = rr;
      rn += (i == k ? 1.0 : 2.0) * rr * rr;
    }
    __syncthreads();
    }
    // off(S) with the diagonal's correction S_ii - lambda_i: the diagonal
    // terms here, the off-diagonal ones below (no per-warp diagonal branch:
    // a binary64 warp instruction costs the pipe the same for one lane)
    double sn = 0;
    float* lamf = reinterpret_cast<float*>(cs);   // binary32 eigenvalues (cs is free until the clean-up)
    for (int i = tid; i < N; i += nt) {
      const double l = S[i * ld + i] / (1.0 - R[i * ld + i]);
      lam[i] = l;
      if (OZ) lamf[i] = (float)l;
      const double d = S[i * ld + i] - l;
      sn = fma(d, d, sn);
    }
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, k = e % N;
      const double sik = i != k ? S[i * ld + k] : 0.0;
      sn = fma(sik, sik, sn);
    }
    sn = warp_sum(sn);
    rn = warp_sum(rn);
    if ((tid & 31) == 0) { red[2 * (tid >> 5)] = sn; red[2 * (tid >> 5) + 1] = rn; }
    __syncthreads();
    if (tid == 0) {
      double a = 0, b = 0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
      red[41] = 2.0 * (sqrt(a) + Hnorm * sqrt(b));  // cluster threshold delta
      red[42] = sqrt(b);                             // |I - W^T W|_F
      red[43] = sqrt(a);                             // |off(S)|_F with the diagonal's correction
    }
    __syncthreads();
    const double delta = red[41];
    if (red[42] <= orth_tol || it >= sweeps) {
      // sweep budget spent: flag only a real failure
      if (red[42] > orth_tol && tid == 0 && !(red[42] <= 1e-10)) raise_status(status, DEV_EIG_NOCONV);
      if (stats && tid == 0) atomicAdd(&stats[0], (unsigned int)it);
      break;
    }
    // E overwrites T.  A pair counts as separated only if it is outside the
    // cluster threshold AND its first-order correction is small (|S_ik| <=
    // kLinear |gap|): a binary32 start can mix two close eigenvectors by a
    // large angle (near an avoided crossing), where the linearised update
    // would destroy orthogonality.  Such pairs only get the orthogonality
    // part R/2 here; the binary64 Jacobi clean-up rotates them exactly.
    constexpr double kLinear = 1e-3;
    if (tid == 0) not_done = red[42] > kDone ? 1 : 0;
    __syncthreads();
    double esq = 0;
    if (OZ) {
      // Relaxed refinement with its W E in binary32: E itself in binary32,
      // straight into the binary32 buffer.  The gaps come from binary32
      // eigenvalues and S_ik + lambda_k R_ik cancels by up to |lambda| / gap,
      // so E_ik carries a relative error of about eps32 |H| / gap (1e-4 at the
      // closest gaps of the workloads); what the update then leaves is that
      // times |E_ik| gap, far below the 1e-9 |H| residual this path is for.
      const float deltaf = (float)delta;
      float esqf = 0.f;
      for (int e = tid; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        const float rik = (float)R[i * ld + k];
        float eik;
        if (i == k) eik = 0.5f * rik;
        else {
          const float gap = lamf[k] - lamf[i];
          const float sik = (float)S[i * ld + k];
          const bool sep = fabsf(gap) > deltaf && fabsf(sik) <= (float)kLinear * fabsf(gap);
          eik = sep ? fmaf(lamf[k], rik, sik) * __frcp_rn(gap) : 0.5f * rik;
          if (!sep) not_done = 1;
          esqf = fmaf(eik, eik, esqf);
        }
        Ef[i * ld + k] = eik;
      }
      esq = (double)esqf;
    } else {
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, k = e % N;
      const double rik = R[i * ld + k];
      double eik;
      if (i == k) eik = 0.5 * rik;
      else {
        const double gap = lam[k] - lam[i];
        const double sik = S[i * ld + k];
        const bool sep = fabs(gap) > delta && fabs(sik) <= kLinear * fabs(gap);
        eik = sep ? (sik + lam[k] * rik) / gap : 0.5 * rik;
        if (!sep || (!relaxed && fabs(eik) > kDone)) not_done = 1;
        esq = fma(eik, eik, esq);
      }
      T[i * ld + k] = eik;
    }
    }
    if (relaxed) {   // |E|_F |off(S)|_F against kRes |H|_F
      esq = warp_sum(esq);
      if ((tid & 31) == 0) red[2 * (tid >> 5)] = esq;
      __syncthreads();
      if (tid == 0) {
        double es = 0;
        for (int w = 0; w < (nt + 31) / 32; ++w) es += red[2 * w];
        if (sqrt(es) * red[43] > kRes * Hnorm) not_done = 1;
      }
    }
    __syncthreads();
    // W <- W + W E (R as scratch for W E).  An update that cannot end the
    // refinement (some |E_ik| or |R|_F above kDone) forms the product in
    // binary32: E is then a correction the next update refines, and the
    // binary32 product is off by about N eps32 |W| |E|, far below the error
    // that update removes.  A finishing update forms it in binary64.
    if (not_done || relaxed) {
      for (int e = tid; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        Wf[i * ld + k] = (float)W[i * ld + k];
        if (!OZ) Ef[i * ld + k] = (float)T[i * ld + k];
      }
      __syncthreads();
      for (int e = tid; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        float acc = 0.f;
        for (int r = 0; r < N; ++r) acc = fmaf(Wf[i * ld + r], Ef[r * ld + k], acc);
        R[i * ld + k] = (double)acc;
      }
    } else {
      for (int e = tid; e < N * N; e += nt) {
        const int i = e / N, k = e % N;
        double acc = 0;
        for (int r = 0; r < N; ++r) acc = fma(W[i * ld + r], T[r * ld + k], acc);
        R[i * ld + k] = acc;
      }
    }
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, k = e % N;
      W[i * ld + k] += R[i * ld + k];
    }
    if (!not_done) {   // uniform across the CTA (read after the barrier above)
      for (int i = tid; i < N; i += nt) S[i * ld + i] = lam[i];
      if (stats && tid == 0) atomicAdd(&stats[0], (unsigned int)(it + 1));
      finished = true;
      __syncthreads();
      break;
    }
    __syncthreads();
  }
  if (!finished) {
  if (stats && tid == 0) atomicAdd(&stats[2], 1u);
  // clean-up: Jacobi on S = W^T H W with V = I (in R)
  for (int e = tid; e < N * N; e += nt) R[(e / N) * ld + (e % N)] = (e / N == e % N) ? 1.0 : 0.0;
  __syncthreads();
  __shared__ int any_rot;
  if (tid == 0) any_rot = 0;
  __syncthreads();
  // stops at no rotation or once off(S) is at the rounding floor of
  // S = W^T H W itself (length-N dot products: about N eps |S|_F; 8 N eps used):
  // a pair still mixed below that is a near-degenerate one whose mixing changes
  // neither the propagator nor the eigenvalues measurably
  const int ok = jacobi_sweeps<double>(S, R, N, ld, N <= 64 ? 12 : 30, angle_tol,
                                       8.0 * 1.12e-16 * (double)N, cs, pr, red);
  if (!ok && tid == 0) raise_status(status, DEV_EIG_NOCONV);
  // did anything rotate?  (V != I)
  for (int e = tid; e < N * N; e += nt) {
    const int i = e / N, k = e % N;
    if (R[i * ld + k] != ((i == k) ? 1.0 : 0.0)) any_rot = 1;
  }
  __syncthreads();
  if (stats && tid == 0 && any_rot) atomicAdd(&stats[1], 1u);
  if (any_rot) {   // W <- W V (Tc as scratch)
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, k = e % N;
      double acc = 0;
      for (int r = 0; r < N; ++r) acc = fma(W[i * ld + r], R[r * ld + k], acc);
      Tc[i * ld + k] = acc;
    }
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) W[(e / N) * ld + (e % N)] = Tc[(e / N) * ld + (e % N)];
    __syncthreads();
  }
  }
  bool bad = false;
  for (int i = tid; i < N; i += nt) bad |= !isfinite(S[i * ld + i]);
  if (bad) raise_status(status, DEV_NONFINITE);
  sort_write<double>(S, W, N, ld, Wg, eig_out + (size_t)j * N);
}

// MAXT: the launch's thread count bound; 256 keeps at least 4 CTAs of
// registers per SM (the binary64 pipe wants every resident warp), 512 is the
// large-N launch.  GWS: storage in the global workspace (a compile-time
// choice, so that the shared-memory instantiation keeps shared-memory loads).
template <int MAXT, bool GWS, bool OZ = false>
__global__ void __launch_bounds__(MAXT, OZ ? 3 : (MAXT <= 256 ? 4 : 1))
k_eig_refine(const double* __restrict__ H0, const double* __restrict__ M,
                             const double* __restrict__ f, int N, int J, int sweeps,
                             double angle_tol, double* __restrict__ W_io,
                             double* __restrict__ eig_out, int* status, unsigned int* stats,
                             double finish_tol, unsigned char* gws, size_t per_cta,
                             const int* __restrict__ order) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int b = blockIdx.x; b < J; b += gridDim.x) {
    int j = order ? order[b] : b;   // a permutation of the steps
    if ((unsigned)j >= (unsigned)J) j = b;
    eig_refine_step<OZ>(H0, M, f, N, j, sweeps, angle_tol, W_io, eig_out, status, stats, finish_tol, base);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Binary32 Jacobi with one warp per matrix (several matrices per CTA): the
// round-robin parallel cyclic scheme of jacobi_sweeps, synchronised by
// __syncwarp only.  In a round every lane updates whole 2 x 2 blocks
// R_k^T A R_l of the full matrix (each element belongs to exactly one block,
// so nothing is mirrored) and rows of V R; the (k, l) and (i, l)
// enumerations advance by a fixed stride with a carry instead of divisions.
// Convergence: no rotation in a sweep, or off(A)^2 <= (4 eps)^2 |A|_F^2.
// ---------------------------------------------------------------------------
__host__ __device__ inline int jacobi32_slot_floats(int N) {
  const int NP = N + (N & 1);
  const int n = 2 * N * (N + 1) + 2 * NP;
  return (n + 3) & ~3;
}

__device__ __forceinline__ float warp_sum_f(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(128) k_eig_jacobi32(const double* __restrict__ H0,
                                                      const double* __restrict__ M,
                                                      const double* __restrict__ f, int N, int J,
                                                      int mpb, double* __restrict__ W_out,
                                                      double* __restrict__ eig_out, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.x * mpb + wid;
  if (wid >= mpb || j >= J) return;   // whole warps leave; only __syncwarp below
  const int ld = N + 1, NP = N + (N & 1), NH = NP / 2;
  float* A = reinterpret_cast<float*>(smem_raw) + (size_t)wid * jacobi32_slot_floats(N);
  float* V = A + N * ld;
  float* cs = V + N * ld;                        // [NP]: c_k, s_k
  int* pr = reinterpret_cast<int*>(cs + NP);     // [NP]: p_k, q_k
  const double fj = f[j];
  for (int p = 0; p < N; ++p)
    for (int q = lane; q < N; q += 32) {
      A[p * ld + q] = (float)(H0[p * N + q] + fj * M[p * N + q]);
      V[p * ld + q] = p == q ? 1.f : 0.f;
    }
  __syncwarp();
  const float eps = 5.96e-8f;
  const float off_tol2 = 16.f * eps * eps;
  const int kstep = 32 % NH, lstep = 32 / NH;    // stride 32 in a (row, col) enumeration over NH
  const int NR = NP - 1;                         // rounds per sweep
  bool converged = false;
  for (int sweep = 0; sweep < 24 && !converged; ++sweep) {
    bool rot = false;
    // round-robin positions of this lane's pair, advanced by one per round
    int pa = (lane + NR - 1) % NR, qa = (NR - 1 - lane + NR) % NR;
    for (int r = 0; r < NR; ++r) {
      if (lane < NH) {
        int p = lane == 0 ? 0 : pa + 1, q = qa + 1;
        if (p > q) { const int t = p; p = q; q = t; }
        float c = 1.f, s = 0.f;
        if (q < N) {
          const float apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          const float thr = eps * 0.01f * sqrtf(fabsf(app) * fabsf(aqq));
          if (fabsf(apq) > thr && apq != 0.f) {
            // binary32 start only (refined in binary64): fast reciprocals suffice
            const float th = __fdividef(aqq - app, 2.f * apq);
            const float t = copysignf(__fdividef(1.f, fabsf(th) + sqrtf(fmaf(th, th, 1.f))), th);
            c = rsqrtf(fmaf(t, t, 1.f));
            s = t * c;
            rot = true;
          }
        }
        pr[2 * lane] = p;
        pr[2 * lane + 1] = q;
        cs[2 * lane] = c;
        cs[2 * lane + 1] = s;
      }
      if (++pa == NR) pa = 0;
      if (++qa == NR) qa = 0;
      __syncwarp();
      if (N == 32) {
        // N = 32 exactly: every lane owns 8 blocks (k, l = lane / 16 + 2 t) and
        // 16 rows of its V column pair, all valid (no dummy index), so a batch
        // of four blocks (eight rows) is loaded before any is stored with no
        // guards; the blocks of a round are disjoint.  (c, s) and the index
        // pair of a rotation are one 8-byte load each.  Same arithmetic as the
        // general path below.
        const int k = lane & 15, lb = lane >> 4;
        const float2 csk = reinterpret_cast<const float2*>(cs)[k];
        const int2 prk = reinterpret_cast<const int2*>(pr)[k];
        const float ck = csk.x, sk = csk.y;
        const int p0 = prk.x, p1 = prk.y;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          float a00[4], a01[4], a10[4], a11[4];
          float2 csl[4];
          int2 prl[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int l = lb + 2 * (4 * h + u);
            csl[u] = reinterpret_cast<const float2*>(cs)[l];
            prl[u] = reinterpret_cast<const int2*>(pr)[l];
            a00[u] = A[p0 * ld + prl[u].x];
            a01[u] = A[p0 * ld + prl[u].y];
            a10[u] = A[p1 * ld + prl[u].x];
            a11[u] = A[p1 * ld + prl[u].y];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int l = lb + 2 * (4 * h + u);
            const float cl = csl[u].x, sl = csl[u].y;
            if (sk == 0.f && sl == 0.f) continue;   // both identity: block unchanged
            const int q0 = prl[u].x, q1 = prl[u].y;
            const float b00 = ck * a00[u] - sk * a10[u], b01 = ck * a01[u] - sk * a11[u];
            const float b10 = sk * a00[u] + ck * a10[u], b11 = sk * a01[u] + ck * a11[u];
            A[p0 * ld + q0] = cl * b00 - sl * b01;
            A[p1 * ld + q1] = sl * b10 + cl * b11;
            if (k == l) {
              A[p0 * ld + q1] = 0.f;
              A[p1 * ld + q0] = 0.f;
            } else {
              A[p0 * ld + q1] = sl * b00 + cl * b01;
              A[p1 * ld + q0] = cl * b10 - sl * b11;
            }
          }
        }
        if (sk != 0.f) {   // V <- V R on column pair k, rows lane / 16 + 2 t
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            float v0[8], v1[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int i = lb + 2 * (8 * h + u);
              v0[u] = V[i * ld + p0];
              v1[u] = V[i * ld + p1];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int i = lb + 2 * (8 * h + u);
              V[i * ld + p0] = ck * v0[u] - sk * v1[u];
              V[i * ld + p1] = sk * v0[u] + ck * v1[u];
            }
          }
        }
        __syncwarp();
        continue;
      }
      if (kstep == 0) {
        // NH divides 32: every lane keeps one row pair k (blocks) and one column pair l (V)
        const int k = lane % NH;
        const float ck = cs[2 * k], sk = cs[2 * k + 1];
        const int p0 = pr[2 * k], p1 = pr[2 * k + 1];
        for (int l = lane / NH; l < NH; l += lstep) {
          const float sl = cs[2 * l + 1];
          if (sk == 0.f && sl == 0.f) continue;
          const float cl = cs[2 * l];
          const int q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (p1 >= N) {
            if (q1 < N) {
              const float x0 = A[p0 * ld + q0], x1 = A[p0 * ld + q1];
              A[p0 * ld + q0] = cl * x0 - sl * x1;
              A[p0 * ld + q1] = sl * x0 + cl * x1;
            }
          } else if (q1 >= N) {
            const float x0 = A[p0 * ld + q0], x1 = A[p1 * ld + q0];
            A[p0 * ld + q0] = ck * x0 - sk * x1;
            A[p1 * ld + q0] = sk * x0 + ck * x1;
          } else {
            const float a00 = A[p0 * ld + q0], a01 = A[p0 * ld + q1];
            const float a10 = A[p1 * ld + q0], a11 = A[p1 * ld + q1];
            const float b00 = ck * a00 - sk * a10, b01 = ck * a01 - sk * a11;
            const float b10 = sk * a00 + ck * a10, b11 = sk * a01 + ck * a11;
            A[p0 * ld + q0] = cl * b00 - sl * b01;
            A[p1 * ld + q1] = sl * b10 + cl * b11;
            if (k == l) {
              A[p0 * ld + q1] = 0.f;
              A[p1 * ld + q0] = 0.f;
            } else {
              A[p0 * ld + q1] = sl * b00 + cl * b01;
              A[p1 * ld + q0] = cl * b10 - sl * b11;
            }
          }
        }
        // V <- V R: this lane's column pair is k, rows i = lane / NH + lstep t
        if (sk != 0.f && p1 < N) {
          for (int i = lane / NH; i < N; i += lstep) {
            const float v0 = V[i * ld + p0], v1 = V[i * ld + p1];
            V[i * ld + p0] = ck * v0 - sk * v1;
            V[i * ld + p1] = sk * v0 + ck * v1;
          }
        }
        __syncwarp();
        continue;
      }
      // A <- R^T A R, block (k, l): rows of pair k, columns of pair l
      for (int k = lane % NH, l = lane / NH; l < NH;) {
        const float sk = cs[2 * k + 1], sl = cs[2 * l + 1];
        if (sk != 0.f || sl != 0.f) {
          const float ck = cs[2 * k], cl = cs[2 * l];
          const int p0 = pr[2 * k], p1 = pr[2 * k + 1], q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (p1 >= N) {          // pair k holds the dummy index of odd N: row p0 only
            if (q1 < N) {
              const float x0 = A[p0 * ld + q0], x1 = A[p0 * ld + q1];
              A[p0 * ld + q0] = cl * x0 - sl * x1;
              A[p0 * ld + q1] = sl * x0 + cl * x1;
            }
          } else if (q1 >= N) {   // pair l holds the dummy: column q0 only
            const float x0 = A[p0 * ld + q0], x1 = A[p1 * ld + q0];
            A[p0 * ld + q0] = ck * x0 - sk * x1;
            A[p1 * ld + q0] = sk * x0 + ck * x1;
          } else {
            const float a00 = A[p0 * ld + q0], a01 = A[p0 * ld + q1];
            const float a10 = A[p1 * ld + q0], a11 = A[p1 * ld + q1];
            const float b00 = ck * a00 - sk * a10, b01 = ck * a01 - sk * a11;
            const float b10 = sk * a00 + ck * a10, b11 = sk * a01 + ck * a11;
            A[p0 * ld + q0] = cl * b00 - sl * b01;
            A[p1 * ld + q1] = sl * b10 + cl * b11;
            if (k == l) {         // the rotated pair: its off-diagonal is zero by construction
              A[p0 * ld + q1] = 0.f;
              A[p1 * ld + q0] = 0.f;
            } else {
              A[p0 * ld + q1] = sl * b00 + cl * b01;
              A[p1 * ld + q0] = cl * b10 - sl * b11;
            }
          }
        }
        k += kstep;
        l += lstep;
        if (k >= NH) { k -= NH; ++l; }
      }
      // V <- V R, row i, pair l
      for (int l = lane % NH, i = lane / NH; i < N;) {
        const float sl = cs[2 * l + 1];
        const int q1 = pr[2 * l + 1];
        if (sl != 0.f && q1 < N) {
          const float cl = cs[2 * l];
          const int q0 = pr[2 * l];
          const float v0 = V[i * ld + q0], v1 = V[i * ld + q1];
          V[i * ld + q0] = cl * v0 - sl * v1;
          V[i * ld + q1] = sl * v0 + cl * v1;
        }
        l += kstep;
        i += lstep;
        if (l >= NH) { l -= NH; ++i; }
      }
      __syncwarp();
    }
    float off = 0.f, tot = 0.f;
    for (int p = 0; p < N; ++p)
      for (int q = lane; q < N; q += 32) {
        const float v = A[p * ld + q];
        tot = fmaf(v, v, tot);
        if (p != q) off = fmaf(v, v, off);
      }
    off = warp_sum_f(off);
    tot = warp_sum_f(tot);
    converged = !__any_sync(0xffffffffu, rot) || off <= off_tol2 * tot || off == 0.f;
  }
  if (!converged && lane == 0) raise_status(status, DEV_EIG_NOCONV);
  // rank-sort the diagonal (ties by index) and write W = V(:, order), lambda
  double* Wj = W_out + (size_t)j * N * N;
  for (int i = lane; i < N; i += 32) {
    const float di = A[i * ld + i];
    int rank = 0;
    for (int k = 0; k < N; ++k) {
      const float dk = A[k * ld + k];
      rank += (dk < di) || (dk == di && k < i);
    }
    eig_out[(size_t)j * N + rank] = (double)di;
    for (int row = 0; row < N; ++row) Wj[row * N + rank] = (double)V[row * ld + i];
  }
}

// rounds per loop body of the register-resident N = 32 start (0: the
// shared-memory kernel below for N = 32 too)
#ifndef QOC_JACOBI32_ROUNDS
#define QOC_JACOBI32_ROUNDS 4
#endif

static int jacobi32_mpb(int N) { return N <= 16 ? 4 : (N <= 40 ? 2 : 1); }

static size_t jacobi_smem(int N, size_t tsize) {
  const int NP = N + (N & 1);
  size_t s = 2 * (size_t)N * (N + 1) * tsize + (size_t)NP * tsize + (size_t)(NP + 2) * sizeof(int);
  s = (s + 15) & ~size_t(15);
  return s + 64 * sizeof(double) + 16;
}
// the tensor-core refinement's layout: W, T (H, then S), R, then the slices
static size_t refine_oz_smem(int N) {
  const int NP = N + (N & 1);
  return (3 * (size_t)N * (N + 1) + N + 1 + 64 + NP) * sizeof(double) + (NP + 2) * sizeof(int) + 16 +
         oz_smem_bytes();
}

static size_t refine_smem(int N) {
  const int NP = N + (N & 1);
  return (5 * (size_t)N * (N + 1) + N + 1 + 64 + NP) * sizeof(double) + (NP + 2) * sizeof(int) + 16 +
         2 * (size_t)N * (N + 1) * sizeof(float);
}

cudaError_t launch_eig(const double* H0, const double* M, const double* f, int N, int J,
                       double* W, double* eig, int* status, int method, int refine_sweeps,
                       double angle_tol, cudaStream_t st, const StepSpace& ws, cudaEvent_t mid,
                       unsigned int* stats, double finish_tol, int phases, int* order) {
  // Jacobi rounds are barrier-bound: few warps per (small) matrix, many CTAs per SM
  const int jthreads = N <= 32 ? 64 : (N <= 64 ? 128 : (N <= 128 ? 256 : 512));
  const int threads = N <= 16 ? 128 : (N <= 128 ? 256 : 512);   // refinement: binary64-bound
  StepGrid g;
  if (method == EIG_JACOBI_FP64) {
    if (!step_grid(jacobi_smem(N, 8), J, ws, (const void*)k_eig_jacobi<double, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_eig_jacobi<double, true><<<g.grid, jthreads, g.smem, st>>>(H0, M, f, N, J, W, eig, status,
                                                                   g.gws, g.per_cta);
    else
      k_eig_jacobi<double, false><<<g.grid, jthreads, g.smem, st>>>(H0, M, f, N, J, W, eig, status,
                                                                    g.gws, g.per_cta);
    if (mid) cudaEventRecord(mid, st);
    return cudaGetLastError();
  }
  if (!(phases & EIG_PHASE_START) || !(N == 32 && QOC_JACOBI32_ROUNDS > 0)) order = nullptr;
  if (!(phases & EIG_PHASE_START)) {
  } else if (N == 32 && QOC_JACOBI32_ROUNDS > 0) {
    if (phases != EIG_PHASE_ALL) order = nullptr;
    const cudaError_t e = launch_eig_jacobi32_reg(H0, M, f, J, W, eig, status, QOC_JACOBI32_ROUNDS, order, st);
    if (e != cudaSuccess) return e;
  } else if (N <= 64) {
    const int mpb = jacobi32_mpb(N);
    const size_t sm = (size_t)mpb * jacobi32_slot_floats(N) * sizeof(float);
    set_max_smem((const void*)k_eig_jacobi32);
    k_eig_jacobi32<<<(J + mpb - 1) / mpb, 32 * mpb, sm, st>>>(H0, M, f, N, J, mpb, W, eig, status);
  } else {
    if (!step_grid(jacobi_smem(N, 4), J, ws, (const void*)k_eig_jacobi<float, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_eig_jacobi<float, true><<<g.grid, jthreads, g.smem, st>>>(H0, M, f, N, J, W, eig, status,
                                                                  g.gws, g.per_cta);
    else
      k_eig_jacobi<float, false><<<g.grid, jthreads, g.smem, st>>>(H0, M, f, N, J, W, eig, status,
                                                                   g.gws, g.per_cta);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (mid) cudaEventRecord(mid, st);
  if (!(phases & EIG_PHASE_REFINE)) return cudaSuccess;
  if (N <= 32 && finish_tol > 0) {
    // relaxed refinement (binary32 sweeps): products on the tensor cores
    const size_t sm = refine_oz_smem(N);
    if (sm <= max_dyn_smem((const void*)k_eig_refine<256, false, true>)) {
      k_eig_refine<256, false, true><<<J, 256, sm, st>>>(H0, M, f, N, J, refine_sweeps, angle_tol, W, eig,
                                                         status, stats, finish_tol, nullptr, 0, order);
      return cudaGetLastError();
    }
  }
  if (threads <= 256) {
    if (!step_grid(refine_smem(N), J, ws, (const void*)k_eig_refine<256, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_eig_refine<256, true><<<g.grid, threads, g.smem, st>>>(H0, M, f, N, J, refine_sweeps, angle_tol,
                                                               W, eig, status, stats, finish_tol, g.gws, g.per_cta, order);
    else
      k_eig_refine<256, false><<<g.grid, threads, g.smem, st>>>(H0, M, f, N, J, refine_sweeps, angle_tol,
                                                                W, eig, status, stats, finish_tol, g.gws, g.per_cta, order);
  } else {
    if (!step_grid(refine_smem(N), J, ws, (const void*)k_eig_refine<512, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_eig_refine<512, true><<<g.grid, threads, g.smem, st>>>(H0, M, f, N, J, refine_sweeps, angle_tol,
                                                               W, eig, status, stats, finish_tol, g.gws, g.per_cta, order);
    else
      k_eig_refine<512, false><<<g.grid, threads, g.smem, st>>>(H0, M, f, N, J, refine_sweeps, angle_tol,
                                                                W, eig, status, stats, finish_tol, g.gws, g.per_cta, order);
  }
  return cudaGetLastError();
}

size_t eig_step_bytes(int N) {
  const size_t a = jacobi_smem(N, 8), b = jacobi_smem(N, 4), c = refine_smem(N);
  return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

}  // namespace qoc
