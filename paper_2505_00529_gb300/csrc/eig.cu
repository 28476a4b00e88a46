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

namespace qoc {

template <typename T> struct JacobiEps;
template <> struct JacobiEps<float> { static constexpr double eps = 5.96e-8; static constexpr int max_sweeps = 24; };
template <> struct JacobiEps<double> { static constexpr double eps = 1.12e-16; static constexpr int max_sweeps = 40; };

// element at position `pos` of the round-robin schedule in round r (NP players)
__device__ __forceinline__ int rr_elem(int pos, int r, int NP) {
  return pos == 0 ? 0 : ((pos - 1 + r) % (NP - 1)) + 1;
}

template <typename T>
__global__ void k_eig_jacobi(const double* __restrict__ H0, const double* __restrict__ M,
                             const double* __restrict__ f, int N, int J,
                             double* __restrict__ W_out, double* __restrict__ eig_out,
                             int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.x;
  if (j >= J) return;
  const int ld = N + 1;
  const int NP = N + (N & 1);
  const int NH = NP / 2;
  T* A = reinterpret_cast<T*>(smem_raw);
  T* V = A + N * ld;
  T* cs = V + N * ld;            // [NH][2] cosine / sine
  int* pr = reinterpret_cast<int*>(cs + 2 * NH);  // [NH][2] pair indices
  double* red = reinterpret_cast<double*>(pr + 2 * NH + 2);
  red = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(red) + 15) & ~uintptr_t(15));

  const int tid = threadIdx.x, nt = blockDim.x;
  const double fj = f[j];
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    A[p * ld + q] = (T)(H0[e] + fj * M[e]);
    V[p * ld + q] = (T)(p == q ? 1.0 : 0.0);
  }
  __syncthreads();

  const T eps = (T)JacobiEps<T>::eps;
  bool converged = false;
  for (int sweep = 0; sweep < JacobiEps<T>::max_sweeps && !converged; ++sweep) {
    for (int r = 0; r < NP - 1; ++r) {
      if (tid < NH) {
        int p = rr_elem(tid, r, NP), q = rr_elem(NP - 1 - tid, r, NP);
        if (p > q) { int t = p; p = q; q = t; }
        T c = 1, s = 0;
        if (q < N) {
          T apq = A[p * ld + q], app = A[p * ld + p], aqq = A[q * ld + q];
          T thr = eps * (T)0.01 * sqrt(fabs(app) * fabs(aqq));
          if (fabs(apq) > thr && apq != (T)0) {
            T th = (aqq - app) / (2 * apq);
            T t = (th >= 0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + 1));
            c = 1 / sqrt(t * t + 1);
            s = t * c;
          }
        }
        pr[2 * tid] = p;
        pr[2 * tid + 1] = q;
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
      }
      __syncthreads();
      // A <- R^T A R on 2x2 blocks (k <= l, mirrored), V <- V R
      const int nblk = NH * (NH + 1) / 2;
      for (int b = tid; b < nblk + N * NH; b += nt) {
        if (b < nblk) {
          // decode upper-triangular block index b -> (k, l), k <= l
          int k = 0, rem = b;
          while (rem >= NH - k) { rem -= NH - k; ++k; }
          int l = k + rem;
          int p0 = pr[2 * k], p1 = pr[2 * k + 1], q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (p1 >= N || q1 >= N) {
            // blocks touching the dummy index of odd N: only the real rows/cols move
            T ck = cs[2 * k], sk = cs[2 * k + 1], cl = cs[2 * l], sl = cs[2 * l + 1];
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
            // both unpaired: only possible for k == l (the dummy pair); A[p0][p0] unchanged
            continue;
          }
          T ck = cs[2 * k], sk = cs[2 * k + 1], cl = cs[2 * l], sl = cs[2 * l + 1];
          T a00 = A[p0 * ld + q0], a01 = A[p0 * ld + q1], a10 = A[p1 * ld + q0], a11 = A[p1 * ld + q1];
          // left: R_k^T [[a00 a01][a10 a11]] with R = [[c s][-s c]] -> R^T = [[c -s][s c]]
          T b00 = ck * a00 - sk * a10, b01 = ck * a01 - sk * a11;
          T b10 = sk * a00 + ck * a10, b11 = sk * a01 + ck * a11;
          // right: [...] R_l
          T c00 = cl * b00 - sl * b01, c01 = sl * b00 + cl * b01;
          T c10 = cl * b10 - sl * b11, c11 = sl * b10 + cl * b11;
          if (k == l) {
            c01 = (T)0.5 * (c01 + c10);  // exact zero in exact arithmetic after the rotation
            if (sk != (T)0) c01 = (T)0;
            c10 = c01;
          }
          A[p0 * ld + q0] = c00; A[p0 * ld + q1] = c01; A[p1 * ld + q0] = c10; A[p1 * ld + q1] = c11;
          if (k != l) {
            A[q0 * ld + p0] = c00; A[q1 * ld + p0] = c01; A[q0 * ld + p1] = c10; A[q1 * ld + p1] = c11;
          }
        } else {
          int e = b - nblk;
          int i = e / NH, l = e % NH;
          int q0 = pr[2 * l], q1 = pr[2 * l + 1];
          if (q1 >= N) continue;
          T cl = cs[2 * l], sl = cs[2 * l + 1];
          T v0 = V[i * ld + q0], v1 = V[i * ld + q1];
          V[i * ld + q0] = cl * v0 - sl * v1;
          V[i * ld + q1] = sl * v0 + cl * v1;
        }
      }
      __syncthreads();
    }
    // convergence: off-diagonal Frobenius^2 vs total
    double off = 0, tot = 0;
    for (int e = tid; e < N * N; e += nt) {
      int p = e / N, q = e % N;
      double v = (double)A[p * ld + q];
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
      red[64] = (o <= (double)eps * (double)eps * t || o == 0.0) ? 1.0 : 0.0;
    }
    __syncthreads();
    converged = red[64] != 0.0;
    __syncthreads();
  }
  if (!converged && tid == 0) raise_status(status, DEV_EIG_NOCONV);

  // sort ascending (rank sort, ties by index) and write W (columns), lambda
  double* Wj = W_out + (size_t)j * N * N;
  double* ej = eig_out + (size_t)j * N;
  for (int i = tid; i < N; i += nt) {
    T di = A[i * ld + i];
    int rank = 0;
    for (int k = 0; k < N; ++k) {
      T dk = A[k * ld + k];
      rank += (dk < di) || (dk == di && k < i);
    }
    ej[rank] = (double)di;
    for (int row = 0; row < N; ++row) Wj[row * N + rank] = (double)V[row * ld + i];
  }
}

// Ogita-Aishima refinement sweeps in binary64 (see the file header).
__global__ void k_eig_refine(const double* __restrict__ H0, const double* __restrict__ M,
                             const double* __restrict__ f, int N, int J, int sweeps,
                             double* __restrict__ W_io, double* __restrict__ eig_out, int* status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int j = blockIdx.x;
  if (j >= J) return;
  const int ld = N + 1;
  double* H = reinterpret_cast<double*>(smem_raw);
  double* W = H + N * ld;
  double* T = W + N * ld;
  double* S = T + N * ld;
  double* R = S + N * ld;
  double* lam = R + N * ld;
  double* red = lam + N + 1;   // [64]
  const int tid = threadIdx.x, nt = blockDim.x;
  const double fj = f[j];
  double* Wg = W_io + (size_t)j * N * N;
  double hn = 0;
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    double h = H0[e] + fj * M[e];
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

  for (int it = 0; it < sweeps; ++it) {
    // T = H W
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      double acc = 0;
      for (int r = 0; r < N; ++r) acc = fma(H[i * ld + r], W[r * ld + k], acc);
      T[i * ld + k] = acc;
    }
    __syncthreads();
    // S = W^T T, R = I - W^T W
    double sn = 0, rn = 0;
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      double s = 0, w = 0;
      for (int r = 0; r < N; ++r) {
        double wri = W[r * ld + i];
        s = fma(wri, T[r * ld + k], s);
        w = fma(wri, W[r * ld + k], w);
      }
      S[i * ld + k] = s;
      double rr = (i == k ? 1.0 : 0.0) - w;
      R[i * ld + k] = rr;
      rn += rr * rr;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nt) lam[i] = S[i * ld + i] / (1.0 - R[i * ld + i]);
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      if (i != k) sn += S[i * ld + k] * S[i * ld + k];
      else { double d = S[i * ld + i] - lam[i]; sn += d * d; }
    }
    sn = warp_sum(sn);
    rn = warp_sum(rn);
    if ((tid & 31) == 0) { red[2 * (tid >> 5)] = sn; red[2 * (tid >> 5) + 1] = rn; }
    __syncthreads();
    if (tid == 0) {
      double a = 0, b = 0;
      for (int w = 0; w < (nt + 31) / 32; ++w) { a += red[2 * w]; b += red[2 * w + 1]; }
      red[41] = 2.0 * (sqrt(a) + Hnorm * sqrt(b));  // cluster threshold delta
    }
    __syncthreads();
    const double delta = red[41];
    // E overwrites S
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      double rik = R[i * ld + k];
      double eik;
      if (i == k) eik = 0.5 * rik;
      else {
        double gap = lam[k] - lam[i];
        eik = fabs(gap) > delta ? (S[i * ld + k] + lam[k] * rik) / gap : 0.5 * rik;
      }
      T[i * ld + k] = eik;
    }
    __syncthreads();
    // W <- W + W E   (R reused as scratch for W E)
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      double acc = 0;
      for (int r = 0; r < N; ++r) acc = fma(W[i * ld + r], T[r * ld + k], acc);
      R[i * ld + k] = acc;
    }
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) {
      int i = e / N, k = e % N;
      W[i * ld + k] += R[i * ld + k];
    }
    __syncthreads();
  }
  // eigenvalues: Rayleigh quotients of the refined vectors (sorted order kept)
  for (int e = tid; e < N * N; e += nt) {
    int i = e / N, k = e % N;
    double acc = 0;
    for (int r = 0; r < N; ++r) acc = fma(H[i * ld + r], W[r * ld + k], acc);
    T[i * ld + k] = acc;
  }
  __syncthreads();
  double* ej = eig_out + (size_t)j * N;
  for (int k = tid; k < N; k += nt) {
    double num = 0, den = 0;
    for (int r = 0; r < N; ++r) {
      num = fma(W[r * ld + k], T[r * ld + k], num);
      den = fma(W[r * ld + k], W[r * ld + k], den);
    }
    double l = num / den;
    if (!isfinite(l)) raise_status(status, DEV_NONFINITE);
    ej[k] = l;
  }
  for (int e = tid; e < N * N; e += nt) {
    int p = e / N, q = e % N;
    Wg[e] = W[p * ld + q];
  }
}

static size_t jacobi_smem(int N, size_t tsize) {
  int NP = N + (N & 1);
  size_t s = 2 * (size_t)N * (N + 1) * tsize + (size_t)NP * tsize + (size_t)(NP + 2) * sizeof(int);
  s = (s + 15) & ~size_t(15);
  return s + 66 * sizeof(double) + 16;
}
static size_t refine_smem(int N) { return (5 * (size_t)N * (N + 1) + N + 1 + 64) * sizeof(double); }

size_t eig_smem_bytes(int N, int method) {
  size_t a = method == EIG_JACOBI_FP64 ? jacobi_smem(N, 8) : jacobi_smem(N, 4);
  size_t b = method == EIG_JACOBI_FP64 ? 0 : refine_smem(N);
  return a > b ? a : b;
}

cudaError_t launch_eig(const double* H0, const double* M, const double* f, int N, int J,
                       double* W, double* eig, int* status, int method, int refine_sweeps,
                       cudaStream_t st) {
  int threads = N <= 16 ? 128 : 256;
  if (method == EIG_JACOBI_FP64) {
    size_t sm = jacobi_smem(N, 8);
    cudaFuncSetAttribute(k_eig_jacobi<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    k_eig_jacobi<double><<<J, threads, sm, st>>>(H0, M, f, N, J, W, eig, status);
    return cudaGetLastError();
  }
  size_t sm = jacobi_smem(N, 4);
  cudaFuncSetAttribute(k_eig_jacobi<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  k_eig_jacobi<float><<<J, threads, sm, st>>>(H0, M, f, N, J, W, eig, status);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  size_t sr = refine_smem(N);
  cudaFuncSetAttribute(k_eig_refine, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
  k_eig_refine<<<J, threads, sr, st>>>(H0, M, f, N, J, refine_sweeps, W, eig, status);
  return cudaGetLastError();
}

}  // namespace qoc
