// Binary32 two-sided Jacobi start of the eigendecomposition H_j = W_j Lambda_j W_j^T
// (Sec. III-A: exp of each step's Hamiltonian H0 + f_j M and its derivatives
// come from that eigendecomposition, stored in the first loop of Alg. 1 and
// Alg. 2) for exactly 32 x 32 matrices, with the matrix held in registers.
//
// One warp per step j.  Lane i holds row i of A and row i of V.  In round r
// (r = 1..31) every index i is paired with i ^ r, so the 16 pairs of a round
// are disjoint and the 31 rounds of a sweep cover each of the 496 pairs once
// (a parallel ordering for a hypercube of 32 nodes).  The rounds run in the
// order r_t = x^t of GF(2^5) = GF(2)[x] / (x^5 + x^2 + 1), which visits all
// 31 non-zero values before it repeats.
//
// Register layout.  At round t0 of a loop body, register k of lane i holds
// the entry of column i ^ (k * x^t0) (GF(2^5) product).  Then:
//   - the diagonal entry A[i][i] is register 0;
//   - in round t0 + s the pair element A[i][i ^ r] is register x^s;
//   - the two columns of each rotated pair sit in registers k and k ^ x^s.
// All three are constants of the unrolled body.  After U rounds the
// registers are renamed by k -> k * x^U, so that the next body starts in the
// same layout.  Cross-lane data moves only by warp shuffles:
//   - the partner's diagonal and pair element;
//   - the (c, s) of the other 15 pairs, for the column rotations of A and V;
//   - the partner's row, for the row rotation of A.
// No shared memory is used between the load and the sorted write-out.
//
// The rotation, its threshold, the convergence test (off(A)^2 <= 16 eps^2
// |A|_F^2, or no rotation in a whole sweep) and the sweep cap match the
// general binary32 kernel; only the pair order and the data layout differ.
// The binary64 refinement that follows does not depend on the start's
// rounding details.
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {
namespace {

constexpr unsigned kFull = 0xffffffffu;

// GF(2^5) modulo x^5 + x^2 + 1 (primitive: x has order 31)
__host__ __device__ constexpr int gf_mulx(int v) { return ((v << 1) & 31) ^ ((v & 16) ? 5 : 0); }
__host__ __device__ constexpr int gf_pow(int s) {
  int v = 1;
  for (int i = 0; i < s; ++i) v = gf_mulx(v);
  return v;
}
__host__ __device__ constexpr int gf_mul(int a, int b) {
  int r = 0;
  for (int i = 0; i < 5; ++i) {
    if (b & (1 << i)) r ^= a;
    a = gf_mulx(a);
  }
  return r;
}
struct Table32 {
  int v[32];
};
__host__ __device__ constexpr Table32 gf_mul_table(int m) {
  Table32 t{};
  for (int k = 0; k < 32; ++k) t.v[k] = gf_mul(k, m);
  return t;
}

// k * base for a compile-time k, from the basis b[j] = base * x^j
__device__ __forceinline__ int gf_lane_mask(int k, const int (&b)[5]) {
  int m = 0;
#pragma unroll
  for (int j = 0; j < 5; ++j)
    if (k & (1 << j)) m ^= b[j];
  return m;
}

constexpr float kEps = 5.96e-8f;

// one round: pairs (i, i ^ r) with r = x^S * base
template <int S>
__device__ __forceinline__ void jac_round(float (&a)[32], float (&v)[32], int lane,
                                          const int (&b)[5], bool& rot) {
  constexpr int G = gf_pow(S);   // register of A[i][i ^ r]
  const int r = gf_lane_mask(G, b);
  const float dii = a[0];
  const float djj = __shfl_xor_sync(kFull, a[0], r);
  const float aij = a[G];
  const float aji = __shfl_xor_sync(kFull, a[G], r);
  // the same (app, aqq, apq) in both lanes of a pair, so the same rotation
  const float apq = 0.5f * (aij + aji);
  const int hb = 1 << (31 - __clz(r));
  const bool lower = (lane & hb) == 0;   // i < i ^ r: this lane is p
  const float app = lower ? dii : djj, aqq = lower ? djj : dii;
  float c = 1.f, s = 0.f;
  const float thr = kEps * 0.01f * sqrtf(fabsf(app) * fabsf(aqq));
  const bool do_rot = fabsf(apq) > thr && apq != 0.f;
  if (do_rot) {
    // binary32 start only (refined in binary64): fast reciprocals suffice
    const float th = __fdividef(aqq - app, 2.f * apq);
    const float t = copysignf(__fdividef(1.f, fabsf(th) + sqrtf(fmaf(th, th, 1.f))), th);
    c = rsqrtf(fmaf(t, t, 1.f));
    s = t * c;
    rot = true;
  }
  // s as seen from this lane's index: column/row p' = c p - s q, q' = c q + s p
  const float st = lower ? s : -s;
  // A <- A R, V <- V R: register pair (k, k ^ G) holds the columns
  // i ^ (k * base) (whose lane computed the rotation) and its partner
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < (k ^ G)) {
      const int m = gf_lane_mask(k, b);
      const float ck = k == 0 ? c : __shfl_xor_sync(kFull, c, m);
      const float sk = k == 0 ? st : __shfl_xor_sync(kFull, st, m);
      const float x0 = a[k], y0 = a[k ^ G];
      a[k] = fmaf(-sk, y0, ck * x0);
      a[k ^ G] = fmaf(sk, x0, ck * y0);
      const float x1 = v[k], y1 = v[k ^ G];
      v[k] = fmaf(-sk, y1, ck * x1);
      v[k ^ G] = fmaf(sk, x1, ck * y1);
    }
  }
  // A <- R^T A: rows i and i ^ r; the partner keeps this lane's column of
  // register k in register k ^ G
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    if (k < (k ^ G)) {
      const float y0 = __shfl_xor_sync(kFull, a[k ^ G], r);
      const float y1 = __shfl_xor_sync(kFull, a[k], r);
      a[k] = fmaf(-st, y0, c * a[k]);
      a[k ^ G] = fmaf(-st, y1, c * a[k ^ G]);
    }
  }
  if (do_rot) a[G] = 0.f;   // the rotated pair: zero by construction
}

template <int S, int U>
__device__ __forceinline__ void jac_rounds(float (&a)[32], float (&v)[32], int lane,
                                           const int (&b)[5], bool& rot) {
  if constexpr (S < U) {
    jac_round<S>(a, v, lane, b, rot);
    jac_rounds<S + 1, U>(a, v, lane, b, rot);
  }
}

constexpr int kWarpsPerCta = 2;

// U rounds per loop body; U = 31 is a whole sweep (no renaming, constant masks)
template <int U>
__global__ void __launch_bounds__(32 * kWarpsPerCta)
    k_eig_jacobi32_reg(const double* __restrict__ H0, const double* __restrict__ M,
                       const double* __restrict__ f, int J, double* __restrict__ W_out,
                       double* __restrict__ eig_out, int* status, int* __restrict__ order) {
  __shared__ float s_mat[kWarpsPerCta][32 * 33];
  __shared__ int s_perm[kWarpsPerCta][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = blockIdx.x * kWarpsPerCta + wid;
  if (j >= J) return;   // whole warps leave; only warp-level synchronisation below
  float* S = s_mat[wid];
  int* perm = s_perm[wid];
  const double fj = f[j];
  // A = H0 + f_j M rounded to binary32, row-major without padding, so that
  // lane i's skewed row A[i][i ^ k] (k = 0..31) falls in 32 different banks
  for (int p = 0; p < 32; ++p)
    S[p * 32 + lane] = (float)(H0[p * 32 + lane] + fj * M[p * 32 + lane]);
  __syncwarp();
  float a[32], v[32];
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    a[k] = S[lane * 32 + (lane ^ k)];
    v[k] = k == 0 ? 1.f : 0.f;
  }
  __syncwarp();
  constexpr bool kWhole = U == 31;
  constexpr int kBodies = (31 + U - 1) / U;   // bodies between convergence tests
  constexpr Table32 kRename = gf_mul_table(gf_pow(U % 31));
  int base = 1;   // x^t0
  const float off_tol2 = 16.f * kEps * kEps;
  bool converged = false;
  for (int sweep = 0; sweep < 24 && !converged; ++sweep) {
    bool rot = false;
    for (int body = 0; body < kBodies; ++body) {
      int b[5];
      b[0] = kWhole ? 1 : base;
#pragma unroll
      for (int q = 1; q < 5; ++q) b[q] = gf_mulx(b[q - 1]);
      jac_rounds<0, U>(a, v, lane, b, rot);
      if constexpr (!kWhole) {
        // rename: new register k holds old register k * x^U
        float ta[32], tv[32];
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          ta[k] = a[kRename.v[k]];
          tv[k] = v[kRename.v[k]];
        }
#pragma unroll
        for (int k = 0; k < 32; ++k) {
          a[k] = ta[k];
          v[k] = tv[k];
        }
        base = gf_mul(base, gf_pow(U % 31));
      }
    }
    float off = 0.f;
#pragma unroll
    for (int k = 1; k < 32; ++k) off = fmaf(a[k], a[k], off);
    float tot = fmaf(a[0], a[0], off);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(kFull, off, o);
      tot += __shfl_xor_sync(kFull, tot, o);
    }
    converged = !__any_sync(kFull, rot) || off <= off_tol2 * tot || off == 0.f;
  }
  if (!converged && lane == 0) raise_status(status, DEV_EIG_NOCONV);
  // rank of this lane's eigenvalue (ties by index), then W = V(:, order)
  const float d = a[0];
  int rank = 0;
  float gap = __int_as_float(0x7f800000);   // distance to the nearest other eigenvalue
#pragma unroll
  for (int m = 1; m < 32; ++m) {
    const float dk = __shfl_xor_sync(kFull, d, m);
    rank += (dk < d) || (dk == d && (lane ^ m) < lane);
    gap = fminf(gap, fabsf(dk - d));
  }
  if (order) {
    // near-degenerate steps (smallest gap <= 1e-3 of the spectral radius) are
    // the ones whose refinement may run its whole update budget and the
    // binary64 clean-up: they go to the front of the refinement's step order,
    // the others to the back, so that no slow step starts in the last wave
    float rad = fabsf(d);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gap = fminf(gap, __shfl_xor_sync(kFull, gap, o));
      rad = fmaxf(rad, __shfl_xor_sync(kFull, rad, o));
    }
    if (lane == 0) {
      const bool hard = !(gap > 1e-3f * rad);
      const int pos = hard ? atomicAdd(&order[J], 1) : J - 1 - atomicAdd(&order[J + 1], 1);
      if (pos >= 0 && pos < J) order[pos] = j;
    }
  }
  perm[lane] = lane;   // stays a valid index even if NaNs broke the ranks
  __syncwarp();
  perm[rank] = lane;
  // V^T into shared memory (column-major V, padded): column i ^ (k * base)
  int b[5];
  b[0] = kWhole ? 1 : base;
#pragma unroll
  for (int q = 1; q < 5; ++q) b[q] = gf_mulx(b[q - 1]);
#pragma unroll
  for (int k = 0; k < 32; ++k) S[(lane ^ gf_lane_mask(k, b)) * 33 + lane] = v[k];
  __syncwarp();
  const int src = perm[lane];
  double* Wj = W_out + (size_t)j * 1024;
  for (int p = 0; p < 32; ++p) Wj[p * 32 + lane] = (double)S[src * 33 + p];
  eig_out[(size_t)j * 32 + rank] = (double)d;
}

}  // namespace

cudaError_t launch_eig_jacobi32_reg(const double* H0, const double* M, const double* f, int J,
                                    double* W, double* eig, int* status, int rounds_per_body,
                                    int* order, cudaStream_t st) {
  if (J <= 0) return cudaSuccess;
  if (order) {
    const cudaError_t e = cudaMemsetAsync(order + J, 0, 2 * sizeof(int), st);
    if (e != cudaSuccess) return e;
  }
  const int grid = (J + kWarpsPerCta - 1) / kWarpsPerCta;
  if (rounds_per_body == 31)
    k_eig_jacobi32_reg<31><<<grid, 32 * kWarpsPerCta, 0, st>>>(H0, M, f, J, W, eig, status, order);
  else if (rounds_per_body == 4)
    k_eig_jacobi32_reg<4><<<grid, 32 * kWarpsPerCta, 0, st>>>(H0, M, f, J, W, eig, status, order);
  else
    k_eig_jacobi32_reg<8><<<grid, 32 * kWarpsPerCta, 0, st>>>(H0, M, f, J, W, eig, status, order);
  return cudaGetLastError();
}

}  // namespace qoc
