// Learned warm start: a small multilayer perceptron that maps a target
// state beta (as [Re beta, Im beta]) to initial control coefficients theta0
// for the trust-region solve.  The paper has no counterpart (it starts the
// trust region from random theta, Sec. IV-B); this is the warm-start pattern
// of the library.  Hand-written kernels:
//   forward   h_{k+1} = gelu(W_k h_k + b_k) (last layer linear), binary32
//   backward  standard reverse mode through the same layers, binary32
//   Adam      m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2, w -= lr mhat / (sqrt(vhat) + eps)
//   inference bfloat16 weights and activations on the tensor cores
//             (mma.sync m16n8k16, binary32 accumulation, bias and GELU in
//             the epilogue), or binary32 throughout
// GELU is the exact form x Phi(x) = x (1 + erf(x / sqrt 2)) / 2.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

__device__ __forceinline__ float gelu_f(float x) { return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f)); }
// d/dx [x Phi(x)] = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_f(float x) {
  const float Phi = 0.5f * (1.0f + erff(x * 0.70710678118654752f));
  const float phi = 0.39894228040143268f * expf(-0.5f * x * x);
  return Phi + x * phi;
}

// C[m][n] = sum_k A(m,k) B(k,n), A(m,k) = A[m*sam + k*sak], B(k,n) = B[k*sbk + n*sbn].
// 32 x 32 output tile per CTA (256 threads, 4 outputs each), K in chunks of 32.
// epilogue: mode 0 plain store (+= when accumulate), 1 bias + store pre-activation
// and gelu output, 2 bias only, 3 multiply by gelu'(pre) (backward through gelu).
template <typename TW>
__global__ void k_gemm(const float* __restrict__ A, long sam, long sak, const TW* __restrict__ B,
                       long sbk, long sbn, float* __restrict__ C, long scm, int M, int N, int K,
                       int mode, const float* __restrict__ bias, float* __restrict__ pre,
                       const float* __restrict__ pre_in, int accumulate) {
  __shared__ float As[32][33];
  __shared__ float Bs[32][33];
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // ty in 0..7: rows ty, ty+8, ...
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int r = ty; r < 32; r += 8) {
      const int m = m0 + r, k = k0 + tx;
      As[r][tx] = (m < M && k < K) ? A[m * sam + k * sak] : 0.f;
      const int kk = k0 + r, n = n0 + tx;
      Bs[r][tx] = (kk < K && n < N) ? (float)B[kk * sbk + n * sbn] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float b = Bs[k][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(As[ty + 8 * q][k], b, acc[q]);
    }
    __syncthreads();
  }
  const int n = n0 + tx;
  if (n >= N) return;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int m = m0 + ty + 8 * q;
    if (m >= M) continue;
    float v = acc[q];
    const long idx = m * scm + n;
    if (mode == 1) {
      v += bias[n];
      pre[idx] = v;
      C[idx] = gelu_f(v);
    } else if (mode == 2) {
      C[idx] = v + bias[n];
    } else if (mode == 3) {
      C[idx] = v * gelu_grad_f(pre_in[idx]);
    } else {
      C[idx] = accumulate ? C[idx] + v : v;
    }
  }
}

// Inference GEMM on the tensor cores: C = A B with A (binary32 activations,
// rounded to bfloat16 as they are staged) and B (bfloat16 weights), binary32
// accumulation; epilogue mode 1 (bias + GELU) or 2 (bias).  32 x 32 output
// tile per CTA of 4 warps, warp w the 16 x 16 block (w / 2, w % 2) as two
// m16n8 tiles; K in chunks of 32 (two k16 steps).  Shared tiles hold A as
// [m][k] and B transposed as [n][k] (k contiguous, as the .col operand
// wants), 40 bfloat16 per row so the fragment loads are free of bank
// conflicts.  Entries outside M, N, K are zero.
__device__ __forceinline__ uint32_t ld_b32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__global__ void __launch_bounds__(128) k_gemm_bf16_tc(const float* __restrict__ A, long sam, long sak,
                                                      const __nv_bfloat16* __restrict__ B, long sbk,
                                                      long sbn, float* __restrict__ C, long scm, int M,
                                                      int N, int K, int mode,
                                                      const float* __restrict__ bias) {
  constexpr int LDT = 40;
  __shared__ __align__(16) __nv_bfloat16 As[32 * LDT];
  __shared__ __align__(16) __nv_bfloat16 Bs[32 * LDT];
  const int m0 = blockIdx.y * 32, n0 = blockIdx.x * 32;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int rm = (warp >> 1) * 16, cw = (warp & 1) * 16;
  float acc[2][4] = {{0.f, 0.f, 0.f, 0.f}, {0.f, 0.f, 0.f, 0.f}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int idx = tid; idx < 32 * 32; idx += 128) {
      const int r = idx >> 5, c = idx & 31;
      const int m = m0 + r, ka = k0 + c;
      As[r * LDT + c] = __float2bfloat16_rn((m < M && ka < K) ? A[m * sam + ka * sak] : 0.f);
      const int kb = k0 + r, n = n0 + c;   // B(kb, n) -> Bs[n][kb]
      Bs[c * LDT + r] = (kb < K && n < N) ? B[kb * sbk + n * sbn] : __float2bfloat16_rn(0.f);
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      const uint32_t a0 = ld_b32(As + (rm + g) * LDT + kk + 2 * t);
      const uint32_t a1 = ld_b32(As + (rm + g + 8) * LDT + kk + 2 * t);
      const uint32_t a2 = ld_b32(As + (rm + g) * LDT + kk + 2 * t + 8);
      const uint32_t a3 = ld_b32(As + (rm + g + 8) * LDT + kk + 2 * t + 8);
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        const int cn = cw + nt * 8;
        const uint32_t b0 = ld_b32(Bs + (cn + g) * LDT + kk + 2 * t);
        const uint32_t b1 = ld_b32(Bs + (cn + g) * LDT + kk + 2 * t + 8);
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(acc[nt][0]), "+f"(acc[nt][1]), "+f"(acc[nt][2]), "+f"(acc[nt][3])
            : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = m0 + rm + g + (q >= 2 ? 8 : 0), n = n0 + cw + nt * 8 + 2 * t + (q & 1);
      if (m >= M || n >= N) continue;
      const float v = acc[nt][q] + bias[n];
      C[m * scm + n] = mode == 1 ? gelu_f(v) : v;
    }
  }
}

// bias gradient: db[n] = sum_b dY[b][n]
__global__ void k_colsum(const float* __restrict__ dY, int Bn, int N, float* __restrict__ db) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  float s = 0.f;
  for (int b = 0; b < Bn; ++b) s += dY[(size_t)b * N + n];
  db[n] = s;
}

// loss = 1/(2B) sum |y - t|^2 over the batch; dY = (y - t) / B
__global__ void k_mse(const float* __restrict__ Y, const float* __restrict__ T, int n, float inv_b,
                      float* __restrict__ dY, float* __restrict__ loss) {
  __shared__ float red[32];
  float s = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float d = Y[i] - T[i];
    dY[i] = d * inv_b;
    s += d * d;
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < (blockDim.x + 31) / 32; ++w) t += red[w];
    atomicAdd(loss, 0.5f * t * inv_b);
  }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, int n, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void k_to_bf16(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// ---------------------------------------------------------------------------
// host-side launchers (used by api.cu)
// ---------------------------------------------------------------------------
static dim3 gemm_grid(int M, int N) { return dim3((N + 31) / 32, (M + 31) / 32); }

cudaError_t mlp_gemm(const float* A, long sam, long sak, const void* B, int b_bf16, long sbk,
                     long sbn, float* C, long scm, int M, int N, int K, int mode, const float* bias,
                     float* pre, const float* pre_in, int accumulate, cudaStream_t st) {
  if (b_bf16)
    k_gemm<__nv_bfloat16><<<gemm_grid(M, N), 256, 0, st>>>(A, sam, sak, (const __nv_bfloat16*)B, sbk,
                                                           sbn, C, scm, M, N, K, mode, bias, pre,
                                                           pre_in, accumulate);
  else
    k_gemm<float><<<gemm_grid(M, N), 256, 0, st>>>(A, sam, sak, (const float*)B, sbk, sbn, C, scm, M,
                                                   N, K, mode, bias, pre, pre_in, accumulate);
  return cudaGetLastError();
}

cudaError_t mlp_gemm_bf16_tc(const float* A, long sam, long sak, const void* B, long sbk, long sbn,
                             float* C, long scm, int M, int N, int K, int mode, const float* bias,
                             cudaStream_t st) {
  k_gemm_bf16_tc<<<gemm_grid(M, N), 128, 0, st>>>(A, sam, sak, (const __nv_bfloat16*)B, sbk, sbn, C, scm,
                                                  M, N, K, mode, bias);
  return cudaGetLastError();
}

cudaError_t mlp_colsum(const float* dY, int Bn, int N, float* db, cudaStream_t st) {
  k_colsum<<<(N + 127) / 128, 128, 0, st>>>(dY, Bn, N, db);
  return cudaGetLastError();
}

cudaError_t mlp_mse(const float* Y, const float* T, int n, float inv_b, float* dY, float* loss,
                    cudaStream_t st) {
  const int blocks = (n + 255) / 256 > 128 ? 128 : (n + 255) / 256;
  k_mse<<<blocks, 256, 0, st>>>(Y, T, n, inv_b, dY, loss);
  return cudaGetLastError();
}

cudaError_t mlp_adam(float* w, const float* g, float* m, float* v, int n, float lr, float b1,
                     float b2, float eps, float c1, float c2, cudaStream_t st) {
  k_adam<<<(n + 255) / 256, 256, 0, st>>>(w, g, m, v, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t mlp_to_bf16(const float* x, void* y, int n, cudaStream_t st) {
  k_to_bf16<<<(n + 255) / 256, 256, 0, st>>>(x, (__nv_bfloat16*)y, n);
  return cudaGetLastError();
}

}  // namespace qoc

namespace qoc {
__global__ void k_gather(const float* __restrict__ src, const int* __restrict__ idx, int rows,
                         int cols, float* __restrict__ dst) {
  const long n = (long)rows * cols;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x) {
    const int r = (int)(e / cols), c = (int)(e % cols);
    dst[e] = src[(long)idx[r] * cols + c];
  }
}
cudaError_t mlp_gather(const float* src, const int* idx, int rows, int cols, float* dst,
                       cudaStream_t st) {
  const long n = (long)rows * cols;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 1024) blocks = 1024;
  k_gather<<<blocks, 256, 0, st>>>(src, idx, rows, cols, dst);
  return cudaGetLastError();
}
}  // namespace qoc
