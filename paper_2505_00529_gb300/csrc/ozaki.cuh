// Products of 32 x 32 binary64 matrices on the tensor cores by error-free
// splitting (Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012:
// "Error-free transformations of matrix multiplication by using fast
// routines of matrix multiplication and its applications").
//
// Every row of the left factor A and every column of the right factor B is
// scaled by a power of two 2^e with all its entries below 2^e in magnitude;
// the scaled entries a = sum_s a_s 2^(-8 s) are cut into NS signed 8-bit
// slices a_s in [-255, 255] (taken from the binary64 bits with integer
// operations), each of which bfloat16 holds exactly.  A slice product
// sum_k a_s,ik b_t,kj has 32 terms below 2^16, so it is an exact integer
// below 2^21 and binary32 accumulation on the tensor cores is exact; so is
// the sum of the up to NS products of one level L = s + t (< 2^24).  The
// levels L = 2 .. NS + 1 (NS <= 6) are recombined exactly in 64-bit integers and
// scaled once in binary64: C_ij = 2^(e_i + f_j) sum_L acc_L 2^(-8L).  The
// slices dropped (levels above NS + 1, bits below 2^(-8 NS) of each line's
// scale) bound the error by about 32 * 2^(-8 NS) |A_row| |B_col| in
// magnitude terms: 2^-43 relative to the scales for NS = 6.
//
// Layout: slices in shared memory as [NS][32 lines][LD] bfloat16 with the
// inner index (k) contiguous: a row of A, or a column of B (B stored
// transposed), per line, so that one split serves both as the left factor of
// a product with its transpose's rows and as the right factor with its
// columns.  mma.sync m16n8k16 (bf16 x bf16 -> f32) on 8 warps: warp w owns
// the 16 x 8 output tile (w / 4, w % 4).
#pragma once

#include <cuda_bf16.h>
#include <stdint.h>

namespace qoc {
namespace oz {

constexpr int LD = 40;   // bfloat16 stride of a line: 80 bytes, conflict-free fragment loads

// |x| < 2^e for every entry of the line; -1022 for an all-zero line
__device__ __forceinline__ int line_exponent_bits(double x) {
  const long long b = __double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  return E == 0 ? -1022 : E - 1022;   // subnormals are treated as zero-scale (below 2^-1022)
}

// Split the n x n (n <= 32) binary64 matrix M (entry (r, c) at M[(r ld + c) es],
// es = 2 for one plane of an interleaved complex array) into NS slices per line:
// byrow: line i = row i, inner k = column; else line j = column j, inner k = row.
// Entries beyond n are zero.  exps[32] receives the line exponents.  All
// threads of the CTA take part (256 threads); ends with a barrier.
template <int NS>
__device__ void split32(const double* M, int ld, int n, bool byrow, __nv_bfloat16* slc, int* exps,
                        int es = 1) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int line = warp; line < 32; line += nw) {
    int e = -1022;
    if (line < n && lane < n) {
      const double x = byrow ? M[(line * ld + lane) * es] : M[(lane * ld + line) * es];
      e = line_exponent_bits(x);   // integer operations only (-1022 for zero)
    }
    for (int o = 16; o > 0; o >>= 1) e = max(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (lane == 0) exps[line] = e;
  }
  __syncthreads();
  for (int idx = tid; idx < 32 * 32; idx += blockDim.x) {
    const int line = idx >> 5, k = idx & 31;
    double x = 0.0;
    if (line < n && k < n) x = byrow ? M[(line * ld + k) * es] : M[(k * ld + line) * es];
    const long long b = __double_as_longlong(x);
    const int E = (int)((b >> 52) & 0x7ff);
    unsigned long long F = 0;   // |x| 2^(56 - e), below 2^56
    if (E != 0) {
      const unsigned long long m = (unsigned long long)(b & 0xfffffffffffffLL) | (1ull << 52);
      const int sh = E - 1019 - exps[line];   // <= 3
      F = sh >= 0 ? (m << sh) : (sh > -64 ? (m >> (-sh)) : 0ull);
    }
    const bool neg = b < 0;
#pragma unroll
    for (int s = 1; s <= NS; ++s) {
      const int d = (int)((F >> (56 - 8 * s)) & 0xffull);
      slc[((s - 1) * 32 + line) * LD + k] = __float2bfloat16_rn((float)(neg ? -d : d));
    }
  }
  __syncthreads();
}

// v 2^ex as a binary64, rounded to nearest even, with integer operations only
// (the conversion and scaling instructions would share the binary64 pipe)
__device__ __forceinline__ double scaled_i64_to_double(long long v, int ex) {
  if (v == 0) return 0.0;
  const unsigned long long a = v < 0 ? 0ull - (unsigned long long)v : (unsigned long long)v;
  int msb = 63 - __clzll((long long)a);
  unsigned long long m;
  if (msb <= 52) {
    m = a << (52 - msb);
  } else {
    const int sh = msb - 52;
    const unsigned long long rem = a & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
    m = a >> sh;
    if (rem > half || (rem == half && (m & 1ull))) {
      ++m;
      if (m >> 53) { m >>= 1; ++msb; }
    }
  }
  const int E = msb + ex + 1023;
  if (E <= 0 || E >= 2047) return ldexp((double)v, ex);   // outside the normal range
  return __longlong_as_double((long long)(((unsigned long long)(v < 0) << 63) |
                                          ((unsigned long long)E << 52) | (m & 0xfffffffffffffull)));
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16* p) {
  return *reinterpret_cast<const uint32_t*>(p);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// C (32 x 32, binary64, entry (i, j) at C[(i ldc + j) cs]; entries beyond n not
// written) = A B with A's slices by row (As, ea) and B's by column (Bs, eb).
// Must be called by all 8 warps of the CTA (warp w: output tile w); no
// barrier inside.
template <int NS>
__device__ void mm32(const __nv_bfloat16* As, const int* ea, const __nv_bfloat16* Bs, const int* eb,
                     double* C, int ldc, int n, int cs = 1) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int r0 = (warp >> 2) * 16, c0 = (warp & 3) * 8;
  float acc[NS][4];
#pragma unroll
  for (int L = 0; L < NS; ++L) acc[L][0] = acc[L][1] = acc[L][2] = acc[L][3] = 0.f;
#pragma unroll
  for (int s = 1; s <= NS; ++s) {
    const __nv_bfloat16* A = As + (size_t)(s - 1) * 32 * LD;
#pragma unroll
    for (int kk = 0; kk < 32; kk += 16) {
      const uint32_t a0 = ld32(A + (r0 + g) * LD + kk + 2 * t);
      const uint32_t a1 = ld32(A + (r0 + g + 8) * LD + kk + 2 * t);
      const uint32_t a2 = ld32(A + (r0 + g) * LD + kk + 2 * t + 8);
      const uint32_t a3 = ld32(A + (r0 + g + 8) * LD + kk + 2 * t + 8);
#pragma unroll
      for (int tt = 1; tt + s <= NS + 1; ++tt) {
        const __nv_bfloat16* B = Bs + (size_t)(tt - 1) * 32 * LD;
        const uint32_t b0 = ld32(B + (c0 + g) * LD + kk + 2 * t);
        const uint32_t b1 = ld32(B + (c0 + g) * LD + kk + 2 * t + 8);
        mma_bf16(acc[s + tt - 2], a0, a1, a2, a3, b0, b1);   // level s + tt
      }
    }
  }
  // exact recombination: sum_L acc_L 2^(8 (NS + 1 - L)) < 2^(8 (NS - 1) + 24)
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = r0 + g + (q >= 2 ? 8 : 0), j = c0 + 2 * t + (q & 1);
    long long v = 0;
#pragma unroll
    for (int L = 0; L < NS; ++L)   // each level is an exact integer below 2^24: int32 conversion
      v += (long long)__float2int_rn(acc[L][q]) * (1ll << (8 * (NS - 1 - L)));
    if (i < n && j < n)   // v carries 2^(-8 (NS + 1)) of the scaled product
      C[(i * ldc + j) * cs] = scaled_i64_to_double(v, ea[i] + eb[j] - 8 * (NS + 1));
  }
}

}  // namespace oz
}  // namespace qoc
