// Time-stepped sweeps (Alg. 2, the sequential loops over j).
//
// Every recursion of the method has the same shape: a state panel X (N x kc
// complex columns) is pushed through one step propagator and receives a
// rank-one source,
//   forward  (Eq. discTDSE, Eq. gradatheta):  X <- U_j X + s_j b_j^T
//   backward (Eq. lambdaevolve, Eq. musys):   X <- U_j^H X + s_j b_j^T
// In a frame rotating with the fixed spectral shift m, U_j = e^{-i dt m}(I + D_j)
// and (U_j is complex symmetric, W_j being real) U_j^H = e^{i dt m}(I + conj D_j);
// the phase factors are folded into the stored sources, so the sweep applies
//   X <- X + D_j X + s^_j b_j^T   or   X <- X + conj(D_j) X + s^_j b_j^T.
// Before each update a per-column contraction Re(c_j^H X) is taken (the
// u_j of the tangent panel, the v_j of the second-order adjoint panel).
//
// The columns are independent (the paper vectorises over them with vmap),
// so a CTA owns kc columns and runs all J steps alone: no grid-wide
// synchronisation.  One thread (or RS lanes) owns one (row, column) entry.
// D_j, s^_j, c_j and row j of B are staged by one elected thread with bulk
// async copies into an NS-deep shared-memory ring (mbarrier completion,
// bounded waits), so the step loop never waits on global memory.
//
// Precision: with TD = double2 everything is binary64.  With TD = float2
// the product D_j X is binary32 and the state is an unevaluated float pair
// (hi + lo) updated with TwoSum; since |D_j| ~ dt |lambda - m| << 1 the
// binary32 rounding enters only through the small increment.
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

template <bool MIX> struct SweepT;
template <> struct SweepT<false> {
  using D = double2; using V = double2; using B = double; using R = double;
};
template <> struct SweepT<true> {
  using D = float2; using V = float2; using B = float; using R = float;
};

// DIRECT: step data read straight from global memory (large N) instead of the
// shared-memory ring; a template flag so that the ring instantiation keeps
// shared-memory (not generic) loads.
template <bool MIX, int RS, bool BWD, bool DIRECT>
__global__ void __launch_bounds__(1024) k_sweep(const SweepArgs a, const int nstage) {
  extern __shared__ __align__(128) unsigned char smem[];
  using TD = typename SweepT<MIX>::D;
  using TV = typename SweepT<MIX>::V;
  using TB = typename SweepT<MIX>::B;
  using R = typename SweepT<MIX>::R;
  const int N = a.N, kc = a.kc, J = a.J;
  constexpr int RPW = 32 / RS;
  const int WPC = (N + RPW - 1) / RPW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = warp / WPC, rb = warp % WPC;
  const int rsub = lane % RS;
  const int i = rb * RPW + lane / RS;
  const int col0 = blockIdx.x * kc;
  const int ncols = min(kc, a.K - col0);
  const bool active = (l < ncols) && (i < N);
  const bool owner = active && rsub == 0;

  // ---- shared memory layout ----
  const uint32_t dbytes = (uint32_t)a.dstride;
  const uint32_t sbytes = a.src ? (uint32_t)(sizeof(TV) * N + 15) / 16 * 16 : 0u;
  const uint32_t cbytes = a.ctr ? (uint32_t)(sizeof(TV) * N + 15) / 16 * 16 : 0u;
  const uint32_t bbytes = a.Brow ? (uint32_t)(sizeof(TB) * a.Kp) : 0u;
  const uint32_t stage = dbytes + sbytes + cbytes + bbytes;
  unsigned char* ring = smem;
  TD* X = reinterpret_cast<TD*>(ring + (size_t)nstage * stage);      // [2][kc][N] (hi part)
  R* red = reinterpret_cast<R*>(X + 2 * kc * N);                      // [2][kc][WPC]
  uint64_t* bar = reinterpret_cast<uint64_t*>(red + 2 * kc * WPC + 2);
  bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(bar) + 7) & ~uintptr_t(7));
  __shared__ int abort_flag;

  const unsigned char* gsrc = reinterpret_cast<const unsigned char*>(a.src);
  const unsigned char* gctr = reinterpret_cast<const unsigned char*>(a.ctr);
  const unsigned char* gb = reinterpret_cast<const unsigned char*>(a.Brow);
  auto issue = [&](int it) {
    const int jj = BWD ? J - 1 - it : it;
    const int s = it % nstage;
    unsigned char* dst = ring + (size_t)s * stage;
    mbar_arrive_expect_tx(&bar[s], stage);
    bulk_g2s(dst, a.D + (size_t)jj * a.dstride, dbytes, &bar[s]);
    dst += dbytes;
    if (sbytes) { bulk_g2s(dst, gsrc + (size_t)jj * sbytes, sbytes, &bar[s]); dst += sbytes; }
    if (cbytes) { bulk_g2s(dst, gctr + (size_t)jj * cbytes, cbytes, &bar[s]); dst += cbytes; }
    if (bbytes) { bulk_g2s(dst, gb + (size_t)jj * bbytes, bbytes, &bar[s]); }
  };

  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstage; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  // initial state
  double2 x0 = make_double2(0.0, 0.0);
  if (active && a.init) {
    x0 = a.init[(size_t)(col0 + l) * N + i];
    x0.x *= a.init_scale;
    x0.y *= a.init_scale;
  }
  R hx = (R)x0.x, hy = (R)x0.y;   // state (binary64) or its hi part
  float lx = 0.f, ly = 0.f;        // lo part (mixed only)
  if (MIX) {
    lx = (float)(x0.x - (double)hx);
    ly = (float)(x0.y - (double)hy);
  }
  if (owner) {
    TD v;
    v.x = hx; v.y = hy;
    X[(0 * kc + l) * N + i] = v;
  }
  __syncthreads();
  // direct mode (large N): the step data is read from global memory
  constexpr bool ring_mode = !DIRECT;
  if (threadIdx.x == 0 && ring_mode) {
    const int pre = min(nstage - 1, J);
    for (int it = 0; it < pre; ++it) issue(it);
  }

  int cur = 0;
  int it = 0;
  int s = 0;                 // ring slot of step it
  uint32_t par = 0;          // mbarrier phase parity of that slot
  int s_issue = nstage - 1;  // ring slot the next prefetch goes to
  const TD* dcol0 = nullptr;
  for (; it < J; ++it) {
    const int jj = BWD ? J - 1 - it : it;
    if (threadIdx.x == 0 && ring_mode && it + nstage - 1 < J) {
      fence_proxy_async_smem();
      issue(it + nstage - 1);
    }
    if (a.states && owner && l == 0) {
      // vector chains store the state entering step j (a_j forward, lambda_{j+1} backward)
      const size_t row = (size_t)(BWD ? jj + 1 : jj) * N + i;
      if (MIX) reinterpret_cast<float4*>(a.states)[row] = make_float4((float)hx, (float)hy, lx, ly);
      else reinterpret_cast<double2*>(a.states)[row] = make_double2((double)hx, (double)hy);
    }
    // a thread whose wait gives up flags the CTA; the data it then reads is
    // never used (the loop ends at the step-end barrier)
    const TD* Ds;
    const TV* srcs;
    const TV* ctrs;
    const TB* brow;
    if (ring_mode) {
      if (!mbar_wait_bounded(&bar[s], par)) abort_flag = 1;
      const unsigned char* sp = ring + (size_t)s * stage;
      Ds = reinterpret_cast<const TD*>(sp);
      srcs = reinterpret_cast<const TV*>(sp + dbytes);
      ctrs = reinterpret_cast<const TV*>(sp + dbytes + sbytes);
      brow = reinterpret_cast<const TB*>(sp + dbytes + sbytes + cbytes);
    } else {
      Ds = reinterpret_cast<const TD*>(a.D + (size_t)jj * a.dstride);
      srcs = reinterpret_cast<const TV*>(gsrc + (size_t)jj * sbytes);
      ctrs = reinterpret_cast<const TV*>(gctr + (size_t)jj * cbytes);
      brow = reinterpret_cast<const TB*>(gb + (size_t)jj * bbytes);
    }
    const TD* Xc = X + (size_t)cur * kc * N + (size_t)l * N;

    // contraction on the entering state: Re(c^H x), summed over rows
    if (a.ctr) {
      R v = 0;
      if (owner) {
        const TV c = ctrs[i];
        v = c.x * hx + c.y * hy;
      }
      v = warp_sum(v);
      if (WPC == 1) {
        if (lane == 0 && l < ncols) reinterpret_cast<R*>(a.contr)[(size_t)jj * a.K + col0 + l] = v;
      } else if (lane == 0 && l < ncols) {
        red[((it & 1) * kc + l) * WPC + rb] = v;
      }
    }
    // matvec: acc_i = sum_q D[q][i] X[q]   (D symmetric), 4x unrolled over q
    R ax0 = 0, ay0 = 0, ax1 = 0, ay1 = 0;
    if (active) {
      dcol0 = Ds + i;
      int q = rsub;
      for (; q + 3 * RS < N; q += 4 * RS) {
        TD d0 = dcol0[(size_t)q * N], d1 = dcol0[(size_t)(q + RS) * N];
        TD d2 = dcol0[(size_t)(q + 2 * RS) * N], d3 = dcol0[(size_t)(q + 3 * RS) * N];
        const TD x0v = Xc[q], x1v = Xc[q + RS], x2v = Xc[q + 2 * RS], x3v = Xc[q + 3 * RS];
        if (BWD) { d0.y = -d0.y; d1.y = -d1.y; d2.y = -d2.y; d3.y = -d3.y; }
        ax0 = fma(d0.x, x0v.x, ax0); ax0 = fma(-d0.y, x0v.y, ax0);
        ay0 = fma(d0.x, x0v.y, ay0); ay0 = fma(d0.y, x0v.x, ay0);
        ax1 = fma(d1.x, x1v.x, ax1); ax1 = fma(-d1.y, x1v.y, ax1);
        ay1 = fma(d1.x, x1v.y, ay1); ay1 = fma(d1.y, x1v.x, ay1);
        ax0 = fma(d2.x, x2v.x, ax0); ax0 = fma(-d2.y, x2v.y, ax0);
        ay0 = fma(d2.x, x2v.y, ay0); ay0 = fma(d2.y, x2v.x, ay0);
        ax1 = fma(d3.x, x3v.x, ax1); ax1 = fma(-d3.y, x3v.y, ax1);
        ay1 = fma(d3.x, x3v.y, ay1); ay1 = fma(d3.y, x3v.x, ay1);
      }
      for (; q < N; q += RS) {
        TD d0 = dcol0[(size_t)q * N];
        const TD x0v = Xc[q];
        if (BWD) d0.y = -d0.y;
        ax0 = fma(d0.x, x0v.x, ax0); ax0 = fma(-d0.y, x0v.y, ax0);
        ay0 = fma(d0.x, x0v.y, ay0); ay0 = fma(d0.y, x0v.x, ay0);
      }
    }
    R ax = ax0 + ax1, ay = ay0 + ay1;
#pragma unroll
    for (int o = 1; o < RS; o <<= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (owner) {
      if (a.src) {
        const TV sv = srcs[i];
        const R b = a.Brow ? (R)brow[col0 + l] : (R)1;
        ax = fma(sv.x, b, ax);
        ay = fma(sv.y, b, ay);
      }
      if (MIX) {
        float fx = (float)hx, fy = (float)hy;
        pair_add(fx, lx, (float)ax);
        pair_add(fy, ly, (float)ay);
        hx = (R)fx;
        hy = (R)fy;
      } else {
        hx += ax;
        hy += ay;
      }
      TD v;
      v.x = hx; v.y = hy;
      X[(size_t)(cur ^ 1) * kc * N + (size_t)l * N + i] = v;
    }
    __syncthreads();
    if (abort_flag) break;
    if (a.ctr && WPC > 1 && rb == 0 && lane == 0 && l < ncols) {
      R v = 0;
      for (int w = 0; w < WPC; ++w) v += red[((it & 1) * kc + l) * WPC + w];
      reinterpret_cast<R*>(a.contr)[(size_t)jj * a.K + col0 + l] = v;
    }
    cur ^= 1;
    if (++s == nstage) { s = 0; par ^= 1u; }
    (void)s_issue;
  }
  if (abort_flag) {
    if (threadIdx.x == 0) {
      raise_status(a.status, DEV_TIMEOUT);
      // drain copies still in flight (bounded) before the CTA retires
      for (int k = it; k < min(J, it + nstage - 1); ++k)
        mbar_wait_bounded(&bar[k % nstage], (uint32_t)((k / nstage) & 1), 100000000ull);
    }
    return;
  }
  const double fx = (double)hx + (double)lx, fy = (double)hy + (double)ly;
  if (owner) {
    if (a.final_out) a.final_out[(size_t)(col0 + l) * N + i] = make_double2(fx, fy);
    if (a.states && l == 0) {
      const size_t row = (size_t)(BWD ? 0 : J) * N + i;
      if (MIX) reinterpret_cast<float4*>(a.states)[row] = make_float4((float)hx, (float)hy, lx, ly);
      else reinterpret_cast<double2*>(a.states)[row] = make_double2(fx, fy);
    }
    if (!(isfinite(fx) && isfinite(fy))) raise_status(a.status, DEV_NONFINITE);
  }
}

template <bool MIX, int RS, bool BWD>
static cudaError_t launch_one(const SweepArgs& a, cudaStream_t st) {
  using TD = typename SweepT<MIX>::D;
  using TV = typename SweepT<MIX>::V;
  using TB = typename SweepT<MIX>::B;
  const int RPW = 32 / RS;
  const int WPC = (a.N + RPW - 1) / RPW;
  const int threads = 32 * WPC * a.kc;
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  const uint32_t vb = (uint32_t)(sizeof(TV) * a.N + 15) / 16 * 16;
  const uint32_t stage = (uint32_t)a.dstride + (a.src ? vb : 0u) + (a.ctr ? vb : 0u) +
                         (a.Brow ? (uint32_t)(sizeof(TB) * a.Kp) : 0u);
  const size_t fixed = 2 * (size_t)a.kc * a.N * sizeof(TD) + (2 * (size_t)a.kc * WPC + 2) * 8 + 8;
  const size_t budget = 200 * 1024;
  int ns = 8;
  while (ns > 2 && (size_t)ns * stage + fixed + 8 * ns > budget) --ns;
  if (2 * (size_t)stage + fixed + 16 > budget) ns = 0;   // direct mode (large N)
  const size_t smem = (size_t)ns * stage + fixed + 8 * ns + 16;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  const int grid = (a.K + a.kc - 1) / a.kc;
  if (ns == 0) {
    set_max_smem((const void*)k_sweep<MIX, RS, BWD, true>);
    k_sweep<MIX, RS, BWD, true><<<grid, threads, smem, st>>>(a, ns);
  } else {
    set_max_smem((const void*)k_sweep<MIX, RS, BWD, false>);
    k_sweep<MIX, RS, BWD, false><<<grid, threads, smem, st>>>(a, ns);
  }
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepArgs& a, int d_fp64, cudaStream_t st) {
  // Each dot product is split over 4 lanes so that a column spreads over
  // four warps (all four sub-partitions) and the per-step dependent chain is
  // N/4 terms long; binary64 is issue-limited on GB300 (one warp instruction
  // per 64 cycles per sub-partition), binary32 is latency-limited.
  if (d_fp64) {
    if (a.backward) return launch_one<false, 4, true>(a, st);
    return launch_one<false, 4, false>(a, st);
  }
  if (a.backward) return launch_one<true, 4, true>(a, st);
  return launch_one<true, 4, false>(a, st);
}

}  // namespace qoc

namespace qoc {

// ---------------------------------------------------------------------------
// Blocked sweep: one dependent step per block of bs time steps (see block.cu):
//   X <- X + Delta X + Q B_blk,   Delta applied as y_i = sum_q M[q][i] x_q,
// block-start states stored for the contractions (panels) or the
// intermediate-state fill (vector chains).  Per block, M (N x N), Q (bs
// columns) and the bs rows of B are staged by bulk copies into the ring.
// ---------------------------------------------------------------------------
template <bool MIX, int RS, bool DIRECT>
__device__ __forceinline__ void bsweep_body(const BSweepArgs& a, const int cta, const int nstage,
                                            unsigned char* smem) {
  using TD = typename SweepT<MIX>::D;
  using TB = typename SweepT<MIX>::B;
  using R = typename SweepT<MIX>::R;
  const int N = a.N, kc = a.kc, J = a.J, bs = a.bs;
  const int nblk = (J + bs - 1) / bs;
  const int b0 = a.blk0, b1 = a.blk1 > 0 ? a.blk1 : nblk;   // this launch's blocks
  constexpr int RPW = 32 / RS;
  const int WPC = (N + RPW - 1) / RPW;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = warp / WPC, rb = warp % WPC;
  const int rsub = lane % RS;
  const int i = rb * RPW + lane / RS;
  const int col0 = cta * kc;
  const int ncols = min(kc, a.K - col0);
  const bool active = (l < ncols) && (i < N);
  const bool owner = active && rsub == 0;

  const uint32_t mbytes = (uint32_t)a.mstride;
  const uint32_t qbytes = a.Q ? (uint32_t)a.qstride : 0u;
  const uint32_t browb = (uint32_t)(sizeof(TB) * a.Kp);
  const uint32_t bmax = a.Brow ? browb * bs : 0u;
  const uint32_t stage = mbytes + qbytes + bmax;
  unsigned char* ring = smem;
  TD* X = reinterpret_cast<TD*>(ring + (size_t)nstage * stage);      // [2][kc][N]
  uint64_t* bar = reinterpret_cast<uint64_t*>(X + 2 * kc * N);
  __shared__ int abort_flag;

  const unsigned char* gB = reinterpret_cast<const unsigned char*>(a.Brow);
  auto issue = [&](int it) {
    const int s = (it - b0) % nstage;
    const int t0 = it * bs, bl = min(bs, J - t0);
    const int row0 = a.backward ? J - t0 - bl : t0;     // rows of this block, ascending in memory
    const uint32_t bb = a.Brow ? browb * bl : 0u;
    unsigned char* dst = ring + (size_t)s * stage;
    mbar_arrive_expect_tx(&bar[s], mbytes + qbytes + bb);
    bulk_g2s(dst, a.M + (size_t)it * a.mstride, mbytes, &bar[s]);
    if (qbytes) bulk_g2s(dst + mbytes, a.Q + (size_t)it * a.qstride, qbytes, &bar[s]);
    if (bb) bulk_g2s(dst + mbytes + qbytes, gB + (size_t)row0 * browb, bb, &bar[s]);
  };

  // direct mode (large N, a block does not fit the ring twice): the block
  // data is read straight from global memory (L2), no copies
  constexpr bool ring_mode = !DIRECT;
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int s = 0; s < nstage; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  double2 x0 = make_double2(0.0, 0.0);
  if (active && a.init && !a.resume) {
    x0 = a.init[(size_t)(col0 + l) * N + i];
    x0.x *= a.init_scale;
    x0.y *= a.init_scale;
  }
  R hx = (R)x0.x, hy = (R)x0.y;
  float lx = 0.f, ly = 0.f;
  if (MIX) {
    lx = (float)(x0.x - (double)hx);
    ly = (float)(x0.y - (double)hy);
  }
  if (active && a.resume) {   // the state a previous launch left at block b0
    const size_t e = ((size_t)b0 * a.K + col0 + l) * N + i;
    if (a.xblk_pairs) {
      const float4 v = reinterpret_cast<const float4*>(a.Xblk)[e];
      hx = (R)v.x; hy = (R)v.y; lx = v.z; ly = v.w;
    } else {
      const TD v = reinterpret_cast<const TD*>(a.Xblk)[e];
      hx = v.x; hy = v.y;
    }
  }
  if (owner) {
    TD v;
    v.x = hx; v.y = hy;
    X[(size_t)l * N + i] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0 && ring_mode) {
    const int pre = min(nstage - 1, b1 - b0);
    for (int it = b0; it < b0 + pre; ++it) issue(it);
  }
  int cur = 0, it = b0, s = 0;
  uint32_t par = 0;
  for (; it < b1; ++it) {
    const int t0 = it * bs, bl = min(bs, J - t0);
    if (threadIdx.x == 0 && ring_mode && it + nstage - 1 < b1) {
      fence_proxy_async_smem();
      issue(it + nstage - 1);
    }
    if (owner) {   // block-start state
      if (a.xblk_pairs) {
        reinterpret_cast<float4*>(a.Xblk)[((size_t)it * a.K + col0 + l) * N + i] =
            make_float4((float)hx, (float)hy, lx, ly);
      } else {
        TD v;
        v.x = hx; v.y = hy;
        reinterpret_cast<TD*>(a.Xblk)[((size_t)it * a.K + col0 + l) * N + i] = v;
      }
    }
    const TD* Ms;
    const TD* Qs;
    const TB* Bs;
    if (ring_mode) {
      if (!mbar_wait_bounded(&bar[s], par)) abort_flag = 1;
      const unsigned char* sp = ring + (size_t)s * stage;
      Ms = reinterpret_cast<const TD*>(sp);
      Qs = reinterpret_cast<const TD*>(sp + mbytes);
      Bs = reinterpret_cast<const TB*>(sp + mbytes + qbytes);
    } else {
      const int row0 = a.backward ? J - t0 - bl : t0;
      Ms = reinterpret_cast<const TD*>(a.M + (size_t)it * a.mstride);
      Qs = a.Q ? reinterpret_cast<const TD*>(a.Q + (size_t)it * a.qstride) : nullptr;
      Bs = a.Brow ? reinterpret_cast<const TB*>(gB + (size_t)row0 * browb) : nullptr;
    }
    const TD* Xc = X + (size_t)cur * kc * N + (size_t)l * N;
    R ax0 = 0, ay0 = 0, ax1 = 0, ay1 = 0;
    if (active) {
      const TD* mcol = Ms + i;
      int q = rsub;
      for (; q + 3 * RS < N; q += 4 * RS) {
        const TD d0 = mcol[(size_t)q * N], d1 = mcol[(size_t)(q + RS) * N];
        const TD d2 = mcol[(size_t)(q + 2 * RS) * N], d3 = mcol[(size_t)(q + 3 * RS) * N];
        const TD x0v = Xc[q], x1v = Xc[q + RS], x2v = Xc[q + 2 * RS], x3v = Xc[q + 3 * RS];
        ax0 = fma(d0.x, x0v.x, ax0); ax0 = fma(-d0.y, x0v.y, ax0);
        ay0 = fma(d0.x, x0v.y, ay0); ay0 = fma(d0.y, x0v.x, ay0);
        ax1 = fma(d1.x, x1v.x, ax1); ax1 = fma(-d1.y, x1v.y, ax1);
        ay1 = fma(d1.x, x1v.y, ay1); ay1 = fma(d1.y, x1v.x, ay1);
        ax0 = fma(d2.x, x2v.x, ax0); ax0 = fma(-d2.y, x2v.y, ax0);
        ay0 = fma(d2.x, x2v.y, ay0); ay0 = fma(d2.y, x2v.x, ay0);
        ax1 = fma(d3.x, x3v.x, ax1); ax1 = fma(-d3.y, x3v.y, ax1);
        ay1 = fma(d3.x, x3v.y, ay1); ay1 = fma(d3.y, x3v.x, ay1);
      }
      for (; q < N; q += RS) {
        const TD d0 = mcol[(size_t)q * N];
        const TD x0v = Xc[q];
        ax0 = fma(d0.x, x0v.x, ax0); ax0 = fma(-d0.y, x0v.y, ax0);
        ay0 = fma(d0.x, x0v.y, ay0); ay0 = fma(d0.y, x0v.x, ay0);
      }
      // rank-bl source update (spread over the RS lanes of the row)
      if (a.Q) {
        for (int m = rsub; m < bl; m += RS) {
          const TD qv = Qs[(size_t)m * N + i];
          const int lr = a.backward ? bl - 1 - m : m;
          const R b = (R)Bs[(size_t)lr * a.Kp + col0 + l];
          ax1 = fma(qv.x, b, ax1);
          ay1 = fma(qv.y, b, ay1);
        }
      }
    }
    R ax = ax0 + ax1, ay = ay0 + ay1;
#pragma unroll
    for (int o = 1; o < RS; o <<= 1) {
      ax += __shfl_xor_sync(0xffffffffu, ax, o);
      ay += __shfl_xor_sync(0xffffffffu, ay, o);
    }
    if (owner) {
      if (MIX) {
        float fx = (float)hx, fy = (float)hy;
        pair_add(fx, lx, (float)ax);
        pair_add(fy, ly, (float)ay);
        hx = (R)fx;
        hy = (R)fy;
      } else {
        hx += ax;
        hy += ay;
      }
      TD v;
      v.x = hx; v.y = hy;
      X[(size_t)(cur ^ 1) * kc * N + (size_t)l * N + i] = v;
    }
    __syncthreads();
    if (abort_flag) break;
    cur ^= 1;
    if (++s == nstage) { s = 0; par ^= 1u; }
  }
  if (abort_flag) {
    if (threadIdx.x == 0) {
      raise_status(a.status, DEV_TIMEOUT);
      for (int k = it; k < min(b1, it + nstage - 1); ++k)
        mbar_wait_bounded(&bar[(k - b0) % nstage], (uint32_t)(((k - b0) / nstage) & 1), 100000000ull);
    }
    return;
  }
  if (b1 < nblk) {   // a chunk: hand the end state to the launch that resumes at b1
    if (owner) {
      const size_t e = ((size_t)b1 * a.K + col0 + l) * N + i;
      if (a.xblk_pairs) {
        reinterpret_cast<float4*>(a.Xblk)[e] = make_float4((float)hx, (float)hy, lx, ly);
      } else {
        TD v;
        v.x = hx; v.y = hy;
        reinterpret_cast<TD*>(a.Xblk)[e] = v;
      }
    }
    return;
  }
  const double fx = (double)hx + (double)lx, fy = (double)hy + (double)ly;
  if (owner) {
    if (a.final_out) a.final_out[(size_t)(col0 + l) * N + i] = make_double2(fx, fy);
    if (a.states) {   // final state of a vector chain: a_J forward, lambda_0 backward
      const size_t row = (size_t)(a.backward ? 0 : J) * N + i;
      if (MIX) reinterpret_cast<float4*>(a.states)[row] = make_float4((float)hx, (float)hy, lx, ly);
      else reinterpret_cast<double2*>(a.states)[row] = make_double2(fx, fy);
    }
    if (!(isfinite(fx) && isfinite(fy))) raise_status(a.status, DEV_NONFINITE);
  }
}

// ---------------------------------------------------------------------------
// Blocked sweep with binary32 increments for N <= RS * NQ, warp-specialised.
// One producer warp keeps the ring full: an elected lane refills a slot with
// bulk copies as soon as every consumer warp has released it on the slot's
// "empty" barrier.  The consumer warps own the state: RS lanes per row i,
// lane r taking the terms q = r, r + RS, ...  A warp covers 32 / RS rows with
// r in the high lane bits, so each half-warp reads 16 (RS = 2) or 8 (RS = 4)
// consecutive rows of M: its shared-memory loads are free of (RS = 2) or have
// at most two-way (RS = 4) bank conflicts.  Each lane loads its M (and Q, B)
// entries of the NEXT block into registers right after the current block's
// X, so that the dependent part of a block step is: read X (shared,
// broadcast), the FMA chain, log2(RS) shuffle rounds, two additions, write
// X, one named barrier; the test that a block has landed runs a step ahead.
// NF = N when N = RS * NQ is fixed at compile time (constant offsets), else 0.
// X layout per column: entry q at run (q mod RS), position (q div RS); runs
// are XS = NQ + 2 float2 apart so the runs a warp reads sit in different
// banks.
// State update: with the state an unevaluated pair (hi, lo), the increment d
// is first added to lo (t = d + lo, one binary32 rounding of the order of the
// increment's own) and TwoSum(hi, t) gives the new pair exactly; only hi
// enters the next product.
// ---------------------------------------------------------------------------
template <int RS, int NQ>
struct FastRegs {
  static constexpr int UQ = (8 + RS - 1) / RS;   // source terms per lane (bs <= 8)
  float2 m[NQ];
  float2 q[UQ];
  float b[UQ];
};

// the entries one lane needs of one block (zeros where q >= N or the lane is idle)
template <int RS, int NQ, int NF>
__device__ __forceinline__ void fast_load(FastRegs<RS, NQ>& r, const unsigned char* sp, int Nrt,
                                          uint32_t mbytes, uint32_t qbytes, bool has_q, int bl,
                                          bool bwd, int Kp, int rsub, int i, int col, int kq,
                                          bool active) {
  const int N = NF ? NF : Nrt;
  const float2* Ms = reinterpret_cast<const float2*>(sp) + rsub * N + i;
#pragma unroll
  for (int k = 0; k < NQ; ++k)
    r.m[k] = (active && k < kq) ? Ms[RS * k * N] : make_float2(0.f, 0.f);
  if (has_q) {
    const float2* Qs = reinterpret_cast<const float2*>(sp + mbytes);
    const float* Bs = reinterpret_cast<const float*>(sp + mbytes + qbytes);
#pragma unroll
    for (int u = 0; u < FastRegs<RS, NQ>::UQ; ++u) {
      const int mm = rsub + RS * u;
      if (active && mm < bl) {
        const int lr = bwd ? bl - 1 - mm : mm;
        r.q[u] = Qs[mm * N + i];
        r.b[u] = Bs[lr * Kp + col];
      } else {
        r.q[u] = make_float2(0.f, 0.f);
        r.b[u] = 0.f;
      }
    }
  }
}

template <int RS, int NQ, int NF>
__device__ __forceinline__ void bsweep_fast_body(const BSweepArgs& a, const int cta, const int nstage,
                                                 unsigned char* smem) {
  constexpr int RPW = 32 / RS, XS = NQ + 2, UQ = FastRegs<RS, NQ>::UQ;
  const int N = NF ? NF : a.N;
  const int kc = a.kc, J = a.J, bs = a.bs, K = a.K, Kp = a.Kp;
  const bool bwd = a.backward != 0, has_q = a.Q != nullptr, has_b = a.Brow != nullptr;
  const bool pairs = a.xblk_pairs != 0;
  const int nblk = (J + bs - 1) / bs;
  const int b0 = a.blk0, nloc = (a.blk1 > 0 ? a.blk1 : nblk) - b0;   // blocks b0 .. b0 + nloc - 1
  const bool last = b0 + nloc == nblk;
  const int WPC = (N + RPW - 1) / RPW;
  const int ncw = WPC * kc;                       // consumer warps
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t mbytes = (uint32_t)a.mstride;
  const uint32_t qbytes = has_q ? (uint32_t)a.qstride : 0u;
  const uint32_t browb = (uint32_t)(sizeof(float) * Kp);
  const uint32_t stage = mbytes + qbytes + (has_b ? browb * bs : 0u);
  unsigned char* ring = smem;
  float2* Xs = reinterpret_cast<float2*>(ring + (size_t)nstage * stage);   // [2][kc][RS][XS]
  const int xbuf = kc * RS * XS;
  uint64_t* full = reinterpret_cast<uint64_t*>(Xs + 2 * xbuf);
  uint64_t* empty = full + nstage;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + nstage);

  for (int e = threadIdx.x; e < 2 * xbuf; e += blockDim.x) Xs[e] = make_float2(0.f, 0.f);
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int s = 0; s < nstage; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], ncw);
    }
    mbar_fence_init();
  }
  __syncthreads();
  if (warp > ncw) return;

  if (warp == ncw) {   // ---- producer ----
    if (lane != 0) return;
    const unsigned char* gM = a.M;
    const unsigned char* gQ = a.Q;
    const unsigned char* gB = reinterpret_cast<const unsigned char*>(a.Brow);
    const size_t ms = a.mstride, qs = a.qstride;
    int s = 0, round = 0, issued = 0;
    for (int li = 0; li < nloc; ++li) {
      const int it = b0 + li;
      if (*abort_flag) break;
      if (li >= nstage && !mbar_wait_or_flag(&empty[s], (uint32_t)((round - 1) & 1), abort_flag)) {
        *abort_flag = 1;
        break;
      }
      const int t0 = it * bs, bl = min(bs, J - t0);
      const int row0 = bwd ? J - t0 - bl : t0;
      const uint32_t qb = has_q ? (((uint32_t)(bl * N) * 8u + 15u) & ~15u) : 0u;
      const uint32_t bb = has_b ? browb * (uint32_t)bl : 0u;
      unsigned char* dst = ring + (size_t)s * stage;
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&full[s], mbytes + qb + bb);
      bulk_g2s(dst, gM + (size_t)it * ms, mbytes, &full[s]);
      if (qb) bulk_g2s(dst + mbytes, gQ + (size_t)it * qs, qb, &full[s]);
      if (bb) bulk_g2s(dst + mbytes + qbytes, gB + (size_t)row0 * browb, bb, &full[s]);
      issued = li + 1;
      if (++s == nstage) { s = 0; ++round; }
    }
    // the copies issued last (each the latest phase of its slot) have landed
    // before the CTA may exit, also when the consumers stopped early
    for (int k = max(0, issued - nstage); k < issued; ++k)
      mbar_wait_bounded(&full[k % nstage], (uint32_t)((k / nstage) & 1), 100000000ull);
    return;
  }

  // ---- consumers ----
  const int l = warp / WPC, rb = warp % WPC;
  const int rsub = lane / RPW;
  const int i = rb * RPW + (lane % RPW);
  const int col = cta * kc + l;
  const bool active = col < K && i < N;
  const bool owner = active && rsub == 0;
  const int kq = (N - rsub + RS - 1) / RS;        // terms q = rsub + RS k < N
  const int nthr = 32 * ncw;
  const int xw = (i % RS) * XS + i / RS;          // this row's entry in the permuted layout
  float2* Xl = Xs + l * RS * XS;
  const float4* Xr = reinterpret_cast<const float4*>(Xl + rsub * XS);

  double2 x0 = make_double2(0.0, 0.0);
  if (active && a.init && !a.resume) {
    x0 = a.init[(size_t)col * N + i];
    x0.x *= a.init_scale;
    x0.y *= a.init_scale;
  }
  float hx = (float)x0.x, hy = (float)x0.y;
  float lx = (float)(x0.x - (double)hx), ly = (float)(x0.y - (double)hy);
  const size_t xb_stride = (size_t)K * N;
  float4* xb4 = reinterpret_cast<float4*>(a.Xblk) + ((size_t)b0 * K + col) * N + i;
  float2* xb2 = reinterpret_cast<float2*>(a.Xblk) + ((size_t)b0 * K + col) * N + i;
  if (active && a.resume && pairs) {   // the state a previous launch left at block b0
    const float4 v = *xb4;
    hx = v.x; hy = v.y; lx = v.z; ly = v.w;
  }
  if (owner) {
    Xl[xw] = make_float2(hx, hy);
    if (pairs) *xb4 = make_float4(hx, hy, lx, ly);
    else *xb2 = make_float2(hx, hy);
  }

  // Every consumer takes the same exit decision: the OR, over the consumers,
  // of a failed wait, formed by the step's barrier itself.
  // Readiness runs one block ahead of use: step it tests block it + 2 (the
  // producer can always issue it once block it is released, even with two
  // slots) and consumes the test only at its end, so the test's latency is
  // off the dependent path; step it + 1 then loads block it + 2.
  FastRegs<RS, NQ> ra, rb2;
  int s = 0;
  uint32_t par = 0;
  bool bad = false;
  if (!mbar_wait_or_flag(&full[0], 0u, abort_flag)) {
    bad = true;
    *abort_flag = 1;
  }
  fast_load<RS, NQ, NF>(ra, ring, N, mbytes, qbytes, has_q, min(bs, J - b0 * bs), bwd, Kp, rsub, i, col,
                        kq, active);
  if (nloc > 1 &&
      !mbar_wait_or_flag(&full[1 % nstage], (uint32_t)((1 / nstage) & 1), abort_flag)) {
    bad = true;
    *abort_flag = 1;
  }
  int s2 = 2 % nstage;                              // slot and parity of block it + 2
  uint32_t par2 = (uint32_t)((2 / nstage) & 1);
  bool ok = !named_barrier_or(1, nthr, bad);

  int cur = 0;
  // one block step with `r` holding this block's data; `nx` receives the next block's
  auto step = [&](int it, const FastRegs<RS, NQ>& r, FastRegs<RS, NQ>& nx) -> bool {
    int s1 = s + 1;
    uint32_t par1 = par;
    if (s1 == nstage) { s1 = 0; par1 ^= 1u; }
    const bool more = it + 1 < nloc;            // it: the block's index within this launch
    const bool next_start = b0 + it + 1 < nblk;  // a block follows (here or in a later launch)
    // release this block's slot: its entries were loaded before the last barrier
    if (lane == 0) mbar_arrive(&empty[s]);
    const float4* xp = Xr + cur * (xbuf / 2);
    float4 xv[NQ / 2];
#pragma unroll
    for (int k = 0; k < NQ / 2; ++k) xv[k] = xp[k];
    const bool look = it + 2 < nloc;
    const uint32_t rdy = look ? mbar_try_wait(&full[s2], par2) : 1u;
    // the next block (independent of X, landed as tested one step earlier)
    if (more) {
      const int t1 = (b0 + it + 1) * bs;
      fast_load<RS, NQ, NF>(nx, ring + (size_t)s1 * stage, N, mbytes, qbytes, has_q, min(bs, J - t1),
                            bwd, Kp, rsub, i, col, kq, active);
    }
    float ax[4] = {0.f, 0.f, 0.f, 0.f}, ay[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
      const float xr = (k & 1) ? xv[k >> 1].z : xv[k >> 1].x;
      const float xi = (k & 1) ? xv[k >> 1].w : xv[k >> 1].y;
      ax[k & 3] = fmaf(r.m[k].x, xr, ax[k & 3]);
      ay[k & 3] = fmaf(r.m[k].x, xi, ay[k & 3]);
      ax[k & 3] = fmaf(-r.m[k].y, xi, ax[k & 3]);
      ay[k & 3] = fmaf(r.m[k].y, xr, ay[k & 3]);
    }
    if (has_q) {
#pragma unroll
      for (int u = 0; u < UQ; ++u) {
        ax[u & 3] = fmaf(r.q[u].x, r.b[u], ax[u & 3]);
        ay[u & 3] = fmaf(r.q[u].y, r.b[u], ay[u & 3]);
      }
    }
    float sx = (ax[0] + ax[1]) + (ax[2] + ax[3]);
    float sy = (ay[0] + ay[1]) + (ay[2] + ay[3]);
#pragma unroll
    for (int o = RPW; o < 32; o <<= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
    }
    if (owner) {
      two_sum(hx, __fadd_rn(sx, lx), hx, lx);
      two_sum(hy, __fadd_rn(sy, ly), hy, ly);
      Xl[(cur ^ 1) * xbuf + xw] = make_float2(hx, hy);
      if (next_start) {
        xb4 += xb_stride;
        xb2 += xb_stride;
        if (pairs) *xb4 = make_float4(hx, hy, lx, ly);
        else *xb2 = make_float2(hx, hy);
      }
    }
    if (!rdy && !mbar_wait_or_flag(&full[s2], par2, abort_flag)) {
      bad = true;
      *abort_flag = 1;
    }
    const bool stop = named_barrier_or(1, nthr, bad);
    cur ^= 1;
    s = s1;
    par = par1;
    if (++s2 == nstage) { s2 = 0; par2 ^= 1u; }
    return !stop;
  };
  int it = 0;
  for (; ok && it + 1 < nloc; it += 2) {
    ok = step(it, ra, rb2);
    if (ok) ok = step(it + 1, rb2, ra);
  }
  if (ok && it < nloc) ok = step(it, ra, rb2);
  if (!ok) {
    if (threadIdx.x == 0) raise_status(a.status, DEV_TIMEOUT);
    *abort_flag = 1;   // stops the producer
    return;
  }
  if (!last) return;   // a chunk: its end state is in Xblk[b0 + nloc]
  const double fx = (double)hx + (double)lx, fy = (double)hy + (double)ly;
  if (owner) {
    if (a.final_out) a.final_out[(size_t)col * N + i] = make_double2(fx, fy);
    if (a.states) {   // final state of a vector chain: a_J forward, lambda_0 backward
      const size_t row = (size_t)(bwd ? 0 : J) * N + i;
      reinterpret_cast<float4*>(a.states)[row] = make_float4(hx, hy, lx, ly);
    }
    if (!(isfinite(fx) && isfinite(fy))) raise_status(a.status, DEV_NONFINITE);
  }
}

// The two warp-specialised variants: kSmallRS lanes per row for N <= 32,
// four for N <= 64, with their CTA thread cap (two blocks of entries in
// registers).  Two lanes per row measured fastest at N = 32 (four and eight
// spread a column over more warps but lose more to the kernels that share
// the SMs during the panel sweeps).
constexpr int kFastThreads = 384;
constexpr int kSmallRS = 2;
enum { SWEEP_GENERAL = 0, SWEEP_FAST_SMALL = 1, SWEEP_FAST_R4 = 2 };

template <int RS, int NQ, int NF>
__global__ void __launch_bounds__(kFastThreads) k_bsweep_fast(const BSweepArgs a, const int nstage) {
  extern __shared__ __align__(128) unsigned char smem[];
  bsweep_fast_body<RS, NQ, NF>(a, blockIdx.x, nstage, smem);
}

template <int RS, int NQ>
__global__ void __launch_bounds__(kFastThreads) k_bsweep_fast_batch(const BSweepArgs* __restrict__ args,
                                                                 const int* __restrict__ cta_off,
                                                                 int nprob, const int nstage) {
  extern __shared__ __align__(128) unsigned char smem[];
  int lo = 0, hi = nprob;   // largest p with cta_off[p] <= blockIdx.x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
  }
  const BSweepArgs a = args[lo];
  bsweep_fast_body<RS, NQ, 0>(a, (int)blockIdx.x - cta_off[lo], nstage, smem);
}

template <bool MIX, int RS, bool DIRECT>
__global__ void __launch_bounds__(1024) k_bsweep(const BSweepArgs a, const int nstage) {
  extern __shared__ __align__(128) unsigned char smem[];
  bsweep_body<MIX, RS, DIRECT>(a, blockIdx.x, nstage, smem);
}

// Many problems in one launch: CTA b belongs to the problem p with
// cta_off[p] <= b < cta_off[p + 1]; every CTA runs its own dependent chain.
template <bool MIX, int RS, bool DIRECT>
__global__ void __launch_bounds__(1024) k_bsweep_batch(const BSweepArgs* __restrict__ args,
                                                       const int* __restrict__ cta_off, int nprob,
                                                       const int nstage) {
  extern __shared__ __align__(128) unsigned char smem[];
  int lo = 0, hi = nprob;   // largest p with cta_off[p] <= blockIdx.x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (cta_off[mid] <= (int)blockIdx.x) lo = mid; else hi = mid;
  }
  const BSweepArgs a = args[lo];
  bsweep_body<MIX, RS, DIRECT>(a, (int)blockIdx.x - cta_off[lo], nstage, smem);
}

// launch geometry of one problem's blocked sweep: threads, ring stages, smem
template <bool MIX, int RS>
static void bsweep_geometry(const BSweepArgs& a, int& threads, size_t& stage, size_t& fixed) {
  using TD = typename SweepT<MIX>::D;
  using TB = typename SweepT<MIX>::B;
  const int RPW = 32 / RS;
  const int WPC = (a.N + RPW - 1) / RPW;
  threads = 32 * WPC * a.kc;
  stage = a.mstride + (a.Q ? a.qstride : 0) + (a.Brow ? sizeof(TB) * a.Kp * a.bs : 0);
  fixed = 2 * (size_t)a.kc * a.N * sizeof(TD) + 16;
}

// Ring depth of a blocked-sweep launch: as deep as 16 stages when the grid
// fits one CTA per SM (bulk-copy latency is what the chain waits on), else
// shallow enough that ceil(grid / SMs) CTAs share an SM's shared memory.
static int ring_stages(size_t stage, size_t fixed, int threads, int total_ctas) {
  if (2 * stage + fixed + 16 + 16 > 200 * 1024) return 0;   // direct mode (large N)
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 1;
  }
  int cps = (total_ctas + nsm - 1) / nsm;
  const int by_threads = 2048 / (threads > 0 ? threads : 32);
  if (cps > by_threads) cps = by_threads;
  if (cps > 32) cps = 32;
  if (cps < 1) cps = 1;
  size_t budget = (size_t)(228 * 1024) / cps;
  budget = budget > 1024 + 16 ? budget - 1024 - 16 : 0;
  if (budget > 200 * 1024) budget = 200 * 1024;
  int ns = 16;
  while (ns > 2 && (size_t)ns * stage + fixed + 8 * ns > budget) --ns;
  return ns;
}

template <bool MIX, int RS>
static cudaError_t launch_bb(const BSweepArgs* host_args, const BSweepArgs* dev_args,
                             const int* dev_cta_off, int nprob, int total_ctas, cudaStream_t st) {
  int threads = 32;
  size_t stage = 16, fixed = 16;
  for (int p = 0; p < nprob; ++p) {
    int t;
    size_t s, f;
    bsweep_geometry<MIX, RS>(host_args[p], t, s, f);
    threads = t > threads ? t : threads;
    stage = s > stage ? s : stage;
    fixed = f > fixed ? f : fixed;
  }
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  const int ns = ring_stages(stage, fixed, threads, total_ctas);
  const size_t smem = (size_t)ns * stage + fixed + 8 * ns + 16;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (ns == 0) {
    set_max_smem((const void*)k_bsweep_batch<MIX, RS, true>);
    k_bsweep_batch<MIX, RS, true><<<total_ctas, threads, smem, st>>>(dev_args, dev_cta_off, nprob, ns);
  } else {
    set_max_smem((const void*)k_bsweep_batch<MIX, RS, false>);
    k_bsweep_batch<MIX, RS, false><<<total_ctas, threads, smem, st>>>(dev_args, dev_cta_off, nprob, ns);
  }
  return cudaGetLastError();
}

// geometry of the warp-specialised binary32 sweep (consumer warps + producer)
template <int RS, int NQ>
static void fast_geometry(const BSweepArgs& a, int& threads, size_t& stage, size_t& fixed) {
  threads = 32 * (((a.N + 32 / RS - 1) / (32 / RS)) * a.kc + 1);
  stage = a.mstride + (a.Q ? a.qstride : 0) + (a.Brow ? sizeof(float) * a.Kp * a.bs : 0);
  fixed = 2 * (size_t)a.kc * RS * (NQ + 2) * sizeof(float2) + 16;
}

// ring depth and shared memory of a warp-specialised launch; 0 if it does not apply
static int fast_plan(int threads, size_t stage, size_t fixed, int total_ctas, size_t& smem) {
  if (threads > kFastThreads) return 0;
  const int ns = ring_stages(stage, fixed + 8 * 16, threads, total_ctas);
  if (ns < 2) return 0;
  smem = (size_t)ns * stage + fixed + 16 * (size_t)ns + 16;
  return smem <= 227 * 1024 ? ns : 0;
}

template <int RS, int NQ>
static cudaError_t launch_fast(const BSweepArgs& a, cudaStream_t st) {
  int threads;
  size_t stage, fixed, smem = 0;
  fast_geometry<RS, NQ>(a, threads, stage, fixed);
  const int grid = (a.K + a.kc - 1) / a.kc;
  const int ns = fast_plan(threads, stage, fixed, grid, smem);
  if (!ns) return cudaErrorInvalidConfiguration;
  if (a.N == NQ * RS) {   // N = 32 or 64: offsets fixed at compile time
    set_max_smem((const void*)k_bsweep_fast<RS, NQ, NQ * RS>);
    k_bsweep_fast<RS, NQ, NQ * RS><<<grid, threads, smem, st>>>(a, ns);
  } else {
    set_max_smem((const void*)k_bsweep_fast<RS, NQ, 0>);
    k_bsweep_fast<RS, NQ, 0><<<grid, threads, smem, st>>>(a, ns);
  }
  return cudaGetLastError();
}

template <int RS, int NQ>
static cudaError_t launch_fast_batch(const BSweepArgs* host_args, const BSweepArgs* dev_args,
                                     const int* dev_cta_off, int nprob, int total_ctas,
                                     cudaStream_t st) {
  int threads = 32;
  size_t stage = 16, fixed = 16, smem = 0;
  for (int p = 0; p < nprob; ++p) {
    int t;
    size_t sg, f;
    fast_geometry<RS, NQ>(host_args[p], t, sg, f);
    threads = t > threads ? t : threads;
    stage = sg > stage ? sg : stage;
    fixed = f > fixed ? f : fixed;
  }
  const int ns = fast_plan(threads, stage, fixed, total_ctas, smem);
  if (!ns) return cudaErrorInvalidConfiguration;
  set_max_smem((const void*)k_bsweep_fast_batch<RS, NQ>);
  k_bsweep_fast_batch<RS, NQ><<<total_ctas, threads, smem, st>>>(dev_args, dev_cta_off, nprob, ns);
  return cudaGetLastError();
}

int bsweep_variant(const BSweepArgs& a, int mixed) {
  if (!mixed || a.N > 64) return SWEEP_GENERAL;
  int threads;
  size_t stage, fixed, smem = 0;
  if (a.N <= 32) {
    fast_geometry<kSmallRS, 32 / kSmallRS>(a, threads, stage, fixed);
    return fast_plan(threads, stage, fixed, 1, smem) > 0 ? SWEEP_FAST_SMALL : SWEEP_GENERAL;
  }
  fast_geometry<4, 16>(a, threads, stage, fixed);
  return fast_plan(threads, stage, fixed, 1, smem) > 0 ? SWEEP_FAST_R4 : SWEEP_GENERAL;
}

// The problems of one batched launch share the variant (the caller groups
// them so: a single evaluation of each takes the same one).
cudaError_t launch_bsweep_batch(const BSweepArgs* host_args, const BSweepArgs* dev_args,
                                const int* dev_cta_off, int nprob, int total_ctas, int mixed,
                                cudaStream_t st) {
  const int v = nprob > 0 ? bsweep_variant(host_args[0], mixed) : SWEEP_GENERAL;
  for (int p = 1; p < nprob; ++p)
    if (bsweep_variant(host_args[p], mixed) != v) return cudaErrorInvalidValue;
  if (v == SWEEP_FAST_SMALL)
    return launch_fast_batch<kSmallRS, 32 / kSmallRS>(host_args, dev_args, dev_cta_off, nprob,
                                                      total_ctas, st);
  if (v == SWEEP_FAST_R4)
    return launch_fast_batch<4, 16>(host_args, dev_args, dev_cta_off, nprob, total_ctas, st);
  if (mixed) return launch_bb<true, 4>(host_args, dev_args, dev_cta_off, nprob, total_ctas, st);
  return launch_bb<false, 4>(host_args, dev_args, dev_cta_off, nprob, total_ctas, st);
}

template <bool MIX, int RS>
static cudaError_t launch_b(const BSweepArgs& a, cudaStream_t st) {
  using TD = typename SweepT<MIX>::D;
  using TB = typename SweepT<MIX>::B;
  const int RPW = 32 / RS;
  const int WPC = (a.N + RPW - 1) / RPW;
  const int threads = 32 * WPC * a.kc;
  if (threads > 1024) return cudaErrorInvalidConfiguration;
  const size_t stage = a.mstride + (a.Q ? a.qstride : 0) + (a.Brow ? sizeof(TB) * a.Kp * a.bs : 0);
  const size_t fixed = 2 * (size_t)a.kc * a.N * sizeof(TD) + 16;
  const int grid = (a.K + a.kc - 1) / a.kc;
  const int ns = ring_stages(stage, fixed, threads, grid);
  const size_t smem = (size_t)ns * stage + fixed + 8 * ns + 16;
  if (smem > 227 * 1024) return cudaErrorInvalidConfiguration;
  if (ns == 0) {
    set_max_smem((const void*)k_bsweep<MIX, RS, true>);
    k_bsweep<MIX, RS, true><<<grid, threads, smem, st>>>(a, ns);
  } else {
    set_max_smem((const void*)k_bsweep<MIX, RS, false>);
    k_bsweep<MIX, RS, false><<<grid, threads, smem, st>>>(a, ns);
  }
  return cudaGetLastError();
}

cudaError_t launch_bsweep(const BSweepArgs& a, int mixed, cudaStream_t st) {
  if (mixed) {
    const int v = bsweep_variant(a, mixed);
    if (v == SWEEP_FAST_SMALL) return launch_fast<kSmallRS, 32 / kSmallRS>(a, st);
    if (v == SWEEP_FAST_R4) return launch_fast<4, 16>(a, st);
    return launch_b<true, 4>(a, st);
  }
  return launch_b<false, 4>(a, st);
}

}  // namespace qoc
