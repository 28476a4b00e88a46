// Time blocking of the sweeps: b consecutive steps folded into one.
//
// In sweep order (forward: t = j; backward: t = J-1-j), every recursion of
// the method reads  X_{t+1} = (I + E_t) X_t + s_t b_t^T  with the contraction
// c_t = Re(z_t^H X_t) taken on the entering state, where E_t = D_j forward and
// E_t = conj(D_j) backward (U_j^H in the rotating frame).  For a block of bl
// steps t0 .. t0+bl-1 write P_k = (I + E_{t0+k-1}) ... (I + E_{t0}) (P_0 = I):
//
//   X_{t0+bl}  = (I + Delta) X_{t0} + Q B_blk,        Delta = P_bl - I,
//   q_m        = (I + E_{t0+bl-1}) ... (I + E_{t0+m+1}) s_{t0+m}          (N x bl)
//   c_{t0+k}   = Re(w_k^H X_{t0}) + sum_{m<k} Re(Gamma_{k,m}) b_{t0+m},
//   w_k        = P_k^H z_{t0+k},     Gamma_{k,m} = z_{t0+k}^H (I + E_{t0+k-1}) ... (I + E_{t0+m+1}) s_{t0+m}.
//
// Delta, Q, W, Gamma depend only on the step data, so they are computed here
// in parallel over blocks; the sequential sweep then takes J/bl steps of one
// matrix-panel product each, storing only block-start states, and the
// contractions and intermediate states are recovered afterwards, again in
// parallel over blocks.  Everything uses only the single-step increments
// E_t, each block product in the increment form Delta_{k+1} = Delta_k + E_k
// + E_k Delta_k (binary32 rounding scales with |Delta|, not with |P| = 1).
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

template <bool MIX> struct BlkT;
template <> struct BlkT<false> { using C = double2; using R = double; };
template <> struct BlkT<true> { using C = float2; using R = float; };

template <typename C> __device__ __forceinline__ C cz();
template <> __device__ __forceinline__ double2 cz<double2>() { return make_double2(0.0, 0.0); }
template <> __device__ __forceinline__ float2 cz<float2>() { return make_float2(0.f, 0.f); }

template <typename C> __device__ __forceinline__ C cmk(double x, double y);
template <> __device__ __forceinline__ double2 cmk<double2>(double x, double y) { return make_double2(x, y); }
template <> __device__ __forceinline__ float2 cmk<float2>(double x, double y) { return make_float2((float)x, (float)y); }

// E_t element (p, q) of block step k in sweep order (conj for backward)
template <typename C>
__device__ __forceinline__ C load_E(const unsigned char* D, size_t dstride, int j, int N, int p, int q, bool bwd) {
  C v = reinterpret_cast<const C*>(D + (size_t)j * dstride)[p * N + q];
  if (bwd) v.y = -v.y;
  return v;
}

// ---------------------------------------------------------------------------
// Delta per block and direction (one CTA per block, blocks in sweep order).
// Writes M[q][i] = Delta[i][q], the layout the blocked sweep reads
// column-wise (y_i = sum_q M[q][i] x_q).
// ---------------------------------------------------------------------------
template <bool MIX>
__device__ __forceinline__ void block_delta_step(const unsigned char* __restrict__ D, size_t dstride,
                                                 int N, int J, int bsteps, int bwd,
                                                 unsigned char* __restrict__ Mo, size_t mstride,
                                                 int blk, unsigned char* smem_raw) {
  using C = typename BlkT<MIX>::C;
  const int t0 = blk * bsteps;
  if (t0 >= J) return;
  const int bl = min(bsteps, J - t0);
  const int ld = N + 1;
  C* Dl = reinterpret_cast<C*>(smem_raw);       // [N][ld] Delta
  C* Tm = Dl + N * ld;                           // [N][ld] E_k Delta
  C* Ek = Tm + N * ld;                           // [N][ld] E_k
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < N * N; e += nt) Dl[(e / N) * ld + e % N] = cz<C>();
  __syncthreads();
  for (int k = 0; k < bl; ++k) {
    const int j = bwd ? J - 1 - (t0 + k) : t0 + k;
    for (int e = tid; e < N * N; e += nt) Ek[(e / N) * ld + e % N] = load_E<C>(D, dstride, j, N, e / N, e % N, bwd);
    __syncthreads();
    // Tm = E_k Delta   (E symmetric: E[i][r] = E[r][i])
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, c = e % N;
      C acc = cz<C>();
      for (int r = 0; r < N; ++r) cfma(acc, Ek[r * ld + i], Dl[r * ld + c]);
      Tm[i * ld + c] = acc;
    }
    __syncthreads();
    for (int e = tid; e < N * N; e += nt) {
      const int i = e / N, c = e % N;
      C v = Dl[i * ld + c];
      const C a = Ek[i * ld + c], b = Tm[i * ld + c];
      v.x += a.x + b.x;
      v.y += a.y + b.y;
      Dl[i * ld + c] = v;
    }
    __syncthreads();
  }
  C* mo = reinterpret_cast<C*>(Mo + (size_t)blk * mstride);
  for (int e = tid; e < N * N; e += nt) {
    const int q = e / N, i = e % N;
    mo[q * N + i] = Dl[i * ld + q];
  }
}

// one block per CTA in shared memory, or a persistent grid over a global workspace
template <bool MIX, bool GWS>   // GWS: storage in the global workspace (compile-time)
__global__ void k_block_delta(const unsigned char* __restrict__ D, size_t dstride, int N, int J,
                              int bsteps, int bwd, unsigned char* __restrict__ Mo, size_t mstride,
                              int nblk, unsigned char* gws, size_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    block_delta_step<MIX>(D, dstride, N, J, bsteps, bwd, Mo, mstride, blk, base);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Q, W, Gamma per block for one direction (one CTA per block).
//   forward recursion  Qk <- Qk + E_k Qk + s_k e_k^T, Gamma_{k,.} = z_k^H Qk (before)
//   backward recursion R  <- R + E_k^H R + z_k e_k^T (k from bl-1 down), W = R at k = 0
// Layouts (per block, stride vbstride bytes):  Q[m][i], W[k][i] (bsteps x N
// each, columns contiguous), Gamma[k][m] (bsteps x bsteps).  Source and
// contraction vectors are indexed by step j in memory order with byte stride
// vstride; block step k in sweep order is step j = t0 + k forward, J-1-t0-k
// backward.
// ---------------------------------------------------------------------------
template <bool MIX>
__device__ __forceinline__ void block_src_step(const unsigned char* __restrict__ D, size_t dstride,
                                               int N, int J, int bsteps, int bwd,
                                               const unsigned char* __restrict__ src,
                                               const unsigned char* __restrict__ ctr, size_t vstride,
                                               unsigned char* __restrict__ Qo,
                                               unsigned char* __restrict__ Wo,
                                               unsigned char* __restrict__ Go, size_t qstride,
                                               size_t gstride, int what, int blk,
                                               unsigned char* smem_raw) {
  using C = typename BlkT<MIX>::C;
  const bool wq = what & BS_Q, wg = what & BS_WG;
  const int t0 = blk * bsteps;
  if (t0 >= J) return;
  const int bl = min(bsteps, J - t0);
  const int ld = N + 1;
  C* Ek = reinterpret_cast<C*>(smem_raw);        // [N][ld]
  C* Pn = Ek + N * ld;                           // [bsteps][N] panel (Q or R), column-major
  C* Tn = Pn + bsteps * N;                       // [bsteps][N] scratch
  C* Gm = Tn + bsteps * N;                       // [bsteps][bsteps]
  const int tid = threadIdx.x, nt = blockDim.x;
  auto stepj = [&](int k) { return bwd ? J - 1 - (t0 + k) : t0 + k; };
  auto vec = [&](const unsigned char* base, int j, int i) {
    return reinterpret_cast<const C*>(base + (size_t)j * vstride)[i];
  };
  for (int e = tid; e < bsteps * N; e += nt) Pn[e] = cz<C>();
  for (int e = tid; e < bsteps * bsteps; e += nt) Gm[e] = cz<C>();
  __syncthreads();
  // forward recursion: Q and Gamma
  for (int k = 0; k < bl; ++k) {
    const int j = stepj(k);
    for (int e = tid; e < N * N; e += nt) Ek[(e / N) * ld + e % N] = load_E<C>(D, dstride, j, N, e / N, e % N, bwd);
    __syncthreads();
    // Gamma_{k,m} = z_k^H Q[:, m] for m < k  (one warp per m)
    const int warp = tid >> 5, lane = tid & 31, nwarp = (nt + 31) >> 5;
    for (int m = warp; wg && m < k; m += nwarp) {
      typename BlkT<MIX>::R gx = 0, gy = 0;
      for (int i = lane; i < N; i += 32) {
        const C z = vec(ctr, j, i), q = Pn[m * N + i];
        gx += z.x * q.x + z.y * q.y;
        gy += z.x * q.y - z.y * q.x;
      }
      gx = warp_sum(gx);
      gy = warp_sum(gy);
      if (lane == 0) Gm[k * bsteps + m] = cmk<C>(gx, gy);
    }
    // Tn = E_k Q (columns m < k)
    for (int e = tid; e < k * N; e += nt) {
      const int m = e / N, i = e % N;
      C acc = cz<C>();
      for (int r = 0; r < N; ++r) cfma(acc, Ek[r * ld + i], Pn[m * N + r]);
      Tn[m * N + i] = acc;
    }
    __syncthreads();
    for (int e = tid; e < (k + 1) * N; e += nt) {
      const int m = e / N, i = e % N;
      if (m < k) {
        C v = Pn[m * N + i];
        v.x += Tn[m * N + i].x;
        v.y += Tn[m * N + i].y;
        Pn[m * N + i] = v;
      } else {
        Pn[m * N + i] = vec(src, j, i);
      }
    }
    __syncthreads();
  }
  if (wq) {
    C* qo = reinterpret_cast<C*>(Qo + (size_t)blk * qstride);
    for (int e = tid; e < bsteps * N; e += nt) qo[e] = (e / N) < bl ? Pn[e] : cz<C>();
  }
  if (!wg) return;
  C* go = reinterpret_cast<C*>(Go + (size_t)blk * gstride);
  for (int e = tid; e < bsteps * bsteps; e += nt) go[e] = Gm[e];
  __syncthreads();
  // backward recursion: W (w_k = P_k^H z_k)
  for (int e = tid; e < bsteps * N; e += nt) Pn[e] = cz<C>();
  __syncthreads();
  for (int k = bl - 1; k >= 0; --k) {
    const int j = stepj(k);
    // R <- R + E_k^H R for the columns already present (k' > k), then column k = z_k
    for (int e = tid; e < N * N; e += nt) Ek[(e / N) * ld + e % N] = load_E<C>(D, dstride, j, N, e / N, e % N, bwd);
    __syncthreads();
    for (int e = tid; e < (bl - 1 - k) * N; e += nt) {
      const int m = k + 1 + e / N, i = e % N;
      C acc = cz<C>();
      for (int r = 0; r < N; ++r) cfma_conj(acc, Ek[r * ld + i], Pn[m * N + r]);   // E^H = conj(E) (symmetric)
      Tn[m * N + i] = acc;
    }
    __syncthreads();
    for (int e = tid; e < (bl - k) * N; e += nt) {
      const int m = k + e / N, i = e % N;
      if (m > k) {
        C v = Pn[m * N + i];
        v.x += Tn[m * N + i].x;
        v.y += Tn[m * N + i].y;
        Pn[m * N + i] = v;
      } else {
        Pn[m * N + i] = vec(ctr, j, i);
      }
    }
    __syncthreads();
  }
  C* wo = reinterpret_cast<C*>(Wo + (size_t)blk * qstride);
  for (int e = tid; e < bsteps * N; e += nt) wo[e] = (e / N) < bl ? Pn[e] : cz<C>();
}

template <bool MIX, bool GWS>   // GWS: storage in the global workspace (compile-time)
__global__ void k_block_src(const unsigned char* __restrict__ D, size_t dstride, int N, int J,
                            int bsteps, int bwd, const unsigned char* __restrict__ src,
                            const unsigned char* __restrict__ ctr, size_t vstride,
                            unsigned char* __restrict__ Qo, unsigned char* __restrict__ Wo,
                            unsigned char* __restrict__ Go, size_t qstride, size_t gstride,
                            int what, int nblk, unsigned char* gws, size_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    block_src_step<MIX>(D, dstride, N, J, bsteps, bwd, src, ctr, vstride, Qo, Wo, Go, qstride,
                        gstride, what, blk, base);
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Contractions from block-start states (parallel over blocks x columns):
//   c_{t0+k} = Re(w_k^H X_{t0}) + sum_{m<k} Re(Gamma_{k,m}) b_{t0+m}
// X_blk: [nblk+1][K][N] block-start states (C).  contr: J x K (double, or
// float when mixed), written at step j of block step k.
// ---------------------------------------------------------------------------
template <bool MIX>
__global__ void k_block_contract(const unsigned char* __restrict__ Xblk, const unsigned char* __restrict__ Wb,
                                 const unsigned char* __restrict__ Gb, size_t qstride, size_t gstride,
                                 const void* __restrict__ Brow, int Kp, int N, int K, int J, int bsteps,
                                 int bwd, void* __restrict__ contr) {
  using C = typename BlkT<MIX>::C;
  using R = typename BlkT<MIX>::R;
  const int blk = blockIdx.x;
  const int t0 = blk * bsteps;
  if (t0 >= J) return;
  const int bl = min(bsteps, J - t0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const C* X = reinterpret_cast<const C*>(Xblk) + (size_t)blk * K * N;
  const C* W = reinterpret_cast<const C*>(Wb + (size_t)blk * qstride);
  const C* G = reinterpret_cast<const C*>(Gb + (size_t)blk * gstride);
  const R* B = reinterpret_cast<const R*>(Brow);
  // one warp per (column l, block step k)
  for (int task = blockIdx.y * nwarp + warp; task < K * bl; task += gridDim.y * nwarp) {
    const int l = task / bl, k = task % bl;
    R v = 0;
    for (int i = lane; i < N; i += 32) {
      const C w = W[k * N + i], x = X[(size_t)l * N + i];
      v += w.x * x.x + w.y * x.y;
    }
    v = warp_sum(v);
    if (lane == 0) {
      for (int m = 0; m < k; ++m) {
        const int jm = bwd ? J - 1 - (t0 + m) : t0 + m;
        v += G[k * bsteps + m].x * B[(size_t)jm * Kp + l];
      }
      const int j = bwd ? J - 1 - (t0 + k) : t0 + k;
      reinterpret_cast<R*>(contr)[(size_t)j * K + l] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// Intermediate states of a vector chain from its block-start states (one CTA
// per block): x <- x + E_k x for k = 0 .. bl-2, writing every entering state.
// States use the chain layout: forward writes row j = t0 + k (a_j), backward
// writes row j + 1 (lambda_{j+1}).  Binary64, or float pairs (float4) when mixed.
// ---------------------------------------------------------------------------
template <bool MIX>
__global__ void k_block_fill(const unsigned char* __restrict__ D, size_t dstride, int N, int J,
                             int bsteps, int bwd, const unsigned char* __restrict__ Xblk,
                             void* __restrict__ states) {
  using C = typename BlkT<MIX>::C;
  using R = typename BlkT<MIX>::R;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int blk = blockIdx.x;
  const int t0 = blk * bsteps;
  if (t0 >= J) return;
  const int bl = min(bsteps, J - t0);
  C* xs = reinterpret_cast<C*>(smem_raw);     // [N] hi parts
  const int i = threadIdx.x;                  // one thread per row (N <= blockDim)
  R hx = 0, hy = 0;
  float lx = 0.f, ly = 0.f;
  if (i < N) {
    if (MIX) {
      const float4 v = reinterpret_cast<const float4*>(Xblk)[(size_t)blk * N + i];
      hx = v.x; hy = v.y; lx = v.z; ly = v.w;
    } else {
      const double2 v = reinterpret_cast<const double2*>(Xblk)[(size_t)blk * N + i];
      hx = v.x; hy = v.y;
    }
    C c;
    c.x = hx; c.y = hy;
    xs[i] = c;
  }
  __syncthreads();
  for (int k = 0; k < bl; ++k) {
    const int j = bwd ? J - 1 - (t0 + k) : t0 + k;
    if (i < N) {
      const size_t row = (size_t)(bwd ? j + 1 : j) * N + i;
      if (MIX) reinterpret_cast<float4*>(states)[row] = make_float4((float)hx, (float)hy, lx, ly);
      else reinterpret_cast<double2*>(states)[row] = make_double2((double)hx, (double)hy);
    }
    if (k == bl - 1) break;
    R ax = 0, ay = 0;
    if (i < N) {
      const C* Dj = reinterpret_cast<const C*>(D + (size_t)j * dstride);
      for (int q = 0; q < N; ++q) {
        C d = Dj[(size_t)q * N + i];
        if (bwd) d.y = -d.y;
        const C x = xs[q];
        ax = fma(d.x, x.x, fma(-d.y, x.y, ax));
        ay = fma(d.x, x.y, fma(d.y, x.x, ay));
      }
    }
    __syncthreads();
    if (i < N) {
      if (MIX) {
        float fx = (float)hx, fy = (float)hy;
        pair_add(fx, lx, (float)ax);
        pair_add(fy, ly, (float)ay);
        hx = fx; hy = fy;
      } else {
        hx += ax;
        hy += ay;
      }
      C c;
      c.x = hx; c.y = hy;
      xs[i] = c;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
size_t block_delta_bytes(int N, int mixed) { return 3 * (size_t)N * (N + 1) * (mixed ? 8 : 16); }
size_t block_src_bytes(int N, int bsteps, int mixed) {
  return ((size_t)N * (N + 1) + 2 * (size_t)bsteps * N + (size_t)bsteps * bsteps) * (mixed ? 8 : 16);
}

cudaError_t launch_block_delta(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                               int mixed, void* M, size_t mstride, cudaStream_t st,
                               const StepSpace& ws) {
  const int nblk = (J + bsteps - 1) / bsteps;
  const int threads = N <= 16 ? 128 : (N <= 128 ? 256 : 512);
  StepGrid g;
  if (mixed) {
    if (!step_grid(block_delta_bytes(N, 1), nblk, ws, (const void*)k_block_delta<true, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_block_delta<true, true><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps,
                                                           bwd, (unsigned char*)M, mstride, nblk, g.gws,
                                                           g.per_cta);
    else
      k_block_delta<true, false><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps,
                                                           bwd, (unsigned char*)M, mstride, nblk, g.gws,
                                                           g.per_cta);
  } else {
    if (!step_grid(block_delta_bytes(N, 0), nblk, ws, (const void*)k_block_delta<false, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_block_delta<false, true><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps,
                                                            bwd, (unsigned char*)M, mstride, nblk, g.gws,
                                                            g.per_cta);
    else
      k_block_delta<false, false><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps,
                                                            bwd, (unsigned char*)M, mstride, nblk, g.gws,
                                                            g.per_cta);
  }
  return cudaGetLastError();
}
cudaError_t launch_block_src(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                             int mixed, const void* src, const void* ctr, size_t vstride, void* Q,
                             void* W, void* G, size_t qstride, size_t gstride, int what,
                             cudaStream_t st, const StepSpace& ws) {
  const int nblk = (J + bsteps - 1) / bsteps;
  const int threads = N <= 128 ? 256 : 512;
  StepGrid g;
  if (mixed) {
    if (!step_grid(block_src_bytes(N, bsteps, 1), nblk, ws, (const void*)k_block_src<true, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_block_src<true, true><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                         (const unsigned char*)src, (const unsigned char*)ctr,
                                                         vstride, (unsigned char*)Q, (unsigned char*)W,
                                                         (unsigned char*)G, qstride, gstride, what, nblk,
                                                         g.gws, g.per_cta);
    else
      k_block_src<true, false><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                         (const unsigned char*)src, (const unsigned char*)ctr,
                                                         vstride, (unsigned char*)Q, (unsigned char*)W,
                                                         (unsigned char*)G, qstride, gstride, what, nblk,
                                                         g.gws, g.per_cta);
  } else {
    if (!step_grid(block_src_bytes(N, bsteps, 0), nblk, ws, (const void*)k_block_src<false, false>, g))
      return cudaErrorInvalidConfiguration;
    if (g.gws)
      k_block_src<false, true><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                          (const unsigned char*)src, (const unsigned char*)ctr,
                                                          vstride, (unsigned char*)Q, (unsigned char*)W,
                                                          (unsigned char*)G, qstride, gstride, what, nblk,
                                                          g.gws, g.per_cta);
    else
      k_block_src<false, false><<<g.grid, threads, g.smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                          (const unsigned char*)src, (const unsigned char*)ctr,
                                                          vstride, (unsigned char*)Q, (unsigned char*)W,
                                                          (unsigned char*)G, qstride, gstride, what, nblk,
                                                          g.gws, g.per_cta);
  }
  return cudaGetLastError();
}
cudaError_t launch_block_contract(const void* Xblk, const void* W, const void* G, size_t qstride,
                                  size_t gstride, const void* Brow, int Kp, int N, int K, int J,
                                  int bsteps, int bwd, int mixed, void* contr, cudaStream_t st) {
  const int nblk = (J + bsteps - 1) / bsteps;
  const int threads = 256;
  const int gy = (K * bsteps + 7) / 8;
  dim3 grid(nblk, gy > 64 ? 64 : gy);
  if (mixed)
    k_block_contract<true><<<grid, threads, 0, st>>>((const unsigned char*)Xblk, (const unsigned char*)W,
                                                     (const unsigned char*)G, qstride, gstride, Brow, Kp,
                                                     N, K, J, bsteps, bwd, contr);
  else
    k_block_contract<false><<<grid, threads, 0, st>>>((const unsigned char*)Xblk, (const unsigned char*)W,
                                                      (const unsigned char*)G, qstride, gstride, Brow,
                                                      Kp, N, K, J, bsteps, bwd, contr);
  return cudaGetLastError();
}

cudaError_t launch_block_fill(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                              int mixed, const void* Xblk, void* states, cudaStream_t st) {
  const int nblk = (J + bsteps - 1) / bsteps;
  const int threads = ((N + 31) / 32) * 32;
  const size_t smem = (size_t)N * (mixed ? 8 : 16);
  if (mixed)
    k_block_fill<true><<<nblk, threads, smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                    (const unsigned char*)Xblk, states);
  else
    k_block_fill<false><<<nblk, threads, smem, st>>>((const unsigned char*)D, dstride, N, J, bsteps, bwd,
                                                     (const unsigned char*)Xblk, states);
  return cudaGetLastError();
}

}  // namespace qoc
