// Per-step contractions that need only the state a_j and costate
// lambda_{j+1} (parallel over j, after the two vector chains):
//
//   a~ = W^T a_j,  l~ = W^T lambda_{j+1}           (eigen-coordinates)
//   p_j = G_j a_j       = W (P~ a~)                (source of the tangent panel, Eq. gradatheta)
//   y_j = G_j^H l_{j+1} = W (conj(P~) l~)          (source of the mu panel, Eq. musys)
//   g_j = Re(l_{j+1}^H G_j a_j)   = Re(l~^H P~ a~)   (gradient, Eq. dLdf)
//   c_j = Re(l_{j+1}^H G2_j a_j)  = Re(l~^H X' a~)   (Hessian diagonal term, Eq. d2Ldf2)
//
// with P~ = Gamma1 o M~ and X' from the spectral preparation.  The stored
// states are in the frame rotating with the spectral shift m (a^_j =
// e^{i j dt m} a_j, likewise lambda^), so with kappa = e^{i dt m}:
//   p^_j = kappa W (P~ a~^),  y^_j = conj(kappa) W (conj(P~) l~^),
//   g_j = Re(kappa l~^H P~ a~),  c_j = Re(kappa l~^H X' a~).
// Everything here is binary64; one CTA per step.
#include "common.cuh"
#include "kernels.hpp"

namespace qoc {

__device__ __forceinline__ double2 load_state(const void* base, int mixed, size_t idx) {
  if (mixed) {
    float4 v = reinterpret_cast<const float4*>(base)[idx];
    return make_double2((double)v.x + (double)v.z, (double)v.y + (double)v.w);
  }
  return reinterpret_cast<const double2*>(base)[idx];
}

__device__ __forceinline__ void pointwise_step(const double* __restrict__ Wg,
                                               const double2* __restrict__ Ptil,
                                               const double2* __restrict__ Xp, const void* a_hat,
                                               const void* l_hat, int mixed, int N, int j,
                                               double2 kappa, void* p_hat, void* y_hat,
                                               size_t vstride, double* __restrict__ g,
                                               double* __restrict__ c, int what,
                                               double2* __restrict__ rbuf,
                                               unsigned char* smem_raw) {
  const bool wp = what & PW_P, wy = what & PW_Y, wc = what & PW_C;
  const bool reuse = (what & PW_RUSE) && rbuf && wy && !wp;   // r_j stored by an earlier PW_P
  const bool need_l = wy || wc;
  const bool need_a = wp || wc || (wy && !reuse);
  const int ld = N + 1;
  double* W = reinterpret_cast<double*>(smem_raw);                     // [N][ld]
  // N (N + 1) is even, so the double2 arrays after W stay 16-byte aligned
  double2* av = reinterpret_cast<double2*>(W + N * ld);                // a~
  double2* lv = av + N;                                                // l~
  double2* at = lv + N;                                                // a^ raw, then P~ a~
  double2* lt = at + N;                                                // lambda^ raw, then conj(P~) l~
  double* red = reinterpret_cast<double*>(lt + N);                     // [2][32]
  const int tid = threadIdx.x, nt = blockDim.x;
  const double* Wj = Wg + (size_t)j * N * N;
  for (int e = tid; e < N * N; e += nt) W[(e / N) * ld + (e % N)] = Wj[e];
  for (int p = tid; p < N; p += nt) {
    if (need_a) at[p] = load_state(a_hat, mixed, (size_t)j * N + p);
    if (need_l) lt[p] = load_state(l_hat, mixed, (size_t)(j + 1) * N + p);
  }
  __syncthreads();
  // eigen-coordinates
  for (int p = tid; p < N; p += nt) {
    double2 sa = make_double2(0, 0), sl = make_double2(0, 0);
    for (int r = 0; r < N; ++r) {
      double w = W[r * ld + p];
      if (need_a) { sa.x = fma(w, at[r].x, sa.x); sa.y = fma(w, at[r].y, sa.y); }
      if (need_l) { sl.x = fma(w, lt[r].x, sl.x); sl.y = fma(w, lt[r].y, sl.y); }
    }
    av[p] = sa;
    lv[p] = sl;
  }
  __syncthreads();
  const double2* Pj = Ptil + (size_t)j * N * N;
  const double2* Xj = Xp + (size_t)j * N * N;
  double gpart = 0, cpart = 0;
  for (int p = tid; p < N; p += nt) {
    double2 r = make_double2(0, 0), s = make_double2(0, 0), x = make_double2(0, 0);
    for (int q = 0; q < N; ++q) {
      if (wp || wy) {
        const double2 P = Pj[(size_t)q * N + p];          // symmetric: P[p][q] = P[q][p]
        if (!reuse) cfma(r, P, av[q]);
        if (wy) cfma_conj(s, P, lv[q]);
      }
      if (wc) cfma(x, Xj[(size_t)q * N + p], av[q]);
    }
    if (reuse) r = rbuf[(size_t)j * N + p];
    else if (wp && rbuf) rbuf[(size_t)j * N + p] = r;
    // Re(kappa conj(l~_p) r_p), Re(kappa conj(l~_p) x_p)
    if (wy) gpart += cmul(kappa, cconjmul(lv[p], r)).x;
    if (wc) cpart += cmul(kappa, cconjmul(lv[p], x)).x;
    at[p] = r;   // a^ no longer needed
    lt[p] = s;
  }
  if (wy || wc) {
    gpart = warp_sum(gpart);
    cpart = warp_sum(cpart);
    if ((tid & 31) == 0) { red[tid >> 5] = gpart; red[32 + (tid >> 5)] = cpart; }
  }
  __syncthreads();
  if (tid == 0 && (wy || wc)) {
    double gs = 0, cs = 0;
    for (int w = 0; w < (nt + 31) / 32; ++w) { gs += red[w]; cs += red[32 + w]; }
    if (wy) g[j] = gs;
    if (wc) c[j] = cs;
  }
  if (!wp && !wy) return;
  // p^ = kappa W r, y^ = conj(kappa) W s
  const double2 ck = cconj(kappa);
  for (int p = tid; p < N; p += nt) {
    double2 pv = make_double2(0, 0), yv = make_double2(0, 0);
    for (int q = 0; q < N; ++q) {
      double w = W[p * ld + q];
      if (wp) { pv.x = fma(w, at[q].x, pv.x); pv.y = fma(w, at[q].y, pv.y); }
      if (wy) { yv.x = fma(w, lt[q].x, yv.x); yv.y = fma(w, lt[q].y, yv.y); }
    }
    pv = cmul(kappa, pv);
    yv = cmul(ck, yv);
    unsigned char* pb = reinterpret_cast<unsigned char*>(p_hat) + (size_t)j * vstride;
    unsigned char* yb = reinterpret_cast<unsigned char*>(y_hat) + (size_t)j * vstride;
    if (mixed) {
      if (wp) reinterpret_cast<float2*>(pb)[p] = make_float2((float)pv.x, (float)pv.y);
      if (wy) reinterpret_cast<float2*>(yb)[p] = make_float2((float)yv.x, (float)yv.y);
    } else {
      if (wp) reinterpret_cast<double2*>(pb)[p] = pv;
      if (wy) reinterpret_cast<double2*>(yb)[p] = yv;
    }
  }
}

// GWS: storage in the global workspace (compile-time, so that the
// shared-memory instantiation keeps shared-memory loads)
template <bool GWS>
__global__ void k_pointwise(const double* __restrict__ Wg, const double2* __restrict__ Ptil,
                            const double2* __restrict__ Xp, const void* a_hat, const void* l_hat,
                            int mixed, int N, int J, double2 kappa, void* p_hat, void* y_hat,
                            size_t vstride, double* __restrict__ g, double* __restrict__ c,
                            int what, double2* __restrict__ rbuf, unsigned char* gws, size_t per_cta) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  unsigned char* base = GWS ? gws + (size_t)blockIdx.x * per_cta : smem_raw;
  for (int j = blockIdx.x; j < J; j += gridDim.x) {
    pointwise_step(Wg, Ptil, Xp, a_hat, l_hat, mixed, N, j, kappa, p_hat, y_hat, vstride, g, c,
                   what, rbuf, base);
    __syncthreads();
  }
}

// max_j | |a_j| - 1 |, j = 0..J, as a non-negative binary64 reduced with an
// integer atomicMax on its bit pattern (monotone for non-negative values);
// *drift must hold +0.0 before the launch.
__global__ void k_drift(const void* a_hat, int mixed, int N, int J, double* drift) {
  double d = 0.0;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int j = warp; j <= J; j += nwarps) {
    double n2 = 0;
    for (int p = lane; p < N; p += 32) {
      const double2 v = load_state(a_hat, mixed, (size_t)j * N + p);
      n2 += v.x * v.x + v.y * v.y;
    }
    n2 = warp_sum(n2);
    d = fmax(d, fabs(sqrt(n2) - 1.0));
  }
  if (lane == 0 && d > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(drift), (unsigned long long)__double_as_longlong(d));
}

cudaError_t launch_drift(const void* a_hat, int mixed, int N, int J, double* drift, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(drift, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  const int blocks = (J + 1 + 7) / 8 < 1024 ? (J + 1 + 7) / 8 : 1024;
  k_drift<<<blocks, 256, 0, st>>>(a_hat, mixed, N, J, drift);
  return cudaGetLastError();
}

size_t pointwise_step_bytes(int N) { return (size_t)N * (N + 1) * 8 + 4 * (size_t)N * 16 + 64 * 8; }

cudaError_t launch_pointwise(const double* W, const double2* Ptil, const double2* Xp,
                             const void* a_hat, const void* l_hat, int mixed, int N, int J,
                             double2 kappa, void* p_hat, void* y_hat, double* g, double* c,
                             int what, cudaStream_t st, const StepSpace& ws, double2* rbuf) {
  const int threads = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
  const size_t vstride = ((mixed ? 8 : 16) * (size_t)N + 15) / 16 * 16;
  StepGrid sg;
  if (!step_grid(pointwise_step_bytes(N), J, ws, (const void*)k_pointwise<false>, sg))
    return cudaErrorInvalidConfiguration;
  if (sg.gws)
    k_pointwise<true><<<sg.grid, threads, sg.smem, st>>>(W, Ptil, Xp, a_hat, l_hat, mixed, N, J, kappa,
                                                         p_hat, y_hat, vstride, g, c, what, rbuf,
                                                         sg.gws, sg.per_cta);
  else
    k_pointwise<false><<<sg.grid, threads, sg.smem, st>>>(W, Ptil, Xp, a_hat, l_hat, mixed, N, J, kappa,
                                                          p_hat, y_hat, vstride, g, c, what, rbuf,
                                                          sg.gws, sg.per_cta);
  return cudaGetLastError();
}

}  // namespace qoc
