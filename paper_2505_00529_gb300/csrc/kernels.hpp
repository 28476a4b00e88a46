// Internal launch interface between the C ABI (api.cu) and the kernels.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include <mutex>
#include <map>
#include <set>
#include <utility>

namespace qoc {

// Largest dynamic shared memory of a kernel on the current device (the opt-in
// limit minus its static shared memory), raised to that as the kernel's
// attribute once per (kernel, device).  Setting it per launch to the launch's
// own size would let a concurrent host thread lower it between another
// thread's set and launch.
inline size_t max_dyn_smem(const void* fn) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> done;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = done.find({fn, dev});
  if (it != done.end()) return it->second;
  int mx = 0;
  if (cudaDeviceGetAttribute(&mx, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) return 0;
  const int lim = mx - (int)fa.sharedSizeBytes;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, lim) != cudaSuccess) return 0;
  done[{fn, dev}] = (size_t)lim;
  return (size_t)lim;
}
inline cudaError_t set_max_smem(const void* fn) {
  return max_dyn_smem(fn) ? cudaSuccess : cudaErrorInvalidValue;
}

// Working storage of a per-step kernel whose matrices do not fit in shared
// memory (large N): a global workspace.  The launch then uses a persistent
// grid in which every CTA owns one slice and loops over the steps.
struct StepSpace {
  unsigned char* base = nullptr;
  size_t bytes = 0;
};
struct StepGrid {
  int grid = 0;
  size_t smem = 0;
  unsigned char* gws = nullptr;
  size_t per_cta = 0;
};
// streaming multiprocessors of the current device (cached)
inline int num_sms() {
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1)
      nsm = 1;
  }
  return nsm;
}
// `units` work units (steps or blocks), `need` bytes of storage each.
inline bool step_grid(size_t need, int units, const StepSpace& ws, const void* fn, StepGrid& g) {
  if (need <= max_dyn_smem(fn)) {
    g.grid = units; g.smem = need; g.gws = nullptr; g.per_cta = 0;
    return true;
  }
  if (!ws.base) return false;
  const size_t per = (need + 255) & ~size_t(255);
  size_t n = ws.bytes / per;
  if (n < 1) return false;
  // no more CTAs than keep the slices L2-resident (96 MB), but at least one per SM
  const int nsm = num_sms();
  size_t cap = (size_t)(96u << 20) / per;
  if (cap < (size_t)nsm) cap = (size_t)nsm;
  if (n > cap) n = cap;
  if (n > (size_t)units) n = (size_t)units;
  g.grid = (int)n; g.smem = 0; g.gws = ws.base; g.per_cta = per;
  return true;
}
// bytes per CTA that the per-step kernels ask of a workspace for this N (0 if all fit)
size_t step_workspace_per_cta(int N, int K, int bs_max, int mixed);

// Device status bits, OR-ed into a word the host reads after each evaluation.
enum : int {
  DEV_OK = 0,
  DEV_EIG_NOCONV = 1,   // Jacobi sweep cap reached
  DEV_TIMEOUT = 2,      // a bounded wait gave up
  DEV_NONFINITE = 4,    // a non-finite value was produced
  DEV_BADSHAPE = 8      // a kernel was launched with a shape it does not support
};

enum { EIG_REFINED = 0, EIG_JACOBI_FP64 = 1 };
enum { PREC_FP64 = 0, PREC_MIXED = 1 };

// second divided difference: dt*|hi - lo| at or below which the series is used
constexpr double TAU_DD2 = 1e-3;

// stats (optional, device): [0] += refinement updates, [1] += steps whose clean-up rotated,
// [2] += steps that took the final residual pass (no early finish)
// method EIG_REFINED: binary32 Jacobi, `refine_sweeps` binary64 Ogita-Aishima
// sweeps, then binary64 Jacobi clean-up rotating only angles above angle_tol.
// finish_tol > 0: the refinement ends after the first update with no cluster
// pairs whose |I - W^T W|_F and largest correction are <= finish_tol (W then
// accurate to about finish_tol^2); 0: refinement to the binary64 floor.
// the parts of a refined eigendecomposition a launch_eig call enqueues: the
// binary32 start, the binary64 refinement (which reads the start from W), or
// both; the refinement of steps [j0, j1) alone takes f + j0, W + j0 N^2,
// eig + j0 N and J = j1 - j0.  order (optional, device, J + 2 ints): with
// both phases in one call, the binary32 start may write a step order for the
// refinement into it (near-degenerate steps first)
enum { EIG_PHASE_START = 1, EIG_PHASE_REFINE = 2, EIG_PHASE_ALL = 3 };
cudaError_t launch_eig(const double* H0, const double* M, const double* f, int N, int J,
                       double* W, double* eig, int* status, int method, int refine_sweeps,
                       double angle_tol, cudaStream_t st, const StepSpace& ws,
                       cudaEvent_t mid = nullptr, unsigned int* stats = nullptr,
                       double finish_tol = 0.0, int phases = EIG_PHASE_ALL, int* order = nullptr);
size_t eig_step_bytes(int N);   // largest per-matrix storage of the eigensolver kernels
// binary32 Jacobi start for N = 32 exactly, the matrix in registers (one warp
// per step); rounds_per_body 4, 8 or 31 (the unrolled loop body).  order
// (optional, device, J + 2 ints): receives a permutation of the steps with the
// near-degenerate ones first ([J], [J + 1] are its counters, zeroed here)
cudaError_t launch_eig_jacobi32_reg(const double* H0, const double* M, const double* f, int J,
                                    double* W, double* eig, int* status, int rounds_per_body,
                                    int* order, cudaStream_t st);

size_t prep_smem_bytes(int N);
// parts (bit mask): 1 -> D_j = W diag(exp(-i dt (lambda - m)) - 1) W^T
// (binary64 when d_fp64, else binary32) at byte stride dstride;
// 2 -> P~_j = Gamma1 o M~_j and X'_j = 2 sum_r M~_pr M~_rq phi[l_p, l_r, l_q].
// parts: PREP_D (increments D_j), PREP_P (M~, P~ = Gamma1 o M~; M~ stored in Mtil when
// non-null), PREP_X (X'; alone it reads M~ and P~ back from Mtil and Ptil)
enum { PREP_D = 1, PREP_P = 2, PREP_X = 4 };
cudaError_t launch_prep(const double* W, const double* eig, const double* M, int N, int J,
                        double dt, double mshift, void* D, size_t dstride, int d_fp64,
                        int parts, double2* Ptil, double2* Xp, double* Mtil, int* status,
                        cudaStream_t st, const StepSpace& ws);

struct SweepArgs {
  int N, K, Kp, J;       // Kp: row stride of the basis copy (multiple of 4)
  int kc;                // columns per CTA
  int backward;          // 0: X <- X + D X + src b^T ; 1: X <- X + conj(D) X + src b^T, j descending
  const unsigned char* D;
  size_t dstride;        // bytes per step of D (multiple of 16)
  // element types: binary64 sweeps use double2 vectors / double basis rows;
  // mixed sweeps use float2 / float.
  const void* src;       // J x N source vectors (null: none)
  const void* ctr;       // J x N contraction vectors (null: none)
  const void* Brow;      // J x Kp basis rows (null: b = 1 for the single column)
  const double2* init;   // [K][N] initial state, or null for zero
  double init_scale;
  double2* final_out;    // [K][N] final state (may be null)
  void* states;          // (J+1) x N states of column 0 (double2, or float4 hi/lo pairs), or null
  void* contr;           // J x K contraction output (u or v): double, or float when mixed; or null
  int* status;
};
cudaError_t launch_sweep(const SweepArgs& a, int d_fp64, cudaStream_t st);

// ---- time blocking (block.cu, blocked sweep in sweep.cu) ----
struct BSweepArgs {
  int N, K, Kp, J;
  int bs;                // time steps per block
  int kc;                // columns per CTA
  int backward;          // sweep order: j descending (B rows of a block reversed)
  const unsigned char* M;   // per block [N][N] (M[q][i] = Delta[i][q]), stride mstride bytes
  size_t mstride;
  const unsigned char* Q;   // per block [bs][N] propagated sources, stride qstride bytes (or null)
  size_t qstride;
  const void* Brow;      // J x Kp basis rows (double, or float when mixed), or null
  const double2* init;   // [K][N] initial state or null
  double init_scale;
  double2* final_out;    // [K][N] final state or null
  void* Xblk;            // [nblk][K][N] block-start states (C, or float4 pairs when xblk_pairs)
  int xblk_pairs;
  void* states;          // vector chains: final state row (J forward, 0 backward), or null
  int* status;
  // Block range [blk0, blk1) of this launch (blk1 = 0: to the last block);
  // final_out and states are written only by the launch that ends at the last
  // block.  resume != 0: start from the block-start state Xblk[blk0] (exact:
  // binary64 states, or binary32 pairs with xblk_pairs) instead of init; a
  // launch that stops before the last block leaves its end state in
  // Xblk[blk1] for the next one.
  int blk0, blk1;
  int resume;
};
cudaError_t launch_bsweep(const BSweepArgs& a, int mixed, cudaStream_t st);
// which sweep kernel launch_bsweep takes for `a`: 0 the general one, 1 or 2
// a warp-specialised binary32 one (N <= 32 / N <= 64, CTA within its thread
// cap); kernels differ in the order of their sums
int bsweep_variant(const BSweepArgs& a, int mixed);
constexpr int kSweepVariants = 3;
// one launch for many problems: CTAs cta_off[p] .. cta_off[p+1]-1 run problem p
cudaError_t launch_bsweep_batch(const BSweepArgs* host_args, const BSweepArgs* dev_args,
                                const int* dev_cta_off, int nprob, int total_ctas, int mixed,
                                cudaStream_t st);
cudaError_t launch_block_delta(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                               int mixed, void* M, size_t mstride, cudaStream_t st,
                               const StepSpace& ws);
size_t block_delta_bytes(int N, int mixed);
size_t block_src_bytes(int N, int bsteps, int mixed);
// what: BS_Q (propagated sources Q, from src only), BS_WG (W and Gamma, needs ctr)
enum { BS_Q = 1, BS_WG = 2 };
cudaError_t launch_block_src(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                             int mixed, const void* src, const void* ctr, size_t vstride, void* Q,
                             void* W, void* G, size_t qstride, size_t gstride, int what,
                             cudaStream_t st, const StepSpace& ws);
cudaError_t launch_block_contract(const void* Xblk, const void* W, const void* G, size_t qstride,
                                  size_t gstride, const void* Brow, int Kp, int N, int K, int J,
                                  int bsteps, int bwd, int mixed, void* contr, cudaStream_t st);
cudaError_t launch_block_fill(const void* D, size_t dstride, int N, int J, int bsteps, int bwd,
                              int mixed, const void* Xblk, void* states, cudaStream_t st);

// p^_j, y^_j, g_j, c_j for all steps from the stored states/costates
// states / costates as written by the vector chains (double2, or float4 pairs
// when mixed); p^, y^ written as double2 (binary64 sweeps) or float2 (mixed)
// what: PW_P (p^ from a^), PW_Y (y^ and g from lambda^ and a^), PW_C (c from X', a^, lambda^);
// with r (J x N): PW_P also stores r_j = P~ a~_j there, and PW_Y | PW_RUSE
// takes g's r_j from it instead of forming a~_j and r_j again (same values)
enum { PW_P = 1, PW_Y = 2, PW_C = 4, PW_RUSE = 8 };
cudaError_t launch_pointwise(const double* W, const double2* Ptil, const double2* Xp,
                             const void* a_hat, const void* l_hat, int mixed, int N, int J,
                             double2 kappa, void* p_hat, void* y_hat, double* g, double* c,
                             int what, cudaStream_t st, const StepSpace& ws, double2* r = nullptr);
size_t pointwise_step_bytes(int N);
// max_j | |a_j| - 1 | over the stored states j = 0..J into *drift (zeroed here)
cudaError_t launch_drift(const void* a_hat, int mixed, int N, int J, double* drift, cudaStream_t st);

cudaError_t launch_control(const double* B, int Kp, const double* theta, int J, int K, double* f,
                           cudaStream_t st);
// lambda^_J = 2 w_t (a^_J - e^{i theta_J} beta); J value; norm drift; returns into out
cudaError_t launch_terminal(const double* f, int J, const void* a_hat, int mixed,
                            const double2* beta, int N, double2 phaseJ, double w_f, double w_t,
                            double2* lamJ, double* cost_out, double* drift_out, cudaStream_t st);
// grad = B^T (2 w_f f + g); Hess (see qoc.h) into out = [J, grad, Hess], raw Hessian, asymmetry
// V, U: J x K contractions, double (uv_f32 = 0) or float (uv_f32 = 1)
// identity != 0: B = I (K = J), the maximal model -- same results without the
// contraction over j
cudaError_t launch_assemble(const double* B, int Kp, const double* f, const double* g,
                            const double* c, const void* V, const void* U, int uv_f32,
                            const double2* SJ, int N, int J, int K, double w_f, double w_t,
                            int method, int want_hess, double* work, double* out,
                            double* hess_raw, double* asym, cudaStream_t st, int identity = 0);
size_t assemble_work_doubles(int J, int K);

// trust-region subproblem on the device (K x K, binary64).  K < kTriMin: from
// the Hessian's eigendecomposition, expected in work as [gt (K) | st (K) |
// eigenvalues d (K) | eigenvectors Q (K*K)]; K >= kTriMin: from the Hessian in
// out_gh itself by tridiagonal reduction (no eigendecomposition needed;
// work then holds that method's 8K + K*K scratch)
constexpr int kTriMin = 48;
__host__ __device__ inline bool tr_needs_eig(int K) { return K < kTriMin; }
size_t tr_work_doubles(int K);
cudaError_t launch_axpy(const double* x, const double* s, int K, double* y, cudaStream_t st);
// method: 0 by K, 1 eigendecomposition (expected in work), 2 tridiagonal reduction
cudaError_t launch_tr_subproblem(const double* out_gh, int K, double radius, double* work,
                                 double* step, double* info, int* status, cudaStream_t st,
                                 int method = 0);

// BFGS update of the K x K model Hessian B from the step s and the gradients
// (state[0]: 0 until the first update with positive curvature scales B, then 1);
// scratch: K doubles
cudaError_t launch_bfgs_update(double* B, const double* s, const double* g_old, const double* g_new, int K,
                               double* state, double min_curv, double* scratch, cudaStream_t st);
cudaError_t launch_set_identity(double* B, int K, cudaStream_t st);
// one CTA waits (bounded, limit_ns) on an mbarrier that nothing completes and
// raises DEV_TIMEOUT in *status when it gives up
cudaError_t launch_wait_selftest(int* status, unsigned long long limit_ns, cudaStream_t st);

// one problem of a batched trust-region solve (device array, one CTA each)
struct TrSlot {
  int K;
  double* gh;               // [J, grad, Hess] at theta (1 + K + K*K)
  double* work;             // tr_work_doubles(K): [gt | st | d | Q] of the current Hessian
  double* step;             // K
  double* info;             // [pred, |s|, sigma, |g|]
  double* theta;            // K: current point
  double* theta_trial;      // K: trial point (the batched evaluation reads it)
  const double* gh_trial;   // [J, grad, Hess] at the trial point
  const double* eig_trial;  // [d (K) | Q (K*K)] of the trial Hessian
  int* status;              // the problem's device status word (read and cleared)
  double radius;
  int active, stop, iters, n_eval_J, n_eval_gh, fail;
};
struct TrBatchOptions {
  double gtol, xtol, radius0, radius_max, eta;
  int max_iter;
  int kmax = 0;          // largest K among the problems (sizes the subproblem's shared memory)
};
// phase 0: take the evaluated initial point; 1: propose (gtol test,
// subproblem, trial point); 2: update (ratio test, radius, acceptance, xtol
// and iteration cap) -- iteration `it`
cudaError_t launch_tr_batch(int phase, TrSlot* slots, int n, int it, const TrBatchOptions& o,
                            cudaStream_t st);

// set the text qoc_last_error() returns on this thread
void note_error(const char* msg);

}  // namespace qoc
