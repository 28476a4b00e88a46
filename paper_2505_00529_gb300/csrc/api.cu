// C ABI of the library (see include/qoc.h): problem objects, device memory,
// the evaluation pipeline of Alg. 2 and the trust-region driver.
//
// One evaluation at theta enqueues, on the problem's stream:
//   control       f = B theta
//   eig           H_j = W_j diag(lambda_j) W_j^T for all j          (parallel over j)
//   prep          D_j, P~_j = Gamma1 o M~_j, X'_j                    (parallel over j)
//   state chain   a_0 .. a_J                                         (sequential)
//   terminal      J, lambda_J = 2 w_t (a_J - beta)
//   costate chain lambda_J .. lambda_0                               (sequential)
//   pointwise     p_j, y_j, g_j, c_j                                 (parallel over j)
//   tangent panel S_0 .. S_J with u_j = Re(y_j^H S_j)                (sequential, K-parallel)
//   mu panel      mu_J .. mu_0 with v_j = Re(mu_{j+1}^H p_j)         (sequential, K-parallel)
//   assembly      grad, Hess
// The host synchronises only when results go back to host memory.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.hpp"
#include "qoc.h"

using namespace qoc;

namespace {
constexpr int kMaxN = 256;      // largest basis (above 64 the per-step kernels use a global workspace)
constexpr int kMaxK = 4096;
constexpr int kMaxKTR = 256;    // trust region: K x K Hessian eigensolver
}  // namespace

struct qoc_problem {
  int N = 0, K = 0, J = 0, Kp = 0;
  double dt = 0, w_f = 0, w_t = 0, mshift = 0;
  int precision = 0, hess_method = QOC_HESS_SECOND_ORDER_ADJOINT, eig_method = QOC_EIG_REFINED;
  int requested_precision = 0;          // as passed to qoc_create_problem
  int identity_basis = 0;               // B = I (the maximal model): assembly without the j-sums
  double err_sigma = 0;                 // sigma of the binary32 error estimate (see qoc.h)
  int refine_sweeps = 2;
  double angle_tol = 1e-13;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  cudaStream_t side = nullptr;          // high-priority stream: the latency-bound chains run here
                                        // while the binary64 derivative preparation fills the GPU
  cudaStream_t pstream = nullptr;       // high-priority stream of the panel sweeps
  cudaEvent_t fork = nullptr, join = nullptr;
  cudaEvent_t ev_state = nullptr, ev_ptil = nullptr, ev_panels = nullptr;
  cudaEvent_t ev_bprod = nullptr;       // backward block products done (panel stream)
  cudaEvent_t ev_fprod = nullptr;       // forward block products done (panel stream)
  cudaEvent_t ev_yhat = nullptr;        // y^ and g done (chain stream)
  cudaEvent_t ev_phat = nullptr;        // p^ (and r_j) done (panel stream)
  cudaEvent_t ev_tangent = nullptr;     // tangent panel swept (panel stream)
  cudaEvent_t ev_musrc = nullptr;       // second-order sources done (chain stream, unsplit adjoint)
  int timing = 0;
  int sched = 0;                        // 0 sequential, 1 three-stream (time-blocked, order >= 1)
  // forward pipeline: the refinement and increments in chunks of steps, the
  // state chain following chunk by chunk on the chain stream
  static constexpr int kMaxChunks = 8;
  int pipeline = -1;                    // chunks (qoc_set_pipeline); -1 the built-in choice
  int piped = 0;                        // chunks of the last evaluation (0: not pipelined)
  // the next time-blocked evaluation with gradients is at the theta of the
  // evaluation just enqueued, whose samples f, eigendecompositions,
  // increments, forward block products and state chain it reuses (set by the
  // trust region after an accepted step; consumed by that evaluation)
  int reuse_fwd = 0;
  int fwd_reused = 0;                   // the last evaluation did
  cudaEvent_t ev_chunk[kMaxChunks] = {};
  cudaEvent_t evp[2 * kMaxChunks] = {}; // timing mode: after each chunk's refinement / increments
  cudaEvent_t trev[4] = {};             // timing mode: around a trust-region iteration's phases
  double trphase_ms[3] = {0, 0, 0};     // last solve: subproblem, cost evaluations, grad + Hess evaluations
  cudaEvent_t ev[14] = {};
  double phase_ms[6] = {0, 0, 0, 0, 0, 0};
  double kphase_ms[QOC_N_PHASES] = {};
  double diag[2] = {0, 0};
  int last_order = -1;
  size_t dstride = 0, vstride = 0, dev_bytes = 0;
  std::vector<void*> allocs;
  // device buffers
  double *H0 = nullptr, *M = nullptr, *B = nullptr, *theta = nullptr, *theta_trial = nullptr;
  float* Bf = nullptr;
  double *f = nullptr, *W = nullptr, *eig = nullptr, *g = nullptr, *c = nullptr;
  double *V = nullptr, *U = nullptr, *work = nullptr, *out = nullptr, *out_trial = nullptr;
  double *hess_raw = nullptr, *scal = nullptr;
  unsigned int* eigstats = nullptr;     // refinement counters (timing mode)
  int* eigorder = nullptr;              // J + 2 ints: the refinement's step order and its counters
  // second-order adjoint on the three-stream schedule: the mu sweep starts
  // from zero and the terminal part of its contraction, 2 w_t Re(S_J^H S_J),
  // is added in the assembly (1), or the sweep starts from mu_J = 2 w_t S_J
  // (0); -1: 1 for binary64 sweeps, 0 for binary32 ones
  int mu_split = -1;
  double2 *alpha = nullptr, *beta = nullptr, *Ptil = nullptr, *Xp = nullptr, *SJ = nullptr,
          *lamJ = nullptr;
  double* Mtil = nullptr;               // M~_j = W_j^T M W_j (three-stream schedule)
  StepSpace ws[3];                      // per-step storage beyond shared memory, one region per
                                        // stream (main, chains, panels); empty for N <= 64
  void *D = nullptr, *a_hat = nullptr, *l_hat = nullptr, *p_hat = nullptr, *y_hat = nullptr;
  double2* rvec = nullptr;              // r_j = P~ a~_j (J x N), from p^ for g
  int* status = nullptr;
  double *trwork = nullptr, *trstep = nullptr, *trinfo = nullptr, *trzero = nullptr;
  // time blocking (bs steps per block; bs == 1: per-step sweeps)
  int bs = 8, nblk = 0;
  int kc = 0;                           // panel columns per CTA (0: built-in choice)
  size_t mstride = 0, qstride = 0, gstride = 0;
  void *Mf = nullptr, *Mb = nullptr, *Qf = nullptr, *Wf = nullptr, *Gf = nullptr, *Qb = nullptr,
       *Wb = nullptr, *Gb = nullptr, *Xa = nullptr, *Xl = nullptr, *XS = nullptr, *Xmu = nullptr;
  // pinned host staging
  double* hbuf = nullptr;
  size_t hbuf_len = 0;
  int* hstatus = nullptr;
};

namespace {

thread_local char g_last_error[256] = "";

qoc_status from_cuda(cudaError_t e, int line = 0) {
  if (e == cudaSuccess) return QOC_OK;
  std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s (api.cu:%d)", cudaGetErrorName(e),
                cudaGetErrorString(e), line);
  if (e == cudaErrorMemoryAllocation) return QOC_ENOMEM;
  if (e == cudaErrorInvalidConfiguration) return QOC_EUNSUPPORTED;
  return QOC_ECUDA;
}

#define QOC_TRY(expr)                         \
  do {                                        \
    cudaError_t e_ = (expr);                  \
    if (e_ != cudaSuccess) return from_cuda(e_, __LINE__); \
  } while (0)

template <typename T>
cudaError_t dalloc(qoc_problem* p, T** ptr, size_t bytes) {
  void* v = nullptr;
  bytes = (bytes + 255) & ~size_t(255);
  cudaError_t e = cudaMalloc(&v, bytes);
  if (e != cudaSuccess) return e;
  p->allocs.push_back(v);
  p->dev_bytes += bytes;
  *ptr = reinterpret_cast<T*>(v);
  return cudaSuccess;
}

bool finite_all(const double* x, size_t n) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(x[i])) return false;
  return true;
}

bool symmetric(const double* A, int N) {
  double nrm = 0;
  for (int i = 0; i < N * N; ++i) nrm = std::fmax(nrm, std::fabs(A[i]));
  for (int i = 0; i < N; ++i)
    for (int k = i + 1; k < N; ++k)
      if (std::fabs(A[i * N + k] - A[k * N + i]) > 1e-12 * std::fmax(nrm, 1e-300)) return false;
  return true;
}

double2 cexpi_h(double x) { return make_double2(std::cos(x), std::sin(x)); }

// Rms spread of the spectra of H_j - m for theta ~ N(0, I):
// sigma^2 = (|H0 - m I|_F^2 + |M|_F^2 mean_j |b_j|^2) / N  (see qoc_precision in qoc.h)
double spectral_sigma(int N, const double* H0, const double* M, const double* basis, int K, int J,
                      double m) {
  double a = 0, c = 0, s2 = 0;
  for (int i = 0; i < N; ++i)
    for (int k = 0; k < N; ++k) {
      const double h = H0[i * N + k] - (i == k ? m : 0.0);
      a += h * h;
      c += M[i * N + k] * M[i * N + k];
    }
  for (size_t e = 0; e < (size_t)J * K; ++e) s2 += basis[e] * basis[e];
  s2 /= (double)J;
  return std::sqrt((a + c * s2) / N);
}

// estimated relative error of binary32 increments at block length bs
constexpr double kMixedTarget = 1e-6;
double mixed_error_estimate(const qoc_problem* p, int bs) {
  return 0.3 * 5.9604644775390625e-8 * p->dt * p->err_sigma *
         std::sqrt((double)p->J * (double)p->N * (double)(bs < 1 ? 1 : bs));
}

// Relaxed finish of the eigenvector refinement for binary32 sweeps: their
// results need the eigendecomposition's residual only to ~1e-9 |H| (binary32
// increments round at 6e-8), which the first binary64 Ogita-Aishima update
// from the binary32 Jacobi start reaches on most steps (orthogonality defect
// <= 3e-5, whose square is what the update leaves); binary64 sweeps refine
// to the binary64 floor.
// relaxed refinement finish for problems on binary32 sweeps: |I - W^T W|_F at
// most 3e-5 before the finishing update.  A looser 1e-4, which would end
// most steps after one update, measured a 1.6e-6 mixed Hessian error on an
// avoided crossing (N = 48, J = 4000): the orthogonality left behind
// accumulates over the steps.
double eig_finish_tol(const qoc_problem* p) { return p->precision == QOC_MIXED_FP32 ? 3e-5 : 0.0; }

// panel columns per CTA: one by default, which spreads a panel over K SMs
// (binary64 is throughput-limited per SM; the binary32 sweep is latency-bound
// per dependent step, which more columns per CTA only lengthen)
int sweep_kc(const qoc_problem* p) {
  return p->kc > 0 ? p->kc : 1;
}

qoc_status device_status(qoc_problem* p) {
  int s = *p->hstatus;
  *p->hstatus = 0;
  if (s == 0) return QOC_OK;
  std::snprintf(g_last_error, sizeof(g_last_error),
                "device status 0x%x (1: eigensolver not converged, 2: bounded wait gave up, "
                "4: non-finite value, 8: unsupported shape)", s);
  if (s & DEV_TIMEOUT) return QOC_ETIMEOUT;
  if (s & DEV_BADSHAPE) return QOC_EUNSUPPORTED;
  return QOC_ENUMERIC;
}

// The time-blocked evaluation (see block.cu): everything after the spectral
// preparation, with the sequential sweeps taking J / bs dependent steps.
BSweepArgs chain_sweep_args(qoc_problem* p, int bwd) {
  BSweepArgs a{};
  const int mixed = p->precision == QOC_MIXED_FP32;
  a.N = p->N; a.K = 1; a.Kp = p->Kp; a.J = p->J; a.bs = p->bs; a.kc = 1; a.backward = bwd;
  a.M = reinterpret_cast<const unsigned char*>(bwd ? p->Mb : p->Mf); a.mstride = p->mstride;
  a.init = bwd ? p->lamJ : p->alpha; a.init_scale = 1.0;
  a.Xblk = bwd ? p->Xl : p->Xa; a.xblk_pairs = mixed;
  a.states = bwd ? p->l_hat : p->a_hat; a.status = p->status;
  return a;
}

// Whether the second-order adjoint's terminal part is split off (qoc_set_mu_split).
// Built-in choice: binary64 sweeps only.  With binary32 sweeps the split costs
// accuracy where the Hessian is a small difference of large terms: mu0 can be
// larger than mu (the source and terminal parts partly cancel), and the
// binary32 sweep's rounding scales with it.  Measured on the avoided crossing
// of the batched workload (N = 48, K = 32, J = 4000, |B^T V| ~ 600 against
// |H| ~ 50): Hessian error 7.6e-7 unsplit, 1.22e-6 split (target 1e-6); the
// bench problem (N = 32, K = 64, J = 4000) went 2.91 -> 2.73 ms.
bool mu_split_on(const qoc_problem* p) {
  if (p->hess_method != QOC_HESS_SECOND_ORDER_ADJOINT) return false;
  return p->mu_split < 0 ? p->precision != QOC_MIXED_FP32 : p->mu_split != 0;
}

BSweepArgs panel_sweep_args(qoc_problem* p, int bwd, bool mu_split = false) {
  BSweepArgs s{};
  const int mixed = p->precision == QOC_MIXED_FP32;
  s.N = p->N; s.K = p->K; s.Kp = p->Kp; s.J = p->J; s.bs = p->bs; s.kc = sweep_kc(p); s.backward = bwd;
  s.M = reinterpret_cast<const unsigned char*>(bwd ? p->Mb : p->Mf); s.mstride = p->mstride;
  s.Q = reinterpret_cast<const unsigned char*>(bwd ? p->Qb : p->Qf); s.qstride = p->qstride;
  s.Brow = mixed ? static_cast<const void*>(p->Bf) : static_cast<const void*>(p->B);
  s.status = p->status;
  if (bwd) {
    s.init = mu_split ? nullptr : p->SJ; s.init_scale = 2.0 * p->w_t; s.Xblk = p->Xmu;
  } else {
    s.final_out = p->SJ; s.Xblk = p->XS;
  }
  return s;
}


// Time-blocked evaluation on three streams (order >= 1):
//   main: derivative preparation P~ (then X' for the Hessian); after the
//       costate: pointwise c_j, drift, the forward contraction (W, Gamma,
//       U); assembly
//   chains (high priority): state chain (after the forward block products)
//       + fill, terminal; costate chain (after the backward ones) + fill;
//       order 2, after the costate and p^: y^, g -> second-order adjoint
//       sources (and, split, its sweep and contraction V)
//   panels (high priority): forward, then backward block products at the
//       fork; order 2, as soon as the state and P~ exist: p^ -> propagated
//       sources -> tangent panel sweep; unsplit, then the second-order
//       adjoint sweep (its sources ready beside the tangent sweep) ->
//       contraction V
// so that the latency-bound sweeps overlap the binary64 X' preparation and
// each other instead of following them, and the chain state -> costate ->
// second-order adjoint carries nothing it does not need.
qoc_status enqueue_blocked(qoc_problem* p, int order, double* out_dev) {
  cudaStream_t st = p->stream;
  const int N = p->N, K = p->K, J = p->J, bs = p->bs;
  const int mixed = p->precision == QOC_MIXED_FP32 ? 1 : 0;
  const double thetaJ = (double)J * p->dt * p->mshift;
  const double2 kappa = cexpi_h(p->dt * p->mshift);
  const bool soa = p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT;
  const void* Bsrc = mixed ? static_cast<const void*>(p->Bf) : static_cast<const void*>(p->B);
  if (order == 0) {
    p->sched = 0;
    if (p->piped) {   // the chain ran chunk by chunk on the chain stream
      QOC_TRY(cudaEventRecord(p->join, p->side));
      QOC_TRY(cudaStreamWaitEvent(st, p->join, 0));
    } else {
      QOC_TRY(launch_block_delta(p->D, p->dstride, N, J, bs, 0, mixed, p->Mf, p->mstride, st, p->ws[0]));
      QOC_TRY(launch_bsweep(chain_sweep_args(p, 0), mixed, st));
    }
    QOC_TRY(launch_block_fill(p->D, p->dstride, N, J, bs, 0, mixed, p->Xa, p->a_hat, st));
    QOC_TRY(launch_terminal(p->f, J, p->a_hat, mixed, p->beta, N, cexpi_h(thetaJ), p->w_f, p->w_t,
                            p->lamJ, p->scal + 0, nullptr, st));
    QOC_TRY(launch_drift(p->a_hat, mixed, N, J, p->scal + 1, st));
    QOC_TRY(cudaMemcpyAsync(out_dev, p->scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (p->timing) for (int k : {9, 3, 4, 5, 6}) cudaEventRecord(p->ev[k], st);
    return QOC_OK;
  }
  p->sched = 1;
  cudaStream_t cs = p->side, ps = p->pstream;
  // The block products depend on the increments only: both run on the panel
  // stream at the fork, the forward ones first, so that the state chain
  // waits for them alone and the costate chain finds its products done;
  // neither sits on the chain stream, and the derivative preparation on the
  // main stream starts at the fork.
  const bool fwd_here = !p->piped && !p->fwd_reused;   // else chunked behind the refinement, or reused
  QOC_TRY(cudaEventRecord(p->fork, st));
  QOC_TRY(cudaStreamWaitEvent(ps, p->fork, 0));
  if (fwd_here) {
    QOC_TRY(launch_block_delta(p->D, p->dstride, N, J, bs, 0, mixed, p->Mf, p->mstride, ps, p->ws[2]));
    QOC_TRY(cudaEventRecord(p->ev_fprod, ps));
  }
  QOC_TRY(launch_block_delta(p->D, p->dstride, N, J, bs, 1, mixed, p->Mb, p->mstride, ps, p->ws[2]));
  QOC_TRY(cudaEventRecord(p->ev_bprod, ps));
  // ---- chains ----
  QOC_TRY(cudaStreamWaitEvent(cs, p->fork, 0));
  if (p->timing) cudaEventRecord(p->ev[10], cs);
  if (fwd_here) {
    QOC_TRY(cudaStreamWaitEvent(cs, p->ev_fprod, 0));
    QOC_TRY(launch_bsweep(chain_sweep_args(p, 0), mixed, cs));
  }
  QOC_TRY(launch_block_fill(p->D, p->dstride, N, J, bs, 0, mixed, p->Xa, p->a_hat, cs));
  QOC_TRY(launch_terminal(p->f, J, p->a_hat, mixed, p->beta, N, cexpi_h(thetaJ), p->w_f, p->w_t,
                          p->lamJ, p->scal + 0, nullptr, cs));
  QOC_TRY(cudaMemcpyAsync(out_dev, p->scal, sizeof(double), cudaMemcpyDeviceToDevice, cs));
  QOC_TRY(cudaEventRecord(p->ev_state, cs));
  QOC_TRY(cudaStreamWaitEvent(cs, p->ev_bprod, 0));
  QOC_TRY(launch_bsweep(chain_sweep_args(p, 1), mixed, cs));
  QOC_TRY(launch_block_fill(p->D, p->dstride, N, J, bs, 1, mixed, p->Xl, p->l_hat, cs));
  if (p->timing) cudaEventRecord(p->ev[11], cs);
  QOC_TRY(cudaEventRecord(p->join, cs));
  // ---- main: P~ ----
  QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, mixed ? 0 : 1,
                      PREP_P, p->Ptil, p->Xp, p->Mtil, p->status, st, p->ws[0]));
  QOC_TRY(cudaEventRecord(p->ev_ptil, st));
  const bool split = order >= 2 && soa && mu_split_on(p);
  if (order >= 2 && split) {
    // ---- panels, split second-order adjoint ----
    // The mu sweep starts from zero, so it needs the costate and y^ but not
    // the tangent panel: the tangent sweep runs on the panel stream while the
    // chain stream, after the costate, goes on to y^ and the mu sweep.
    QOC_TRY(cudaStreamWaitEvent(ps, p->ev_ptil, 0));
    QOC_TRY(cudaStreamWaitEvent(ps, p->ev_state, 0));
    if (p->timing) cudaEventRecord(p->ev[12], ps);
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_P, ps, p->ws[2], p->rvec));
    QOC_TRY(cudaEventRecord(p->ev_phat, ps));
    QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 0, mixed, p->p_hat, p->y_hat, p->vstride,
                             p->Qf, p->Wf, p->Gf, p->qstride, p->gstride, BS_Q, ps, p->ws[2]));
    QOC_TRY(launch_bsweep(panel_sweep_args(p, 0), mixed, ps));
    QOC_TRY(cudaEventRecord(p->ev_tangent, ps));
    // chain stream: y^ (r_j from the p^ pass), the mu sources, sweep and V
    QOC_TRY(cudaStreamWaitEvent(cs, p->ev_phat, 0));
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_Y | PW_RUSE, cs, p->ws[1], p->rvec));
    QOC_TRY(cudaEventRecord(p->ev_yhat, cs));
    QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 1, mixed, p->y_hat, p->p_hat, p->vstride,
                             p->Qb, p->Wb, p->Gb, p->qstride, p->gstride, BS_Q | BS_WG, cs, p->ws[1]));
    QOC_TRY(launch_bsweep(panel_sweep_args(p, 1, true), mixed, cs));
    QOC_TRY(launch_block_contract(p->Xmu, p->Wb, p->Gb, p->qstride, p->gstride, Bsrc, p->Kp, N, K,
                                  J, bs, 1, mixed, p->V, cs));
    if (p->timing) cudaEventRecord(p->ev[13], cs);
    QOC_TRY(cudaEventRecord(p->ev_panels, cs));
    // ---- main: X', c_j, the forward contraction ----
    QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, mixed ? 0 : 1,
                        PREP_X, p->Ptil, p->Xp, p->Mtil, p->status, st, p->ws[0]));
    if (p->timing) cudaEventRecord(p->ev[3], st);
    QOC_TRY(cudaStreamWaitEvent(st, p->join, 0));
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_C, st, p->ws[0]));
    QOC_TRY(launch_drift(p->a_hat, mixed, N, J, p->scal + 1, st));
    if (p->timing) cudaEventRecord(p->ev[4], st);
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_yhat, 0));
    QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 0, mixed, p->p_hat, p->y_hat, p->vstride,
                             p->Qf, p->Wf, p->Gf, p->qstride, p->gstride, BS_WG, st, p->ws[0]));
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_tangent, 0));
    QOC_TRY(launch_block_contract(p->XS, p->Wf, p->Gf, p->qstride, p->gstride, Bsrc, p->Kp, N, K, J,
                                  bs, 0, mixed, p->U, st));
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_panels, 0));
  } else if (order >= 2) {
    // ---- panels ----
    QOC_TRY(cudaStreamWaitEvent(ps, p->ev_ptil, 0));
    QOC_TRY(cudaStreamWaitEvent(ps, p->ev_state, 0));
    if (p->timing) cudaEventRecord(p->ev[12], ps);
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_P, ps, p->ws[2], p->rvec));
    QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 0, mixed, p->p_hat, p->y_hat, p->vstride,
                             p->Qf, p->Wf, p->Gf, p->qstride, p->gstride, BS_Q, ps, p->ws[2]));
    QOC_TRY(cudaEventRecord(p->ev_phat, ps));
    QOC_TRY(launch_bsweep(panel_sweep_args(p, 0), mixed, ps));
    QOC_TRY(cudaEventRecord(p->ev_tangent, ps));
    // y^, g and the second-order sources need the costate and p^ but not the
    // tangent panel: the chain stream takes them after the costate, beside
    // the tangent sweep, and the mu sweep follows the tangent sweep directly
    QOC_TRY(cudaStreamWaitEvent(cs, p->ev_phat, 0));
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_Y | PW_RUSE, cs, p->ws[1], p->rvec));
    // the forward contraction (W, Gamma and U) is not on the way to the
    // second-order adjoint sweep: the main stream takes it, beside that sweep
    QOC_TRY(cudaEventRecord(p->ev_yhat, cs));
    if (soa) {
      QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 1, mixed, p->y_hat, p->p_hat, p->vstride,
                               p->Qb, p->Wb, p->Gb, p->qstride, p->gstride, BS_Q | BS_WG, cs, p->ws[1]));
      QOC_TRY(cudaEventRecord(p->ev_musrc, cs));
      QOC_TRY(cudaStreamWaitEvent(ps, p->ev_musrc, 0));
      QOC_TRY(launch_bsweep(panel_sweep_args(p, 1), mixed, ps));
      QOC_TRY(launch_block_contract(p->Xmu, p->Wb, p->Gb, p->qstride, p->gstride, Bsrc, p->Kp, N, K,
                                    J, bs, 1, mixed, p->V, ps));
    }
    if (p->timing) cudaEventRecord(p->ev[13], ps);
    QOC_TRY(cudaEventRecord(p->ev_panels, ps));
    // ---- main: X', c_j ----
    QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, mixed ? 0 : 1,
                        PREP_X, p->Ptil, p->Xp, p->Mtil, p->status, st, p->ws[0]));
    if (p->timing) cudaEventRecord(p->ev[3], st);
    QOC_TRY(cudaStreamWaitEvent(st, p->join, 0));
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_C, st, p->ws[0]));
    QOC_TRY(launch_drift(p->a_hat, mixed, N, J, p->scal + 1, st));
    if (p->timing) cudaEventRecord(p->ev[4], st);
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_yhat, 0));
    QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 0, mixed, p->p_hat, p->y_hat, p->vstride,
                             p->Qf, p->Wf, p->Gf, p->qstride, p->gstride, BS_WG, st, p->ws[0]));
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_tangent, 0));
    QOC_TRY(launch_block_contract(p->XS, p->Wf, p->Gf, p->qstride, p->gstride, Bsrc, p->Kp, N, K, J,
                                  bs, 0, mixed, p->U, st));
    QOC_TRY(cudaStreamWaitEvent(st, p->ev_panels, 0));
  } else {
    if (p->timing) {
      cudaEventRecord(p->ev[3], st);
      cudaEventRecord(p->ev[12], st);
      cudaEventRecord(p->ev[13], st);
    }
    QOC_TRY(cudaStreamWaitEvent(st, p->join, 0));
    QOC_TRY(launch_drift(p->a_hat, mixed, N, J, p->scal + 1, st));
    QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                             p->y_hat, p->g, p->c, PW_Y, st, p->ws[0]));
    if (p->timing) cudaEventRecord(p->ev[4], st);
  }
  if (p->timing) cudaEventRecord(p->ev[5], st);
  QOC_TRY(launch_assemble(p->B, p->Kp, p->f, p->g, p->c, p->V, p->U, mixed, p->SJ, N, J, K,
                          p->w_f, p->w_t, soa ? (split ? 2 : 0) : 1, order >= 2, p->work, out_dev, p->hess_raw,
                          p->scal + 2, st, p->identity_basis));
  if (p->timing) cudaEventRecord(p->ev[6], st);
  return QOC_OK;
}

// Chunks of the forward pipeline for an evaluation (0: none).  Time-blocked
// evaluations with the refined eigensolver only, on request: measured at
// N = 32, J = 4000, the refinement in four chunks of 1000 steps loses more
// to its part-empty last waves and to the chain sharing the SMs (0.68 ->
// 1.00 ms) than the chain gains, so the built-in choice is off.
int pipeline_chunks(const qoc_problem* p, int /*order*/) {
  if (p->bs <= 1 || p->eig_method != QOC_EIG_REFINED) return 0;
  const int nblk = (p->J + p->bs - 1) / p->bs;
  int c = p->pipeline < 0 ? 0 : p->pipeline;
  if (c > qoc_problem::kMaxChunks) c = qoc_problem::kMaxChunks;
  if (c > nblk) c = nblk;
  return c >= 2 ? c : 0;
}

// The eigendecompositions, increments D_j and the forward state chain of a
// pipelined evaluation.  The binary32 start runs over all steps at once (it
// needs every step to fill the GPU); the refinement and the increments then
// run in chunks of whole blocks on the main stream, and the chain stream
// takes each chunk's forward block products and state-chain blocks as soon
// as that chunk's increments exist, resuming from the block-start state the
// previous chunk left: bit for bit the unchunked evaluation, with the chain's
// latency hidden behind the refinement of the later chunks.
qoc_status enqueue_pipelined_start(qoc_problem* p) {
  cudaStream_t st = p->stream, cs = p->side;
  const int N = p->N, J = p->J, bs = p->bs, C = p->piped;
  const int nblk = (J + bs - 1) / bs;
  const int mixed = p->precision == QOC_MIXED_FP32 ? 1 : 0;
  const size_t NN = (size_t)N * N;
  unsigned int* stats = p->timing ? p->eigstats : nullptr;
  QOC_TRY(launch_eig(p->H0, p->M, p->f, N, J, p->W, p->eig, p->status, EIG_REFINED, p->refine_sweeps,
                     p->angle_tol, st, p->ws[0], p->timing ? p->ev[8] : nullptr, stats, eig_finish_tol(p),
                     EIG_PHASE_START));
  for (int c = 0; c < C; ++c) {
    const int b0 = (int)((long long)c * nblk / C), b1 = (int)((long long)(c + 1) * nblk / C);
    const int j0 = b0 * bs, j1 = b1 * bs < J ? b1 * bs : J, jn = j1 - j0;
    QOC_TRY(launch_eig(p->H0, p->M, p->f + j0, N, jn, p->W + j0 * NN, p->eig + (size_t)j0 * N, p->status,
                       EIG_REFINED, p->refine_sweeps, p->angle_tol, st, p->ws[0], nullptr, stats,
                       eig_finish_tol(p), EIG_PHASE_REFINE));
    if (p->timing) cudaEventRecord(p->evp[2 * c], st);
    unsigned char* Dc = static_cast<unsigned char*>(p->D) + (size_t)j0 * p->dstride;
    QOC_TRY(launch_prep(p->W + j0 * NN, p->eig + (size_t)j0 * N, p->M, N, jn, p->dt, p->mshift, Dc,
                        p->dstride, mixed ? 0 : 1, PREP_D, p->Ptil, p->Xp, nullptr, p->status, st, p->ws[0]));
    if (p->timing) cudaEventRecord(p->evp[2 * c + 1], st);
    QOC_TRY(cudaEventRecord(p->ev_chunk[c], st));
    QOC_TRY(cudaStreamWaitEvent(cs, p->ev_chunk[c], 0));
    QOC_TRY(launch_block_delta(Dc, p->dstride, N, jn, bs, 0, mixed,
                               static_cast<unsigned char*>(p->Mf) + (size_t)b0 * p->mstride, p->mstride,
                               cs, p->ws[1]));
    BSweepArgs a = chain_sweep_args(p, 0);
    a.blk0 = b0;
    a.blk1 = b1;
    a.resume = c > 0;
    QOC_TRY(launch_bsweep(a, mixed, cs));
  }
  if (p->timing) cudaEventRecord(p->ev[1], st);
  return QOC_OK;
}

// Enqueue one evaluation.  order 0: J; 1: J + grad; 2: J + grad + Hess.
// theta_dev: K doubles on the device.  out_dev: 1 + K (+ K*K) doubles.
qoc_status enqueue_eval(qoc_problem* p, const double* theta_dev, int order, double* out_dev) {
  cudaStream_t st = p->stream;
  const int N = p->N, K = p->K, J = p->J;
  const int mixed = p->precision == QOC_MIXED_FP32 ? 1 : 0;
  const int d_fp64 = mixed ? 0 : 1;
  if (p->timing) cudaEventRecord(p->ev[0], st);
  p->fwd_reused = p->reuse_fwd && p->bs > 1 && order >= 1;
  p->reuse_fwd = 0;
  if (p->fwd_reused) {   // f, W, lambda, D, the forward products and chain are current
    p->piped = 0;
    if (p->timing)
      for (int k : {7, 8, 1, 2}) cudaEventRecord(p->ev[k], st);
    return enqueue_blocked(p, order, out_dev);
  }
  // theta_dev == nullptr: the samples f are already in p->f (a model evaluation)
  if (theta_dev) QOC_TRY(launch_control(p->B, p->Kp, theta_dev, J, K, p->f, st));
  if (p->timing) {
    cudaEventRecord(p->ev[7], st);
    QOC_TRY(cudaMemsetAsync(p->eigstats, 0, 4 * sizeof(unsigned int), st));
  }
  p->piped = pipeline_chunks(p, order);
  if (p->piped) {
    const qoc_status ps = enqueue_pipelined_start(p);
    if (ps != QOC_OK) return ps;
  } else {
    QOC_TRY(launch_eig(p->H0, p->M, p->f, N, J, p->W, p->eig, p->status,
                       p->eig_method == QOC_EIG_JACOBI_FP64 ? EIG_JACOBI_FP64 : EIG_REFINED,
                       p->refine_sweeps, p->angle_tol, st, p->ws[0], p->timing ? p->ev[8] : nullptr,
                       p->timing ? p->eigstats : nullptr, eig_finish_tol(p), EIG_PHASE_ALL, p->eigorder));
    if (p->timing) cudaEventRecord(p->ev[1], st);
    QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, d_fp64, PREP_D,
                        p->Ptil, p->Xp, nullptr, p->status, st, p->ws[0]));
  }
  if (p->timing) cudaEventRecord(p->ev[2], st);
  if (p->bs > 1) return enqueue_blocked(p, order, out_dev);
  p->sched = 0;
  if (order >= 1)
    QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, d_fp64,
                        PREP_P | PREP_X, p->Ptil, p->Xp, nullptr, p->status, st, p->ws[0]));
  if (p->timing) cudaEventRecord(p->ev[9], st);
  SweepArgs a{};
  a.N = N; a.K = 1; a.Kp = p->Kp; a.J = J; a.kc = 1; a.backward = 0;
  a.D = reinterpret_cast<const unsigned char*>(p->D); a.dstride = p->dstride;
  a.init = p->alpha; a.init_scale = 1.0; a.states = p->a_hat; a.status = p->status;
  QOC_TRY(launch_sweep(a, d_fp64, st));
  const double thetaJ = (double)J * p->dt * p->mshift;
  QOC_TRY(launch_terminal(p->f, J, p->a_hat, mixed, p->beta, N, cexpi_h(thetaJ), p->w_f, p->w_t,
                          p->lamJ, p->scal + 0, p->scal + 1, st));
  QOC_TRY(cudaMemcpyAsync(out_dev, p->scal, sizeof(double), cudaMemcpyDeviceToDevice, st));
  if (order == 0) {
    if (p->timing) for (int k = 3; k < 7; ++k) cudaEventRecord(p->ev[k], st);
    return QOC_OK;
  }
  SweepArgs l = a;
  l.backward = 1; l.init = p->lamJ; l.states = p->l_hat;
  QOC_TRY(launch_sweep(l, d_fp64, st));
  if (p->timing) cudaEventRecord(p->ev[3], st);
  const double2 kappa = cexpi_h(p->dt * p->mshift);
  QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J, kappa, p->p_hat,
                           p->y_hat, p->g, p->c, PW_P | PW_Y | (order >= 2 ? PW_C : 0), st, p->ws[0]));
  if (p->timing) cudaEventRecord(p->ev[4], st);
  if (order >= 2) {
    SweepArgs s{};
    s.N = N; s.K = K; s.Kp = p->Kp; s.J = J; s.kc = sweep_kc(p); s.backward = 0;
    s.D = reinterpret_cast<const unsigned char*>(p->D); s.dstride = p->dstride;
    s.src = p->p_hat; s.ctr = p->y_hat;
    s.Brow = mixed ? static_cast<const void*>(p->Bf) : static_cast<const void*>(p->B);
    s.init = nullptr; s.final_out = p->SJ; s.contr = p->U; s.status = p->status;
    QOC_TRY(launch_sweep(s, d_fp64, st));
    if (p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT) {
      SweepArgs m = s;
      m.backward = 1; m.src = p->y_hat; m.ctr = p->p_hat;
      m.init = p->SJ; m.init_scale = 2.0 * p->w_t; m.final_out = nullptr; m.contr = p->V;
      QOC_TRY(launch_sweep(m, d_fp64, st));
    }
  }
  if (p->timing) cudaEventRecord(p->ev[5], st);
  QOC_TRY(launch_assemble(p->B, p->Kp, p->f, p->g, p->c, p->V, p->U, mixed, p->SJ, N, J, K,
                          p->w_f, p->w_t, p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT ? 0 : 1,
                          order >= 2, p->work, out_dev, p->hess_raw, p->scal + 2, st, p->identity_basis));
  if (p->timing) cudaEventRecord(p->ev[6], st);
  return QOC_OK;
}

void collect_timing(qoc_problem* p) {
  if (!p->timing) return;
  auto el = [&](int a, int b) {
    float ms = 0;
    return cudaEventElapsedTime(&ms, p->ev[a], p->ev[b]) == cudaSuccess ? (double)ms : 0.0;
  };
  // events: 0 start, 7 control, 8 binary32 Jacobi, 1 refinement, 2 increments D_j,
  // sequential schedule: 9 derivative preparation, 3 chains, 4 pointwise, 5 panels, 6 assembly;
  // three-stream schedule: 3 P~ and X' (main), 4 c_j (main), 5 panels joined, 6 assembly,
  // 10/11 chains (chain stream), 12/13 panels (panel stream)
  double* k = p->kphase_ms;
  k[9] = el(0, 6);
  k[0] = el(0, 7); k[1] = el(7, 8); k[2] = el(8, 1); k[3] = el(1, 2); k[8] = el(5, 6);
  if (p->piped) {   // refinement and increments interleaved by chunk on the main stream
    auto elp = [&](cudaEvent_t a, cudaEvent_t b) {
      float ms = 0;
      return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : 0.0;
    };
    k[2] = k[3] = 0;
    for (int c = 0; c < p->piped; ++c) {
      k[2] += elp(c ? p->evp[2 * c - 1] : p->ev[8], p->evp[2 * c]);
      k[3] += elp(p->evp[2 * c], p->evp[2 * c + 1]);
    }
  }
  if (p->sched == 1) {
    k[4] = el(2, 3); k[5] = el(10, 11); k[6] = el(3, 4); k[7] = el(12, 13);
    const double ph[6] = {el(0, 1), el(1, 3), el(10, 11), el(3, 4), el(12, 13), el(5, 6)};
    for (int i = 0; i < 6; ++i) p->phase_ms[i] = ph[i];
  } else {
    k[4] = el(2, 9); k[5] = el(9, 3); k[6] = el(3, 4); k[7] = el(4, 5);
    for (int i = 0; i < 6; ++i) p->phase_ms[i] = el(i, i + 1);
  }
}

// host-pointer evaluation: theta in, [J, grad, Hess] out
qoc_status eval_host(qoc_problem* p, const double* theta, int order, double* J, double* grad,
                     double* hess) {
  if (!p || !theta || !J) return QOC_EINVAL;
  if ((order >= 1 && !grad) || (order >= 2 && !hess)) return QOC_EINVAL;
  if (!finite_all(theta, p->K)) return QOC_EINVAL;
  const int K = p->K;
  const size_t nout = 1 + (order >= 1 ? K : 0) + (order >= 2 ? (size_t)K * K : 0);
  std::memcpy(p->hbuf, theta, sizeof(double) * K);
  QOC_TRY(cudaMemcpyAsync(p->theta, p->hbuf, sizeof(double) * K, cudaMemcpyHostToDevice, p->stream));
  qoc_status s = enqueue_eval(p, p->theta, order, p->out);
  if (s != QOC_OK) return s;
  QOC_TRY(cudaMemcpyAsync(p->hbuf + K, p->out, sizeof(double) * nout, cudaMemcpyDeviceToHost,
                          p->stream));
  QOC_TRY(cudaMemcpyAsync(p->hbuf + K + nout, p->scal, 3 * sizeof(double), cudaMemcpyDeviceToHost,
                          p->stream));
  QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
  QOC_TRY(cudaStreamSynchronize(p->stream));
  collect_timing(p);
  p->last_order = order;
  p->diag[0] = p->hbuf[K + nout + 1];
  p->diag[1] = order >= 2 ? p->hbuf[K + nout + 2] : 0.0;
  s = device_status(p);
  const double* o = p->hbuf + K;
  *J = o[0];
  if (order >= 1) std::memcpy(grad, o + 1, sizeof(double) * K);
  if (order >= 2) std::memcpy(hess, o + 1 + K, sizeof(double) * K * K);
  if (s != QOC_OK) return s;
  if (!finite_all(o, nout)) return QOC_ENUMERIC;
  return QOC_OK;
}

}  // namespace

// a non-CUDA failure reason for qoc_last_error (entry points in other files)
void qoc::note_error(const char* msg) { std::snprintf(g_last_error, sizeof(g_last_error), "%s", msg); }

extern "C" {

int qoc_version(void) { return 200; }

const char* qoc_last_error(void) { return g_last_error; }
int qoc_max_basis_size(void) { return kMaxN; }

const char* qoc_status_string(qoc_status s) {
  switch (s) {
    case QOC_OK: return "ok";
    case QOC_EINVAL: return "invalid argument";
    case QOC_ENOMEM: return "out of memory";
    case QOC_ECUDA: return "CUDA error";
    case QOC_ENUMERIC: return "numerical failure (non-finite value or eigensolver not converged)";
    case QOC_ENOTCONV: return "trust region did not converge within max_iter";
    case QOC_ETIMEOUT: return "bounded device wait timed out";
    case QOC_EUNSUPPORTED: return "unsupported size or option in this build";
  }
  return "unknown status";
}

void qoc_destroy_problem(qoc_problem* p) {
  if (!p) return;
  if (p->stream) cudaStreamSynchronize(p->stream);
  for (void* v : p->allocs) cudaFree(v);
  if (p->hbuf) cudaFreeHost(p->hbuf);
  if (p->hstatus) cudaFreeHost(p->hstatus);
  for (auto& e : p->ev)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->ev_chunk)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->evp)
    if (e) cudaEventDestroy(e);
  for (auto& e : p->trev)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t* sp : {&p->side, &p->pstream})
    if (*sp) {
      cudaStreamSynchronize(*sp);
      cudaStreamDestroy(*sp);
    }
  for (cudaEvent_t e : {p->fork, p->join, p->ev_state, p->ev_ptil, p->ev_panels, p->ev_bprod, p->ev_fprod, p->ev_yhat, p->ev_phat, p->ev_tangent, p->ev_musrc})
    if (e) cudaEventDestroy(e);
  if (p->own_stream && p->stream) cudaStreamDestroy(p->stream);
  delete p;
}

qoc_status qoc_create_problem(int N, const double* H0, const double* M, const double* a0,
                              const double* a_target, int K, const double* basis, double dt,
                              int steps, double w_ctrl, double w_term, int precision,
                              void* cuda_stream, qoc_problem** out) {
  if (!out) return QOC_EINVAL;
  *out = nullptr;
  if (!H0 || !M || !a0 || !a_target || !basis) return QOC_EINVAL;
  if (N < 1 || K < 1 || steps < 1) return QOC_EINVAL;
  if (N > kMaxN || K > kMaxK) return QOC_EUNSUPPORTED;
  if (!(dt > 0) || !std::isfinite(dt) || !(w_ctrl >= 0) || !(w_term >= 0) ||
      !std::isfinite(w_ctrl) || !std::isfinite(w_term))
    return QOC_EINVAL;
  if (precision != QOC_FP64 && precision != QOC_MIXED_FP32 && precision != QOC_MIXED_FP32_ALWAYS)
    return QOC_EINVAL;
  const size_t NN = (size_t)N * N;
  if (!finite_all(H0, NN) || !finite_all(M, NN) || !finite_all(a0, 2 * (size_t)N) ||
      !finite_all(a_target, 2 * (size_t)N) || !finite_all(basis, (size_t)steps * K))
    return QOC_EINVAL;
  if (!symmetric(H0, N) || !symmetric(M, N)) return QOC_EINVAL;

  qoc_problem* p = new (std::nothrow) qoc_problem();
  if (!p) return QOC_ENOMEM;
  p->N = N; p->K = K; p->J = steps; p->Kp = (K + 3) / 4 * 4;
  p->dt = dt; p->w_f = w_ctrl; p->w_t = w_term; p->requested_precision = precision;
  // the eigendecomposition is binary64-accurate on both paths: refinement
  // until W is orthonormal to the binary64 floor (at most 4 updates), then a
  // clean-up of every rotation angle above 1e-13 (smaller angles move the
  // propagators by less than 1e-13 dt |lambda_p - lambda_q|)
  // binary64 refinement updates allowed per step: the binary32 start is
  // coarser relative to the eigenvalue gaps at large N
  p->refine_sweeps = N <= 64 ? 4 : 8;
  p->angle_tol = 1e-13;
  double tr = 0;
  for (int i = 0; i < N; ++i) tr += H0[i * N + i];
  p->mshift = tr / N;
  const int J = steps;
  // precision policy: binary32 increments unless their estimated error at
  // the default block length exceeds the mixed-precision target
  p->err_sigma = spectral_sigma(N, H0, M, basis, K, J, p->mshift);
  if (K == J) {
    bool id = true;
    for (int j = 0; j < J && id; ++j)
      for (int l = 0; l < K; ++l)
        if (basis[(size_t)j * K + l] != (j == l ? 1.0 : 0.0)) { id = false; break; }
    p->identity_basis = id ? 1 : 0;
  }
  if (precision == QOC_MIXED_FP32_ALWAYS) p->precision = QOC_MIXED_FP32;
  else if (precision == QOC_MIXED_FP32)
    p->precision = mixed_error_estimate(p, J >= 16 ? 4 : 1) <= kMixedTarget ? QOC_MIXED_FP32 : QOC_FP64;
  else p->precision = QOC_FP64;
  precision = p->precision;
  const int mixed = precision == QOC_MIXED_FP32;
  p->dstride = ((mixed ? 8 : 16) * NN + 15) / 16 * 16;
  p->vstride = ((mixed ? 8 : 16) * (size_t)N + 15) / 16 * 16;

  cudaError_t e = cudaSuccess;
  auto fail = [&](cudaError_t err) {
    qoc_destroy_problem(p);
    return from_cuda(err);
  };
  if (cuda_stream) {
    p->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if ((e = cudaStreamCreateWithFlags(&p->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    p->own_stream = true;
  }
  for (auto& ev : p->ev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e);
  for (auto& ev : p->evp)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e);
  for (auto& ev : p->trev)
    if ((e = cudaEventCreate(&ev)) != cudaSuccess) return fail(e);
  for (auto& ev : p->ev_chunk)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if ((e = cudaStreamCreateWithPriority(&p->side, cudaStreamNonBlocking, hi)) != cudaSuccess) return fail(e);
    if ((e = cudaStreamCreateWithPriority(&p->pstream, cudaStreamNonBlocking, hi)) != cudaSuccess)
      return fail(e);
  }
  for (cudaEvent_t* ep : {&p->fork, &p->join, &p->ev_state, &p->ev_ptil, &p->ev_panels, &p->ev_bprod, &p->ev_fprod, &p->ev_yhat, &p->ev_phat, &p->ev_tangent, &p->ev_musrc})
    if ((e = cudaEventCreateWithFlags(ep, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
#define ALLOC(ptr, bytes) \
  if ((e = dalloc(p, &(ptr), (bytes))) != cudaSuccess) return fail(e)
  ALLOC(p->H0, 8 * NN);
  ALLOC(p->M, 8 * NN);
  ALLOC(p->B, 8 * (size_t)J * p->Kp);
  ALLOC(p->Bf, 4 * (size_t)J * p->Kp);
  ALLOC(p->theta, 8 * (size_t)K);
  ALLOC(p->theta_trial, 8 * (size_t)K);
  ALLOC(p->f, 8 * (size_t)J);
  ALLOC(p->W, 8 * (size_t)J * NN);
  ALLOC(p->eig, 8 * (size_t)J * N);
  ALLOC(p->g, 8 * (size_t)J);
  ALLOC(p->c, 8 * (size_t)J);
  ALLOC(p->V, 8 * (size_t)J * K);
  ALLOC(p->U, 8 * (size_t)J * K);
  ALLOC(p->work, 8 * assemble_work_doubles(J, K));
  ALLOC(p->out, 8 * (1 + (size_t)K + (size_t)K * K));
  ALLOC(p->out_trial, 8 * (1 + (size_t)K + (size_t)K * K));
  ALLOC(p->hess_raw, 8 * (size_t)K * K);
  ALLOC(p->scal, 8 * 8);
  ALLOC(p->eigstats, 4 * sizeof(unsigned int));
  ALLOC(p->eigorder, sizeof(int) * ((size_t)J + 2));
  ALLOC(p->alpha, 16 * (size_t)N);
  ALLOC(p->beta, 16 * (size_t)N);
  ALLOC(p->lamJ, 16 * (size_t)N);
  ALLOC(p->Ptil, 16 * (size_t)J * NN);
  ALLOC(p->Mtil, 8 * (size_t)J * NN);
  ALLOC(p->Xp, 16 * (size_t)J * NN);
  ALLOC(p->SJ, 16 * (size_t)K * N);
  ALLOC(p->D, (size_t)J * p->dstride);
  ALLOC(p->a_hat, 16 * (size_t)(J + 1) * N);
  ALLOC(p->l_hat, 16 * (size_t)(J + 1) * N);
  ALLOC(p->p_hat, (size_t)J * p->vstride);
  ALLOC(p->rvec, 16 * (size_t)J * N);
  ALLOC(p->y_hat, (size_t)J * p->vstride);
  ALLOC(p->status, sizeof(int));
  // block size: binary32 rounding of the block increment grows ~ sqrt(bs), so
  // the mixed path keeps 4 (Hessian error ~5e-7 on the N=32 workload, 8e-7 at 8)
  p->bs = J >= 16 ? (mixed ? 4 : 8) : 1;
  p->nblk = (J + p->bs - 1) / p->bs;
  {
    const size_t cs = mixed ? 8 : 16;
    // per-block buffers sized for the smallest blocked size (2 steps) and
    // the largest (8 sources per block)
    p->mstride = (cs * NN + 15) / 16 * 16;
    p->qstride = (cs * 8 * (size_t)N + 15) / 16 * 16;
    p->gstride = (cs * 64 + 15) / 16 * 16;
    const size_t nbp = ((size_t)J + 1) / 2 + 1;
    ALLOC(p->Mf, nbp * p->mstride);
    ALLOC(p->Mb, nbp * p->mstride);
    ALLOC(p->Qf, nbp * p->qstride);
    ALLOC(p->Wf, nbp * p->qstride);
    ALLOC(p->Gf, nbp * p->gstride);
    ALLOC(p->Qb, nbp * p->qstride);
    ALLOC(p->Wb, nbp * p->qstride);
    ALLOC(p->Gb, nbp * p->gstride);
    ALLOC(p->Xa, 16 * nbp * N);
    ALLOC(p->Xl, 16 * nbp * N);
    ALLOC(p->XS, cs * nbp * (size_t)K * N);
    ALLOC(p->Xmu, cs * nbp * (size_t)K * N);
  }
  if (K <= kMaxKTR) {
    ALLOC(p->trwork, 8 * tr_work_doubles(K));
    ALLOC(p->trstep, 8 * (size_t)K);
    ALLOC(p->trinfo, 8 * 8);
    ALLOC(p->trzero, 8 * ((size_t)K * K + 1));
  }
  {
    // Per-step storage for matrices that do not fit in shared memory (N > 64,
    // or the trust region's K x K eigensolver for K > 64): one region per
    // stream, each a slice per CTA of a persistent grid.
    const int mx = precision == QOC_MIXED_FP32 ? 1 : 0;
    size_t need = 0;
    for (size_t v : {eig_step_bytes(N), prep_smem_bytes(N), pointwise_step_bytes(N),
                     block_delta_bytes(N, mx), block_src_bytes(N, 8, mx)})
      need = v > need ? v : need;
    const size_t need_tr = K <= kMaxKTR ? eig_step_bytes(K) : 0;
    int nsm = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const size_t big = 200 * 1024;
    for (int r = 0; r < 3; ++r) {
      size_t per = need;
      if (r == 0 && need_tr > per) per = need_tr;
      if (per <= big) continue;
      per = (per + 255) & ~size_t(255);
      const size_t nct = (r == 0 ? 2 : 1) * (size_t)nsm;
      ALLOC(p->ws[r].base, per * nct);
      p->ws[r].bytes = per * nct;
    }
  }
#undef ALLOC
  p->hbuf_len = 2 * (1 + (size_t)K + (size_t)K * K) + 2 * (size_t)K + 2 * (size_t)N + 64;
  if ((e = cudaMallocHost(&p->hbuf, 8 * p->hbuf_len)) != cudaSuccess) return fail(e);
  if ((e = cudaMallocHost(&p->hstatus, sizeof(int))) != cudaSuccess) return fail(e);
  *p->hstatus = 0;

  // upload inputs (the basis is padded to Kp columns, plus a binary32 copy)
  std::vector<double> Bp((size_t)J * p->Kp, 0.0);
  std::vector<float> Bfp((size_t)J * p->Kp, 0.0f);
  for (int j = 0; j < J; ++j)
    for (int l = 0; l < K; ++l) {
      Bp[(size_t)j * p->Kp + l] = basis[(size_t)j * K + l];
      Bfp[(size_t)j * p->Kp + l] = (float)basis[(size_t)j * K + l];
    }
  if ((e = cudaMemcpy(p->H0, H0, 8 * NN, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->M, M, 8 * NN, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->B, Bp.data(), 8 * Bp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->Bf, Bfp.data(), 4 * Bfp.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->alpha, a0, 16 * (size_t)N, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemcpy(p->beta, a_target, 16 * (size_t)N, cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(p->status, 0, sizeof(int))) != cudaSuccess) return fail(e);
  if ((e = cudaMemset(p->V, 0, 8 * (size_t)J * K)) != cudaSuccess) return fail(e);
  if (p->trzero && (e = cudaMemset(p->trzero, 0, 8 * ((size_t)K * K + 1))) != cudaSuccess) return fail(e);
  *out = p;
  return QOC_OK;
}

qoc_status qoc_set_target(qoc_problem* p, const double* a_target) {
  if (!p || !a_target || !finite_all(a_target, 2 * (size_t)p->N)) return QOC_EINVAL;
  std::memcpy(p->hbuf, a_target, 16 * (size_t)p->N);
  QOC_TRY(cudaMemcpyAsync(p->beta, p->hbuf, 16 * (size_t)p->N, cudaMemcpyHostToDevice, p->stream));
  return from_cuda(cudaStreamSynchronize(p->stream));
}

qoc_status qoc_set_hess_method(qoc_problem* p, int method) {
  if (!p || (method != QOC_HESS_SECOND_ORDER_ADJOINT && method != QOC_HESS_TANGENT)) return QOC_EINVAL;
  p->hess_method = method;
  return QOC_OK;
}

qoc_status qoc_set_eig_method(qoc_problem* p, int method) {
  if (!p || (method != QOC_EIG_REFINED && method != QOC_EIG_JACOBI_FP64)) return QOC_EINVAL;
  p->eig_method = method;
  return QOC_OK;
}

qoc_status qoc_get_precision(const qoc_problem* p, int* effective, double* estimate) {
  if (!p) return QOC_EINVAL;
  if (effective) *effective = p->precision;
  if (estimate) *estimate = mixed_error_estimate(p, p->bs);
  return QOC_OK;
}

qoc_status qoc_set_block_steps(qoc_problem* p, int steps) {
  if (!p || steps < 1 || steps > 8 || (steps > 1 && p->J < steps)) return QOC_EINVAL;
  if (p->requested_precision == QOC_MIXED_FP32 && p->precision == QOC_MIXED_FP32 &&
      mixed_error_estimate(p, steps) > kMixedTarget) {
    std::snprintf(g_last_error, sizeof(g_last_error),
                  "qoc_set_block_steps: %d steps per block raise the binary32 error estimate to %.2e, "
                  "above the mixed-precision target %.0e", steps, mixed_error_estimate(p, steps),
                  kMixedTarget);
    return QOC_EINVAL;
  }
  p->bs = steps;
  p->nblk = (p->J + steps - 1) / steps;
  return QOC_OK;
}

qoc_status qoc_set_panel_columns(qoc_problem* p, int kc) {
  if (!p || kc < 0 || kc > 4) return QOC_EINVAL;
  if (kc > 0 && 32 * ((p->N + 7) / 8) * kc > 1024) return QOC_EUNSUPPORTED;
  p->kc = kc;
  return QOC_OK;
}

qoc_status qoc_get_tr_phase_times(const qoc_problem* p, double* out) {
  if (!p || !out) return QOC_EINVAL;
  for (int k = 0; k < 3; ++k) out[k] = p->trphase_ms[k];
  return QOC_OK;
}

qoc_status qoc_set_pipeline(qoc_problem* p, int chunks) {
  if (!p || chunks < -1 || chunks > qoc_problem::kMaxChunks) return QOC_EINVAL;
  p->pipeline = chunks;
  return QOC_OK;
}

qoc_status qoc_set_mu_split(qoc_problem* p, int split) {
  if (!p || split < -1 || split > 1) return QOC_EINVAL;
  p->mu_split = split;
  return QOC_OK;
}

qoc_status qoc_set_refine_sweeps(qoc_problem* p, int sweeps) {
  if (!p || sweeps < 0 || sweeps > 16) return QOC_EINVAL;
  p->refine_sweeps = sweeps;
  return QOC_OK;
}

qoc_status qoc_selftest_bounded_wait(qoc_problem* p, unsigned long long limit_ns) {
  if (!p || limit_ns < 1000ull || limit_ns > 10000000000ull) return QOC_EINVAL;
  QOC_TRY(launch_wait_selftest(p->status, limit_ns, p->stream));
  return qoc_sync_status(p);
}

qoc_status qoc_enable_timing(qoc_problem* p, int on) {
  if (!p) return QOC_EINVAL;
  p->timing = on ? 1 : 0;
  return QOC_OK;
}

qoc_status qoc_eval_J(qoc_problem* p, const double* theta, double* J) {
  return eval_host(p, theta, 0, J, nullptr, nullptr);
}

qoc_status qoc_eval_grad(qoc_problem* p, const double* theta, double* J, double* grad) {
  return eval_host(p, theta, 1, J, grad, nullptr);
}

qoc_status qoc_eval_grad_hess(qoc_problem* p, const double* theta, double* J, double* grad,
                              double* hess) {
  return eval_host(p, theta, 2, J, grad, hess);
}

qoc_status qoc_eval_grad_hess_model(qoc_problem* p, const double* f, const double* jac, double* J,
                                    double* grad, double* hess, double* dJdf) {
  if (!p || !f || !jac || !J || !grad || !hess || !dJdf) return QOC_EINVAL;
  const int K = p->K, Jn = p->J, Kp = p->Kp;
  if (!finite_all(f, Jn) || !finite_all(jac, (size_t)Jn * K)) return QOC_EINVAL;
  // the Jacobian becomes the problem's basis (padded to Kp columns, with its binary32 copy)
  std::vector<double> Bp((size_t)Jn * Kp, 0.0);
  std::vector<float> Bfp((size_t)Jn * Kp, 0.0f);
  bool id = K == Jn;
  for (int j = 0; j < Jn; ++j)
    for (int l = 0; l < K; ++l) {
      const double v = jac[(size_t)j * K + l];
      Bp[(size_t)j * Kp + l] = v;
      Bfp[(size_t)j * Kp + l] = (float)v;
      if (v != (j == l ? 1.0 : 0.0)) id = false;
    }
  QOC_TRY(cudaStreamSynchronize(p->stream));
  QOC_TRY(cudaMemcpy(p->B, Bp.data(), 8 * Bp.size(), cudaMemcpyHostToDevice));
  QOC_TRY(cudaMemcpy(p->Bf, Bfp.data(), 4 * Bfp.size(), cudaMemcpyHostToDevice));
  QOC_TRY(cudaMemcpy(p->f, f, 8 * (size_t)Jn, cudaMemcpyHostToDevice));
  p->identity_basis = id ? 1 : 0;
  const size_t nout = 1 + (size_t)K + (size_t)K * K;
  qoc_status s = enqueue_eval(p, nullptr, 2, p->out);
  if (s != QOC_OK) return s;
  std::vector<double> o(nout), g(Jn);
  QOC_TRY(cudaMemcpyAsync(o.data(), p->out, 8 * nout, cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaMemcpyAsync(g.data(), p->g, 8 * (size_t)Jn, cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
  QOC_TRY(cudaStreamSynchronize(p->stream));
  collect_timing(p);
  p->last_order = 2;
  s = device_status(p);
  if (s != QOC_OK) return s;
  *J = o[0];
  std::memcpy(grad, o.data() + 1, 8 * (size_t)K);
  std::memcpy(hess, o.data() + 1 + K, 8 * (size_t)K * K);
  for (int j = 0; j < Jn; ++j) dJdf[j] = 2.0 * p->w_f * f[j] + g[j];
  if (!finite_all(o.data(), nout)) return QOC_ENUMERIC;
  return QOC_OK;
}

qoc_status qoc_eval_grad_hess_dev(qoc_problem* p, const double* theta_dev, double* out_dev) {
  if (!p || !theta_dev || !out_dev) return QOC_EINVAL;
  p->last_order = 2;
  return enqueue_eval(p, theta_dev, 2, out_dev);
}

qoc_status qoc_sync_status(qoc_problem* p) {
  if (!p) return QOC_EINVAL;
  QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), p->stream));
  QOC_TRY(cudaStreamSynchronize(p->stream));
  collect_timing(p);
  return device_status(p);
}

qoc_status qoc_get_diagnostics(const qoc_problem* p, double* norm_drift, double* hess_asym,
                               double* phase_ms) {
  if (!p) return QOC_EINVAL;
  if (norm_drift) *norm_drift = p->diag[0];
  if (hess_asym) *hess_asym = p->diag[1];
  if (phase_ms)
    for (int k = 0; k < 6; ++k) phase_ms[k] = p->timing ? p->phase_ms[k] : 0.0;
  return QOC_OK;
}

qoc_status qoc_get_eig_stats(qoc_problem* p, double* out) {
  if (!p || !out) return QOC_EINVAL;
  unsigned int h[3] = {0, 0, 0};
  QOC_TRY(cudaMemcpyAsync(h, p->eigstats, sizeof(h), cudaMemcpyDeviceToHost, p->stream));
  QOC_TRY(cudaStreamSynchronize(p->stream));
  for (int i = 0; i < 3; ++i) out[i] = p->timing ? (double)h[i] / p->J : 0.0;
  return QOC_OK;
}

qoc_status qoc_get_phase_times(const qoc_problem* p, double* out, int n) {
  if (!p || !out || n < 0) return QOC_EINVAL;
  for (int k = 0; k < n && k < QOC_N_PHASES; ++k) out[k] = p->timing ? p->kphase_ms[k] : 0.0;
  return QOC_OK;
}

size_t qoc_device_bytes(const qoc_problem* p) { return p ? p->dev_bytes : 0; }

qoc_status qoc_read_buffer(const qoc_problem* p, int which, double* host_out, size_t count) {
  if (!p || !host_out || p->last_order < 0) return QOC_EINVAL;
  const int N = p->N, K = p->K, J = p->J;
  const bool mixed = p->precision == QOC_MIXED_FP32;
  const double m = p->mshift, dt = p->dt;
  auto need = [&](size_t n) { return count >= n; };
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return from_cuda(e);
  // states are stored in the frame rotating with the shift m: x_j = e^{-i j dt m} x^_j
  auto unframe_rows = [&](const void* dev, int rows) -> qoc_status {
    const size_t n = (size_t)rows * N;
    std::vector<double> raw(4 * n);
    cudaError_t err = cudaMemcpy(raw.data(), dev, 16 * n, cudaMemcpyDeviceToHost);
    if (err != cudaSuccess) return from_cuda(err);
    for (int j = 0; j < rows; ++j) {
      const double2 ph = cexpi_h(-(double)j * dt * m);
      for (int i = 0; i < N; ++i) {
        double xr, xi;
        const size_t k = (size_t)j * N + i;
        if (mixed) {
          const float* fr = reinterpret_cast<const float*>(raw.data());
          xr = (double)fr[4 * k] + (double)fr[4 * k + 2];
          xi = (double)fr[4 * k + 1] + (double)fr[4 * k + 3];
        } else {
          xr = raw[2 * k];
          xi = raw[2 * k + 1];
        }
        host_out[2 * k] = ph.x * xr - ph.y * xi;
        host_out[2 * k + 1] = ph.x * xi + ph.y * xr;
      }
    }
    return QOC_OK;
  };
  switch (which) {
    case QOC_BUF_F:
      if (!need(J)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->f, 8 * (size_t)J, cudaMemcpyDeviceToHost));
    case QOC_BUF_EIGVAL:
      if (!need((size_t)J * N)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->eig, 8 * (size_t)J * N, cudaMemcpyDeviceToHost));
    case QOC_BUF_EIGVEC:
      if (!need((size_t)J * N * N)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->W, 8 * (size_t)J * N * N, cudaMemcpyDeviceToHost));
    case QOC_BUF_STATE:
      if (!need(2 * (size_t)(J + 1) * N)) return QOC_EINVAL;
      return unframe_rows(p->a_hat, J + 1);
    case QOC_BUF_COSTATE:
      if (p->last_order < 1 || !need(2 * (size_t)(J + 1) * N)) return QOC_EINVAL;
      return unframe_rows(p->l_hat, J + 1);
    case QOC_BUF_G:
      if (p->last_order < 1 || !need(J)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->g, 8 * (size_t)J, cudaMemcpyDeviceToHost));
    case QOC_BUF_C:
      if (p->last_order < 2 || !need(J)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->c, 8 * (size_t)J, cudaMemcpyDeviceToHost));
    case QOC_BUF_V:
    case QOC_BUF_U: {
      if (p->last_order < 2 || !need((size_t)J * K)) return QOC_EINVAL;
      const void* src = which == QOC_BUF_V ? static_cast<const void*>(p->V) : static_cast<const void*>(p->U);
      if (!mixed)
        return from_cuda(cudaMemcpy(host_out, src, 8 * (size_t)J * K, cudaMemcpyDeviceToHost));
      std::vector<float> tmp((size_t)J * K);
      e = cudaMemcpy(tmp.data(), src, 4 * (size_t)J * K, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return from_cuda(e);
      for (size_t k = 0; k < tmp.size(); ++k) host_out[k] = (double)tmp[k];
      return QOC_OK;
    }
    case QOC_BUF_SJ: {
      if (p->last_order < 2 || !need(2 * (size_t)N * K)) return QOC_EINVAL;
      std::vector<double> raw(2 * (size_t)N * K);
      e = cudaMemcpy(raw.data(), p->SJ, 16 * (size_t)N * K, cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) return from_cuda(e);
      const double2 ph = cexpi_h(-(double)J * dt * m);
      for (int l = 0; l < K; ++l)
        for (int i = 0; i < N; ++i) {
          double xr = raw[2 * ((size_t)l * N + i)], xi = raw[2 * ((size_t)l * N + i) + 1];
          host_out[2 * ((size_t)i * K + l)] = ph.x * xr - ph.y * xi;
          host_out[2 * ((size_t)i * K + l) + 1] = ph.x * xi + ph.y * xr;
        }
      return QOC_OK;
    }
    case QOC_BUF_HESS_RAW:
      if (p->last_order < 2 || !need((size_t)K * K)) return QOC_EINVAL;
      return from_cuda(cudaMemcpy(host_out, p->hess_raw, 8 * (size_t)K * K, cudaMemcpyDeviceToHost));
    default:
      return QOC_EINVAL;
  }
}

qoc_status qoc_trust_region_solve(qoc_problem* p, const double* theta0, const qoc_tr_options* opt,
                                  double* theta_out, qoc_tr_report* report) {
  if (!p || !theta0 || !opt || !theta_out || !report) return QOC_EINVAL;
  if (!p->trwork) return QOC_EUNSUPPORTED;
  if (!(opt->radius0 > 0) || !(opt->radius_max >= opt->radius0) || opt->max_iter < 1 ||
      !(opt->eta >= 0 && opt->eta < 0.25) || !(opt->gtol >= 0) || !(opt->xtol >= 0))
    return QOC_EINVAL;
  if (!finite_all(theta0, p->K)) return QOC_EINVAL;
  const int K = p->K;
  cudaStream_t st = p->stream;
  std::memset(report, 0, sizeof(*report));
  double radius = opt->radius0;
  std::memcpy(p->hbuf, theta0, 8 * (size_t)K);
  QOC_TRY(cudaMemcpyAsync(p->theta, p->hbuf, 8 * (size_t)K, cudaMemcpyHostToDevice, st));
  double* hs = p->hbuf + K;   // [J, |g|] and [pred, |s|, sigma, |g|, J_trial]
  for (double& t : p->trphase_ms) t = 0.0;
  auto elapsed = [](cudaEvent_t a, cudaEvent_t b) {
    float ms = 0;
    return cudaEventElapsedTime(&ms, a, b) == cudaSuccess ? (double)ms : 0.0;
  };
  // evaluate grad/Hess at theta and factor the Hessian; device status checked here
  auto eval_gh = [&]() -> qoc_status {
    if (p->timing) cudaEventRecord(p->trev[0], st);
    qoc_status s = enqueue_eval(p, p->theta, 2, p->out);
    if (s != QOC_OK) return s;
    if (tr_needs_eig(K))
      QOC_TRY(launch_eig(p->out + 1 + K, p->trzero, p->trzero, K, 1, p->trwork + 3 * K,
                         p->trwork + 2 * K, p->status, EIG_JACOBI_FP64, 0, 0.0, st, p->ws[0]));
    if (p->timing) cudaEventRecord(p->trev[1], st);
    QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), st));
    QOC_TRY(cudaStreamSynchronize(st));
    if (p->timing) p->trphase_ms[2] += elapsed(p->trev[0], p->trev[1]);
    return device_status(p);
  };
  qoc_status s = eval_gh();
  if (s != QOC_OK) return s;
  report->n_eval_gh = 1;
  double Jc = 0;
  int it = 0;
  int stop = 2;
  for (it = 1; it <= opt->max_iter; ++it) {
    if (p->timing) cudaEventRecord(p->trev[0], st);
    QOC_TRY(launch_tr_subproblem(p->out, K, radius, p->trwork, p->trstep, p->trinfo, p->status, st));
    QOC_TRY(launch_axpy(p->theta, p->trstep, K, p->theta_trial, st));
    if (p->timing) cudaEventRecord(p->trev[2], st);
    s = enqueue_eval(p, p->theta_trial, 0, p->out_trial);
    if (s != QOC_OK) return s;
    if (p->timing) cudaEventRecord(p->trev[3], st);
    QOC_TRY(cudaMemcpyAsync(hs, p->trinfo, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(hs + 4, p->out_trial, sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(hs + 5, p->out, sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), st));
    QOC_TRY(cudaStreamSynchronize(st));
    s = device_status(p);
    if (s == QOC_ETIMEOUT || s == QOC_EUNSUPPORTED) return s;
    if (p->timing) {
      p->trphase_ms[0] += elapsed(p->trev[0], p->trev[2]);
      p->trphase_ms[1] += elapsed(p->trev[2], p->trev[3]);
    }
    const double pred = hs[0], snorm = hs[1], gnorm = hs[3], Jt = hs[4];
    // a trial point whose evaluation failed numerically is a rejected step
    const bool trial_ok = s == QOC_OK && std::isfinite(Jt);
    Jc = hs[5];
    report->n_eval_J++;
    report->grad_norm = gnorm;
    if (gnorm < opt->gtol) { stop = 0; --it; report->n_eval_J--; break; }
    if (!(pred > 0) || !std::isfinite(pred)) { stop = 3; break; }
    const double rho = trial_ok ? (Jc - Jt) / pred : -1.0;
    if (rho < 0.25) radius *= 0.25;
    else if (rho > 0.75 && std::fabs(snorm - radius) <= 1e-8 * radius)
      radius = std::fmin(2.0 * radius, opt->radius_max);
    if (rho > opt->eta) {
      QOC_TRY(cudaMemcpyAsync(p->theta, p->theta_trial, 8 * (size_t)K, cudaMemcpyDeviceToDevice, st));
      p->reuse_fwd = trial_ok;   // the trial's cost evaluation left its forward part in place
      s = eval_gh();
      if (s != QOC_OK) return s;
      report->n_eval_gh++;
    }
    if (radius < opt->xtol) { stop = 1; break; }
  }
  if (it > opt->max_iter) it = opt->max_iter;
  // final state: theta, J, |grad|
  QOC_TRY(cudaMemcpyAsync(p->hbuf, p->theta, 8 * (size_t)K, cudaMemcpyDeviceToHost, st));
  QOC_TRY(cudaMemcpyAsync(hs, p->out, 8 * (1 + (size_t)K), cudaMemcpyDeviceToHost, st));
  QOC_TRY(cudaStreamSynchronize(st));
  std::memcpy(theta_out, p->hbuf, 8 * (size_t)K);
  double gn = 0;
  for (int l = 0; l < K; ++l) gn += hs[1 + l] * hs[1 + l];
  report->iters = it;
  report->J = hs[0];
  report->grad_norm = std::sqrt(gn);
  report->radius = radius;
  report->stop_reason = stop;
  p->last_order = 2;
  return stop == 2 ? QOC_ENOTCONV : QOC_OK;
}

qoc_status qoc_trust_region_solve_bfgs(qoc_problem* p, const double* theta0, const qoc_tr_options* opt,
                                       double* theta_out, qoc_tr_report* report) {
  if (!p || !theta0 || !opt || !theta_out || !report) return QOC_EINVAL;
  if (!p->trwork) return QOC_EUNSUPPORTED;
  if (!(opt->radius0 > 0) || !(opt->radius_max >= opt->radius0) || opt->max_iter < 1 ||
      !(opt->eta >= 0 && opt->eta < 0.25) || !(opt->gtol >= 0) || !(opt->xtol >= 0))
    return QOC_EINVAL;
  if (!finite_all(theta0, p->K)) return QOC_EINVAL;
  const int K = p->K;
  cudaStream_t st = p->stream;
  std::memset(report, 0, sizeof(*report));
  double radius = opt->radius0;
  // the model Hessian B sits in the Hessian slot of out (gradient-only
  // evaluations leave it alone); the trial's Hessian slot is the update's
  // scratch; trinfo[4] flags the first (scaling) update
  double* Bm = p->out + 1 + K;
  std::memcpy(p->hbuf, theta0, 8 * (size_t)K);
  QOC_TRY(cudaMemcpyAsync(p->theta, p->hbuf, 8 * (size_t)K, cudaMemcpyHostToDevice, st));
  QOC_TRY(cudaMemsetAsync(p->trinfo + 4, 0, sizeof(double), st));
  qoc_status s = enqueue_eval(p, p->theta, 1, p->out);
  if (s != QOC_OK) return s;
  QOC_TRY(launch_set_identity(Bm, K, st));
  double* hs = p->hbuf + K;
  int it = 0, stop = 2;
  for (it = 1; it <= opt->max_iter; ++it) {
    if (tr_needs_eig(K))
      QOC_TRY(launch_eig(Bm, p->trzero, p->trzero, K, 1, p->trwork + 3 * K, p->trwork + 2 * K, p->status,
                         EIG_JACOBI_FP64, 0, 0.0, st, p->ws[0]));
    QOC_TRY(launch_tr_subproblem(p->out, K, radius, p->trwork, p->trstep, p->trinfo, p->status, st));
    QOC_TRY(launch_axpy(p->theta, p->trstep, K, p->theta_trial, st));
    s = enqueue_eval(p, p->theta_trial, 1, p->out_trial);
    if (s != QOC_OK) return s;
    QOC_TRY(launch_bfgs_update(Bm, p->trstep, p->out + 1, p->out_trial + 1, K, p->trinfo + 4, 1e-8,
                               p->out_trial + 1 + K, st));
    QOC_TRY(cudaMemcpyAsync(hs, p->trinfo, 4 * sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(hs + 4, p->out_trial, sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(hs + 5, p->out, sizeof(double), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemcpyAsync(p->hstatus, p->status, sizeof(int), cudaMemcpyDeviceToHost, st));
    QOC_TRY(cudaMemsetAsync(p->status, 0, sizeof(int), st));
    QOC_TRY(cudaStreamSynchronize(st));
    s = device_status(p);
    if (s == QOC_ETIMEOUT || s == QOC_EUNSUPPORTED) return s;
    const double pred = hs[0], snorm = hs[1], gnorm = hs[3], Jt = hs[4], Jc = hs[5];
    const bool trial_ok = s == QOC_OK && std::isfinite(Jt);
    report->n_eval_J++;
    report->grad_norm = gnorm;
    if (gnorm < opt->gtol) { stop = 0; --it; report->n_eval_J--; break; }
    if (!(pred > 0) || !std::isfinite(pred)) { stop = 3; break; }
    const double rho = trial_ok ? (Jc - Jt) / pred : -1.0;
    if (rho < 0.25) radius *= 0.25;
    else if (rho > 0.75 && std::fabs(snorm - radius) <= 1e-8 * radius)
      radius = std::fmin(2.0 * radius, opt->radius_max);
    if (rho > opt->eta) {
      QOC_TRY(cudaMemcpyAsync(p->theta, p->theta_trial, 8 * (size_t)K, cudaMemcpyDeviceToDevice, st));
      QOC_TRY(cudaMemcpyAsync(p->out, p->out_trial, 8 * (1 + (size_t)K), cudaMemcpyDeviceToDevice, st));
    }
    if (radius < opt->xtol) { stop = 1; break; }
  }
  if (it > opt->max_iter) it = opt->max_iter;
  QOC_TRY(cudaMemcpyAsync(p->hbuf, p->theta, 8 * (size_t)K, cudaMemcpyDeviceToHost, st));
  QOC_TRY(cudaMemcpyAsync(hs, p->out, 8 * (1 + (size_t)K), cudaMemcpyDeviceToHost, st));
  QOC_TRY(cudaStreamSynchronize(st));
  std::memcpy(theta_out, p->hbuf, 8 * (size_t)K);
  double gn = 0;
  for (int l = 0; l < K; ++l) gn += hs[1 + l] * hs[1 + l];
  report->iters = it;
  report->J = hs[0];
  report->grad_norm = std::sqrt(gn);
  report->radius = radius;
  report->stop_reason = stop;
  report->n_eval_gh = 0;
  p->last_order = 1;
  return stop == 2 ? QOC_ENOTCONV : QOC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches of uneven problems (different N, K, J and sweep precision).  Each
// problem's parallel phases run on its own stream; the four latency-bound
// sweeps (states, costates, tangent panels, second-order adjoint panels) run
// as one launch each over all problems.  The fork/join graph of one batched
// evaluation is captured once into a CUDA graph and replayed.
// ---------------------------------------------------------------------------
struct qoc_batch {
  int n = 0;
  std::vector<qoc_problem*> P;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<cudaEvent_t> ev;         // per problem: 5 phase events; then 5 batch events
  // the four batched sweeps, each split into groups by the sweep precision
  // and the sweep kernel a single evaluation of the problem takes
  // (bsweep_variant), one launch per group: index GPS * sweep + gi with
  // gi = kSweepVariants * mixed + variant
  static constexpr int GPS = 2 * kSweepVariants;
  static constexpr int NG = 4 * GPS;
  std::vector<BSweepArgs> hargs[NG];
  std::vector<int> hoff[NG];
  BSweepArgs* dargs[NG] = {};
  int* doff[NG] = {};
  int nargs[NG] = {}, total[NG] = {};
  cudaStream_t aux[GPS] = {};              // each group's stream (0 is the batch stream)
  cudaEvent_t fork[4] = {};                // per sweep: fork of the groups
  cudaEvent_t gjoin[NG] = {};              // per group: its join
  std::vector<size_t> toff, ooff;
  std::vector<char> split;             // per problem: split second-order adjoint (at creation)
  size_t ntheta = 0, nout = 0;
  double *theta = nullptr, *out = nullptr, *hbuf = nullptr;
  int* hstat = nullptr;
  int use_graph = 1;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

// one phase of problem i of the batch on stream s (see the header comment)
qoc_status batch_phase(qoc_batch* b, int i, int phase, cudaStream_t s) {
  qoc_problem* p = b->P[i];
  const int N = p->N, K = p->K, J = p->J, bs = p->bs, mixed = p->precision == QOC_MIXED_FP32 ? 1 : 0;
  double* out = b->out + b->ooff[i];
  const void* Bsrc = mixed ? static_cast<const void*>(p->Bf) : static_cast<const void*>(p->B);
  switch (phase) {
    case 0:
      QOC_TRY(cudaMemcpyAsync(p->theta, b->theta + b->toff[i], 8 * (size_t)K, cudaMemcpyDeviceToDevice, s));
      QOC_TRY(launch_control(p->B, p->Kp, p->theta, J, K, p->f, s));
      QOC_TRY(launch_eig(p->H0, p->M, p->f, N, J, p->W, p->eig, p->status,
                         p->eig_method == QOC_EIG_JACOBI_FP64 ? EIG_JACOBI_FP64 : EIG_REFINED,
                         p->refine_sweeps, p->angle_tol, s, p->ws[0], nullptr, nullptr, eig_finish_tol(p),
                         EIG_PHASE_ALL, p->eigorder));
      QOC_TRY(launch_prep(p->W, p->eig, p->M, N, J, p->dt, p->mshift, p->D, p->dstride, mixed ? 0 : 1,
                          PREP_D | PREP_P | PREP_X, p->Ptil, p->Xp, nullptr, p->status, s, p->ws[0]));
      QOC_TRY(launch_block_delta(p->D, p->dstride, N, J, bs, 0, mixed, p->Mf, p->mstride, s, p->ws[0]));
      QOC_TRY(launch_block_delta(p->D, p->dstride, N, J, bs, 1, mixed, p->Mb, p->mstride, s, p->ws[0]));
      return QOC_OK;
    case 1: {
      QOC_TRY(launch_block_fill(p->D, p->dstride, N, J, bs, 0, mixed, p->Xa, p->a_hat, s));
      const double thetaJ = (double)J * p->dt * p->mshift;
      QOC_TRY(launch_terminal(p->f, J, p->a_hat, mixed, p->beta, N, cexpi_h(thetaJ), p->w_f, p->w_t,
                              p->lamJ, p->scal + 0, p->scal + 1, s));
      QOC_TRY(cudaMemcpyAsync(out, p->scal, sizeof(double), cudaMemcpyDeviceToDevice, s));
      return QOC_OK;
    }
    case 2:
      QOC_TRY(launch_block_fill(p->D, p->dstride, N, J, bs, 1, mixed, p->Xl, p->l_hat, s));
      QOC_TRY(launch_pointwise(p->W, p->Ptil, p->Xp, p->a_hat, p->l_hat, mixed, N, J,
                               cexpi_h(p->dt * p->mshift), p->p_hat, p->y_hat, p->g, p->c, PW_P | PW_Y | PW_C, s, p->ws[0]));
      QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 0, mixed, p->p_hat, p->y_hat, p->vstride,
                               p->Qf, p->Wf, p->Gf, p->qstride, p->gstride, BS_Q | BS_WG, s, p->ws[0]));
      return QOC_OK;
    case 3:
      QOC_TRY(launch_block_contract(p->XS, p->Wf, p->Gf, p->qstride, p->gstride, Bsrc, p->Kp, N, K, J,
                                    bs, 0, mixed, p->U, s));
      if (p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT)
        QOC_TRY(launch_block_src(p->D, p->dstride, N, J, bs, 1, mixed, p->y_hat, p->p_hat, p->vstride,
                                 p->Qb, p->Wb, p->Gb, p->qstride, p->gstride, BS_Q | BS_WG, s, p->ws[0]));
      return QOC_OK;
    default:
      if (p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT)
        QOC_TRY(launch_block_contract(p->Xmu, p->Wb, p->Gb, p->qstride, p->gstride, Bsrc, p->Kp, N, K,
                                      J, bs, 1, mixed, p->V, s));
      QOC_TRY(launch_assemble(p->B, p->Kp, p->f, p->g, p->c, p->V, p->U, mixed, p->SJ, N, J, K,
                              p->w_f, p->w_t,
                              p->hess_method == QOC_HESS_SECOND_ORDER_ADJOINT ? (b->split[i] ? 2 : 0) : 1,
                              1, p->work, out, p->hess_raw, p->scal + 2, s, p->identity_basis));
      return QOC_OK;
  }
}

// the whole batched evaluation, enqueued on b->st with forks to the problems' streams
qoc_status enqueue_batch(qoc_batch* b) {
  const int n = b->n;
  cudaEvent_t* bev = b->ev.data() + 5 * (size_t)n;
  QOC_TRY(cudaEventRecord(bev[0], b->st));
  for (int phase = 0; phase < 5; ++phase) {
    // fork: every problem stream waits for the batch stream, runs its phase
    for (int i = 0; i < n; ++i) {
      cudaStream_t s = b->P[i]->stream;
      QOC_TRY(cudaStreamWaitEvent(s, bev[phase], 0));
      qoc_status r = batch_phase(b, i, phase, s);
      if (r != QOC_OK) return r;
      QOC_TRY(cudaEventRecord(b->ev[5 * (size_t)i + phase], s));
    }
    // join, then the batched sweep of this stage
    for (int i = 0; i < n; ++i) QOC_TRY(cudaStreamWaitEvent(b->st, b->ev[5 * (size_t)i + phase], 0));
    if (phase < 4) {
      // one launch per kernel group, the groups side by side on their streams
      const int g0 = qoc_batch::GPS * phase;
      bool forked = false;
      for (int v = 0; v < qoc_batch::GPS; ++v) {
        const int g = g0 + v;
        if (!b->nargs[g]) continue;
        cudaStream_t s = b->st;
        if (v > 0) {
          if (!forked) {
            QOC_TRY(cudaEventRecord(b->fork[phase], b->st));
            forked = true;
          }
          s = b->aux[v];
          QOC_TRY(cudaStreamWaitEvent(s, b->fork[phase], 0));
        }
        QOC_TRY(launch_bsweep_batch(b->hargs[g].data(), b->dargs[g], b->doff[g], b->nargs[g],
                                    b->total[g], v >= kSweepVariants ? 1 : 0, s));
        if (v > 0) QOC_TRY(cudaEventRecord(b->gjoin[g], s));
      }
      for (int v = 1; v < qoc_batch::GPS; ++v)
        if (b->nargs[g0 + v]) QOC_TRY(cudaStreamWaitEvent(b->st, b->gjoin[g0 + v], 0));
      QOC_TRY(cudaEventRecord(bev[phase + 1], b->st));
    }
  }
  return QOC_OK;
}

}  // namespace

extern "C" {

void qoc_batch_destroy(qoc_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto a : b->aux)
    if (a) cudaStreamSynchronize(a);
  for (auto e : b->ev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k < qoc_batch::NG; ++k) {
    cudaFree(b->dargs[k]);
    cudaFree(b->doff[k]);
    if (b->gjoin[k]) cudaEventDestroy(b->gjoin[k]);
  }
  for (auto e : b->fork)
    if (e) cudaEventDestroy(e);
  for (auto a : b->aux)
    if (a) cudaStreamDestroy(a);
  cudaFree(b->theta);
  cudaFree(b->out);
  if (b->hbuf) cudaFreeHost(b->hbuf);
  if (b->hstat) cudaFreeHost(b->hstat);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  delete b;
}

qoc_status qoc_batch_create(qoc_problem* const* problems, int n, void* cuda_stream, qoc_batch** out) {
  if (!out || !problems || n < 1) return QOC_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    if (!problems[i]) return QOC_EINVAL;
    if (problems[i]->bs < 2) return QOC_EUNSUPPORTED;
    for (int k = 0; k < i; ++k)
      if (problems[k] == problems[i]) return QOC_EINVAL;
  }
  qoc_batch* b = new (std::nothrow) qoc_batch();
  if (!b) return QOC_ENOMEM;
  b->n = n;
  b->P.assign(problems, problems + n);
  cudaError_t e;
  auto fail = [&](cudaError_t err) { qoc_batch_destroy(b); return from_cuda(err, __LINE__); };
  if (cuda_stream) b->st = (cudaStream_t)cuda_stream;
  else {
    if ((e = cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    b->own_stream = true;
  }
  b->ev.assign(5 * (size_t)n + 5, nullptr);
  for (auto& ev : b->ev)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  for (auto& ev : b->gjoin)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  for (auto& ev : b->fork)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e);
  for (int v = 1; v < qoc_batch::GPS; ++v)
    if ((e = cudaStreamCreateWithFlags(&b->aux[v], cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
  for (int i = 0; i < n; ++i) {
    qoc_problem* p = problems[i];
    b->toff.push_back(b->ntheta);
    b->ooff.push_back(b->nout);
    b->ntheta += p->K;
    b->nout += 1 + (size_t)p->K + (size_t)p->K * p->K;
    // descriptor lists of the four batched sweeps
    const bool split = mu_split_on(p);
    b->split.push_back(split ? 1 : 0);
    BSweepArgs args[4] = {chain_sweep_args(p, 0), chain_sweep_args(p, 1), panel_sweep_args(p, 0),
                           panel_sweep_args(p, 1, split)};
    for (int k = 0; k < 4; ++k) {
      if (k == 3 && p->hess_method != QOC_HESS_SECOND_ORDER_ADJOINT) continue;
      const int mx = p->precision == QOC_MIXED_FP32 ? 1 : 0;
      const int g = qoc_batch::GPS * k + kSweepVariants * mx + bsweep_variant(args[k], mx);
      b->hoff[g].push_back(b->total[g]);
      b->hargs[g].push_back(args[k]);
      b->total[g] += (args[k].K + args[k].kc - 1) / args[k].kc;
    }
  }
  for (int k = 0; k < qoc_batch::NG; ++k) {
    b->nargs[k] = (int)b->hargs[k].size();
    b->hoff[k].push_back(b->total[k]);
    if (!b->nargs[k]) continue;
    if ((e = cudaMalloc(&b->dargs[k], sizeof(BSweepArgs) * b->nargs[k])) != cudaSuccess) return fail(e);
    if ((e = cudaMalloc(&b->doff[k], sizeof(int) * (b->nargs[k] + 1))) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(b->dargs[k], b->hargs[k].data(), sizeof(BSweepArgs) * b->nargs[k],
                        cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
    if ((e = cudaMemcpy(b->doff[k], b->hoff[k].data(), sizeof(int) * (b->nargs[k] + 1),
                        cudaMemcpyHostToDevice)) != cudaSuccess) return fail(e);
  }
  if ((e = cudaMalloc(&b->theta, 8 * b->ntheta)) != cudaSuccess) return fail(e);
  if ((e = cudaMalloc(&b->out, 8 * b->nout)) != cudaSuccess) return fail(e);
  if ((e = cudaMallocHost(&b->hbuf, 8 * (b->ntheta + b->nout))) != cudaSuccess) return fail(e);
  if ((e = cudaMallocHost(&b->hstat, sizeof(int) * n)) != cudaSuccess) return fail(e);
  *out = b;
  return QOC_OK;
}

qoc_status qoc_batch_set_graph(qoc_batch* b, int on) {
  if (!b) return QOC_EINVAL;
  b->use_graph = on ? 1 : 0;
  return QOC_OK;
}

qoc_status qoc_batch_eval_grad_hess_dev(qoc_batch* b, const double* thetas_dev, double* outs_dev) {
  if (!b || !thetas_dev || !outs_dev) return QOC_EINVAL;
  if (thetas_dev != b->theta)
    QOC_TRY(cudaMemcpyAsync(b->theta, thetas_dev, 8 * b->ntheta, cudaMemcpyDeviceToDevice, b->st));
  if (b->use_graph && b->exec) {
    QOC_TRY(cudaGraphLaunch(b->exec, b->st));
  } else {
    // the first call runs eagerly (one-time kernel attribute set-up happens
    // outside any capture), then records the same work as a graph for replay
    qoc_status r = enqueue_batch(b);
    if (r != QOC_OK) return r;
    if (b->use_graph) {
      QOC_TRY(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal));
      r = enqueue_batch(b);
      cudaGraph_t g = nullptr;
      cudaError_t ec = cudaStreamEndCapture(b->st, &g);
      if (r != QOC_OK) {
        if (g) cudaGraphDestroy(g);
        return r;
      }
      QOC_TRY(ec);
      b->graph = g;
      QOC_TRY(cudaGraphInstantiate(&b->exec, b->graph, 0));
    }
  }
  if (outs_dev != b->out)
    QOC_TRY(cudaMemcpyAsync(outs_dev, b->out, 8 * b->nout, cudaMemcpyDeviceToDevice, b->st));
  for (qoc_problem* p : b->P) p->last_order = 2;
  return QOC_OK;
}

qoc_status qoc_batch_eval_grad_hess(qoc_batch* b, const double* thetas, double* outs) {
  if (!b || !thetas || !outs) return QOC_EINVAL;
  if (!finite_all(thetas, b->ntheta)) return QOC_EINVAL;
  std::memcpy(b->hbuf, thetas, 8 * b->ntheta);
  QOC_TRY(cudaMemcpyAsync(b->theta, b->hbuf, 8 * b->ntheta, cudaMemcpyHostToDevice, b->st));
  qoc_status r = qoc_batch_eval_grad_hess_dev(b, b->theta, b->out);
  if (r != QOC_OK) return r;
  QOC_TRY(cudaMemcpyAsync(b->hbuf + b->ntheta, b->out, 8 * b->nout, cudaMemcpyDeviceToHost, b->st));
  for (int i = 0; i < b->n; ++i) {
    QOC_TRY(cudaMemcpyAsync(b->hstat + i, b->P[i]->status, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    QOC_TRY(cudaMemsetAsync(b->P[i]->status, 0, sizeof(int), b->st));
  }
  QOC_TRY(cudaStreamSynchronize(b->st));
  std::memcpy(outs, b->hbuf + b->ntheta, 8 * b->nout);
  for (int i = 0; i < b->n; ++i) {
    if (b->hstat[i] == 0) continue;
    *b->P[i]->hstatus = b->hstat[i];
    return device_status(b->P[i]);
  }
  if (!finite_all(outs, b->nout)) return QOC_ENUMERIC;
  return QOC_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched trust region: every problem runs the basic trust region of
// qoc_trust_region_solve, all of them advancing together.  One iteration is
// enqueued as: propose (device: gtol test, exact subproblem, trial point) ->
// one batched gradient + Hessian evaluation of every trial point (the batch's
// CUDA graph) -> eigendecomposition of each trial Hessian -> update (device:
// ratio test, radius, acceptance, xtol and iteration cap).  The host then
// reads the per-problem state once for the whole batch and, when problems
// have stopped, rebuilds the batch over those still running.
// ---------------------------------------------------------------------------
namespace {

struct TrBatchRun {
  std::vector<qoc_problem*> P;
  std::vector<TrSlot> slot;              // host copy of every problem's state
  std::vector<int> act;                  // indices of the problems in the current batch
  TrSlot* dslots = nullptr;              // device slots of the current batch
  double* etrial = nullptr;              // per problem [d (K) | Q (K*K)] of its trial Hessian
  double* thcur = nullptr;               // per problem its current point (K); the batched
                                         // evaluation copies each trial point into the
                                         // problem's own theta buffer, so that one cannot hold it
  std::vector<size_t> eoff, toff;
  qoc_batch* b = nullptr;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  ~TrBatchRun() {
    if (st) cudaStreamSynchronize(st);
    if (b) qoc_batch_destroy(b);
    cudaFree(dslots);
    cudaFree(etrial);
    cudaFree(thcur);
    if (own_stream && st) cudaStreamDestroy(st);
  }
};

// (re)build the batch over run.act and upload its slots
qoc_status tr_rebuild(TrBatchRun& run) {
  if (run.b) {
    QOC_TRY(cudaStreamSynchronize(run.st));
    qoc_batch_destroy(run.b);
    run.b = nullptr;
  }
  std::vector<qoc_problem*> ps;
  for (int i : run.act) ps.push_back(run.P[i]);
  qoc_status s = qoc_batch_create(ps.data(), (int)ps.size(), run.st, &run.b);
  if (s != QOC_OK) return s;
  std::vector<TrSlot> dev(run.act.size());
  for (size_t k = 0; k < run.act.size(); ++k) {
    TrSlot& t = run.slot[run.act[k]];
    t.theta_trial = run.b->theta + run.b->toff[k];
    t.gh_trial = run.b->out + run.b->ooff[k];
    dev[k] = t;
  }
  QOC_TRY(cudaMemcpyAsync(run.dslots, dev.data(), sizeof(TrSlot) * dev.size(), cudaMemcpyHostToDevice,
                          run.st));
  return QOC_OK;
}

// evaluate the current batch at its trial points and factor each trial Hessian
qoc_status tr_eval_trials(TrBatchRun& run) {
  qoc_status s = qoc_batch_eval_grad_hess_dev(run.b, run.b->theta, run.b->out);
  if (s != QOC_OK) return s;
  for (size_t k = 0; k < run.act.size(); ++k) {
    qoc_problem* p = run.P[run.act[k]];
    const int K = p->K;
    if (!tr_needs_eig(K)) continue;   // the subproblem reduces the Hessian itself
    double* e = run.etrial + run.eoff[run.act[k]];
    QOC_TRY(launch_eig(run.b->out + run.b->ooff[k] + 1 + K, p->trzero, p->trzero, K, 1, e + K, e,
                       p->status, EIG_JACOBI_FP64, 0, 0.0, run.st, p->ws[0]));
  }
  return QOC_OK;
}

// read the batch's slots back into run.slot (synchronises)
qoc_status tr_pull(TrBatchRun& run) {
  std::vector<TrSlot> dev(run.act.size());
  QOC_TRY(cudaMemcpyAsync(dev.data(), run.dslots, sizeof(TrSlot) * dev.size(), cudaMemcpyDeviceToHost,
                          run.st));
  QOC_TRY(cudaStreamSynchronize(run.st));
  for (size_t k = 0; k < run.act.size(); ++k) run.slot[run.act[k]] = dev[k];
  return QOC_OK;
}

}  // namespace

extern "C" qoc_status qoc_batch_trust_region_solve(qoc_problem* const* problems, int n,
                                                   const double* theta0s, const qoc_tr_options* opt,
                                                   double* theta_out, qoc_tr_report* reports,
                                                   void* cuda_stream) {
  if (!problems || n < 1 || !theta0s || !opt || !theta_out || !reports) return QOC_EINVAL;
  if (!(opt->radius0 > 0) || !(opt->radius_max >= opt->radius0) || opt->max_iter < 1 ||
      !(opt->eta >= 0 && opt->eta < 0.25) || !(opt->gtol >= 0) || !(opt->xtol >= 0))
    return QOC_EINVAL;
  size_t ntheta = 0;
  for (int i = 0; i < n; ++i) {
    qoc_problem* p = problems[i];
    if (!p) return QOC_EINVAL;
    for (int k = 0; k < i; ++k)
      if (problems[k] == p) return QOC_EINVAL;
    if (!p->trwork || p->bs < 2) return QOC_EUNSUPPORTED;
    ntheta += p->K;
  }
  if (!finite_all(theta0s, ntheta)) return QOC_EINVAL;
  TrBatchRun run;
  run.P.assign(problems, problems + n);
  if (cuda_stream) run.st = static_cast<cudaStream_t>(cuda_stream);
  else {
    QOC_TRY(cudaStreamCreateWithFlags(&run.st, cudaStreamNonBlocking));
    run.own_stream = true;
  }
  size_t ne = 0, nt = 0;
  run.slot.resize(n);
  for (int i = 0; i < n; ++i) {
    qoc_problem* p = run.P[i];
    run.eoff.push_back(ne);
    run.toff.push_back(nt);
    ne += (size_t)p->K + (size_t)p->K * p->K;
    nt += (size_t)p->K;
    TrSlot& t = run.slot[i];
    std::memset(&t, 0, sizeof(t));
    t.K = p->K; t.gh = p->out; t.work = p->trwork; t.step = p->trstep; t.info = p->trinfo;
    t.status = p->status; t.active = 1;
    run.act.push_back(i);
  }
  QOC_TRY(cudaMalloc(&run.dslots, sizeof(TrSlot) * n));
  QOC_TRY(cudaMalloc(&run.etrial, 8 * ne));
  QOC_TRY(cudaMalloc(&run.thcur, 8 * nt));
  for (int i = 0; i < n; ++i) {
    run.slot[i].eig_trial = run.etrial + run.eoff[i];
    run.slot[i].theta = run.thcur + run.toff[i];
  }
  TrBatchOptions o{opt->gtol, opt->xtol, opt->radius0, opt->radius_max, opt->eta, opt->max_iter};
  for (int i = 0; i < n; ++i) o.kmax = run.P[i]->K > o.kmax ? run.P[i]->K : o.kmax;
  qoc_status s = tr_rebuild(run);
  if (s != QOC_OK) return s;
  // initial point: theta0 into the trial slots, evaluated and taken as current
  {
    std::vector<double> th(run.b->ntheta);
    std::memcpy(th.data(), theta0s, 8 * ntheta);
    QOC_TRY(cudaMemcpyAsync(run.b->theta, th.data(), 8 * ntheta, cudaMemcpyHostToDevice, run.st));
    for (int i = 0; i < n; ++i) QOC_TRY(cudaMemsetAsync(run.P[i]->status, 0, sizeof(int), run.st));
    if ((s = tr_eval_trials(run)) != QOC_OK) return s;
    QOC_TRY(launch_tr_batch(0, run.dslots, n, 0, o, run.st));
    if ((s = tr_pull(run)) != QOC_OK) return s;
  }
  for (int it = 1; it <= opt->max_iter; ++it) {
    std::vector<int> still;
    for (int i : run.act)
      if (run.slot[i].active) still.push_back(i);
    if (still.empty()) break;
    if (still.size() != run.act.size()) {
      run.act = still;
      if ((s = tr_rebuild(run)) != QOC_OK) return s;
    }
    const int na = (int)run.act.size();
    QOC_TRY(launch_tr_batch(1, run.dslots, na, it, o, run.st));
    if ((s = tr_eval_trials(run)) != QOC_OK) return s;
    QOC_TRY(launch_tr_batch(2, run.dslots, na, it, o, run.st));
    if ((s = tr_pull(run)) != QOC_OK) return s;
  }
  // results: theta, J and |grad| of the final iterates; status words of
  // problems evaluated after they stopped are cleared
  for (int i = 0; i < n; ++i) QOC_TRY(cudaMemsetAsync(run.P[i]->status, 0, sizeof(int), run.st));
  QOC_TRY(cudaStreamSynchronize(run.st));
  qoc_status worst = QOC_OK;
  size_t off = 0;
  for (int i = 0; i < n; ++i) {
    qoc_problem* p = run.P[i];
    const int K = p->K;
    std::vector<double> gh(1 + (size_t)K);
    QOC_TRY(cudaMemcpy(theta_out + off, run.thcur + run.toff[i], 8 * (size_t)K, cudaMemcpyDeviceToHost));
    QOC_TRY(cudaMemcpy(p->theta, run.thcur + run.toff[i], 8 * (size_t)K, cudaMemcpyDeviceToDevice));
    QOC_TRY(cudaMemcpy(gh.data(), p->out, 8 * (1 + (size_t)K), cudaMemcpyDeviceToHost));
    off += K;
    const TrSlot& t = run.slot[i];
    double gn = 0;
    for (int l = 0; l < K; ++l) gn += gh[1 + l] * gh[1 + l];
    qoc_tr_report& r = reports[i];
    std::memset(&r, 0, sizeof(r));
    r.iters = t.iters; r.n_eval_J = t.n_eval_J; r.n_eval_gh = t.n_eval_gh;
    r.J = gh[0]; r.grad_norm = std::sqrt(gn); r.radius = t.radius; r.stop_reason = t.stop;
    p->last_order = 2;
    if (t.stop == 4) {
      *p->hstatus = t.fail;
      qoc_status e = device_status(p);
      if (e == QOC_OK) e = QOC_ENUMERIC;
      if (worst == QOC_OK || worst == QOC_ENOTCONV) worst = e;
    } else if (t.stop == 2 && worst == QOC_OK) {
      worst = QOC_ENOTCONV;
    }
  }
  return worst;
}
