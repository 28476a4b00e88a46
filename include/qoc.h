/*
 * qoc.h -- C ABI of the GB300 (sm_103a) library for the exact gradient and
 * Hessian of the discrete quantum-optimal-control cost by the first- and
 * second-order adjoint method (H. S. Bhat, "Second-Order Adjoint Method for
 * Quantum Optimal Control", arXiv 2505.00529).
 *
 * The problem (Sec. II, Eqs. Zdef, discTDSE, discretecost, with weights):
 *
 *   f   = B theta                       (linear control model, f_j = f(j dt))
 *   H_j = H0 + f_j M,   U_j = exp(-i dt H_j),   a_{j+1} = U_j a_j,  a_0 = alpha
 *   J(theta) = w_ctrl * sum_j f_j^2 + w_term * |a_J - beta|^2
 *
 * The paper's cost is w_ctrl = 1/2, w_term = rho/2.  The library computes
 * J, dJ/dtheta (first-order adjoint, Eqs. lambdasys, dLdf; Alg. 1) and the
 * full K x K Hessian (second-order adjoint, Eqs. musys, gradatheta, d2Ldf2;
 * Alg. 2), and runs an exact-Hessian trust-region iteration on top of them
 * (Sec. IV-B).  Every step of an evaluation runs in CUDA kernels on the
 * device; the host only validates arguments, moves theta in and the results
 * out, and sequences launches.
 *
 * Conventions for every entry point:
 *   - All floating point arguments are IEEE binary64 (double).
 *   - Matrices are row-major.  Complex vectors are interleaved (re, im):
 *     a complex vector of length N is 2N doubles.
 *   - Host pointers are read during the call only; the caller keeps
 *     ownership.  Output buffers are caller-allocated.
 *   - Entry points with the suffix _dev take DEVICE pointers, enqueue work on
 *     the problem's stream and return without synchronising.
 *   - Errors are returned as qoc_status, never thrown; the library never
 *     exits the process and never traps on the device.  After QOC_ECUDA the
 *     CUDA context may be unusable.
 *   - A problem object is not thread-safe: calls on one problem must not
 *     overlap.  Distinct problems may be used from distinct threads.
 */
#ifndef QOC_H
#define QOC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qoc_problem qoc_problem; /* opaque; owns all of its device memory */

typedef enum {
  QOC_OK = 0,
  QOC_EINVAL = 1,       /* bad argument: null pointer, size out of range, non-symmetric H0/M, ... */
  QOC_ENOMEM = 2,       /* device or host allocation failed */
  QOC_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  QOC_ENUMERIC = 4,     /* non-finite input/output or an eigensolver that did not converge */
  QOC_ENOTCONV = 5,     /* trust region hit max_iter (best iterate still returned) */
  QOC_ETIMEOUT = 6,     /* a bounded device wait gave up (kernel returned early) */
  QOC_EUNSUPPORTED = 7  /* valid request this build does not implement (e.g. N too large) */
} qoc_status;

/* Arithmetic of the per-step propagator products (the time-stepped sweeps).
 *   QOC_FP64       : every operation in binary64 ("plain FP64").
 *   QOC_MIXED_FP32 : mixed precision held to a relative error of 1e-6 in J,
 *                    the gradient and the Hessian.  The propagator-times-panel
 *                    products run in binary32 on the increment
 *                    D_j = exp(-i dt (H_j - m)) - I with the state carried as
 *                    an unevaluated float pair, while the eigendecomposition,
 *                    divided differences, contractions and the gradient /
 *                    Hessian accumulation stay binary64 -- unless the a priori
 *                    estimate of the binary32 rounding error (below) exceeds
 *                    1e-6, in which case the sweeps run in binary64 as with
 *                    QOC_FP64.  qoc_get_precision reports which was chosen.
 *   QOC_MIXED_FP32_ALWAYS : binary32 increments whatever the estimate (the
 *                    error then follows the estimate and may exceed 1e-6).
 *
 * The binary32 rounding of the increments accumulates like a random walk
 * over the J steps and the N-term sums of every product, so the relative
 * error of the Hessian (the most sensitive result) is estimated as
 *     err = 0.3 eps32 dt sigma sqrt(J N b),   eps32 = 2^-24,
 * b the time-block length (qoc_set_block_steps) and sigma the rms spread of
 * the spectra of H_j - m for theta ~ N(0, I) (the random start of Sec. IV-A):
 *     sigma^2 = ( |H0 - m I|_F^2 + |M|_F^2 mean_j |b_j|^2 ) / N,
 * with m = tr(H0)/N and b_j the rows of the basis.  The constant 0.3 is the
 * measured one (0.24 at N = 32, J = 4000; 0.28 at N = 256, J = 10^4, block
 * lengths 1 to 8).  The choice is made at qoc_create_problem with the default
 * block length. */
typedef enum { QOC_FP64 = 0, QOC_MIXED_FP32 = 1, QOC_MIXED_FP32_ALWAYS = 2 } qoc_precision;

/* Which exact form of the Hessian to assemble (both are Eq. d2Ldf2):
 *   QOC_HESS_SECOND_ORDER_ADJOINT : Alg. 2 -- forward tangent panel S_j and
 *       backward second-order adjoint panel mu_j,
 *       Hess = B^T diag(2w+c) B + B^T V + B^T U.
 *   QOC_HESS_TANGENT : the mu recursion unrolled (no backward panel),
 *       Hess = B^T diag(2w+c) B + 2 w_term Re(S_J^H S_J) + B^T U + U^T B. */
typedef enum { QOC_HESS_SECOND_ORDER_ADJOINT = 0, QOC_HESS_TANGENT = 1 } qoc_hess_method;

/* Eigensolver for the per-step H_j (Alg. 2 first loop).
 *   QOC_EIG_REFINED      : binary32 cyclic Jacobi followed by binary64
 *                          Ogita-Aishima refinement sweeps (default).
 *   QOC_EIG_JACOBI_FP64  : binary64 cyclic Jacobi throughout. */
typedef enum { QOC_EIG_REFINED = 0, QOC_EIG_JACOBI_FP64 = 1 } qoc_eig_method;

/* Create a problem.  Sec. II / Eq. discretecost.
 *   N          basis size, 1 <= N <= qoc_max_basis_size().
 *   H0, M      N*N real symmetric (checked to 1e-12 relative), row-major.
 *   a0, a_target  N complex, interleaved (2N doubles): alpha and beta.
 *   K          number of control coefficients (>= 1).
 *   basis      steps*K row-major: basis[j*K + l] = d f_j / d theta_l.
 *   dt         time step (> 0); steps = J >= 1 (T = J dt).
 *   w_ctrl, w_term  cost weights (>= 0).
 *   precision  a qoc_precision value.
 *   cuda_stream  cudaStream_t to run on, or NULL for a library-owned stream.
 *   out        receives the new problem.
 * Device memory for every intermediate (O(J N^2)) is allocated here; no later
 * call allocates. */
qoc_status qoc_create_problem(int N, const double* H0, const double* M,
                              const double* a0, const double* a_target,
                              int K, const double* basis, double dt, int steps,
                              double w_ctrl, double w_term, int precision,
                              void* cuda_stream, qoc_problem** out);

/* Select the Hessian form (qoc_hess_method) / eigensolver (qoc_eig_method). */
qoc_status qoc_set_hess_method(qoc_problem* p, int method);
qoc_status qoc_set_eig_method(qoc_problem* p, int method);

/* Time blocking of the sequential sweeps (no counterpart in the paper; an
 * exact regrouping of Alg. 2's loops): `steps` consecutive time steps are
 * folded into one dependent step X <- (I + Delta) X + Q B_blk, with the
 * block propagators, propagated sources and the contractions at the
 * intermediate steps computed in parallel over blocks.  1 <= steps <= 8;
 * 1 selects one dependent step per time step.  Default when J >= 16: 8 for
 * binary64 sweeps, 4 for binary32 ones (the binary32 rounding of the block
 * propagator grows like sqrt(steps)); 1 when J < 16.  QOC_EINVAL otherwise,
 * and for a QOC_MIXED_FP32 problem on binary32 sweeps when the new length
 * would raise the error estimate above 1e-6. */
qoc_status qoc_set_block_steps(qoc_problem* p, int steps);

/* Forward pipeline of a time-blocked evaluation (no
 * counterpart in the paper; a reordering of Alg. 2's first loops that
 * changes no result): after the binary32 eigensolver start over all steps,
 * the binary64 refinement and the increments D_j run in `chunks` chunks of
 * whole time blocks, and the forward state sweep follows chunk by chunk on
 * its own stream, resuming each chunk from the block-start state the
 * previous one stored, so that its dependent steps overlap the refinement of
 * the later chunks.  Results are bit-identical to the unchunked schedule.
 * chunks: 0 or 1 off, 2..8 the chunk count (at most one block each), -1 the
 * built-in choice, off: at N = 32, J = 4000 four chunks measured 4.20 ms per
 * gradient + Hessian evaluation against 3.94 ms unchunked (the chunked
 * refinement's part-empty waves and the SMs the chain shares cost more than
 * the chain's overlap gains).  QOC_EINVAL otherwise. */
qoc_status qoc_set_pipeline(qoc_problem* p, int chunks);

/* Terminal part of the second-order adjoint in closed form (Sec. III-B,
 * Eq. musys with its terminal condition mu_J = 2 w_t S_J; a regrouping of
 * Alg. 2's Hessian sum that changes no result beyond rounding).  The mu
 * recursion is linear, so mu = mu0 + mu_T: mu0 from the sources y_j with
 * mu0_J = 0, mu_T the terminal value carried back by the adjoint propagators
 * alone.  The contraction of mu_T with the tangent sources telescopes to
 * Re(S_J^H mu_J), so the Hessian is
 *   B^T diag(2 w_f + c) B + B^T V0 + 2 w_t Re(S_J^H S_J) + B^T U
 * with V0 from mu0, and the mu sweep no longer waits for the tangent sweep:
 * on the three-stream schedule (time blocking, Hessian requested) the two
 * panels run side by side.
 *   split  1 on: QOC_BUF_V then holds the contraction of mu0;
 *          0 off: mu starts from mu_J = 2 w_t S_J and QOC_BUF_V holds the full
 *          contraction;
 *          -1 (default) the built-in choice: on for binary64 sweeps, off for
 *          binary32 ones.  Binary32 sweeps round in proportion to the swept
 *          values, and mu0 can exceed mu where the Hessian is a small
 *          difference of large terms: on the batched workload's avoided
 *          crossing (N = 48, K = 32, J = 4000) the split measured a Hessian
 *          error of 1.22e-6 against 7.6e-7 unsplit, while saving 0.18 ms of
 *          2.91 at N = 32, K = 64, J = 4000.
 *          Other values: QOC_EINVAL.
 * Takes effect at the next evaluation; a batch takes each problem's setting
 * when it is created (qoc_batch_create).  The per-step (block steps 1)
 * schedule and the tangent form are unaffected. */
qoc_status qoc_set_mu_split(qoc_problem* p, int split);

/* Panel columns per CTA of the tangent and second-order adjoint sweeps
 * (1, 2 or 4; 0 restores the built-in choice, 1).  A launch-shape knob; the
 * autotuner in the Python package picks it together with the block steps.
 * It leaves the arithmetic unchanged except for binary32 panels with
 * 32 < N <= 64 whose CTA exceeds the warp-specialised sweep's thread cap
 * (32 (ceil(N/8) kc + 1) > 384): those run the general sweep, whose sums are
 * ordered differently (results agree to rounding).
 * QOC_EUNSUPPORTED when 32 ceil(N/8) kc > 1024 threads. */
qoc_status qoc_set_panel_columns(qoc_problem* p, int kc);

/* Cap on the binary64 refinement updates per step of the eigensolver
 * (QOC_EIG_REFINED; 0 <= sweeps <= 16; default 4 for N <= 64, 8 above).  A
 * step whose refinement has not reached its tolerance within the cap marks
 * the evaluation's device status "eigensolver not converged", which the call
 * returns as QOC_ENUMERIC (the results are then not to be used).  Takes effect
 * for evaluations enqueued after the call; a batch keeps the value captured
 * when it was built.  QOC_EINVAL outside the range. */
qoc_status qoc_set_refine_sweeps(qoc_problem* p, int sweeps);

/* Failure-detection self-test.  Runs the library's bounded device wait (the
 * one every sweep uses on its shared-memory ring) on an mbarrier that nothing
 * completes and with no copy in flight, giving up after limit_ns nanoseconds
 * (1e3 <= limit_ns <= 1e10), on the problem's stream; then synchronises the
 * stream and returns what the status check reports: QOC_ETIMEOUT when the
 * wait gave up and the kernel returned, as any evaluation whose wait ran out
 * would.  The device status is cleared and the problem stays usable.
 * QOC_EINVAL for a limit outside the range. */
qoc_status qoc_selftest_bounded_wait(qoc_problem* p, unsigned long long limit_ns);

/* The arithmetic a problem's sweeps use (*effective: QOC_FP64 or
 * QOC_MIXED_FP32) and the estimated relative error of binary32 increments
 * at the current block length (*estimate, see qoc_precision; computed for
 * every precision).  Either pointer may be NULL. */
qoc_status qoc_get_precision(const qoc_problem* p, int* effective, double* estimate);

/* Replace the target state beta (N complex, interleaved host doubles). */
qoc_status qoc_set_target(qoc_problem* p, const double* a_target);

/* J(theta), Eq. discretecost.  theta: K host doubles.  J: one host double. */
qoc_status qoc_eval_J(qoc_problem* p, const double* theta, double* J);

/* J and dJ/dtheta (K host doubles), Eqs. lambdasys and dLdf (Alg. 1). */
qoc_status qoc_eval_grad(qoc_problem* p, const double* theta, double* J, double* grad);

/* J, gradient and the symmetrised K*K row-major Hessian (Alg. 2, Eq. d2Ldf2). */
qoc_status qoc_eval_grad_hess(qoc_problem* p, const double* theta, double* J,
                              double* grad, double* hess);

/* Control models that are not linear in theta (f(t; theta), e.g. a neural
 * network in t, Sec. III-D; Eq. d2Ldf2 with its d^2 f / dtheta^2 terms).
 * The caller gives, at its current theta, the samples f (steps doubles, f_j =
 * f(j dt; theta)) and the Jacobian jac (steps x K row-major, jac[j*K + l] =
 * d f_j / d theta_l).  Returns J, grad = jac^T d, the symmetrised Hessian
 * WITHOUT the model's second-derivative term,
 *   hess = jac^T diag(2 w_ctrl + c) jac + jac^T V + jac^T U,
 * and dJdf (steps doubles): d_j = dJ/df_j = 2 w_ctrl f_j + g_j.  The full
 * Hessian is hess + sum_j d_j d^2 f_j / dtheta^2, the last term being the
 * model's own (its second derivatives, which only the caller knows).  The
 * Jacobian replaces the problem's basis: later theta-evaluations use it as
 * the linear model.  The precision of QOC_MIXED_FP32 was chosen at
 * qoc_create_problem from the basis given there, so create the problem with
 * a representative Jacobian (e.g. the model's at its starting theta) as the
 * basis.  Synchronises; host pointers. */
qoc_status qoc_eval_grad_hess_model(qoc_problem* p, const double* f, const double* jac, double* J,
                                    double* grad, double* hess, double* dJdf);

/* Device-pointer form of qoc_eval_grad_hess: theta_dev (K doubles) is read
 * and out_dev (1 + K + K*K doubles: J, grad, Hess row-major) written on the
 * problem's stream; returns after enqueueing.  Device-side failures
 * (eigensolver non-convergence, bounded-wait timeouts) are reported by the
 * next qoc_sync_status call. */
qoc_status qoc_eval_grad_hess_dev(qoc_problem* p, const double* theta_dev, double* out_dev);

/* Wait for the problem's stream and report any device-side status raised
 * since the last call (clears it). */
qoc_status qoc_sync_status(qoc_problem* p);

/* Exact-Hessian trust-region iteration (Sec. IV-B; textbook basic trust
 * region with the exact subproblem; stop rule of Alg. 1/2: |grad| < gtol or
 * trust radius < xtol).  theta0, theta_out: K host doubles (may alias). */
typedef struct {
  double gtol;        /* stop when |grad J| < gtol */
  double xtol;        /* stop when the trust radius (bound on |step|) < xtol */
  double radius0;     /* initial radius (> 0) */
  double radius_max;  /* radius cap (>= radius0) */
  double eta;         /* accept a step when actual/predicted decrease > eta (0 <= eta < 1/4) */
  int max_iter;       /* iteration cap (>= 1) */
} qoc_tr_options;

typedef struct {
  int iters;          /* iterations performed */
  int n_eval_J;       /* trial-point cost evaluations */
  int n_eval_gh;      /* gradient+Hessian evaluations */
  double J;           /* final cost */
  double grad_norm;   /* final |grad| */
  double radius;      /* final trust radius */
  int stop_reason;    /* 0 gtol, 1 xtol, 2 max_iter (status QOC_ENOTCONV), 3 no predicted decrease */
} qoc_tr_report;

qoc_status qoc_trust_region_solve(qoc_problem* p, const double* theta0,
                                  const qoc_tr_options* opt, double* theta_out,
                                  qoc_tr_report* report);

/* Gradient-only trust region (Alg. 1 with a quasi-Newton model: the
 * baseline of Sec. IV-B, where the optimiser builds a Hessian approximation
 * from gradients by BFGS updates).  The iteration of qoc_trust_region_solve
 * with the exact Hessian replaced by B: B = I until the first trial with
 * positive curvature y^T s, which first sets B = (y^T y / y^T s) I; every
 * evaluated trial (accepted or not) then updates
 *   B <- B - (B s)(B s)^T / (s^T B s) + y y^T / (y^T s)
 * with s its step and y its gradient minus the current one, skipped unless
 * y^T s > 1e-8 |s| |y| (Nocedal & Wright, Eq. 6.19).  Each trial evaluation
 * is J and the gradient (qoc_eval_grad's work); no Hessian is evaluated.
 * The report's n_eval_J counts the trial evaluations and n_eval_gh is 0.
 * Arguments and statuses as qoc_trust_region_solve. */
qoc_status qoc_trust_region_solve_bfgs(qoc_problem* p, const double* theta0,
                                       const qoc_tr_options* opt, double* theta_out,
                                       qoc_tr_report* report);

/* One trust-region subproblem (the step both trust regions take, Sec. IV-B;
 * Nocedal & Wright Sec. 4.3): s minimising g^T s + s^T H s / 2 subject to
 * |s| <= radius, exactly (secular equation |s(sigma)| = radius with
 * s(sigma) = -(H + sigma I)^-1 g, sigma >= max(0, -lambda_min(H)), and the
 * hard case), in binary64 on the device.
 *   K        size (1 <= K <= 4096); g: K host doubles; H: K*K symmetric host doubles.
 *   method   0: as the solvers choose it (1 for K < 48, 2 from 48);
 *            1: through the eigendecomposition of H (binary64 Jacobi);
 *            2: through the Householder tridiagonal reduction of H, Sturm
 *               bisection for lambda_min and tridiagonal LDL^T solves.
 *   s        K host doubles (output).
 *   info     4 host doubles (output): predicted decrease -(g^T s + s^T H s / 2),
 *            |s|, sigma, |g|.
 * Allocates and frees its device memory; synchronises. */
qoc_status qoc_tr_subproblem(int K, const double* g, const double* H, double radius, int method,
                             double* s, double* info);

/* Diagnostics of the last evaluation (host doubles; each pointer may be NULL):
 *   norm_drift   max_j | |a_j| - 1 |   (norm drift of the propagated state)
 *   hess_asym    |Hess - Hess^T|_F / |Hess|_F before symmetrisation
 *   phase_ms[6]  milliseconds of the phases eig, prep, chains, pointwise,
 *                panels, assembly (only when timing was enabled, else 0). */
qoc_status qoc_get_diagnostics(const qoc_problem* p, double* norm_drift, double* hess_asym,
                               double* phase_ms /* [6] */);

/* Per-kernel timing of the last evaluation (timing enabled), milliseconds
 * between events, in this order:
 *   0 control (f = B theta)         1 binary32 Jacobi (k_eig_jacobi32_reg at N = 32, else k_eig_jacobi32)
 *   2 binary64 refinement or the binary64 Jacobi (k_eig_refine / k_eig_jacobi)
 *   3 propagator increments D_j     4 derivative preparation (M~, P~, X')
 *   5 state and costate chains      6 pointwise contractions
 *   7 tangent and second-order adjoint panels    8 gradient/Hessian assembly
 *   9 the whole evaluation (first to last event on the problem's stream)
 * With time blocking and a gradient or Hessian request the chains, the
 * panels and the derivative preparation run concurrently on three streams
 * (5 and 7 are then measured on their own streams and overlap 4 and 6).
 * Writes min(n, QOC_N_PHASES) values. */
#define QOC_N_PHASES 10
qoc_status qoc_get_phase_times(const qoc_problem* p, double* out, int n);

/* Work counters of the last evaluation's refined eigensolver (timing
 * enabled; 0 otherwise), after the evaluation has completed:
 *   out[0] = mean binary64 Ogita-Aishima updates per step
 *   out[1] = fraction of steps whose binary64 Jacobi clean-up rotated
 *   out[2] = fraction of steps that took the final residual pass and the
 *            clean-up (the others finish early after their last update)
 * Synchronises the problem's stream. */
qoc_status qoc_get_eig_stats(qoc_problem* p, double* out /* [3] */);

/* Device time of the phases of the last qoc_trust_region_solve, in
 * milliseconds, taken with CUDA events when timing is enabled
 * (qoc_enable_timing; zeros otherwise):
 *   out[0] = subproblems and trial points, summed over the iterations
 *   out[1] = cost-only evaluations at the trial points
 *   out[2] = gradient + Hessian evaluations (and their eigendecompositions
 *            for the subproblem when K < 48)
 * The rest of the solve's wall time is host work and synchronisation. */
qoc_status qoc_get_tr_phase_times(const qoc_problem* p, double* out /* [3] */);
qoc_status qoc_enable_timing(qoc_problem* p, int on);

/* Copy an intermediate of the last evaluation to the host, for parity
 * tests against an independent implementation.  `which` and the layout of
 * the `count` doubles it writes:
 *   QOC_BUF_F       J doubles: f_j
 *   QOC_BUF_EIGVAL  J*N: eigenvalues of H_j, ascending
 *   QOC_BUF_EIGVEC  J*N*N: W_j row-major, column q = eigenvector q
 *   QOC_BUF_STATE   (J+1)*2N: a_0..a_J (interleaved complex)
 *   QOC_BUF_COSTATE (J+1)*2N: lambda_1..lambda_J in rows 1..J (row 0 = lambda_0)
 *   QOC_BUF_G       J: g_j = Re(lambda_{j+1}^H G_j a_j)
 *   QOC_BUF_C       J: c_j = Re(lambda_{j+1}^H G2_j a_j)
 *   QOC_BUF_V       J*K: Re(mu_{j+1,l}^H G_j a_j)   (second-order-adjoint form only; mu0
 *                   in place of mu when the terminal part is split, qoc_set_mu_split)
 *   QOC_BUF_U       J*K: Re(lambda_{j+1}^H G_j S_{j,l})
 *   QOC_BUF_SJ      N*K*2: S_J = da_J/dtheta (interleaved complex, row-major N x K)
 *   QOC_BUF_HESS_RAW K*K: Hessian before symmetrisation
 * Returns QOC_EINVAL if count is smaller than the buffer. */
enum {
  QOC_BUF_F = 0, QOC_BUF_EIGVAL = 1, QOC_BUF_EIGVEC = 2, QOC_BUF_STATE = 3,
  QOC_BUF_COSTATE = 4, QOC_BUF_G = 5, QOC_BUF_C = 6, QOC_BUF_V = 7, QOC_BUF_U = 8,
  QOC_BUF_SJ = 9, QOC_BUF_HESS_RAW = 10
};
qoc_status qoc_read_buffer(const qoc_problem* p, int which, double* host_out, size_t count);

/* ---------------------------------------------------------------------------
 * Learned warm start (no counterpart in the paper, whose trust region starts
 * from random theta, Sec. IV-B): a multilayer perceptron
 *   theta0 = W_L gelu(... gelu(W_1 x + b_1) ...) + b_L,  gelu(x) = x (1 + erf(x/sqrt 2))/2,
 * mapping features x of a target (e.g. [Re beta, Im beta]) to initial
 * control coefficients.  binary32 training (own forward/backward/Adam
 * kernels), bfloat16-weight inference.  Parameters are one flat binary32
 * vector: for each layer k, W_k (d_k x d_{k+1}, row-major, y = x W_k) then b_k.
 * ------------------------------------------------------------------------- */
typedef struct qoc_mlp qoc_mlp;

/* Number of parameters of the layout above (0 on invalid sizes). */
size_t qoc_mlp_param_count(int n_in, int hidden, int n_hidden_layers, int n_out);

/* Create with initial parameters params_init (host, qoc_mlp_param_count
 * floats, copied) and buffers for minibatches of up to max_batch rows. */
qoc_status qoc_mlp_create(int n_in, int hidden, int n_hidden_layers, int n_out,
                          const float* params_init, int max_batch, void* cuda_stream,
                          qoc_mlp** out);

/* Upload the training set: X (n x n_in), T (n x n_out), row-major host floats. */
qoc_status qoc_mlp_set_dataset(qoc_mlp* m, const float* X, const float* T, int n);

/* Train: for each of `epochs` epochs, minibatches of `batch` rows taken in
 * the order perm[ep*n .. ep*n+n-1] (host ints, a permutation of 0..n-1);
 * loss 1/(2B) sum |y - t|^2; Adam(lr, 0.9, 0.999, 1e-8).  losses[ep] receives
 * the mean minibatch loss of the epoch. */
qoc_status qoc_mlp_train(qoc_mlp* m, const int* perm, int epochs, int batch, float lr,
                         float* losses);

/* Loss and its gradient with respect to the flat parameter vector for one
 * minibatch (X batch x n_in, T batch x n_out; host floats). */
qoc_status qoc_mlp_gradient(qoc_mlp* m, const float* X, const float* T, int batch, float* loss,
                            float* grad);

/* Inference on n rows of X into Y (n x n_out).  bf16 != 0: every layer on
 * the tensor cores with bfloat16 weights and bfloat16 activations (rounded
 * from binary32 as each layer reads them), binary32 accumulation, bias and
 * GELU in binary32 (relative error against a binary64 evaluation of the same
 * network of order 1e-2 of the output scale); bf16 == 0: binary32 throughout. */
qoc_status qoc_mlp_predict(qoc_mlp* m, const float* X, int n, float* Y, int bf16);

/* Copy the current parameters to the host. */
qoc_status qoc_mlp_get_params(const qoc_mlp* m, float* params);

void qoc_mlp_destroy(qoc_mlp* m);

/* ---------------------------------------------------------------------------
 * Batches of uneven problems (different N, K, J and sweep precision; time
 * blocking on).  One batched evaluation = the gradient and Hessian of every
 * problem at its own theta: the parallel phases of each problem run on that
 * problem's stream, each of the four sequential sweeps runs as one launch
 * per sweep precision and kernel over all problems that take it (binary32
 * N <= 32, binary32 N <= 64, the general binary32 one, binary64; side by
 * side on their own streams), and the
 * whole evaluation is captured once into a CUDA graph (qoc_batch_set_graph(b,
 * 0) disables the graph).  Every problem takes the kernel a single
 * evaluation of it takes, so batched results equal single ones bit for bit.
 * The batch references the problems (caller keeps them alive and must not
 * use them concurrently).
 *   thetas: concatenation of the problems' theta (sum K_i doubles)
 *   outs:   concatenation of [J, grad (K_i), Hess (K_i^2)] per problem
 * ------------------------------------------------------------------------- */
typedef struct qoc_batch qoc_batch;
qoc_status qoc_batch_create(qoc_problem* const* problems, int n, void* cuda_stream, qoc_batch** out);
qoc_status qoc_batch_set_graph(qoc_batch* b, int on);
qoc_status qoc_batch_eval_grad_hess(qoc_batch* b, const double* thetas, double* outs);
/* device-pointer form: enqueues on the batch stream and returns */
qoc_status qoc_batch_eval_grad_hess_dev(qoc_batch* b, const double* thetas_dev, double* outs_dev);
void qoc_batch_destroy(qoc_batch* b);

/* Batched exact-Hessian trust region (Sec. IV-B runs one solve per trial;
 * the batching pattern runs many at once): every problem takes the basic
 * trust region of qoc_trust_region_solve from its own theta0 with the same
 * options, all advancing together.  One iteration is: on the device, per
 * problem, the gtol test, the exact subproblem and the trial point; one
 * batched gradient + Hessian evaluation of every trial point (a qoc_batch
 * with its CUDA graph); the eigendecomposition of each trial Hessian; on the
 * device, the ratio test, radius update, acceptance (theta, J, gradient,
 * Hessian and its eigendecomposition taken over from the trial) and the
 * xtol / iteration-cap tests.  The host reads the problems' states once per
 * iteration for the whole batch and, when some have stopped, rebuilds the
 * batch over the others.  Each trial point is evaluated with its gradient
 * and Hessian, so an accepted step costs no further evaluation; the
 * iterates are those of qoc_trust_region_solve.
 *   problems  n distinct problems with time blocking (steps >= 16) and
 *             K <= 256; the caller keeps them alive, unused meanwhile.
 *   theta0s   concatenation of the starting points (sum K_i host doubles).
 *   theta_out concatenation of the final points (may alias theta0s).
 *   reports   n reports: iters, n_eval_J (trial evaluations), n_eval_gh
 *             (1 + accepted steps), final J, |grad|, radius, stop_reason
 *             (0 gtol, 1 xtol, 2 max_iter, 3 no predicted decrease,
 *             4 device failure of that problem's evaluation).
 *   cuda_stream  stream to run on, or NULL for a temporary one.
 * Returns QOC_OK when every problem stopped by 0, 1 or 3; QOC_ENOTCONV if
 * one hit max_iter; the failing problem's status (QOC_ETIMEOUT, ...) if one
 * failed (the others' results are still written).  Allocates a small state
 * array and each problem's trial eigendecomposition for the call. */
qoc_status qoc_batch_trust_region_solve(qoc_problem* const* problems, int n, const double* theta0s,
                                        const qoc_tr_options* opt, double* theta_out,
                                        qoc_tr_report* reports, void* cuda_stream);

/* ---------------------------------------------------------------------------
 * Gradient and Hessian assembly that allocates no device memory.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc when they need the result (code running during a
 * CUDA-graph capture that forbids allocation, frameworks whose memory pool
 * owns all device memory, latency-bound loops that cannot take an
 * allocation's implicit synchronisation).  It computes, from per-step
 * contractions the caller already holds on the device (for example read back
 * with qoc_read_buffer from a qoc_problem evaluated with the second-order
 * adjoint Hessian),
 *   grad = B^T (2 w_ctrl f + g),
 *   Hess = sym( B^T diag(2 w_ctrl + c) B + B^T V + B^T U ),
 * the same arithmetic as the assembly step of qoc_eval_grad_hess.
 *
 *   basis_dev   steps x K row-major binary64 (device)
 *   f_dev, g_dev, c_dev   steps binary64 each (device)
 *   U_dev, V_dev          steps x K row-major binary64 (device)
 *   out_dev     1 + K + K*K binary64 (device): out[0] is not written, grad
 *               at out[1..K], the symmetrised Hessian row-major after it
 *   cuda_stream stream of the current device (NULL: legacy default stream);
 *               the call enqueues and returns
 * Intermediate partial sums go to one file-scope device array of
 * QOC_NOALLOC_SCRATCH_DOUBLES doubles (4 MiB) that every GPU loading the
 * library keeps until process exit.  The call needs
 * qoc_assemble_noalloc_scratch_doubles(steps, K) of them and returns
 * QOC_EINVAL (with the reason in qoc_last_error) when that is above the
 * maximum, e.g. K = 64 allows steps <= 8000.  The first call on a device
 * looks up the array's device address with that device current, and every
 * later call made while cuda_stream is not being captured looks it up again
 * (the address changes if the device's context is destroyed and recreated);
 * make that first call before any stream capture.  All calls
 * share the array and it keeps the previous call's contents (nothing needs
 * clearing: each call writes every element it reads), so calls that may
 * overlap on the GPU race: order them on one stream or with events.
 * Errors: QOC_EINVAL (bad size, NULL pointer, too large), QOC_ECUDA.
 * ------------------------------------------------------------------------- */
#define QOC_NOALLOC_SCRATCH_DOUBLES 524288
size_t qoc_assemble_noalloc_scratch_doubles(int steps, int K);
qoc_status qoc_assemble_grad_hess_noalloc(int steps, int K, const double* basis_dev, const double* f_dev,
                                          const double* g_dev, const double* c_dev, const double* U_dev,
                                          const double* V_dev, double w_ctrl, double* out_dev,
                                          void* cuda_stream);

/* Measured binary64 FMA rate of the current device (no counterpart in the
 * paper; the denominator of the roofline of the binary64-bound kernels):
 * a kernel of independent FMA chains on ctas_per_sm x 256 threads per SM,
 * timed `repeats` times with CUDA events after one warm-up launch; the
 * fastest launch gives *tflops (2 flops per FMA) and *ms (may be NULL).
 * Allocates and frees a small output buffer; synchronises the device. */
qoc_status qoc_measure_fp64_rate(int ctas_per_sm, int repeats, double* tflops, double* ms);

/* Bytes of device memory the problem holds. */
size_t qoc_device_bytes(const qoc_problem* p);

/* Largest N this build supports. */
int qoc_max_basis_size(void);

/* Release everything the problem owns (NULL is a no-op). */
void qoc_destroy_problem(qoc_problem* p);

/* Text of the last failure this thread saw inside the library: the CUDA
 * error, or the device status bits behind QOC_ENUMERIC / QOC_ETIMEOUT, or a
 * size limit (empty if none); valid until the thread's next failing call. */
const char* qoc_last_error(void);

/* Static, human-readable name of a status. */
const char* qoc_status_string(qoc_status s);

/* Library ABI version (major*10000 + minor*100 + patch). */
int qoc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* QOC_H */
