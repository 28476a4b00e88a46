"""Basis sizes above 64 (the upper half of the batched recipe, N up to 128,
and the largest single problem, N = 256): the per-step kernels then keep their
matrices in a per-CTA slice of a global workspace and the sweeps read their
block data straight from global memory.  Parity with the oracle on the same
seeded inputs (small J), the full-size N=256/K=128/J=10^4 problem through
properties that hold at any size, and the trust region at K = 128."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def check(prob, theta, precision, block_steps=None, intermediates=True):
    ref = orc.evaluate(prob, theta, order=2, keep=intermediates)
    tol = TOL[precision]
    with q.Problem(prob, precision=precision, block_steps=block_steps) as P:
        J, g, H = P.eval_grad_hess(theta)
        assert abs(J - ref["J"]) <= tol * abs(ref["J"]), (J, ref["J"])
        assert rel(g, ref["grad"]) <= tol, rel(g, ref["grad"])
        assert rel(H, ref["hess"]) <= tol, rel(H, ref["hess"])
        np.testing.assert_array_equal(H, H.T)
        if intermediates:
            lam = P.buffer(_lib.QOC_BUF_EIGVAL)
            assert np.abs(lam - ref["eig"]).max() <= 1e-13 * max(np.abs(ref["eig"]).max(), 1.0) * prob.N
            a = P.buffer(_lib.QOC_BUF_STATE)
            assert rel(a, ref["a"]) <= (1e-10 if precision == q.QOC_FP64 else 1e-5)


@pytest.mark.parametrize("shape", [(72, 5, 37), (96, 16, 24), (128, 9, 16), (65, 3, 1), (127, 4, 9)],
                         ids=lambda s: "N%d_K%d_J%d" % s)
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_large_n_parity(shape, precision):
    N, K, J = shape
    prob = inputs.small_problem(N, K, J, seed=N + K + J)
    check(prob, inputs.eval_theta(K, N, 0.5), precision)


@pytest.fixture(scope="module")
def largest_truncated():
    """The N=256, K=128 system of the largest workload on its first 8 steps
    (same H0, M, target, basis rows and dt) and its oracle evaluation."""
    full = inputs.config_problem(5)
    prob = inputs.Problem(full.H0, full.M, full.alpha, full.beta, full.B[:8], full.dt, full.w_f,
                          full.w_t, name="largest-8")
    theta = inputs.eval_theta(full.K, 5)
    return prob, theta, orc.evaluate(prob, theta, order=2)


@pytest.mark.parametrize("block_steps", [1, 2], ids=["per_step", "blocked"])
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_largest_system_truncated(largest_truncated, precision, block_steps):
    prob, theta, ref = largest_truncated
    tol = TOL[precision]
    with q.Problem(prob, precision=precision, block_steps=block_steps) as P:
        J, g, H = P.eval_grad_hess(theta)
    assert abs(J - ref["J"]) <= tol * abs(ref["J"]), (J, ref["J"])
    assert rel(g, ref["grad"]) <= tol, rel(g, ref["grad"])
    assert rel(H, ref["hess"]) <= tol, rel(H, ref["hess"])


def test_largest_system_full_size():
    """N=256, K=128, J=10^4: the binary64 gradient against a central difference
    of J along a random direction and the Hessian against a central difference
    of the gradient, Hessian symmetry before symmetrisation, norm drift; mixed
    vs binary64.  At this size the mixed path meets 1e-6 for J and the gradient
    but not for the Hessian: the binary32 rounding of increments |D_j| ~ 0.2
    accumulates over 10^4 steps to about 5e-6 (measured 4.6e-6), so the Hessian
    is held to 1e-5 here; the binary64 path is the one to use for this size."""
    import time
    prob = inputs.config_problem(5)
    theta = inputs.eval_theta(prob.K, 5)
    with q.Problem(prob, precision=q.QOC_FP64) as P:
        t0 = time.perf_counter()
        J64, g64, H64 = P.eval_grad_hess(theta)
        print(f"N=256 K=128 J=10^4 binary64 evaluation: {time.perf_counter() - t0:.2f} s")
        d = P.diagnostics()
        assert d["norm_drift"] < 1e-11 and d["hess_asym"] < 1e-9, d
        v = np.random.default_rng(3).normal(size=prob.K)
        v /= np.linalg.norm(v)
        h = 1e-4
        fd = (P.eval_J(theta + h * v) - P.eval_J(theta - h * v)) / (2 * h)
        assert abs(fd - g64 @ v) <= 1e-6 * max(abs(g64 @ v), np.linalg.norm(g64) * 1e-3)
        # second derivative along v from the gradient
        gp = P.eval_grad(theta + h * v)[1]
        gm = P.eval_grad(theta - h * v)[1]
        assert rel((gp - gm) / (2 * h), H64 @ v) <= 1e-5
    with q.Problem(prob, precision=q.QOC_MIXED_FP32) as P:
        t0 = time.perf_counter()
        J32, g32, H32 = P.eval_grad_hess(theta)
        print(f"N=256 K=128 J=10^4 mixed evaluation: {time.perf_counter() - t0:.2f} s")
    assert abs(J32 - J64) <= 1e-6 * abs(J64)
    assert rel(g32, g64) <= 1e-6 and rel(H32, H64) <= 1e-5, (rel(g32, g64), rel(H32, H64))


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_trust_region_k128(precision):
    """K = 128 (the largest workload's control dimension): the subproblem's
    K x K binary64 eigensolver no longer fits shared memory."""
    prob = inputs.small_problem(6, 128, 256, seed=41, dt=0.02)
    th_o, info_o = orc.trust_region_solve(prob, np.zeros(prob.K), gtol=1e-7, xtol=1e-12)
    with q.Problem(prob, precision=precision) as P:
        th, info = P.trust_region_solve(np.zeros(prob.K), gtol=1e-7 if precision == q.QOC_FP64 else 1e-5,
                                        xtol=1e-12)
    assert abs(info["J"] - info_o["J"]) <= (1e-8 if precision == q.QOC_FP64 else 1e-6) * abs(info_o["J"])
    if precision == q.QOC_FP64:
        assert info["iters"] == info_o["iters"]


def test_batch_with_large_n():
    """Uneven batch with N above and below 64 (ring and direct sweeps in one
    launch) reproduces the per-problem evaluations."""
    shapes = [(72, 16, 40), (8, 32, 60), (128, 8, 33), (40, 12, 50)]
    probs = [inputs.small_problem(N, K, J, seed=3 * i + 1) for i, (N, K, J) in enumerate(shapes)]
    Ps = [q.Problem(p, precision=q.QOC_MIXED_FP32) for p in probs]
    try:
        with q.Batch(Ps) as b:
            thetas = [inputs.eval_theta(p.K, 70 + i, 0.5) for i, p in enumerate(probs)]
            for _ in range(2):
                res = b.eval_grad_hess(thetas)
                for P, th, (J, g, H) in zip(Ps, thetas, res):
                    Ji, gi, Hi = P.eval_grad_hess(th)
                    assert abs(J - Ji) <= 1e-13 * abs(Ji)
                    assert rel(g, gi) <= 1e-13 and rel(H, Hi) <= 1e-13
    finally:
        for P in Ps:
            P.close()
