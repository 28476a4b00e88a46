"""The forward pipeline (refinement and increments in chunks, the state chain
following chunk by chunk from the stored block-start states) reorders work
only: every result (J alone, J and the gradient, J, gradient and Hessian,
the stored states) must equal the unchunked schedule's bit for bit, for each
sweep variant (binary32 warp-specialised at N <= 32 and N <= 64, the general
sweep above, binary64), ragged horizons and every chunk count."""
import numpy as np
import pytest

from paper_2505_00529_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

CASES = [  # (N, K, J), block steps, chunks
    ((5, 4, 203), 4, 3),
    ((32, 9, 400), 4, 8),
    ((40, 6, 333), 3, 2),
    ((72, 5, 130), 2, 4),
    ((16, 7, 64), 8, 8),      # one block per chunk
]


def _run(P, theta, chunks):
    _lib.qoc_set_pipeline(P.handle, chunks)
    J, g, H = P.eval_grad_hess(theta)
    states = P.buffer(_lib.QOC_BUF_STATE)
    costates = P.buffer(_lib.QOC_BUF_COSTATE)
    J1, g1 = P.eval_grad(theta)
    J0 = P.eval_J(theta)
    return J, g, H, states, costates, J1, g1, J0


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%d_K%d_J%d_b%d_c%d" % (*c[0], c[1], c[2]))
@pytest.mark.parametrize("precision", [_lib.QOC_FP64, _lib.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_pipelined_forward_chain_is_bit_identical(case, precision):
    (N, K, J), bs, chunks = case
    prob = inputs.small_problem(N=N, K=K, J=J, seed=300 + N + J, dt=0.05, basis="random")
    theta = inputs.eval_theta(K, 11, 0.7)
    with _lib.Problem(prob, precision=precision, block_steps=bs) as P:
        ref = _run(P, theta, 0)
        got = _run(P, theta, chunks)
        again = _run(P, theta, 0)
    for a, b, c in zip(ref, got, again):
        np.testing.assert_array_equal(np.asarray(b), np.asarray(a))
        np.testing.assert_array_equal(np.asarray(c), np.asarray(a))


def test_pipeline_timing_and_range():
    prob = inputs.small_problem(N=8, K=4, J=256, seed=9, dt=0.05, basis="random")
    theta = inputs.eval_theta(4, 2, 0.5)
    with _lib.Problem(prob, precision=_lib.QOC_MIXED_FP32, block_steps=4) as P:
        _lib.qoc_enable_timing(P.handle, 1)
        _lib.qoc_set_pipeline(P.handle, 4)
        P.eval_grad_hess(theta)
        ph = _lib.qoc_get_phase_times(P.handle)
        assert ph["eig_refine"] > 0 and ph["prep_D"] > 0 and ph["total"] > 0
        for bad in (-2, 9):
            with pytest.raises(_lib.QocError) as e:
                _lib.qoc_set_pipeline(P.handle, bad)
            assert e.value.status == _lib.QOC_EINVAL


@pytest.mark.parametrize("precision", [_lib.QOC_FP64, _lib.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_trust_region_reuses_the_trial_forward_part_exactly(precision):
    """After an accepted step the trust region evaluates the gradient and
    Hessian at the trial point reusing the trial's control samples,
    eigendecompositions, increments and forward chain: the J it reports must
    be a fresh evaluation's at the returned point bit for bit (the gradient
    norm to its summation order)."""
    prob = inputs.small_problem(N=12, K=6, J=240, seed=41, dt=0.05, basis="sine_cosine")
    with _lib.Problem(prob, precision=precision) as P:
        accepted = 0
        for iters in (1, 2, 4, 8):
            th, info = P.trust_region_solve(np.zeros(6), gtol=0.0, xtol=0.0, max_iter=iters)
            J, g, H = P.eval_grad_hess(th)
            assert info["J"] == J
            gn = float(np.linalg.norm(np.asarray(g)))
            assert abs(info["grad_norm"] - gn) <= 1e-14 * max(gn, 1e-300)
            accepted = max(accepted, info["n_eval_gh"] - 1)
        assert accepted >= 2   # the reused evaluations were exercised


def test_trust_region_phase_times():
    """With timing enabled the solve's device phases are measured: each
    positive, together within the solve's wall time."""
    import time
    prob = inputs.small_problem(N=12, K=6, J=240, seed=41, dt=0.05, basis="sine_cosine")
    with _lib.Problem(prob, precision=_lib.QOC_MIXED_FP32) as P:
        _lib.qoc_enable_timing(P.handle, 1)
        t0 = time.perf_counter()
        _, info = P.trust_region_solve(np.zeros(6), gtol=0.0, xtol=0.0, max_iter=6)
        wall_ms = 1e3 * (time.perf_counter() - t0)
        ph = _lib.qoc_get_tr_phase_times(P.handle)
    assert info["iters"] >= 1
    assert all(v > 0 for v in ph.values()), ph
    assert sum(ph.values()) <= wall_ms
