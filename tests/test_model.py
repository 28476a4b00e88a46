"""Control models that are not linear in theta (qoc_eval_grad_hess_model):
a tanh network in t, f(t) = sum_h v_h tanh(w_h t + c_h), through the C ABI
against the oracle's evaluation of the same samples and Jacobian; the full
Hessian adds the model's own term sum_j d_j d^2 f_j / dtheta^2."""
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


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_tanh_network_model_matches_oracle(precision):
    H = 4
    prob = inputs.small_problem(N=6, K=3 * H, J=120, seed=81, dt=0.05)
    t = np.arange(prob.J) * prob.dt
    tol = TOL[precision]
    # the problem is created with the model's Jacobian at the first theta as
    # its basis: the precision policy estimates the binary32 error from it
    prob.B = inputs.tanh_network_control(t, inputs.eval_theta(3 * H, 82, 0.7))[1]
    with q.Problem(prob, precision=precision) as P:
        for seed in (82, 83):     # two calls in a row, different theta
            theta = inputs.eval_theta(3 * H, seed, 0.7)
            f, jac, hf = inputs.tanh_network_control(t, theta)
            ref = orc.evaluate_model(prob, f, jac, order=2)
            J, g, Hb, d = P.eval_grad_hess_model(f, jac)
            assert abs(J - ref["J"]) <= tol * abs(ref["J"])
            assert rel(g, ref["grad"]) <= tol and rel(Hb, ref["hess"]) <= tol, (rel(g, ref["grad"]),
                                                                               rel(Hb, ref["hess"]))
            assert rel(d, ref["d"]) <= (1e-10 if precision == q.QOC_FP64 else 1e-5)
            full = Hb + np.einsum("j,jlm->lm", d, hf)
            full_ref = ref["hess"] + np.einsum("j,jlm->lm", ref["d"], hf)
            assert rel(full, full_ref) <= 10 * tol
        # the last Jacobian is now the basis of the linear evaluations
        th2 = inputs.eval_theta(3 * H, 84, 0.7)
        J2, g2, H2 = P.eval_grad_hess(th2)
        lin = orc.evaluate_samples(prob, jac @ th2, jac, order=2)
        assert rel(H2, lin["hess"]) <= tol and abs(J2 - lin["J"]) <= tol * abs(lin["J"])


def test_model_linear_case_equals_theta_evaluation():
    prob = inputs.small_problem(N=5, K=4, J=80, seed=85, dt=0.05, basis="random")
    theta = inputs.eval_theta(4, 86)
    with q.Problem(prob) as P:
        J1, g1, H1 = P.eval_grad_hess(theta)
        J2, g2, H2, d = P.eval_grad_hess_model(prob.B @ theta, prob.B)
    assert abs(J1 - J2) <= 1e-13 * abs(J1) and rel(g1, g2) <= 1e-13 and rel(H1, H2) <= 1e-13
