"""The second-order adjoint with its terminal part in closed form
(qoc_set_mu_split; by default on binary64 sweeps, on the time-blocked schedule).

Eq. musys is linear in mu, so mu = mu0 + mu_T, with mu0 the recursion from
the sources G_j^H lambda_{j+1} b_j^T and mu0_J = 0, and mu_T the terminal value
2 w_t S_J carried back by U_j^H alone.  The contraction of mu_T with the
tangent sources G_j a_j telescopes into the tangent recursion (Eq.
gradatheta):

    sum_j b_jl Re(mu_T,{j+1},m^H G_j a_j) = Re(S_J,l^H mu_J,m),

so B^T V = B^T V0 + 2 w_t Re(S_J^H S_J).  The CPU test checks that identity
on the oracle's own recursions; the GPU tests check the split evaluation
against the unsplit one and against the oracle (V0 step by step)."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def oracle_V0(prob, ref):
    mu0 = orc.second_adjoints(ref["U_prop"], ref["G"], ref["lam"], np.zeros_like(ref["SJ"]), prob.B,
                              prob.w_t)
    return orc.hessian(prob.B, prob.w_f, ref["G"], ref["G2"], ref["a"], ref["lam"], ref["S"], mu0)[2]


@pytest.mark.parametrize("basis, N, K, J", [("random", 5, 4, 23), ("sine", 6, 3, 40),
                                            ("maximal", 4, 12, 12)])
def test_terminal_part_telescopes_on_the_oracle(basis, N, K, J):
    prob = inputs.small_problem(N=N, K=K, J=J, seed=300 + N, dt=0.05, basis=basis)
    theta = inputs.eval_theta(K, 301 + N)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    V0 = oracle_V0(prob, ref)
    SJ = ref["SJ"]
    gram = 2.0 * prob.w_t * np.real(SJ.conj().T @ SJ)
    lhs = prob.B.T @ ref["V"]
    rhs = prob.B.T @ V0 + gram
    assert np.abs(lhs - rhs).max() <= 1e-12 * np.abs(lhs).max(), np.abs(lhs - rhs).max()
    # and the terminal part is not negligible here, so the check has teeth
    assert np.abs(gram).max() >= 1e-3 * np.abs(lhs).max()
    # the split Hessian equals the oracle's unsymmetrised one
    c, Uc = ref["c"], ref["U"]
    B = prob.B
    Hsplit = B.T @ ((2.0 * prob.w_f + c)[:, None] * B) + B.T @ V0 + gram + B.T @ Uc
    assert rel(Hsplit, ref["hess_raw"]) <= 1e-12


@pytest.fixture(scope="module")
def _built():
    build.build()
    _lib.lib()


TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}
TOL_INTER = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-5}
# split against unsplit: the same arithmetic but for the terminal part's
# rounding (binary64 Gram sum against the swept terminal value)
TOL_SPLIT = {q.QOC_FP64: 1e-12, q.QOC_MIXED_FP32: 1e-6}


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("basis, N, K, J, bs", [("random", 7, 5, 37, 4), ("sine", 9, 6, 64, 2),
                                                ("maximal", 5, 20, 20, 4), ("random", 32, 8, 200, 4)])
def test_split_matches_unsplit_and_oracle(_built, precision, basis, N, K, J, bs):
    prob = inputs.small_problem(N=N, K=K, J=J, seed=400 + N + J, dt=0.05, basis=basis)
    theta = inputs.eval_theta(K, 401 + N)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    out = {}
    for split in (True, False):
        with q.Problem(prob, precision=precision, block_steps=bs, mu_split=split) as P:
            J_, g, H = P.eval_grad_hess(theta)
            out[split] = (J_, g, H, P.buffer(_lib.QOC_BUF_V), P.buffer(_lib.QOC_BUF_HESS_RAW))
            # a second evaluation after the first reuses nothing stale
            J2, g2, H2 = P.eval_grad_hess(theta)
            np.testing.assert_array_equal(H2, H)
    tol = TOL[precision]
    Js, gs, Hs, Vs, Rs = out[True]
    Ju, gu, Hu, Vu, Ru = out[False]
    assert Js == Ju
    np.testing.assert_array_equal(gs, gu)
    assert rel(Hs, Hu) <= TOL_SPLIT[precision], rel(Hs, Hu)
    np.testing.assert_array_equal(Hs, Hs.T)
    assert rel(Hs, ref["hess"]) <= tol, rel(Hs, ref["hess"])
    assert rel(Rs, ref["hess_raw"]) <= tol, rel(Rs, ref["hess_raw"])
    # V: the contraction of mu0 (split) and of mu (unsplit), step by step
    assert rel(Vs, oracle_V0(prob, ref)) <= TOL_INTER[precision], rel(Vs, oracle_V0(prob, ref))
    assert rel(Vu, ref["V"]) <= TOL_INTER[precision], rel(Vu, ref["V"])


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_builtin_choice_and_validation(_built, precision):
    """Built-in choice (-1): split on binary64 sweeps only; the V buffer tells
    which form ran (mu0's contraction or mu's)."""
    prob = inputs.small_problem(N=6, K=4, J=40, seed=9, dt=0.05, basis="random")
    theta = inputs.eval_theta(4, 10)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    with q.Problem(prob, precision=precision, block_steps=4) as P:
        with pytest.raises(q.QocError):
            q.qoc_set_mu_split(P.handle, 2)
        with pytest.raises(q.QocError):
            q.qoc_set_mu_split(P.handle, -2)
        P.eval_grad_hess(theta)
        V = P.buffer(_lib.QOC_BUF_V)
        eff = P.precision()[0]
    exp = oracle_V0(prob, ref) if eff == q.QOC_FP64 else ref["V"]
    other = ref["V"] if eff == q.QOC_FP64 else oracle_V0(prob, ref)
    assert rel(V, exp) <= TOL_INTER[eff], rel(V, exp)
    assert rel(V, other) > 1e3 * TOL_INTER[eff]
    assert q.lib().qoc_set_mu_split(None, 1) != 0
