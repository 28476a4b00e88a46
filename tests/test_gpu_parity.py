"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the
same seeded inputs.  Tolerances: 1e-10 relative for the binary64 path,
1e-6 for mixed precision (the stated targets), per result.

Intermediates are compared only through basis-invariant quantities
(eigenvalues, the propagators rebuilt from (W, lambda), states, costates,
per-step contractions), never eigenvectors themselves."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}
# per-step intermediates (states, contractions) in mixed precision: bilinear
# quantities such as g_j = Re(lambda_{j+1}^H G_j a_j) can lose a digit to
# cancellation, so they are held to 1e-5; J, grad and Hess keep 1e-6
TOL_INTER = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-5}
# eigenvalues (relative to the largest) and the propagators rebuilt from
# (W, lambda): binary64 sweeps refine the eigenvectors to the binary64 floor;
# binary32 sweeps stop the refinement once the residual it leaves is below
# 1e-9 |H| (eigenvalues and smooth functions of H accurate to about that)
TOL_EIG = {q.QOC_FP64: 1e-13, q.QOC_MIXED_FP32: 1e-8}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


# row-wise check of per-step arrays: the worst step's relative error, each
# step's norm floored at ROW_FLOOR x the rms step norm so that a step whose
# value happens to be near zero is measured against the array's scale
ROW_FLOOR = 0.1
TOL_ROW = {q.QOC_FP64: 1e-9, q.QOC_MIXED_FP32: 1e-4}


def rowwise(a, b, floor=ROW_FLOOR):
    a = np.asarray(a).reshape(len(b), -1)
    b = np.asarray(b).reshape(len(b), -1)
    nb = np.linalg.norm(b, axis=1)
    den = np.maximum(nb, floor * max(np.sqrt(np.mean(nb ** 2)), 1e-300))
    return float((np.linalg.norm(a - b, axis=1) / den).max())


def split_applied(P, prob, method, block_steps=None):
    """Whether an evaluation splits the second-order adjoint's terminal part
    off (qoc_set_mu_split, by default on binary64 sweeps): the
    second-order-adjoint form on the time-blocked schedule (block steps > 1;
    by default when J >= 16)."""
    bs = block_steps if block_steps is not None else (1 if prob.J < 16 else 2)
    return (method == q.QOC_HESS_SECOND_ORDER_ADJOINT and bs > 1
            and P.precision()[0] == q.QOC_FP64)


def oracle_V0(prob, ref):
    """V[j, m] = Re(mu0_{j+1,m}^H G_j a_j) for the oracle's mu recursion
    (Eq. musys) started from mu0_J = 0 instead of 2 w_t S_J."""
    mu0 = orc.second_adjoints(ref["U_prop"], ref["G"], ref["lam"], np.zeros_like(ref["SJ"]), prob.B,
                              prob.w_t)
    return orc.hessian(prob.B, prob.w_f, ref["G"], ref["G2"], ref["a"], ref["lam"], ref["S"], mu0)[2]


def check_eval(prob, theta, precision, method=q.QOC_HESS_SECOND_ORDER_ADJOINT, eig=None,
               ref=None, intermediates=True):
    tol = TOL[precision]
    tin = TOL_INTER[precision]
    ref = ref if ref is not None else orc.evaluate(prob, theta, order=2, keep=intermediates)
    with q.Problem(prob, precision=precision, hess_method=method, eig_method=eig) as P:
        J, g, H = P.eval_grad_hess(theta)
        assert abs(J - ref["J"]) <= tol * abs(ref["J"]), (J, ref["J"])
        assert rel(g, ref["grad"]) <= tol, rel(g, ref["grad"])
        assert rel(H, ref["hess"]) <= tol, rel(H, ref["hess"])
        np.testing.assert_array_equal(H, H.T)
        if not intermediates:
            return P.diagnostics()
        # (a1) control
        assert rel(P.buffer(_lib.QOC_BUF_F), ref["f"]) <= 1e-14
        # (a2) eigenvalues, and the propagators rebuilt from (W, lambda)
        lam = P.buffer(_lib.QOC_BUF_EIGVAL)
        W = P.buffer(_lib.QOC_BUF_EIGVEC)
        scale = np.abs(ref["eig"]).max()
        teig = TOL_EIG[precision]
        assert np.abs(lam - ref["eig"]).max() <= teig * max(scale, 1.0) * prob.N
        Ug = np.einsum("jpr,jr,jqr->jpq", W, np.exp(-1j * prob.dt * lam), W)
        assert rel(Ug, ref["U_prop"]) <= teig
        # (a4) states, (a7) costates: whole arrays and step by step
        trow = TOL_ROW[precision]
        a = P.buffer(_lib.QOC_BUF_STATE)
        assert rel(a, ref["a"]) <= tin
        assert rowwise(a, ref["a"]) <= trow, rowwise(a, ref["a"])
        lm = P.buffer(_lib.QOC_BUF_COSTATE)
        assert rel(lm[1:], ref["lam"][1:]) <= tin
        assert rowwise(lm[1:], ref["lam"][1:]) <= trow, rowwise(lm[1:], ref["lam"][1:])
        # (a7/a9) per-step contractions: whole arrays and step by step
        per_step = [(_lib.QOC_BUF_G, "g"), (_lib.QOC_BUF_C, "c"), (_lib.QOC_BUF_U, "U")]
        exp = dict(ref)
        if method == q.QOC_HESS_SECOND_ORDER_ADJOINT:
            per_step.append((_lib.QOC_BUF_V, "V"))
            if split_applied(P, prob, method):
                exp["V"] = oracle_V0(prob, ref)
        for which, key in per_step:
            got = P.buffer(which)
            assert rel(got, exp[key]) <= tin, (key, rel(got, exp[key]))
            assert rowwise(got, exp[key]) <= trow, (key, rowwise(got, exp[key]))
        if method == q.QOC_HESS_SECOND_ORDER_ADJOINT:
            assert rel(P.buffer(_lib.QOC_BUF_HESS_RAW), ref["hess_raw"]) <= tol
        # (a5) final tangent panel
        assert rel(P.buffer(_lib.QOC_BUF_SJ), ref["SJ"]) <= tin
        return P.diagnostics()


SHAPES = [  # (N, K, J): tiny, odd N, ragged tails, single step, N = 1, max N
    (4, 3, 50), (5, 8, 37), (2, 1, 1), (1, 2, 10), (7, 5, 33), (16, 12, 200), (32, 64, 300),
    (33, 6, 41), (64, 5, 60),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "N%d_K%d_J%d" % s)
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_small_parity(shape, precision):
    N, K, J = shape
    prob = inputs.small_problem(N=N, K=K, J=J, seed=100 + N + K + J, dt=0.05, basis="random")
    theta = inputs.eval_theta(K, 7)
    check_eval(prob, theta, precision)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_tangent_form_and_jacobi_eig(precision):
    prob = inputs.small_problem(N=12, K=10, J=120, seed=5, dt=0.04, basis="sine_cosine")
    theta = inputs.eval_theta(10, 8)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    check_eval(prob, theta, precision, method=q.QOC_HESS_TANGENT, ref=ref)
    check_eval(prob, theta, precision, eig=q.QOC_EIG_JACOBI_FP64, ref=ref)


def test_maximal_model():
    """Maximal model f_j = theta_j (Eq. maximal), K = J."""
    J = 64
    prob = inputs.small_problem(N=4, K=J, J=J, seed=9, dt=0.1, basis="maximal")
    theta = inputs.eval_theta(J, 10)
    check_eval(prob, theta, q.QOC_FP64)
    check_eval(prob, theta, q.QOC_MIXED_FP32)


@pytest.mark.parametrize("method", [q.QOC_HESS_SECOND_ORDER_ADJOINT, q.QOC_HESS_TANGENT], ids=["soa", "tangent"])
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_maximal_model_identity_assembly(precision, method):
    """Maximal model at J = K = 300 (several assembly chunks, a ragged last
    one): the identity-basis assembly (no sums over steps) against the
    oracle, both Hessian forms."""
    J = 300
    prob = inputs.small_problem(N=5, K=J, J=J, seed=19, dt=0.05, basis="maximal")
    theta = inputs.eval_theta(J, 20)
    ref = orc.evaluate(prob, theta, order=2)
    tol = TOL[precision]
    with q.Problem(prob, precision=precision, hess_method=method) as P:
        Jv, g, H = P.eval_grad_hess(theta)
        assert abs(Jv - ref["J"]) <= tol * abs(ref["J"])
        assert rel(g, ref["grad"]) <= tol and rel(H, ref["hess"]) <= tol, (rel(g, ref["grad"]), rel(H, ref["hess"]))
        np.testing.assert_array_equal(H, H.T)
        if method == q.QOC_HESS_SECOND_ORDER_ADJOINT:
            assert rel(P.buffer(_lib.QOC_BUF_HESS_RAW), ref["hess_raw"]) <= tol
        assert P.diagnostics()["hess_asym"] < 10 * tol


def test_zero_control_and_degenerate_spectrum():
    """f = 0 (theta = 0) and an exactly degenerate H0 (repeated energies)."""
    N, K, J, dt = 6, 4, 80, 0.05
    prob = inputs.small_problem(N=N, K=K, J=J, seed=12, dt=dt)
    prob.H0 = np.diag([-1.0, -1.0, -0.5, -0.5, 0.0, 0.0])
    for theta in (np.zeros(K), inputs.eval_theta(K, 13)):
        check_eval(prob, theta, q.QOC_FP64)
        check_eval(prob, theta, q.QOC_MIXED_FP32)


def test_doubly_degenerate_spectrum_n32():
    """N = 32 made of two identical decoupled 16 x 16 systems (H0 + f M =
    Q (A ⊕ A) Q^T with a random orthogonal Q): every eigenvalue is exactly
    doubly degenerate at every step and every control value, and every
    entry is dense.  The binary32 start ranks the ties by index, each pair
    is a cluster for the refinement (the binary64 clean-up on every step),
    and the propagator derivatives stay well defined (Daleckii-Krein with
    divided differences at equal points)."""
    rng = np.random.default_rng(3232)
    n, K, J, dt = 16, 4, 48, 0.05
    A0 = np.diag(np.sort(rng.uniform(-2.0, 0.0, n)))
    Bx = rng.normal(0.0, 0.05, (n, n))
    A0 = A0 + (Bx + Bx.T) / 2
    Mx = rng.normal(0.0, 0.3, (n, n))
    M1 = (Mx + Mx.T) / 2
    Q, _ = np.linalg.qr(rng.normal(size=(2 * n, 2 * n)))
    H0 = Q @ np.kron(np.eye(2), A0) @ Q.T
    M = Q @ np.kron(np.eye(2), M1) @ Q.T
    H0 = (H0 + H0.T) / 2
    M = (M + M.T) / 2
    prob = inputs.small_problem(N=2 * n, K=K, J=J, seed=33, dt=dt, basis="random")
    prob.H0, prob.M = H0, M
    lam = np.linalg.eigvalsh(H0)
    assert np.abs(lam[1::2] - lam[0::2]).max() <= 1e-12 * np.abs(lam).max()
    theta = inputs.eval_theta(K, 34)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    check_eval(prob, theta, q.QOC_FP64, ref=ref)
    check_eval(prob, theta, q.QOC_MIXED_FP32, ref=ref)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("N", [8, 32])
def test_avoided_crossing(precision, N):
    """A step lands exactly on an avoided crossing (gap 2e-6 against |H| ~ 5):
    levels 0 and 1 of H0 + f M cross at f = 1 with coupling 1e-6, the whole
    system rotated by a random orthogonal Q so every entry is dense.  The
    binary32 eigenvector start mixes the close pair by a large angle there.
    N = 32 takes the register-resident start and the refinement's step order
    (near-degenerate steps first)."""
    rng = np.random.default_rng(77)
    K, J, dt, c = 3, 120, 0.02, 1e-6
    A = rng.normal(0.0, 0.05, (N - 2, N - 2))
    H0 = np.zeros((N, N)); M = np.zeros((N, N))
    H0[:2, :2] = [[0.0, c], [c, 1.0]]
    M[:2, :2] = [[0.0, 0.0], [0.0, -1.0]]
    H0[2:, 2:] = np.diag(np.linspace(2.0, 5.0, N - 2)) + (A + A.T) / 2
    Bm = rng.normal(0.0, 0.3, (N - 2, N - 2))
    M[2:, 2:] = (Bm + Bm.T) / 2
    Q, _ = np.linalg.qr(rng.normal(size=(N, N)))
    H0 = Q @ H0 @ Q.T; H0 = (H0 + H0.T) / 2
    M = Q @ M @ Q.T; M = (M + M.T) / 2
    j = np.arange(J)
    B = np.stack([j / (J // 2), np.sin(np.pi * j / J), np.sin(2 * np.pi * j / J)], axis=1)
    alpha = np.zeros(N, complex); alpha[0] = 1.0
    beta = rng.normal(size=N) + 1j * rng.normal(size=N); beta /= np.linalg.norm(beta)
    prob = inputs.Problem(H0, M, alpha, beta, B, dt, dt, 1.0, name="avoided-crossing")
    theta = np.array([1.0, 0.0, 0.0])      # f at step J/2 is exactly 1
    lam = np.linalg.eigvalsh(H0 + M)
    assert np.diff(lam).min() < 3e-6
    check_eval(prob, theta, precision)
    check_eval(prob, np.array([1.0, 0.3, -0.2]), precision)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_config1_full_size(precision):
    prob = inputs.config_problem(1)
    for seed in (0, 1):
        theta = inputs.eval_theta(prob.K, seed)
        d = check_eval(prob, theta, precision)
        assert d["norm_drift"] < (1e-12 if precision == q.QOC_FP64 else 1e-6)
        assert d["hess_asym"] < TOL[precision]


@pytest.fixture(scope="module")
def config2_ref():
    prob = inputs.config_problem(2)
    theta = inputs.eval_theta(prob.K, 0)
    return prob, theta, orc.evaluate(prob, theta, order=2, keep=True)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_config2_full_size(config2_ref, precision):
    """The plain-vs-mixed workload at full size (N=32, K=64, J=4000): results
    and every per-step intermediate, whole arrays and step by step."""
    prob, theta, ref = config2_ref
    with q.Problem(prob, precision=precision) as P:
        assert P.precision()[0] == precision      # this workload keeps binary32 increments
    check_eval(prob, theta, precision, ref=ref, intermediates=True)


def test_deterministic():
    prob = inputs.small_problem(N=16, K=8, J=100, seed=3, dt=0.05)
    theta = inputs.eval_theta(8, 4)
    for prec in (q.QOC_FP64, q.QOC_MIXED_FP32):
        with q.Problem(prob, precision=prec) as P:
            r1 = P.eval_grad_hess(theta)
            r2 = P.eval_grad_hess(theta)
        assert r1[0] == r2[0]
        np.testing.assert_array_equal(r1[1], r2[1])
        np.testing.assert_array_equal(r1[2], r2[2])


def test_eval_J_and_grad_entry_points():
    prob = inputs.small_problem(N=8, K=6, J=90, seed=14, dt=0.05)
    theta = inputs.eval_theta(6, 15)
    ref = orc.evaluate(prob, theta, order=1)
    with q.Problem(prob) as P:
        assert abs(P.eval_J(theta) - ref["J"]) <= 1e-10 * abs(ref["J"])
        J, g = P.eval_grad(theta)
        assert rel(g, ref["grad"]) <= 1e-10
        with pytest.raises(q.QocError) as e:
            P.eval_J(np.full(6, np.nan))
        assert e.value.status == _lib.QOC_EINVAL


def test_device_pointer_entry_point():
    torch = pytest.importorskip("torch")
    prob = inputs.small_problem(N=8, K=6, J=90, seed=16, dt=0.05)
    theta = inputs.eval_theta(6, 17)
    stream = torch.cuda.current_stream()
    with q.Problem(prob, cuda_stream=stream.cuda_stream) as P:
        J, g, H = P.eval_grad_hess(theta)
        th = torch.tensor(theta, dtype=torch.float64, device="cuda")
        out = torch.zeros(1 + 6 + 36, dtype=torch.float64, device="cuda")
        q.qoc_eval_grad_hess_dev(P.handle, th.data_ptr(), out.data_ptr())
        q.qoc_sync_status(P.handle)
        o = out.cpu().numpy()
    assert o[0] == J
    np.testing.assert_array_equal(o[1:7], g)
    np.testing.assert_array_equal(o[7:].reshape(6, 6), H)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_trust_region_config1(precision):
    """Exact-Hessian trust region from theta = 0 (Sec. IV-B): both converge to
    the same J, |grad| below tolerance, Hessian positive definite."""
    prob = inputs.config_problem(1)
    th_o, info_o = orc.trust_region_solve(prob, np.zeros(prob.K), gtol=1e-8, xtol=1e-12)
    with q.Problem(prob, precision=precision) as P:
        th, info = P.trust_region_solve(np.zeros(prob.K), gtol=1e-8 if precision == 0 else 1e-5,
                                        xtol=1e-12)
        J, g, H = P.eval_grad_hess(th)
    assert info["stop"] == "gtol", info
    assert abs(info["J"] - info_o["J"]) <= (1e-8 if precision == q.QOC_FP64 else 1e-6) * abs(info_o["J"])
    assert np.linalg.eigvalsh(H).min() > 0
    if precision == q.QOC_FP64:
        assert info["iters"] == info_o["iters"]
        assert rel(th, th_o) < 1e-6


@pytest.mark.parametrize("bs", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_time_blocking(bs, precision):
    """Blocked sweeps (bs steps per dependent step, ragged last block) and the
    per-step sweeps (bs = 1) give the oracle's results, both Hessian forms."""
    prob = inputs.small_problem(N=7, K=5, J=37, seed=77, dt=0.05, basis="random")
    theta = inputs.eval_theta(5, 78)
    ref = orc.evaluate(prob, theta, order=2, keep=True)
    tol = TOL[precision]
    for method in (q.QOC_HESS_SECOND_ORDER_ADJOINT, q.QOC_HESS_TANGENT):
        with q.Problem(prob, precision=precision, hess_method=method, block_steps=bs) as P:
            J, g, H = P.eval_grad_hess(theta)
            assert abs(J - ref["J"]) <= tol * abs(ref["J"])
            assert rel(g, ref["grad"]) <= tol
            assert rel(H, ref["hess"]) <= tol
            tin = TOL_INTER[precision]
            assert rel(P.buffer(_lib.QOC_BUF_STATE), ref["a"]) <= tin
            assert rel(P.buffer(_lib.QOC_BUF_COSTATE)[1:], ref["lam"][1:]) <= tin
            assert rel(P.buffer(_lib.QOC_BUF_U), ref["U"]) <= tin
            if method == q.QOC_HESS_SECOND_ORDER_ADJOINT:
                Vexp = oracle_V0(prob, ref) if split_applied(P, prob, method, bs) else ref["V"]
                assert rel(P.buffer(_lib.QOC_BUF_V), Vexp) <= tin
            # gradient-only and cost-only evaluations (chains without panels)
            J1, g1 = P.eval_grad(theta)
            assert abs(J1 - ref["J"]) <= tol * abs(ref["J"])
            assert rel(g1, ref["grad"]) <= tol
            assert abs(P.eval_J(theta) - ref["J"]) <= tol * abs(ref["J"])


def test_block_steps_validation():
    prob = inputs.small_problem(N=4, K=2, J=5, seed=1, dt=0.05)
    with q.Problem(prob) as P:
        for bad in (0, 9, 6):
            with pytest.raises(q.QocError):
                q.qoc_set_block_steps(P.handle, bad)


@pytest.mark.parametrize("N,K,J", [(32, 9, 64), (20, 7, 45), (40, 7, 50)], ids=lambda v: str(v))
def test_panel_columns(N, K, J):
    """Several panel columns per CTA (ragged last CTA): the oracle's results in
    both precisions; for binary32 panels with N <= 32 the column count leaves
    the arithmetic unchanged (the same warp-specialised kernel), so the
    results equal the one-column ones bit for bit."""
    prob = inputs.small_problem(N=N, K=K, J=J, seed=500 + N, dt=0.05, basis="random")
    theta = inputs.eval_theta(K, 501)
    ref = orc.evaluate(prob, theta, order=2)
    for precision in (q.QOC_FP64, q.QOC_MIXED_FP32):
        tol = TOL[precision]
        res = {}
        for kc in (1, 2, 4):
            with q.Problem(prob, precision=precision, panel_columns=kc) as P:
                res[kc] = P.eval_grad_hess(theta)
            Jv, g, H = res[kc]
            assert abs(Jv - ref["J"]) <= tol * abs(ref["J"]), (precision, kc)
            assert rel(g, ref["grad"]) <= tol and rel(H, ref["hess"]) <= tol, (precision, kc)
        if precision == q.QOC_MIXED_FP32 and N <= 32:
            for kc in (2, 4):
                assert res[kc][0] == res[1][0]
                assert np.array_equal(res[kc][1], res[1][1]) and np.array_equal(res[kc][2], res[1][2])


def _estimate(prob, bs):
    """The binary32 increment error estimate of qoc_precision (include/qoc.h)."""
    N = prob.N
    m = np.trace(prob.H0) / N
    sig2 = (np.sum((prob.H0 - m * np.eye(N)) ** 2) + np.sum(prob.M ** 2) * np.sum(prob.B ** 2) / prob.J) / N
    return 0.3 * 2.0 ** -24 * prob.dt * np.sqrt(sig2) * np.sqrt(prob.J * N * bs)


def test_precision_policy():
    """QOC_MIXED_FP32 keeps binary32 increments only while the estimated
    error stays within 1e-6; QOC_MIXED_FP32_ALWAYS keeps them regardless;
    a block length that would raise the estimate above 1e-6 is refused."""
    small = inputs.small_problem(N=8, K=4, J=200, seed=3, dt=0.05)
    big = inputs.small_problem(N=64, K=16, J=2000, seed=4, dt=0.05)
    assert _estimate(small, 4) < 1e-6 < _estimate(big, 4)
    with q.Problem(small, precision=q.QOC_MIXED_FP32) as P:
        eff, est = P.precision()
        assert eff == q.QOC_MIXED_FP32 and abs(est - _estimate(small, 4)) <= 1e-12 * est
    with q.Problem(big, precision=q.QOC_MIXED_FP32) as P:
        eff, est = P.precision()
        assert eff == q.QOC_FP64 and abs(est - _estimate(big, 8)) <= 1e-12 * est
    with q.Problem(big, precision=q.QOC_MIXED_FP32_ALWAYS) as P:
        assert P.precision()[0] == q.QOC_MIXED_FP32
    with q.Problem(big, precision=q.QOC_FP64) as P:
        assert P.precision()[0] == q.QOC_FP64
    # a time step at which block length 4 stays within 1e-6 but 8 does not
    edge = inputs.small_problem(N=8, K=4, J=200, seed=3, dt=0.05)
    edge.dt *= 0.85e-6 / _estimate(small, 4)
    assert _estimate(edge, 4) < 1e-6 < _estimate(edge, 8)
    with q.Problem(edge, precision=q.QOC_MIXED_FP32) as P:
        assert P.precision()[0] == q.QOC_MIXED_FP32
        q.qoc_set_block_steps(P.handle, 2)
        with pytest.raises(q.QocError) as e:
            q.qoc_set_block_steps(P.handle, 8)
        assert e.value.status == _lib.QOC_EINVAL
    with q.Problem(edge, precision=q.QOC_MIXED_FP32_ALWAYS) as P:
        q.qoc_set_block_steps(P.handle, 8)
