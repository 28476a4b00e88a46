"""Pins of the FP64 oracle against things other than itself: library routines
(scipy expm / expm_frechet / block-matrix Frechet identity), closed forms,
brute force in 50-digit arithmetic, finite differences and exact identities
of the discrete problem.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla

from oracle import qoc_oracle as orc
from paper_2505_00529_gb300 import inputs


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def small():
    return inputs.small_problem(N=5, K=3, J=40, seed=11, dt=0.05)


# --------------------------------------------------------------------------
# divided differences
# --------------------------------------------------------------------------

def test_dd1_against_definition_in_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    rng = np.random.default_rng(0)
    dt = 0.013
    xs = rng.uniform(-20, 5, size=40)
    ys = np.concatenate([xs[:10], xs[10:20] + 1e-9, xs[20:30] + 1e-4, rng.uniform(-20, 5, 10)])
    got = orc.dd1(xs, ys, dt)
    for x, y, g in zip(xs, ys, got):
        X, Y = mp.mpf(float(x)), mp.mpf(float(y))
        phi = lambda u: mp.exp(-1j * mp.mpf(dt) * u)
        if X == Y:
            ref = -1j * mp.mpf(dt) * phi(X)
        else:
            ref = (phi(X) - phi(Y)) / (X - Y)
        ref = complex(ref)
        assert abs(g - ref) <= 1e-14 * abs(ref)


def test_dd2_against_opitz_block_exponential():
    """phi[x,y,z] is the (0,2) entry of phi of the bidiagonal matrix with
    x, y, z on the diagonal and ones above it (Opitz)."""
    rng = np.random.default_rng(1)
    dt = 0.02
    for _ in range(50):
        x, y, z = rng.uniform(-10, 2, size=3)
        A = np.array([[x, 1.0, 0.0], [0.0, y, 1.0], [0.0, 0.0, z]])
        ref = sla.expm(-1j * dt * A)[0, 2]
        got = orc.dd2(x, y, z, dt)
        assert abs(got - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("gap", [0.0, 1e-9, 1e-5, 0.9e-3 / 0.02, 1.1e-3 / 0.02, 0.3])
def test_dd2_against_recursive_definition_in_50_digits(gap):
    """Both branches (series / recursion), straddling the switch at dt*|x-z| = 1e-3."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 60
    dt = 0.02
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = rng.uniform(-8, 0)
        y = x + gap * rng.uniform(0, 1)
        z = x + gap
        X, Y, Z = (mp.mpf(float(v)) for v in (x, y, z))
        d = mp.mpf(dt)

        def f(u):
            return mp.exp(-1j * d * u)

        def f1(u, v):
            return -1j * d * f(u) if u == v else (f(u) - f(v)) / (u - v)

        if X == Z:
            ref = (-1j * d) ** 2 / 2 * f(X)
        elif X == Y:  # phi[x,x,z] = (phi[x,z] - phi'(x)) / (z - x)
            ref = (f1(X, Z) - f1(X, X)) / (Z - X)
        else:
            ref = (f1(X, Y) - f1(Y, Z)) / (X - Z)
        ref = complex(ref)
        got = orc.dd2(x, y, z, dt)
        assert abs(got - ref) <= 2e-12 * abs(ref), (gap, got, ref)
        # symmetric in its arguments
        assert abs(orc.dd2(z, x, y, dt) - got) <= 1e-15 * abs(ref)


# --------------------------------------------------------------------------
# propagators and derivatives of exp against scipy
# --------------------------------------------------------------------------

def _steps(prob, theta):
    f = orc.control_signal(prob.B, theta)
    H = orc.step_hamiltonians(prob.H0, prob.M, f)
    lam, W = orc.eigensystems(H)
    return f, H, lam, W


def test_propagators_against_expm(small):
    th = inputs.eval_theta(small.K, 3)
    f, H, lam, W = _steps(small, th)
    U = orc.propagators(W, lam, small.dt)
    for j in (0, 7, 39):
        ref = sla.expm(-1j * small.dt * H[j])
        assert rel(U[j], ref) < 1e-13


def test_frechet1_against_expm_frechet(small):
    th = inputs.eval_theta(small.K, 4)
    f, H, lam, W = _steps(small, th)
    G = orc.frechet1(W, lam, small.M, small.dt)
    for j in (0, 13, 39):
        Z = -1j * small.dt * H[j]
        E = -1j * small.dt * small.M
        _, ref = sla.expm_frechet(Z, E)
        assert rel(G[j], ref) < 1e-12


def test_frechet2_against_block_expm(small):
    """expm([[Z,E,0],[0,Z,E],[0,0,Z]]) has (1,3) block = 1/2 d^2exp_Z[E,E]."""
    th = inputs.eval_theta(small.K, 5)
    f, H, lam, W = _steps(small, th)
    G2 = orc.frechet2(W, lam, small.M, small.dt)
    N = small.N
    for j in (0, 21, 39):
        Z = -1j * small.dt * H[j]
        E = -1j * small.dt * small.M
        Bk = np.zeros((3 * N, 3 * N), dtype=complex)
        for b in range(3):
            Bk[b * N:(b + 1) * N, b * N:(b + 1) * N] = Z
        Bk[0:N, N:2 * N] = E
        Bk[N:2 * N, 2 * N:3 * N] = E
        ref = 2.0 * sla.expm(Bk)[0:N, 2 * N:3 * N]
        assert rel(G2[j], ref) < 1e-10


def test_frechet2_with_degenerate_spectrum():
    """Exactly degenerate eigenvalues (H0 with repeated energies, f = 0)
    exercise the confluent branches of both divided differences."""
    N, dt = 4, 0.1
    H0 = np.diag([-1.0, -1.0, 0.5, 0.5])
    rng = np.random.default_rng(7)
    M = rng.normal(size=(N, N))
    M = M + M.T
    lam, W = np.linalg.eigh(H0[None])
    G = orc.frechet1(W, lam, M, dt)[0]
    G2 = orc.frechet2(W, lam, M, dt)[0]
    Z = -1j * dt * H0
    E = -1j * dt * M
    _, refG = sla.expm_frechet(Z, E)
    Bk = np.zeros((3 * N, 3 * N), dtype=complex)
    for b in range(3):
        Bk[b * N:(b + 1) * N, b * N:(b + 1) * N] = Z
    Bk[0:N, N:2 * N] = E
    Bk[N:2 * N, 2 * N:3 * N] = E
    refG2 = 2.0 * sla.expm(Bk)[0:N, 2 * N:3 * N]
    assert rel(G, refG) < 1e-12
    assert rel(G2, refG2) < 1e-10


# --------------------------------------------------------------------------
# closed forms
# --------------------------------------------------------------------------

def test_zero_control_closed_form():
    """f == 0: a_J = exp(-i T H0) alpha exactly."""
    prob = inputs.config_problem(1)
    r = orc.evaluate(prob, np.zeros(prob.K), order=0, keep=True)
    aJ_ref = sla.expm(-1j * prob.T * prob.H0) @ prob.alpha
    assert rel(r["a"][-1], aJ_ref) < 1e-12
    d = aJ_ref - prob.beta
    J_ref = prob.w_t * np.vdot(d, d).real
    assert abs(r["J"] - J_ref) < 1e-11 * abs(J_ref)  # 1000 steps of rounding


def test_commuting_case_closed_form():
    """H0 = diag(h), M = diag(m): a_J,p = alpha_p exp(-i (T h_p + m_p F)),
    F = dt 1^T B theta, so J, grad and Hess have closed forms in F."""
    rng = np.random.default_rng(8)
    N, K, J, dt = 3, 4, 60, 0.07
    h = rng.uniform(-2, 0, N)
    m = rng.normal(0, 0.7, N)
    B = rng.normal(size=(J, K))
    alpha = (rng.normal(size=N) + 1j * rng.normal(size=N))
    alpha /= np.linalg.norm(alpha)
    beta = (rng.normal(size=N) + 1j * rng.normal(size=N))
    beta /= np.linalg.norm(beta)
    w_f, w_t = 0.3, 1.7
    prob = inputs.Problem(np.diag(h), np.diag(m), alpha, beta, B, dt, w_f, w_t)
    theta = rng.normal(size=K)
    T = J * dt
    cvec = dt * B.sum(axis=0)
    F = cvec @ theta
    z = np.conj(beta) * alpha * np.exp(-1j * (T * h + m * F))
    # |r_p - beta_p|^2 = |alpha_p|^2 + |beta_p|^2 - 2 Re z_p
    E = w_t * np.sum(np.abs(alpha) ** 2 + np.abs(beta) ** 2 - 2 * z.real)
    dE = w_t * np.sum(-2 * m * z.imag)
    d2E = w_t * np.sum(2 * m ** 2 * z.real)
    Bt = B.T @ B
    J_ref = w_f * theta @ Bt @ theta + E
    g_ref = 2 * w_f * Bt @ theta + dE * cvec
    H_ref = 2 * w_f * Bt + d2E * np.outer(cvec, cvec)
    r = orc.evaluate(prob, theta, order=2)
    assert abs(r["J"] - J_ref) < 1e-12 * abs(J_ref)
    assert rel(r["grad"], g_ref) < 1e-11
    assert rel(r["hess"], H_ref) < 1e-11


def _su2_cost_mp(mp, H0, M, alpha, beta, B, dt, w_f, w_t, theta):
    """J(theta) for N=2 in 50-digit arithmetic: each step is the SU(2)
    closed form exp(-i dt (h0 I + h.sigma)) = exp(-i dt h0)(cos(dt|h|) I -
    i sin(dt|h|) (h.sigma)/|h|), h = ((a-d)/2 -> z, b -> x) for [[a,b],[b,d]]."""
    th = [t if isinstance(t, mp.mpf) else mp.mpf(float(t)) for t in theta]
    a = [mp.mpc(complex(alpha[0])), mp.mpc(complex(alpha[1]))]
    fsq = mp.mpf(0)
    d = mp.mpf(dt)
    for j in range(B.shape[0]):
        fj = mp.fsum(mp.mpf(float(B[j, l])) * th[l] for l in range(len(th)))
        fsq += fj * fj
        A = mp.mpf(float(H0[0, 0])) + fj * mp.mpf(float(M[0, 0]))
        Dd = mp.mpf(float(H0[1, 1])) + fj * mp.mpf(float(M[1, 1]))
        Bo = mp.mpf(float(H0[0, 1])) + fj * mp.mpf(float(M[0, 1]))
        h0 = (A + Dd) / 2
        hz = (A - Dd) / 2
        hx = Bo
        hn = mp.sqrt(hx * hx + hz * hz)
        c, s = mp.cos(d * hn), mp.sin(d * hn)
        ph = mp.exp(-1j * d * h0)
        nx, nz = (hx / hn, hz / hn) if hn != 0 else (mp.mpf(0), mp.mpf(0))
        u00 = ph * (c - 1j * s * nz)
        u11 = ph * (c + 1j * s * nz)
        u01 = ph * (-1j * s * nx)
        a = [u00 * a[0] + u01 * a[1], u01 * a[0] + u11 * a[1]]
    r0 = a[0] - mp.mpc(complex(beta[0]))
    r1 = a[1] - mp.mpc(complex(beta[1]))
    return mp.mpf(w_f) * fsq + mp.mpf(w_t) * (abs(r0) ** 2 + abs(r1) ** 2)


def test_two_level_brute_force_50_digits():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    prob = inputs.small_problem(N=2, K=3, J=25, seed=21, dt=0.08)
    theta = inputs.eval_theta(3, 22)
    args = (prob.H0, prob.M, prob.alpha, prob.beta, prob.B, prob.dt, prob.w_f, prob.w_t)
    J0 = _su2_cost_mp(mp, *args, theta)
    h = mp.mpf("1e-12")
    K = 3
    grad = np.zeros(K)
    hess = np.zeros((K, K))
    e = np.eye(K)

    def Jat(shift):
        th = [mp.mpf(float(t)) for t in theta]
        th = [t + s for t, s in zip(th, shift)]
        return _su2_cost_mp(mp, *args, th)

    for l in range(K):
        sp = [h * e[l, i] for i in range(K)]
        sm = [-h * e[l, i] for i in range(K)]
        grad[l] = float((Jat(sp) - Jat(sm)) / (2 * h))
        for m in range(K):
            spp = [h * (e[l, i] + e[m, i]) for i in range(K)]
            spm = [h * (e[l, i] - e[m, i]) for i in range(K)]
            smp = [h * (-e[l, i] + e[m, i]) for i in range(K)]
            smm = [h * (-e[l, i] - e[m, i]) for i in range(K)]
            hess[l, m] = float((Jat(spp) - Jat(spm) - Jat(smp) + Jat(smm)) / (4 * h * h))
    r = orc.evaluate(prob, theta, order=2)
    assert abs(r["J"] - float(J0)) < 1e-13 * abs(float(J0))
    assert rel(r["grad"], grad) < 1e-12
    assert rel(r["hess"], hess) < 1e-11


# --------------------------------------------------------------------------
# finite differences (gradient of J, Hessian from the gradient)
# --------------------------------------------------------------------------

def _richardson(fun, theta, h):
    K = len(theta)
    out = []
    for l in range(K):
        e = np.zeros(K)
        e[l] = 1.0

        def D(hh):
            return (fun(theta + hh * e) - fun(theta - hh * e)) / (2 * hh)

        out.append((4 * D(h / 2) - D(h)) / 3)
    return np.array(out)


@pytest.mark.parametrize("w", [(None, 1.0), (0.5, 0.5e3)])  # workload weights (dt, 1), paper weights (rho=1e3)
def test_gradient_and_hessian_by_finite_differences(w):
    w_f, w_t = w
    prob = inputs.small_problem(N=4, K=3, J=50, seed=31, dt=0.04, basis="random",
                                w_f=w_f, w_t=w_t)
    theta = inputs.eval_theta(3, 32, scale=0.5)
    r = orc.evaluate(prob, theta, order=2)
    g_fd = _richardson(lambda t: orc.eval_J(prob, t), theta, 1e-3)
    assert rel(r["grad"], g_fd) < 1e-8
    H_fd = np.stack([_richardson(lambda t: orc.eval_grad(prob, t)[1][l], theta, 1e-3)
                     for l in range(3)])
    assert rel(r["hess"], H_fd) < 1e-8
    assert r["asym"] < 1e-12


def test_maximal_model_by_finite_differences():
    """Maximal model f_j = theta_j (Eq. maximal), K = J."""
    J = 12
    prob = inputs.small_problem(N=3, K=J, J=J, seed=41, dt=0.1, basis="maximal")
    theta = inputs.eval_theta(J, 42)
    r = orc.evaluate(prob, theta, order=2)
    g_fd = _richardson(lambda t: orc.eval_J(prob, t), theta, 1e-3)
    assert rel(r["grad"], g_fd) < 1e-8
    H_fd = np.stack([_richardson(lambda t: orc.eval_grad(prob, t)[1][l], theta, 1e-3)
                     for l in range(J)])
    assert rel(r["hess"], H_fd) < 1e-7


# --------------------------------------------------------------------------
# identities and invariants of the discrete problem
# --------------------------------------------------------------------------

def test_forward_tangent_and_tangent_form_identities(small):
    th = inputs.eval_theta(small.K, 51)
    r = orc.evaluate(small, th, order=2, keep=True)
    g2 = orc.gradient_forward_tangent(small, r["f"], r["a"][-1], r["SJ"])
    assert rel(r["grad"], g2) < 1e-12
    H2 = orc.hessian_tangent_form(small, r["c"], r["U"], r["SJ"])
    assert rel(r["hess_raw"], H2) < 1e-12


def test_invariants_along_the_trajectory(small):
    th = inputs.eval_theta(small.K, 52)
    r = orc.evaluate(small, th, order=2, keep=True)
    a, lam, S = r["a"], r["lam"], r["S"]
    J = small.J
    norms = np.linalg.norm(a, axis=1)
    assert np.max(np.abs(norms - 1)) < 1e-13 * J
    # |a_j(theta)| == 1 for all theta => Re(a_j^H S_j) = 0
    assert np.max(np.abs(np.real(np.einsum("jn,jnk->jk", a.conj(), S)))) < 1e-13 * J
    # lambda_j^H a_j is constant in j
    inner = np.einsum("jn,jn->j", lam.conj(), a)
    assert np.max(np.abs(inner - inner[-1])) < 1e-13 * J
    # time reversal recovers alpha
    U = r["U_prop"]
    b = a[-1].copy()
    for j in range(J - 1, -1, -1):
        b = U[j].conj().T @ b
    assert np.linalg.norm(b - small.alpha) < 1e-13 * J


def test_hessian_positive_definite_at_optimum_and_tr_convergence():
    """Config-1 problem solved from theta = 0: converges, and the Hessian at
    the optimum has positive eigenvalues (Sec. IV-B observation)."""
    prob = inputs.config_problem(1)
    theta, info = orc.trust_region_solve(prob, np.zeros(prob.K), gtol=1e-9, xtol=1e-12)
    assert info["stop"] == "gtol", info
    assert np.linalg.eigvalsh(info["hess"]).min() > 0
    r = orc.evaluate(prob, theta, order=1)
    assert r["J"] <= orc.eval_J(prob, np.zeros(prob.K))


# --------------------------------------------------------------------------
# trust-region subproblem and iteration
# --------------------------------------------------------------------------

def _brute_subproblem(g, H, radius, n=20001):
    """K = 2: minimum over a fine polar grid of the disk plus the interior
    Newton point (when it is feasible)."""
    best = None
    ang = np.linspace(0, 2 * np.pi, n)
    for r in np.linspace(0, radius, 401):
        s = np.stack([r * np.cos(ang), r * np.sin(ang)], axis=1)
        v = s @ g + 0.5 * np.einsum("ni,ij,nj->n", s, H, s)
        i = np.argmin(v)
        if best is None or v[i] < best[0]:
            best = (v[i], s[i])
    try:
        sn = -np.linalg.solve(H, g)
        if np.linalg.norm(sn) <= radius and np.all(np.linalg.eigvalsh(H) > 0):
            v = sn @ g + 0.5 * sn @ H @ sn
            if v < best[0]:
                best = (v, sn)
    except np.linalg.LinAlgError:
        pass
    return best


@pytest.mark.parametrize("case", [
    (np.array([1.0, -2.0]), np.array([[2.0, 0.3], [0.3, 1.0]]), 10.0),   # interior
    (np.array([1.0, -2.0]), np.array([[2.0, 0.3], [0.3, 1.0]]), 0.5),    # boundary
    (np.array([0.5, 0.4]), np.array([[-1.0, 0.2], [0.2, 0.5]]), 1.0),    # indefinite
    (np.array([0.0, 0.7]), np.array([[-2.0, 0.0], [0.0, 1.0]]), 1.0),    # hard case
])
def test_tr_subproblem_against_brute_force(case):
    g, H, radius = case
    s, _ = orc.tr_subproblem(g, H, radius)
    assert np.linalg.norm(s) <= radius * (1 + 1e-10)
    v = s @ g + 0.5 * s @ H @ s
    vb, _ = _brute_subproblem(g, H, radius)
    assert v <= vb + 1e-6 * max(1.0, abs(vb))


def test_tr_converges_in_one_step_on_convex_quadratic():
    """w_t = 0 makes J = w_f |B theta|^2 a convex quadratic: one Newton step
    inside the initial radius reaches the minimiser."""
    prob = inputs.small_problem(N=3, K=4, J=30, seed=61, dt=0.05, w_t=0.0)
    theta0 = np.array([0.2, -0.1, 0.3, 0.1])
    theta, info = orc.trust_region_solve(prob, theta0, gtol=1e-10)
    assert info["stop"] == "gtol"
    assert info["n_eval_gh"] == 2 and info["n_eval_J"] == 1
    assert np.linalg.norm(theta) < 1e-10


# --------------------------------------------------------------------------
# Alg. 1 with the BFGS trust region (Sec. IV-B's gradient-only baseline)
# --------------------------------------------------------------------------

def test_bfgs_update_secant_symmetry_and_definiteness():
    """The BFGS update satisfies the secant equation B+ s = y, keeps B
    symmetric and positive definite when y^T s > 0, and is skipped when the
    curvature is not positive (Nocedal & Wright, Sec. 6.1)."""
    rng = np.random.default_rng(5)
    K = 7
    A = rng.normal(size=(K, K))
    B = A @ A.T + K * np.eye(K)
    for _ in range(5):
        s = rng.normal(size=K)
        y = rng.normal(size=K)
        if y @ s <= 0:
            y = -y
        Bp = orc.bfgs_update(B, s, y)
        np.testing.assert_allclose(Bp @ s, y, rtol=1e-12, atol=1e-12 * np.linalg.norm(y))
        np.testing.assert_array_equal(Bp, Bp.T)
        assert np.linalg.eigvalsh(Bp).min() > 0
        assert orc.bfgs_update(B, s, -y) is B
        B = Bp


def test_bfgs_trust_region_on_convex_quadratic():
    """w_t = 0: J = w_f |B theta|^2 is a convex quadratic, every y equals
    A s with A = 2 w_f B^T B; the BFGS trust region must reach the minimiser
    theta = 0 and its last approximation must satisfy the secant equation of
    the quadratic along its last step direction."""
    prob = inputs.small_problem(N=3, K=4, J=30, seed=61, dt=0.05, w_t=0.0)
    A = 2 * prob.w_f * prob.B.T @ prob.B
    theta, info = orc.trust_region_solve_bfgs(prob, np.array([0.2, -0.1, 0.3, 0.1]), gtol=1e-10)
    assert info["stop"] == "gtol", info
    assert np.linalg.norm(theta) < 1e-9
    assert np.linalg.eigvalsh(info["hess_approx"]).min() > 0
    # B reproduces the exact curvature on the span it has explored
    Bk = info["hess_approx"]
    assert np.linalg.norm(Bk - A) < np.linalg.norm(A)


def test_bfgs_trust_region_reaches_the_exact_minimiser():
    """From theta = 0 the BFGS (Alg. 1) and exact-Hessian (Alg. 2) trust
    regions converge to the same local minimiser; the BFGS one needs at
    least as many iterations."""
    prob = inputs.small_problem(N=4, K=3, J=50, seed=62, dt=0.05)
    th2, info2 = orc.trust_region_solve(prob, np.zeros(3), gtol=1e-8, xtol=1e-14)
    th1, info1 = orc.trust_region_solve_bfgs(prob, np.zeros(3), gtol=1e-8, xtol=1e-14)
    assert info1["stop"] == "gtol" and info2["stop"] == "gtol", (info1["stop"], info2["stop"])
    assert np.linalg.norm(th1 - th2) <= 1e-6 * max(1.0, np.linalg.norm(th2))
    assert abs(info1["J"] - info2["J"]) <= 1e-12 * abs(info2["J"])
    assert info1["iters"] >= info2["iters"]


# --------------------------------------------------------------------------
# control models that are not linear in theta (Eq. d2Ldf2 with d^2 f != 0)
# --------------------------------------------------------------------------

def test_model_evaluation_reduces_to_the_linear_one():
    """Samples and Jacobian of a linear model (f = B theta, jac = B) give
    exactly the linear evaluation."""
    prob = inputs.small_problem(N=4, K=3, J=40, seed=71, dt=0.05, basis="random")
    theta = inputs.eval_theta(3, 72)
    a = orc.evaluate(prob, theta, order=2)
    b = orc.evaluate_model(prob, prob.B @ theta, prob.B, order=2)
    assert a["J"] == b["J"]
    np.testing.assert_array_equal(a["grad"], b["grad"])
    np.testing.assert_array_equal(a["hess"], b["hess"])
    np.testing.assert_array_equal(b["d"], 2 * prob.w_f * (prob.B @ theta) + a["g"])


def test_nonlinear_model_gradient_and_hessian_by_finite_differences():
    """f(t) = sum_h v_h tanh(w_h t + c_h): jac^T d is the gradient of
    J(theta) and hess + sum_j d_j d^2 f_j / dtheta^2 its Hessian (central
    differences with Richardson extrapolation)."""
    prob = inputs.small_problem(N=4, K=6, J=60, seed=73, dt=0.05)
    t = np.arange(prob.J) * prob.dt
    theta = np.array([0.7, -0.4, 1.1, 0.3, 0.5, -0.2])

    def full(th):
        f, jac, hf = inputs.tanh_network_control(t, th)
        r = orc.evaluate_model(prob, f, jac, order=2)
        return r["J"], r["grad"], r["hess"] + np.einsum("j,jlm->lm", r["d"], hf)

    def J_of(th):
        f, _, _ = inputs.tanh_network_control(t, th)
        return orc.evaluate_samples(prob, f, np.zeros((prob.J, 1)), order=0)["J"]

    J0, g, H = full(theta)
    g_fd = _richardson(J_of, theta, 1e-3)
    assert np.linalg.norm(g - g_fd) <= 1e-8 * np.linalg.norm(g)
    H_fd = np.stack([_richardson(lambda th, l=l: full(th)[1][l], theta, 1e-3) for l in range(6)])
    assert np.linalg.norm(H - H_fd) <= 1e-6 * np.linalg.norm(H), np.linalg.norm(H - H_fd) / np.linalg.norm(H)
    # the model's own second-derivative term matters here
    f, jac, hf = inputs.tanh_network_control(t, theta)
    r = orc.evaluate_model(prob, f, jac, order=2)
    assert np.linalg.norm(np.einsum("j,jlm->lm", r["d"], hf)) > 1e-3 * np.linalg.norm(H)
