"""Plain FP64 CPU oracle for the second-order adjoint method (Bhat, arXiv 2505.00529).

TEST INFRASTRUCTURE ONLY.  This module is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by ``bench.py``'s CPU-baseline / reference
leg, and by nothing else.  The product path (the CUDA library and its Python
binding) never imports, links or runs it.  It shares no code with the CUDA
path: the two meet only in the seeded input generators and in test asserts.

What it computes (Sec. II, Eqs. Zdef, discTDSE, discretecost; weights
generalised): for a linear control model f = B theta,

    H_j = H0 + f_j M,   U_j = exp(-i dt H_j),   a_{j+1} = U_j a_j,  a_0 = alpha,
    J(theta) = w_f * sum_j f_j^2 + w_t * |a_J - beta|^2,

(the paper's cost is w_f = 1/2, w_t = rho/2), together with its exact
gradient and Hessian by the first- and second-order adjoint recursions of
Alg. 2, storing every intermediate (states, costates, tangents, second-order
adjoints and the per-step derivatives of the matrix exponential) exactly as
that algorithm lays them out.  Every array is float64 / complex128.

Readings of the paper taken here (each is pinned by a test):
  * lambda_J = 2 w_t (a_J - beta): Eq. lambdafc drops the rho that the
    variation (Eq. varLprime) and mu_J = rho da_J/dtheta carry.
  * dU_j/df_j = -i dt dexp_{Z_j}[M] (Eq. Zdef); Eq. gradatheta prints +i dt,
    Alg. 2 prints -i dt: the latter is the derivative.
  * Eq. d2Ldf2 is used as the total theta-derivative of Eq. dLdf, i.e. with
    the same "-Re" bracket as Eq. dLdf; written with G_j = dU_j/df_j and
    G2_j = d^2 U_j / df_j^2 every term is "+Re".
  * The derivatives of exp (omitted in the paper, Sec. III-A/B) are the
    Daleckii-Krein formulas in the eigenbasis of H_j with the divided
    differences of phi(x) = exp(-i dt x).
"""
from __future__ import annotations

import math
import numpy as np

TAU_DD2 = 1e-3  # dt*|x - z| below which the second divided difference uses its series


# ---------------------------------------------------------------------------
# control model and per-step Hamiltonians (Sec. II, Eq. Zdef; linear model)
# ---------------------------------------------------------------------------

def control_signal(B, theta):
    """f_j = f(j dt; theta) = sum_l B[j, l] theta_l (left-endpoint samples)."""
    return np.asarray(B, float) @ np.asarray(theta, float)


def step_hamiltonians(H0, M, f):
    """H_j = H0 + f_j M, so that Z_j = -i dt H_j (Eq. Zdef, one field)."""
    return H0[None, :, :] + f[:, None, None] * M[None, :, :]


def eigensystems(H):
    """Eigendecompositions V_j D_j V_j^T of every step Hamiltonian (Alg. 2,
    first loop).  Library routine (LAPACK syevd via numpy); eigenvalues
    ascending, eigenvectors in the columns of W_j."""
    lam, W = np.linalg.eigh(H)
    return lam, W


# ---------------------------------------------------------------------------
# divided differences of phi(x) = exp(-i dt x)
# ---------------------------------------------------------------------------

def phase(lam, dt):
    """phi(lambda) = exp(-i dt lambda), the eigenvalues of U_j."""
    return np.exp(-1j * dt * lam)


def _sinc(x):
    """sin(x)/x with the removable singularity filled in."""
    out = np.ones_like(x)
    nz = np.abs(x) > 0
    out[nz] = np.sin(x[nz]) / x[nz]
    return out


def dd1(x, y, dt):
    """First divided difference phi[x, y] = (phi(x) - phi(y)) / (x - y),
    phi'(x) = -i dt phi(x) when x == y.  Written in the exactly equivalent
    form -i dt exp(-i dt (x+y)/2) sinc(dt (x-y)/2), which has no cancellation."""
    x = np.asarray(x, float)
    y = np.asarray(y, float)
    return -1j * dt * np.exp(-1j * dt * 0.5 * (x + y)) * _sinc(0.5 * dt * (x - y))


def dd2(x, y, z, dt, tau=TAU_DD2):
    """Second divided difference phi[x, y, z] (symmetric in its arguments).

    With the points sorted lo <= mid <= hi:
      dt*(hi - lo) >  tau: (phi[lo, mid] - phi[mid, hi]) / (lo - hi)
      dt*(hi - lo) <= tau: exp(-i dt c) * sum_{n>=2} (-i dt)^n / n! * h_{n-2}(lo-c, mid-c, hi-c)
    where c is the mean of the three points and h_k is the complete
    homogeneous symmetric polynomial of degree k (the divided difference of
    (u - c)^n over three points).
    """
    x, y, z = np.broadcast_arrays(np.asarray(x, float), np.asarray(y, float),
                                  np.asarray(z, float))
    pts = np.sort(np.stack([x, y, z], axis=-1), axis=-1)
    lo, mid, hi = pts[..., 0], pts[..., 1], pts[..., 2]
    out = np.empty(lo.shape, dtype=np.complex128)
    far = dt * (hi - lo) > tau
    if np.any(far):
        out[far] = (dd1(lo[far], mid[far], dt) - dd1(mid[far], hi[far], dt)) / (lo[far] - hi[far])
    near = ~far
    if np.any(near):
        c = (lo[near] + mid[near] + hi[near]) / 3.0
        u, v, w = lo[near] - c, mid[near] - c, hi[near] - c
        # h_k(u, v, w) by h_k(u,v,w) = h_k(u,v) + w h_{k-1}(u,v,w), h_k(u,v) = sum_i u^i v^(k-i)
        total = np.zeros(u.shape, dtype=np.complex128)
        h2 = [np.ones_like(u)]          # h_k(u, v)
        h3 = [np.ones_like(u)]          # h_k(u, v, w)
        r = np.maximum(np.maximum(np.abs(u), np.abs(v)), np.abs(w))
        for n in range(2, 60):
            k = n - 2
            if k > 0:
                h2.append(h2[-1] * v + u ** k)  # h_k(u,v) = v h_{k-1}(u,v) + u^k
                h3.append(h2[-1] + w * h3[-1])
            coef = (-1j * dt) ** n / math.factorial(n)
            total += coef * h3[k]
            # |h_m| <= C(m+2, 2) r^m, so the next term is bounded by:
            m = k + 1
            nxt = dt ** (n + 1) / math.factorial(n + 1) * (m + 2) * (m + 1) / 2 * r ** m
            if np.all(nxt < 1e-19 * np.maximum(np.abs(total), 1e-300)):
                break
        out[near] = np.exp(-1j * dt * c) * total
    return out


# ---------------------------------------------------------------------------
# propagators and the derivatives of exp (Sec. III-A/B, Alg. 2 third loop)
# ---------------------------------------------------------------------------

def propagators(W, lam, dt):
    """U_j = exp(Z_j) = W_j diag(phi(lambda_j)) W_j^T (Alg. 2, eigen route)."""
    return np.einsum("jpr,jr,jqr->jpq", W, phase(lam, dt), W)


def rotated_dipoles(W, M):
    """M~_j = W_j^T M W_j, the dipole matrix in the eigenbasis of H_j."""
    return np.einsum("jrp,rs,jsq->jpq", W, M, W, optimize=True)


def frechet1(W, lam, M, dt):
    """G_j = dU_j/df_j = -i dt dexp_{Z_j}[M] = W (Gamma1 o M~) W^T with
    Gamma1_pq = phi[lambda_p, lambda_q] (Daleckii-Krein)."""
    Mt = rotated_dipoles(W, M)
    G1 = dd1(lam[:, :, None], lam[:, None, :], dt)
    return np.einsum("jpr,jrs,jqs->jpq", W, G1 * Mt, W, optimize=True)


def frechet2(W, lam, M, dt, chunk=None):
    """G2_j = d^2 U_j / df_j^2 = -dt^2 d^2exp_{Z_j}[M, M] = W X W^T with
    X_pq = 2 sum_r M~_pr M~_rq phi[lambda_p, lambda_r, lambda_q].
    Steps are taken `chunk` at a time (each step on its own; by default as
    many as keep the [chunk, N, N, N] divided-difference array near 2^22
    entries)."""
    J, N = lam.shape
    if chunk is None:
        chunk = max(1, min(64, (1 << 22) // N ** 3))
    out = np.empty((J, N, N), dtype=np.complex128)
    Mt = rotated_dipoles(W, M)
    for j0 in range(0, J, chunk):
        j1 = min(J, j0 + chunk)
        L = lam[j0:j1]
        G2 = dd2(L[:, :, None, None], L[:, None, :, None], L[:, None, None, :], dt)  # [j, p, r, q]
        X = 2.0 * np.einsum("jpr,jrq,jprq->jpq", Mt[j0:j1], Mt[j0:j1], G2)
        out[j0:j1] = np.einsum("jpr,jrs,jqs->jpq", W[j0:j1], X, W[j0:j1], optimize=True)
    return out


# ---------------------------------------------------------------------------
# the recursions of Alg. 2
# ---------------------------------------------------------------------------

def forward_states(U, alpha):
    """a_0 = alpha, a_{j+1} = U_j a_j (Eq. discTDSE).  Returns a_0..a_J."""
    J, N, _ = U.shape
    a = np.empty((J + 1, N), dtype=np.complex128)
    a[0] = alpha
    for j in range(J):
        a[j + 1] = U[j] @ a[j]
    return a


def cost(f, aJ, beta, w_f, w_t):
    """J = w_f sum_j f_j^2 + w_t |a_J - beta|^2 (Eq. discretecost, weighted)."""
    d = aJ - beta
    return float(w_f * np.dot(f, f) + w_t * np.real(np.vdot(d, d)))


def costates(U, aJ, beta, w_t):
    """lambda_J = 2 w_t (a_J - beta), lambda_j = U_j^H lambda_{j+1}
    (Eq. lambdasys with the cost weight restored).  Returns lambda_0..lambda_J."""
    J, N, _ = U.shape
    lam = np.empty((J + 1, N), dtype=np.complex128)
    lam[J] = 2.0 * w_t * (aJ - beta)
    for j in range(J - 1, -1, -1):
        lam[j] = U[j].conj().T @ lam[j + 1]
    return lam


def tangents(U, G, a, B):
    """S_j = d a_j / d theta (N x K): S_0 = 0,
    S_{j+1} = U_j S_j + G_j a_j b_j^T (Eq. gradatheta / Alg. 2 tangent loop,
    all columns l at once).  Returns S_0..S_J."""
    J, N, _ = U.shape
    K = B.shape[1]
    S = np.zeros((J + 1, N, K), dtype=np.complex128)
    for j in range(J):
        S[j + 1] = U[j] @ S[j] + np.outer(G[j] @ a[j], B[j])
    return S


def second_adjoints(U, G, lam, SJ, B, w_t):
    """mu_{j,l} = d lambda_j / d theta_l (N x K): mu_J = 2 w_t S_J,
    mu_j = U_j^H mu_{j+1} + G_j^H lambda_{j+1} b_j^T (Eq. musys with
    G_j = -i dt dexp[M]; Alg. 2 second-order adjoint loop).  Returns mu_0..mu_J."""
    J, N, _ = U.shape
    K = B.shape[1]
    mu = np.empty((J + 1, N, K), dtype=np.complex128)
    mu[J] = 2.0 * w_t * SJ
    for j in range(J - 1, -1, -1):
        mu[j] = U[j].conj().T @ mu[j + 1] + np.outer(G[j].conj().T @ lam[j + 1], B[j])
    return mu


def gradient(B, f, w_f, G, a, lam):
    """Eq. dLdf: dJ/dtheta = B^T (2 w_f f + g), g_j = Re(lambda_{j+1}^H G_j a_j)."""
    J = B.shape[0]
    g = np.array([np.real(np.vdot(lam[j + 1], G[j] @ a[j])) for j in range(J)])
    return B.T @ (2.0 * w_f * f + g), g


def hessian(B, w_f, G, G2, a, lam, S, mu):
    """Eq. d2Ldf2 (linear model, so d^2 f / dtheta^2 = 0):

        Hess = B^T diag(2 w_f + c) B + B^T V + B^T U
        c_j    = Re(lambda_{j+1}^H G2_j a_j)
        V[j,m] = Re(mu_{j+1,m}^H G_j a_j)
        U[j,m] = Re(lambda_{j+1}^H G_j S_{j,m})

    Returns the unsymmetrised Hessian and (c, V, U)."""
    J, K = B.shape
    c = np.empty(J)
    V = np.empty((J, K))
    Uc = np.empty((J, K))
    for j in range(J):
        p = G[j] @ a[j]
        c[j] = np.real(np.vdot(lam[j + 1], G2[j] @ a[j]))
        V[j] = np.real(mu[j + 1].conj().T @ p)
        Uc[j] = np.real((G[j].conj().T @ lam[j + 1]).conj() @ S[j])
    H = B.T @ ((2.0 * w_f + c)[:, None] * B) + B.T @ V + B.T @ Uc
    return H, c, V, Uc


# ---------------------------------------------------------------------------
# one full evaluation in Alg. 2 order
# ---------------------------------------------------------------------------

def evaluate(prob, theta, order=2, keep=False):
    """Alg. 2 (order=2) or Alg. 1 (order=1) for one theta.

    Returns a dict with J, grad, (hess, hess_raw, asym, c, V, U) and, with
    keep=True, every stored intermediate."""
    theta = np.asarray(theta, float)
    return evaluate_samples(prob, control_signal(prob.B, theta), prob.B, order, keep)


def evaluate_model(prob, f, jac, order=2):
    """Alg. 2 for a control model f(t; theta) that need not be linear in
    theta: the samples f_j and the Jacobian rows b_j = df_j/dtheta at the
    current theta are given.  Eq. d2Ldf2 then carries, besides the linear
    model's terms, sum_j d_j d^2 f_j/dtheta^2 with d_j = dJ/df_j =
    2 w_f f_j + g_j (its control-cost part and the dexp.M bracket with the
    second derivative of f); that term belongs to the model.  Returns the
    dict of evaluate() for (f, jac) -- grad = jac^T d and hess the Hessian
    without the model's second-derivative term -- plus "d"."""
    f = np.asarray(f, float)
    jac = np.asarray(jac, float)
    out = evaluate_samples(prob, f, jac, order)
    if order >= 1:
        out["d"] = 2 * prob.w_f * f + out["g"]
    return out


def evaluate_samples(prob, f, B, order=2, keep=False):
    """Alg. 2 / Alg. 1 from the control samples f and the rows b_j of B."""
    H = step_hamiltonians(prob.H0, prob.M, f)
    lam_e, W = eigensystems(H)                       # first loop: store V_j, D_j
    U = propagators(W, lam_e, prob.dt)
    a = forward_states(U, prob.alpha)                # first loop: a_{j+1}
    Jval = cost(f, a[-1], prob.beta, prob.w_f, prob.w_t)
    out = {"J": Jval, "f": f}
    if order == 0:
        if keep:
            out.update(W=W, eig=lam_e, U=U, a=a)
        return out
    lam = costates(U, a[-1], prob.beta, prob.w_t)   # second loop
    G = frechet1(W, lam_e, prob.M, prob.dt)          # third loop: dexp . M
    grad, g = gradient(B, f, prob.w_f, G, a, lam)
    out.update(grad=grad, g=g)
    if order >= 2:
        G2 = frechet2(W, lam_e, prob.M, prob.dt)     # third loop: d^2exp . (M x M)
        S = tangents(U, G, a, B)                # fourth loop
        mu = second_adjoints(U, G, lam, S[-1], B, prob.w_t)  # fifth loop
        Hraw, c, V, Uc = hessian(B, prob.w_f, G, G2, a, lam, S, mu)
        nrm = np.linalg.norm(Hraw)
        out.update(hess=0.5 * (Hraw + Hraw.T), hess_raw=Hraw,
                   asym=float(np.linalg.norm(Hraw - Hraw.T) / max(nrm, 1e-300)),
                   c=c, V=V, U=Uc, SJ=S[-1])
        if keep:
            out.update(G2=G2, S=S, mu=mu)
    if keep:
        out.update(W=W, eig=lam_e, U_prop=U, G=G, a=a, lam=lam)
    return out


def eval_J(prob, theta):
    return evaluate(prob, theta, order=0)["J"]


def eval_grad(prob, theta):
    r = evaluate(prob, theta, order=1)
    return r["J"], r["grad"]


def eval_grad_hess(prob, theta):
    r = evaluate(prob, theta, order=2)
    return r["J"], r["grad"], r["hess"]


# ---------------------------------------------------------------------------
# independent cross-checks (exact identities of the discrete problem)
# ---------------------------------------------------------------------------

def gradient_forward_tangent(prob, f, aJ, SJ):
    """dJ/dtheta = 2 w_f B^T f + 2 w_t Re(S_J^H (a_J - beta)) (forward mode)."""
    return 2.0 * prob.w_f * prob.B.T @ f + 2.0 * prob.w_t * np.real(SJ.conj().T @ (aJ - prob.beta))


def hessian_tangent_form(prob, c, Uc, SJ):
    """The same Hessian without mu: unrolling the mu recursion gives
    B^T V = 2 w_t Re(S_J^H S_J) + U^T B, hence
    Hess = B^T diag(2 w_f + c) B + 2 w_t Re(S_J^H S_J) + B^T U + U^T B."""
    B = prob.B
    return (B.T @ ((2.0 * prob.w_f + c)[:, None] * B) + 2.0 * prob.w_t * np.real(SJ.conj().T @ SJ)
            + B.T @ Uc + Uc.T @ B)


# ---------------------------------------------------------------------------
# trust-region solve (Sec. IV-B couples Alg. 2 with an exact-Hessian trust
# region; the paper does not spell the method out, so this is the textbook
# one: Nocedal & Wright Alg. 4.1 with the exact (More-Sorensen) subproblem)
# ---------------------------------------------------------------------------

def tr_subproblem(g, H, radius):
    """argmin_s g^T s + 1/2 s^T H s subject to |s| <= radius, exactly,
    through the eigendecomposition H = Q diag(d) Q^T and the secular
    equation |s(sigma)| = radius, s(sigma) = -(H + sigma I)^{-1} g, including
    the hard case.  Returns (s, sigma)."""
    d, Q = np.linalg.eigh(H)
    gt = Q.T @ g
    dmin = d[0]
    if dmin > 0:
        s_t = -gt / d
        if np.linalg.norm(s_t) <= radius:
            return Q @ s_t, 0.0
    lo = max(0.0, -dmin)

    def snorm(sig):
        return np.linalg.norm(gt / (d + sig))

    # hard case: g has (numerically) no component along the lowest eigenspace
    mask = np.abs(d - dmin) <= 1e-12 * max(1.0, abs(dmin))
    gperp = gt.copy()
    if np.linalg.norm(gt[mask]) <= 1e-14 * max(1.0, np.linalg.norm(gt)):
        gperp[mask] = 0.0
        dd = d + lo
        s_t = np.zeros_like(gt)
        nm = ~mask
        s_t[nm] = -gperp[nm] / dd[nm]
        ns = np.linalg.norm(s_t)
        if ns <= radius:
            z = np.zeros_like(gt)
            z[np.argmax(mask)] = 1.0
            s_t = s_t + math.sqrt(max(radius ** 2 - ns ** 2, 0.0)) * z
            return Q @ s_t, lo
    # Newton on 1/|s(sigma)| - 1/radius (concave, monotone), safeguarded by bisection
    sig_hi = lo + np.linalg.norm(g) / radius + 1.0
    while snorm(sig_hi) > radius:
        sig_hi *= 2.0
    sig = sig_hi
    sig_lo = lo
    for _ in range(200):
        s_t = -gt / (d + sig)
        ns = np.linalg.norm(s_t)
        phi = 1.0 / ns - 1.0 / radius
        if abs(ns - radius) <= 1e-13 * radius:
            break
        if phi < 0:
            sig_lo = sig
        else:
            sig_hi = sig
        dns = -np.sum(gt ** 2 / (d + sig) ** 3) / ns       # d|s|/dsigma
        dphi = -dns / ns ** 2
        new = sig - phi / dphi
        if not (sig_lo < new < sig_hi):
            new = 0.5 * (sig_lo + sig_hi)
        sig = new
    return Q @ (-gt / (d + sig)), sig


def trust_region_solve(prob, theta0, gtol=1e-10, xtol=1e-10, radius0=1.0,
                       radius_max=1e3, max_iter=10000, eta=0.1):
    """Textbook trust-region Newton iteration with exact gradient and Hessian
    from Alg. 2.  Stops when |grad| < gtol or the trust radius (the bound
    on the step |theta^{m+1} - theta^m|) falls below xtol (Sec. III-A/B stop
    rule with delta = xtol, epsilon = gtol).

    Returns (theta, info)."""
    theta = np.array(theta0, float)
    radius = radius0
    Jc, g, H = eval_grad_hess(prob, theta)
    n_J, n_gh = 0, 1
    stop = "max_iter"
    it = 0
    for it in range(1, max_iter + 1):
        if np.linalg.norm(g) < gtol:
            stop = "gtol"
            it -= 1
            break
        s, _ = tr_subproblem(g, H, radius)
        pred = -(g @ s + 0.5 * s @ H @ s)
        if pred <= 0:
            stop = "no_decrease"
            break
        Jt = eval_J(prob, theta + s)
        n_J += 1
        rho = (Jc - Jt) / pred
        ns = np.linalg.norm(s)
        if rho < 0.25:
            radius = 0.25 * radius
        elif rho > 0.75 and abs(ns - radius) <= 1e-8 * radius:
            radius = min(2.0 * radius, radius_max)
        if rho > eta:
            theta = theta + s
            Jc, g, H = eval_grad_hess(prob, theta)
            n_gh += 1
        if radius < xtol:
            stop = "xtol"
            break
    return theta, {"iters": it, "J": Jc, "grad_norm": float(np.linalg.norm(g)),
                   "stop": stop, "n_eval_J": n_J, "n_eval_gh": n_gh, "hess": H}


# ---------------------------------------------------------------------------
# Alg. 1 with a quasi-Newton trust region (Sec. IV-B: gradients alone, the
# optimiser building its Hessian approximation by BFGS updates)
# ---------------------------------------------------------------------------

def bfgs_update(Bk, s, y, min_curvature=1e-8):
    """BFGS update of a Hessian approximation (Nocedal & Wright, Eq. 6.19):
    B+ = B - (B s)(B s)^T / (s^T B s) + y y^T / (y^T s).  Skipped (B returned
    unchanged) when the curvature y^T s is not above min_curvature |s| |y|,
    the condition under which the update keeps B positive definite."""
    sy = float(y @ s)
    if not sy > min_curvature * np.linalg.norm(s) * np.linalg.norm(y):
        return Bk
    Bs = Bk @ s
    return Bk - np.outer(Bs, Bs) / float(s @ Bs) + np.outer(y, y) / sy


def trust_region_solve_bfgs(prob, theta0, gtol=1e-10, xtol=1e-10, radius0=1.0,
                            radius_max=1e3, max_iter=10000, eta=0.1):
    """The trust region of trust_region_solve with the exact Hessian replaced
    by a BFGS approximation built from Alg. 1 gradients: B = I until the
    first update, which starts from (y^T y / y^T s) I; every evaluated trial
    point updates B with s = its step and y = its gradient minus the current
    one (accepted or not).  Returns (theta, info)."""
    theta = np.array(theta0, float)
    K = theta.size
    radius = radius0
    Jc, g = eval_grad(prob, theta)
    Bk = np.eye(K)
    scaled = False
    n_J = 0
    stop = "max_iter"
    it = 0
    for it in range(1, max_iter + 1):
        if np.linalg.norm(g) < gtol:
            stop = "gtol"
            it -= 1
            break
        s, _ = tr_subproblem(g, Bk, radius)
        pred = -(g @ s + 0.5 * s @ Bk @ s)
        if pred <= 0:
            stop = "no_decrease"
            break
        Jt, gt = eval_grad(prob, theta + s)
        n_J += 1
        y = gt - g
        if not scaled and y @ s > 0:
            Bk = (y @ y) / (y @ s) * np.eye(K)
            scaled = True
        Bk = bfgs_update(Bk, s, y)
        rho = (Jc - Jt) / pred
        ns = np.linalg.norm(s)
        if rho < 0.25:
            radius = 0.25 * radius
        elif rho > 0.75 and abs(ns - radius) <= 1e-8 * radius:
            radius = min(2.0 * radius, radius_max)
        if rho > eta:
            theta = theta + s
            Jc, g = Jt, gt
        if radius < xtol:
            stop = "xtol"
            break
    return theta, {"iters": it, "J": Jc, "grad_norm": float(np.linalg.norm(g)),
                   "stop": stop, "n_eval_grad": n_J + 1, "hess_approx": Bk}
