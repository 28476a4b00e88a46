"""Seeded synthetic inputs for the discrete quantum-optimal-control problem.

This module only draws numbers: it holds none of the method's arithmetic, so
both the CUDA path and the CPU oracle take their inputs from it.  The
paper's molecular full-CI matrices (H2, HeH+ in STO-3G / 6-31G, Sec. II and
Sec. IV) are not available, so CI-shaped synthetic Hamiltonians stand in for
them: a sorted diagonal of "CI energies" plus small (banded) symmetric
couplings, and a dense symmetric dipole matrix M.

Every generator uses ``numpy.random.default_rng(seed)`` with the draw order
energies -> off-diagonals -> M -> target, so a (config, index) pair always
gives the same arrays on any machine.

Layouts (all float64, row-major):
  H0, M      (N, N) real symmetric
  alpha, beta (N,) complex128 (passed to the C ABI as interleaved re/im)
  B          (J, K) control basis, B[j, l] = d f_j / d theta_l
"""
from __future__ import annotations

import dataclasses
import numpy as np


@dataclasses.dataclass
class Problem:
    """One discrete control problem (Sec. II, Eq. discretecost with weights)."""

    H0: np.ndarray
    M: np.ndarray
    alpha: np.ndarray
    beta: np.ndarray
    B: np.ndarray
    dt: float
    w_f: float
    w_t: float
    name: str = ""

    @property
    def N(self) -> int:
        return self.H0.shape[0]

    @property
    def K(self) -> int:
        return self.B.shape[1]

    @property
    def J(self) -> int:
        return self.B.shape[0]

    @property
    def T(self) -> float:
        return self.J * self.dt


# ---------------------------------------------------------------------------
# control bases (f = B theta): pure sampling of known functions on the grid
# t_j = j * dt, j = 0..J-1 (left endpoints, Sec. II: f_j = f(j dt; theta)).
# ---------------------------------------------------------------------------

def sine_basis(J: int, dt: float, K: int) -> np.ndarray:
    """B[j, m-1] = sin(m pi t_j / T), m = 1..K."""
    T = J * dt
    t = np.arange(J) * dt
    m = np.arange(1, K + 1)
    return np.sin(np.pi * np.outer(t, m) / T)


def sine_cosine_basis(J: int, dt: float, K: int) -> np.ndarray:
    """Fourier basis on [0, T): first K/2 columns sin(2 pi m t/T), last K/2
    columns cos(2 pi m t/T), m = 1..K/2.  Orthogonal on the grid (B^T B = J/2 I
    for K/2 < J/2).  (The half-period family sin/cos(m pi t/T) is numerically
    rank-deficient at K = 64 -- rank 49 -- which gives J(theta) exactly flat
    directions.)"""
    assert K % 2 == 0
    T = J * dt
    t = np.arange(J) * dt
    m = np.arange(1, K // 2 + 1)
    arg = 2.0 * np.pi * np.outer(t, m) / T
    return np.concatenate([np.sin(arg), np.cos(arg)], axis=1)


def maximal_basis(J: int) -> np.ndarray:
    """Maximal model f_j = theta_j (Sec. III-D, Eq. maximal): B = I."""
    return np.eye(J)


# ---------------------------------------------------------------------------
# Hamiltonian / dipole / target draws
# ---------------------------------------------------------------------------

def _sym_upper(rng, N, sigma, band=None, diag=True):
    """Symmetric matrix: draw the upper triangle (row by row), mirror it."""
    A = np.zeros((N, N))
    for p in range(N):
        q0 = p if diag else p + 1
        q1 = N if band is None else min(N, p + band + 1)
        if q1 > q0:
            A[p, q0:q1] = rng.normal(0.0, sigma, size=q1 - q0)
    return np.triu(A) + np.triu(A, 1).T


def draw_system(rng, N, e_lo, e_hi, off_sigma, band, m_sigma):
    """H0 = diag(sorted U[e_lo, e_hi]) + symmetric off-diagonals N(0, off_sigma^2)
    nonzero iff 0 < |p - q| <= band (band=None: dense); M dense symmetric
    N(0, m_sigma^2) including the diagonal; target a random unit complex
    vector; alpha = e_1."""
    energies = np.sort(rng.uniform(e_lo, e_hi, size=N))
    off = _sym_upper(rng, N, off_sigma, band=band, diag=False)
    H0 = np.diag(energies) + off
    M = _sym_upper(rng, N, m_sigma, band=None, diag=True)
    x = rng.normal(size=N)
    y = rng.normal(size=N)
    beta = (x + 1j * y) / np.linalg.norm(x + 1j * y)
    alpha = np.zeros(N, dtype=np.complex128)
    alpha[0] = 1.0
    return H0, M, alpha, beta


def random_targets(seed: int, N: int, count: int) -> np.ndarray:
    """`count` random unit complex vectors of length N (rows)."""
    rng = np.random.default_rng(seed)
    z = rng.normal(size=(count, N)) + 1j * rng.normal(size=(count, N))
    return z / np.linalg.norm(z, axis=1, keepdims=True)


def small_problem(N: int, K: int, J: int, seed: int, dt: float = 0.01,
                  basis: str = "sine", w_f: float | None = None,
                  w_t: float = 1.0, m_sigma: float = 0.5) -> Problem:
    """Config-1 recipe at arbitrary sizes (used by tests for ragged shapes)."""
    rng = np.random.default_rng(seed)
    H0, M, alpha, beta = draw_system(rng, N, -2.0, 0.0, 0.05, None, m_sigma)
    if basis == "sine":
        B = sine_basis(J, dt, K)
    elif basis == "sine_cosine":
        B = sine_cosine_basis(J, dt, K)
    elif basis == "maximal":
        assert K == J
        B = maximal_basis(J)
    elif basis == "random":
        B = rng.normal(size=(J, K)) / np.sqrt(K)
    else:
        raise ValueError(basis)
    return Problem(H0, M, alpha, beta, B, dt, dt if w_f is None else w_f, w_t,
                   name=f"small_N{N}_K{K}_J{J}_s{seed}")


def config_problem(cfg: int, index: int = 0) -> Problem:
    """The five synthetic workloads (seed = 1000*cfg + index).

    1: N=4, K=8 sine, T=10, J=1000 (plain FP64, single problem)
    2: N=32, K=64 Fourier sine/cosine, T=20, J=4000 (plain vs mixed precision)
    3: batched uneven problems: N in {8..128 step 8}, K in {16,32,64,128},
       J in {2000,4000,8000}, config-1 recipe, T=10, sine basis
    4: config-2 system (the learned warm start's fixed N=32 system)
    5: N=256, K=128 sine, T=40, J=10000 (largest single problem)
    Cost weights w_f = dt, w_t = 1 (J = dt*sum f^2 + |a_J - beta|^2).
    """
    seed = 1000 * cfg + index
    rng = np.random.default_rng(seed)
    if cfg == 1:
        N, K, T, J = 4, 8, 10.0, 1000
        H0, M, alpha, beta = draw_system(rng, N, -2.0, 0.0, 0.05, None, 0.5)
        B = sine_basis(J, T / J, K)
    elif cfg in (2, 4):
        if cfg == 4:
            rng = np.random.default_rng(1000 * 2 + index)
        N, K, T, J = 32, 64, 20.0, 4000
        H0, M, alpha, beta = draw_system(rng, N, -10.0, 0.0, 0.1, 8, 0.3)
        B = sine_cosine_basis(J, T / J, K)
    elif cfg == 3:
        N = int(rng.choice(np.arange(8, 129, 8)))
        K = int(rng.choice([16, 32, 64, 128]))
        J = int(rng.choice([2000, 4000, 8000]))
        T = 10.0
        H0, M, alpha, beta = draw_system(rng, N, -2.0, 0.0, 0.05, None, 0.5)
        B = sine_basis(J, T / J, K)
    elif cfg == 5:
        N, K, T, J = 256, 128, 40.0, 10000
        H0, M, alpha, beta = draw_system(rng, N, -30.0, 0.0, 0.05, 32, 0.2)
        B = sine_basis(J, T / J, K)
    else:
        raise ValueError(f"unknown config {cfg}")
    dt = T / J
    return Problem(H0, M, alpha, beta, B, dt, dt, 1.0, name=f"config{cfg}_{index}")


def scaling_problem(N: int, J: int, seed: int, dt: float = 0.1) -> Problem:
    """The wall-time scaling experiment's setting (Sec. IV-A, Fig. 1): the
    maximal model f_j = theta_j (K = J), alpha = e_1, beta = e_N, a random
    diagonal H0 and a random symmetric M (real symmetric here; the paper's are
    Hermitian), diagonal energies U[-2, 0] and M entries N(0, 0.5^2) as in
    the small single workload; paper weights (w_f = 1/2, w_t = rho/2 with
    rho = 1)."""
    rng = np.random.default_rng(seed)
    H0 = np.diag(np.sort(rng.uniform(-2.0, 0.0, N)))
    M = _sym_upper(rng, N, 0.5)
    alpha = np.zeros(N, complex)
    alpha[0] = 1.0
    beta = np.zeros(N, complex)
    beta[-1] = 1.0
    return Problem(H0, M, alpha, beta, maximal_basis(J), dt, 0.5, 0.5, name=f"scaling_N{N}_J{J}")


def tanh_network_control(t, theta):
    """A control model that is not linear in its parameters (the neural
    network f(t; theta) the paper proposes for future work, Sec. III-D):
    f(t) = sum_h v_h tanh(w_h t + c_h), theta = [v (H), w (H), c (H)].
    Returns f (J), its Jacobian df/dtheta (J x 3H) and its second
    derivatives d^2 f / dtheta^2 (J x 3H x 3H), all analytic."""
    t = np.asarray(t, float)
    theta = np.asarray(theta, float)
    H = theta.size // 3
    v, w, c = theta[:H], theta[H:2 * H], theta[2 * H:]
    z = np.tanh(np.outer(t, w) + c)                 # J x H
    s = 1.0 - z ** 2                                 # tanh'
    s2 = -2.0 * z * s                                # tanh''
    J = t.size
    f = z @ v
    jac = np.concatenate([z, s * v * t[:, None], s * v], axis=1)
    hess = np.zeros((J, 3 * H, 3 * H))
    for h in range(H):
        iv, iw, ic = h, H + h, 2 * H + h
        hess[:, iv, iw] = hess[:, iw, iv] = s[:, h] * t
        hess[:, iv, ic] = hess[:, ic, iv] = s[:, h]
        hess[:, iw, iw] = v[h] * s2[:, h] * t ** 2
        hess[:, iw, ic] = hess[:, ic, iw] = v[h] * s2[:, h] * t
        hess[:, ic, ic] = v[h] * s2[:, h]
    return f, jac, hess


def batched_shape(index: int):
    """(N, K, J) of problem `index` of the batched workload (config 3), drawn
    exactly as config_problem(3, index) draws them, without the matrices."""
    rng = np.random.default_rng(1000 * 3 + index)
    N = int(rng.choice(np.arange(8, 129, 8)))
    K = int(rng.choice([16, 32, 64, 128]))
    J = int(rng.choice([2000, 4000, 8000]))
    return N, K, J


def eval_theta(K: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Evaluation point theta ~ N(0, scale^2) (Sec. IV-A draws N(0,1))."""
    return scale * np.random.default_rng(seed).normal(size=K)
