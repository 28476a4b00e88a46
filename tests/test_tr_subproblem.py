"""The trust-region subproblem on the device (qoc_tr_subproblem) against the
oracle's exact solution (whose K = 2 cases are pinned by brute force), by
both methods: through the eigendecomposition and through the Householder
tridiagonal reduction (the one the solvers take from K = 48).  Interior,
boundary, indefinite and hard cases at sizes on both sides of the switch."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


def _case(kind, K, seed):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(K, K)))
    if kind == "interior":
        d = rng.uniform(1.0, 5.0, K)
        g = rng.normal(size=K) * 0.01
        radius = 10.0
    elif kind == "boundary":
        d = rng.uniform(0.5, 5.0, K)
        g = rng.normal(size=K)
        radius = 0.1
    elif kind == "indefinite":
        d = rng.uniform(-2.0, 3.0, K)
        g = rng.normal(size=K)
        radius = 1.0
    else:   # hard case: g orthogonal to the lowest eigenvector, radius beyond the limit step
        d = np.sort(rng.uniform(-1.0, 3.0, K))
        d[0] = -2.0
        gt = rng.normal(size=K) * 0.05
        gt[0] = 0.0
        g = Q @ gt
        radius = 5.0
    H = (Q * d) @ Q.T
    return g, (H + H.T) / 2, radius


def model(g, H, s):
    return g @ s + 0.5 * s @ H @ s


@pytest.mark.parametrize("K", [5, 47, 48, 64, 130])
@pytest.mark.parametrize("kind", ["interior", "boundary", "indefinite", "hard"])
@pytest.mark.parametrize("method", [1, 2], ids=["eig", "tridiagonal"])
def test_subproblem_matches_oracle(K, kind, method):
    g, H, radius = _case(kind, K, 1000 * K + len(kind))
    s_ref, sig_ref = orc.tr_subproblem(g, H, radius)
    s, info = q.qoc_tr_subproblem(g, H, radius, method)
    assert np.linalg.norm(s) <= radius * (1 + 1e-10)
    assert abs(info[1] - np.linalg.norm(s)) <= 1e-12 * max(radius, 1.0)
    assert abs(info[3] - np.linalg.norm(g)) <= 1e-12 * np.linalg.norm(g)
    m, m_ref = model(g, H, s), model(g, H, s_ref)
    assert abs(info[0] + m) <= 1e-10 * max(abs(m), 1e-12), (info[0], m)
    assert abs(m - m_ref) <= 1e-10 * max(abs(m_ref), 1e-12), (kind, m, m_ref)
    if kind == "hard":
        assert abs(np.linalg.norm(s) - radius) <= 1e-9 * radius
    else:   # unique minimiser
        assert np.linalg.norm(s - s_ref) <= 1e-8 * max(np.linalg.norm(s_ref), 1e-12), np.linalg.norm(s - s_ref)
        assert abs(info[2] - sig_ref) <= 1e-8 * max(abs(sig_ref), 1.0)


def test_subproblem_size_200_methods_agree():
    g, H, radius = _case("indefinite", 200, 77)
    s1, i1 = q.qoc_tr_subproblem(g, H, radius, 1)
    s2, i2 = q.qoc_tr_subproblem(g, H, radius, 2)
    assert np.linalg.norm(s1 - s2) <= 1e-8 * np.linalg.norm(s1)
    assert abs(i1[0] - i2[0]) <= 1e-10 * abs(i1[0])
