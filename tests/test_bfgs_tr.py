"""The gradient-only trust region (Alg. 1 with BFGS updates, the baseline of
Sec. IV-B) through the C ABI against the oracle's: the same iterations in
binary64, the same minimiser as the exact-Hessian (Alg. 2) solve, with more
iterations."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

CASES = [(4, 6, 80, 0.05, 41), (6, 5, 64, 0.05, 42), (3, 8, 100, 0.1, 43)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("case", CASES, ids=lambda c: "N%d_K%d_J%d" % c[:3])
def test_bfgs_trust_region_matches_oracle(case):
    N, K, J, dt, seed = case
    prob = inputs.small_problem(N, K, J, seed=seed, dt=dt)
    th_o, info_o = orc.trust_region_solve_bfgs(prob, np.zeros(K), gtol=1e-6, xtol=1e-12, max_iter=500)
    th_e, info_e = orc.trust_region_solve(prob, np.zeros(K), gtol=1e-6, xtol=1e-12, max_iter=500)
    with q.Problem(prob, precision=q.QOC_FP64) as P:
        th, info = P.trust_region_solve(np.zeros(K), gtol=1e-6, xtol=1e-12, max_iter=500, hessian="bfgs")
        th2, info2 = P.trust_region_solve(np.zeros(K), gtol=1e-6, xtol=1e-12, max_iter=500)
    assert info["stop"] == info_o["stop"] == "gtol", (info, info_o["stop"])
    assert info["iters"] == info_o["iters"], (info["iters"], info_o["iters"])
    assert info["n_eval_J"] == info_o["n_eval_grad"] - 1 and info["n_eval_gh"] == 0
    assert rel(th, th_o) <= 1e-6 and abs(info["J"] - info_o["J"]) <= 1e-10 * abs(info_o["J"])
    # the same minimiser as the exact-Hessian solve, reached in more iterations
    assert rel(th, th2) <= 1e-5 and info["iters"] > info2["iters"] == info_e["iters"]


def test_bfgs_trust_region_mixed():
    N, K, J, dt, seed = CASES[0]
    prob = inputs.small_problem(N, K, J, seed=seed, dt=dt)
    th_o, info_o = orc.trust_region_solve_bfgs(prob, np.zeros(K), gtol=1e-5, xtol=1e-12, max_iter=500)
    with q.Problem(prob, precision=q.QOC_MIXED_FP32) as P:
        th, info = P.trust_region_solve(np.zeros(K), gtol=1e-5, xtol=1e-12, max_iter=500, hessian="bfgs")
    assert info["stop"] == "gtol"
    assert abs(info["J"] - info_o["J"]) <= 1e-6 * abs(info_o["J"])
