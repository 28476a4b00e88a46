"""Batched trust region (qoc_batch_trust_region_solve): uneven problems
solved together must take the oracle's iterations, problem by problem (the
textbook trust region with the exact subproblem, Sec. IV-B), and agree with
the single-problem solve; problems that stop early leave the batch."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

# (N, K, J, dt): uneven basis sizes, control dimensions and step counts
SHAPES = [(4, 8, 100, 0.1), (6, 5, 64, 0.05), (8, 12, 150, 0.05), (3, 4, 40, 0.1), (12, 6, 90, 0.05)]
# gtol where every problem stops by the gradient test well inside the binary64
# (resp. mixed-precision) rounding of the gradient
OPTS = {q.QOC_FP64: dict(gtol=1e-7, xtol=1e-12, max_iter=300),
        q.QOC_MIXED_FP32: dict(gtol=1e-5, xtol=1e-12, max_iter=300)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


@pytest.fixture(scope="module")
def cases():
    probs = [inputs.small_problem(N, K, J, seed=900 + i, dt=dt) for i, (N, K, J, dt) in enumerate(SHAPES)]
    starts = [np.zeros(p.K) if i % 2 == 0 else inputs.eval_theta(p.K, 950 + i, 0.3) for i, p in enumerate(probs)]
    refs = {prec: [orc.trust_region_solve(p, t0, **o) for p, t0 in zip(probs, starts)]
            for prec, o in OPTS.items()}
    return probs, starts, refs


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_batch_tr_matches_oracle(cases, precision):
    probs, starts, refs = cases
    opts = OPTS[precision]
    Ps = [q.Problem(p, precision=precision) for p in probs]
    try:
        thetas, infos, status = q.qoc_batch_trust_region_solve([P.handle for P in Ps], starts, **opts)
        assert status == _lib.QOC_OK
        for p, th, info, (th_o, info_o) in zip(probs, thetas, infos, refs[precision]):
            assert info["stop"] == info_o["stop"], (p.N, info, info_o["stop"])
            if precision == q.QOC_FP64:
                assert info["iters"] == info_o["iters"], (p.N, info["iters"], info_o["iters"])
                assert info["n_eval_J"] == info_o["n_eval_J"] and info["n_eval_gh"] == info_o["n_eval_gh"]
                assert abs(info["J"] - info_o["J"]) <= 1e-8 * abs(info_o["J"])
                assert rel(th, th_o) <= 1e-6
            else:
                assert abs(info["J"] - info_o["J"]) <= 1e-6 * abs(info_o["J"])
            assert info["stop"] == "gtol" and info["grad_norm"] < opts["gtol"]
        # the problems' own single solves take the same iterations
        if precision == q.QOC_FP64:
            for P, t0, th, info in zip(Ps, starts, thetas, infos):
                th1, info1 = P.trust_region_solve(t0, **opts)
                assert info1["iters"] == info["iters"] and rel(th, th1) <= 1e-9
    finally:
        for P in Ps:
            P.close()


def test_batch_tr_validation():
    a = inputs.small_problem(6, 4, 64, seed=1)
    c = inputs.small_problem(6, 4, 8, seed=2)     # J < 16: no time blocking
    P1 = q.Problem(a)
    P3 = q.Problem(c)
    try:
        with pytest.raises(q.QocError) as e:
            q.qoc_batch_trust_region_solve([P1.handle, P1.handle], [np.zeros(4), np.zeros(4)])
        assert e.value.status == _lib.QOC_EINVAL
        with pytest.raises(q.QocError) as e:
            q.qoc_batch_trust_region_solve([P1.handle, P3.handle], [np.zeros(4), np.zeros(4)])
        assert e.value.status == _lib.QOC_EUNSUPPORTED
        with pytest.raises(q.QocError) as e:
            q.qoc_batch_trust_region_solve([P1.handle], [np.zeros(4)], radius0=-1.0)
        assert e.value.status == _lib.QOC_EINVAL
        # a cap of one iteration: reported as max_iter, status QOC_ENOTCONV
        th, infos, status = q.qoc_batch_trust_region_solve([P1.handle], [np.zeros(4)], gtol=1e-14,
                                                           max_iter=1)
        assert status == _lib.QOC_ENOTCONV and infos[0]["stop"] == "max_iter" and infos[0]["iters"] == 1
    finally:
        P1.close()
        P3.close()
