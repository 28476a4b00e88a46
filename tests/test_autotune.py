"""Launch-shape autotuner: candidate sets (CPU) and a tuned configuration
that is the fastest of its table, cached, and gives results equal to the
oracle's within the path's tolerance (GPU)."""
import json

import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, autotune, build, inputs

TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}


def test_candidates():
    c = autotune.candidates(32, 64, 4000, q.QOC_MIXED_FP32)
    assert set(c) == {(bs, kc) for bs in (2, 4) for kc in (1, 2, 4)}
    c = autotune.candidates(64, 64, 4000, q.QOC_FP64)
    assert all(bs in (2, 4, 8) for bs, _ in c) and all(kc <= 4 for _, kc in c)
    assert (8, 4) in c                          # 32 * 8 * 4 = 1024 threads
    assert autotune.candidates(8, 1, 4000, q.QOC_FP64) == [(2, 1), (4, 1), (8, 1)]   # kc <= K
    assert autotune.candidates(8, 4, 10, q.QOC_FP64) == []                          # J < 16


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_tune_cache_and_parity(tmp_path, precision):
    from oracle import qoc_oracle as orc
    build.build()
    prob = inputs.small_problem(16, 12, 200, seed=5)
    cache = str(tmp_path / "tune.json")
    r = autotune.tune(prob, precision, evals=2, cache=cache)
    assert not r["cached"]
    assert (r["block_steps"], r["panel_columns"]) in autotune.candidates(16, 12, 200, precision)
    assert r["ms"] == min(t[2] for t in r["table"]) and r["ms"] > 0
    again = autotune.tune(prob, precision, cache=cache)
    assert again["cached"] and again["block_steps"] == r["block_steps"]
    assert len(json.load(open(cache))) == 1
    theta = inputs.eval_theta(12, 9, 0.5)
    ref = orc.evaluate(prob, theta, order=2)
    with q.Problem(prob, precision=precision) as P:
        autotune.apply(P, r)
        J, g, H = P.eval_grad_hess(theta)
    tol = TOL[precision]
    assert abs(J - ref["J"]) <= tol * abs(ref["J"])
    assert np.linalg.norm(g - ref["grad"]) <= tol * np.linalg.norm(ref["grad"])
    assert np.linalg.norm(H - ref["hess"]) <= tol * np.linalg.norm(ref["hess"])


@pytest.mark.gpu
def test_panel_columns_do_not_change_results():
    build.build()
    prob = inputs.small_problem(24, 9, 150, seed=6)
    theta = inputs.eval_theta(9, 3, 0.5)
    res = []
    for kc in (1, 2, 4):
        with q.Problem(prob, precision=q.QOC_MIXED_FP32, panel_columns=kc) as P:
            res.append(P.eval_grad_hess(theta))
    for J, g, H in res[1:]:
        assert J == res[0][0]
        np.testing.assert_array_equal(g, res[0][1])
        np.testing.assert_array_equal(H, res[0][2])
    with pytest.raises(q.QocError):
        q.Problem(inputs.small_problem(64, 4, 50, seed=1), precision=q.QOC_FP64, panel_columns=8)
