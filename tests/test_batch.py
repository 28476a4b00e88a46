"""Batched evaluation of uneven problems (the batching pattern): one batched
gradient + Hessian over problems of different N, K, J must reproduce each
problem's own evaluation (same kernels, same arithmetic order) and, through
it, the FP64 oracle; the CUDA-graph replay must track new theta."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

pytestmark = pytest.mark.gpu

TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}
# uneven shapes: N odd/even up to the maximum, ragged last time block, K = 1
SHAPES = [(8, 16, 200), (24, 12, 333), (5, 3, 77), (40, 32, 150), (64, 9, 61), (3, 1, 17)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    build.build()
    _lib.lib()


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def _problems(seed0=0):
    return [inputs.small_problem(N, K, J, seed=seed0 + 11 * i) for i, (N, K, J) in enumerate(SHAPES)]


def _thetas(probs, seed):
    return [inputs.eval_theta(p.K, seed + i, 0.5) for i, p in enumerate(probs)]


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
@pytest.mark.parametrize("graph", [True, False], ids=["graph", "eager"])
def test_batch_matches_individual(precision, graph):
    probs = _problems()
    methods = [q.QOC_HESS_SECOND_ORDER_ADJOINT if i % 3 else q.QOC_HESS_TANGENT for i in range(len(probs))]
    Ps = [q.Problem(p, precision=precision, hess_method=m) for p, m in zip(probs, methods)]
    try:
        with q.Batch(Ps, graph=graph) as b:
            for call, seed in enumerate((5, 6, 6)):      # new theta, then a repeat
                thetas = _thetas(probs, 100 * seed)
                res = b.eval_grad_hess(thetas)
                for P, th, (J, g, H) in zip(Ps, thetas, res):
                    Ji, gi, Hi = P.eval_grad_hess(th)
                    assert abs(J - Ji) <= 1e-13 * abs(Ji), (call, P.N, J, Ji)
                    assert rel(g, gi) <= 1e-13, (call, P.N, rel(g, gi))
                    assert rel(H, Hi) <= 1e-13, (call, P.N, rel(H, Hi))
                    np.testing.assert_array_equal(H, H.T)
    finally:
        for P in Ps:
            P.close()


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_batch_against_oracle(precision):
    probs = _problems(seed0=7)
    Ps = [q.Problem(p, precision=precision) for p in probs]
    tol = TOL[precision]
    try:
        with q.Batch(Ps) as b:
            thetas = _thetas(probs, 900)
            for _ in range(2):    # eager first call, then the graph replay
                res = b.eval_grad_hess(thetas)
                for p, th, (J, g, H) in zip(probs, thetas, res):
                    ref = orc.evaluate(p, th, order=2)
                    assert abs(J - ref["J"]) <= tol * abs(ref["J"]), (p.N, J, ref["J"])
                    assert rel(g, ref["grad"]) <= tol, (p.N, rel(g, ref["grad"]))
                    assert rel(H, ref["hess"]) <= tol, (p.N, rel(H, ref["hess"]))
    finally:
        for P in Ps:
            P.close()


def test_batch_device_pointer_entry():
    torch = pytest.importorskip("torch")
    probs = _problems(seed0=3)[:3]
    Ps = [q.Problem(p, precision=q.QOC_MIXED_FP32) for p in probs]
    try:
        stream = torch.cuda.Stream()
        with q.Batch(Ps, cuda_stream=stream.cuda_stream) as b:
            thetas = _thetas(probs, 40)
            flat = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device="cuda")
            out = torch.zeros(b.n_out, dtype=torch.float64, device="cuda")
            with torch.cuda.stream(stream):
                for _ in range(3):
                    q.qoc_batch_eval_grad_hess_dev(b.handle, flat.data_ptr(), out.data_ptr())
            stream.synchronize()
            for P in Ps:
                q.qoc_sync_status(P.handle)
            res = b.split(out.cpu().numpy())
            for P, th, (J, g, H) in zip(Ps, thetas, res):
                Ji, gi, Hi = P.eval_grad_hess(th)
                assert abs(J - Ji) <= 1e-13 * abs(Ji)
                assert rel(g, gi) <= 1e-13 and rel(H, Hi) <= 1e-13
    finally:
        for P in Ps:
            P.close()


def test_batch_validation():
    a = inputs.small_problem(6, 4, 64, seed=1)
    c = inputs.small_problem(6, 4, 8, seed=2)     # J < 16: per-step path, no time blocking
    P1 = q.Problem(a, precision=q.QOC_FP64)
    P2 = q.Problem(a, precision=q.QOC_MIXED_FP32)
    P3 = q.Problem(c, precision=q.QOC_FP64)
    try:
        with pytest.raises(q.QocError) as e:
            q.Batch([P1, P1])
        assert e.value.status == _lib.QOC_EINVAL
        with pytest.raises(q.QocError) as e:
            q.Batch([P1, P3])
        assert e.value.status == _lib.QOC_EUNSUPPORTED
        with q.Batch([P1]) as b:
            with pytest.raises(ValueError):
                b.eval_grad_hess([np.zeros(5)])
            with pytest.raises(q.QocError) as e:
                b.eval_grad_hess([np.array([0.0, np.nan, 0.0, 0.0])])
            assert e.value.status == _lib.QOC_EINVAL
    finally:
        for P in (P1, P2, P3):
            P.close()


def test_batch_mixed_sweep_precisions():
    """One batch holding binary64-sweep and binary32-sweep problems (the
    sweeps are grouped by precision as well as by kernel): every result
    equals the problem's own evaluation and the oracle's within its tolerance."""
    probs = _problems(seed0=21)[:4]
    precs = [q.QOC_FP64, q.QOC_MIXED_FP32, q.QOC_MIXED_FP32, q.QOC_FP64]
    Ps = [q.Problem(p, precision=pr) for p, pr in zip(probs, precs)]
    try:
        assert [P.precision()[0] for P in Ps] == precs
        with q.Batch(Ps) as b:
            thetas = _thetas(probs, 1300)
            for _ in range(2):
                res = b.eval_grad_hess(thetas)
                for P, p, pr, th, (J, g, H) in zip(Ps, probs, precs, thetas, res):
                    Ji, gi, Hi = P.eval_grad_hess(th)
                    assert abs(J - Ji) <= 1e-13 * abs(Ji) and rel(g, gi) <= 1e-13 and rel(H, Hi) <= 1e-13
                    ref = orc.evaluate(p, th, order=2)
                    assert rel(H, ref["hess"]) <= TOL[pr], (p.N, pr, rel(H, ref["hess"]))
    finally:
        for P in Ps:
            P.close()


@pytest.fixture(scope="module")
def avoided_crossing_ref():
    pr = inputs.config_problem(3, 344)
    th = inputs.eval_theta(pr.K, 167)
    return pr, th, orc.evaluate(pr, th, order=2)


@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_batched_workload_avoided_crossing(avoided_crossing_ref, precision):
    """A problem of the batched-workload recipe (N=48, K=32, J=4000) whose
    trajectory passes an avoided crossing (eigenvalue gap 3e-5 against
    |H| ~ 50 at one step): the refined eigensolver must succeed, and J, the
    gradient and the Hessian must match the oracle (and, for the binary64
    sweeps, the binary64 Jacobi eigensolver path)."""
    pr, th, ref = avoided_crossing_ref
    assert (pr.N, pr.K, pr.J) == (48, 32, 4000)
    tol = TOL[precision]
    with q.Problem(pr, precision=precision) as P:
        J1, g1, H1 = P.eval_grad_hess(th)
    assert abs(J1 - ref["J"]) <= tol * abs(ref["J"])
    assert rel(g1, ref["grad"]) <= tol and rel(H1, ref["hess"]) <= tol, (rel(g1, ref["grad"]), rel(H1, ref["hess"]))
    if precision == q.QOC_FP64:
        with q.Problem(pr, precision=q.QOC_FP64, eig_method=q.QOC_EIG_JACOBI_FP64) as P:
            J0, g0, H0 = P.eval_grad_hess(th)
        assert rel(H1, H0) <= tol and rel(g1, g0) <= tol
