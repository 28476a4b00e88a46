"""Device failure paths reached without faulting the GPU.

* A bounded device wait that gives up: the library's mbarrier wait (the one
  the sweeps use on their shared-memory rings) runs on a barrier that nothing
  completes, with no copy in flight, and a short limit; the kernel returns and
  the status check reports QOC_ETIMEOUT.
* An eigensolver that does not converge: the binary64 refinement capped at
  zero updates leaves the binary32 start's non-orthogonality (~1e-7) above
  what the refinement accepts, and the evaluation reports QOC_ENUMERIC.

After either, the same problem evaluates bit for bit as before: the context
and the problem's buffers stay usable."""
import time

import numpy as np
import pytest

from paper_2505_00529_gb300 import _lib, inputs

pytestmark = pytest.mark.gpu

PRECISIONS = [_lib.QOC_FP64, _lib.QOC_MIXED_FP32]


def _setup(prec):
    prob = inputs.small_problem(8, 4, 200, seed=5, dt=0.05)
    theta = inputs.eval_theta(4, 3, 0.5)
    return _lib.Problem(prob, precision=prec), theta


def _same(a, b):
    (J0, g0, H0), (J1, g1, H1) = a, b
    assert J1 == J0
    np.testing.assert_array_equal(g1, g0)
    np.testing.assert_array_equal(H1, H0)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_bounded_wait_gives_up_with_etimeout(prec):
    P, theta = _setup(prec)
    with P:
        ref = P.eval_grad_hess(theta)
        t0 = time.perf_counter()
        st = _lib.qoc_selftest_bounded_wait(P.handle, 2_000_000)   # 2 ms
        took = time.perf_counter() - t0
        assert st == _lib.QOC_ETIMEOUT
        assert took < 5.0
        _same(ref, P.eval_grad_hess(theta))
        # a generous limit on the same barrier gives up too (nothing completes it)
        assert _lib.qoc_selftest_bounded_wait(P.handle, 20_000_000) == _lib.QOC_ETIMEOUT
        _same(ref, P.eval_grad_hess(theta))


def test_bounded_wait_limit_is_checked():
    P, _ = _setup(_lib.QOC_FP64)
    with P:
        assert _lib.qoc_selftest_bounded_wait(P.handle, 10) == _lib.QOC_EINVAL
        assert _lib.qoc_selftest_bounded_wait(P.handle, 10**11) == _lib.QOC_EINVAL


@pytest.mark.parametrize("prec", PRECISIONS)
def test_capped_refinement_reports_enumeric(prec):
    P, theta = _setup(prec)
    with P:
        ref = P.eval_grad_hess(theta)
        _lib.qoc_set_refine_sweeps(P.handle, 0)
        with pytest.raises(_lib.QocError) as e:
            P.eval_grad_hess(theta)
        assert e.value.status == _lib.QOC_ENUMERIC
        assert "device status 0x1 " in str(e.value)
        _lib.qoc_set_refine_sweeps(P.handle, 4)       # the default for N <= 64
        _same(ref, P.eval_grad_hess(theta))


def test_refine_sweeps_range_is_checked():
    P, _ = _setup(_lib.QOC_FP64)
    with P:
        for bad in (-1, 17):
            with pytest.raises(_lib.QocError) as e:
                _lib.qoc_set_refine_sweeps(P.handle, bad)
            assert e.value.status == _lib.QOC_EINVAL
