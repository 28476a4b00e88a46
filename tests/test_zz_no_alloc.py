"""The assembly entry point that allocates nothing (fixed device scratch
array) against the library's own evaluation and the oracle: the per-step
contractions of an evaluated problem, passed back in, must give the same
gradient and Hessian as qoc_eval_grad_hess and, within the stated tolerance,
as the binary64 oracle, on two calls in a row of different sizes (the shared
array keeps the previous call's contents).  The device's free memory must not
change across a call.  Named to be collected last."""
import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs
from oracle import qoc_oracle as orc

TOL = {q.QOC_FP64: 1e-10, q.QOC_MIXED_FP32: 1e-6}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def test_noalloc_rejects_oversize_before_any_device_call():
    build.build()
    _lib.lib()
    K = 64
    ok = q.qoc_assemble_noalloc_scratch_doubles(8000, K)
    assert ok <= _lib.QOC_NOALLOC_SCRATCH_DOUBLES
    assert q.qoc_assemble_noalloc_scratch_doubles(8001, K) > _lib.QOC_NOALLOC_SCRATCH_DOUBLES
    fake = 256   # never dereferenced: the size check fails first
    with pytest.raises(q.QocError) as e:
        q.qoc_assemble_grad_hess_noalloc(8200, K, fake, fake, fake, fake, fake, fake, 1.0, fake)
    assert e.value.status == _lib.QOC_EINVAL
    assert "maximum" in str(e.value)
    with pytest.raises(q.QocError) as e:
        q.qoc_assemble_grad_hess_noalloc(10, 4, fake, fake, None, fake, fake, fake, 1.0, fake)
    assert e.value.status == _lib.QOC_EINVAL


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [q.QOC_FP64, q.QOC_MIXED_FP32], ids=["fp64", "mixed"])
def test_noalloc_assembly_matches_eval_grad_hess(precision):
    torch = pytest.importorskip("torch")
    build.build()
    _lib.lib()
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream(device=dev)
    # two calls in a row: larger then smaller problem, different theta
    cases = [((24, 48, 700), 11), ((6, 5, 90), 12)]
    for (N, K, J), seed in cases:
        prob = inputs.small_problem(N, K, J, seed=seed)
        theta = inputs.eval_theta(K, seed + 100, 0.5)
        # the no-alloc assembly takes the full contraction V (unsplit adjoint)
        with q.Problem(prob, precision=precision, mu_split=False) as P:
            Jv, g_ref, H_ref = P.eval_grad_hess(theta)
            f = P.buffer(_lib.QOC_BUF_F)
            g = P.buffer(_lib.QOC_BUF_G)
            c = P.buffer(_lib.QOC_BUF_C)
            U = P.buffer(_lib.QOC_BUF_U)
            V = P.buffer(_lib.QOC_BUF_V)
        t = lambda a: torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=dev)
        Bd, fd, gd, cd, Ud, Vd = (t(prob.B), t(f), t(g), t(c), t(U), t(V))
        out = torch.full((1 + K + K * K,), 7.0, dtype=torch.float64, device=dev)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info(dev)[0]
        q.qoc_assemble_grad_hess_noalloc(J, K, Bd.data_ptr(), fd.data_ptr(), gd.data_ptr(), cd.data_ptr(),
                                         Ud.data_ptr(), Vd.data_ptr(), prob.w_f, out.data_ptr(),
                                         stream.cuda_stream)
        stream.synchronize()
        if seed != cases[0][1]:
            # the first call may load the library's module that holds the array;
            # a later call allocates nothing
            assert torch.cuda.mem_get_info(dev)[0] == free0
        o = out.cpu().numpy()
        assert o[0] == 7.0                       # out[0] is not written
        grad, H = o[1:1 + K], o[1 + K:].reshape(K, K)
        tol = TOL[precision]
        assert rel(grad, g_ref) <= tol, rel(grad, g_ref)
        assert rel(H, H_ref) <= tol, rel(H, H_ref)
        np.testing.assert_array_equal(H, H.T)
        ref = orc.evaluate(prob, theta, order=2)
        assert rel(grad, ref["grad"]) <= tol, rel(grad, ref["grad"])
        assert rel(H, ref["hess"]) <= tol, rel(H, ref["hess"])
