"""Thin ctypes binding of ``libqoc.so`` (declared in ``include/qoc.h``).

Argument marshalling only: every step of an evaluation runs in the CUDA
library.  There is no CPU fallback; loading fails loudly when the library
has not been built (``paper_2505_00529_gb300.build.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

QOC_OK, QOC_EINVAL, QOC_ENOMEM, QOC_ECUDA, QOC_ENUMERIC, QOC_ENOTCONV, QOC_ETIMEOUT, QOC_EUNSUPPORTED = range(8)
QOC_FP64, QOC_MIXED_FP32, QOC_MIXED_FP32_ALWAYS = 0, 1, 2
QOC_HESS_SECOND_ORDER_ADJOINT, QOC_HESS_TANGENT = 0, 1
QOC_EIG_REFINED, QOC_EIG_JACOBI_FP64 = 0, 1
(QOC_BUF_F, QOC_BUF_EIGVAL, QOC_BUF_EIGVEC, QOC_BUF_STATE, QOC_BUF_COSTATE, QOC_BUF_G, QOC_BUF_C,
 QOC_BUF_V, QOC_BUF_U, QOC_BUF_SJ, QOC_BUF_HESS_RAW) = range(11)

# every entry point declared in include/qoc.h
EXPORTS = [
    "qoc_create_problem", "qoc_set_hess_method", "qoc_set_eig_method", "qoc_set_block_steps",
    "qoc_eval_J",
    "qoc_eval_grad", "qoc_eval_grad_hess", "qoc_eval_grad_hess_dev", "qoc_sync_status",
    "qoc_trust_region_solve", "qoc_get_diagnostics", "qoc_enable_timing", "qoc_read_buffer",
    "qoc_device_bytes", "qoc_max_basis_size", "qoc_destroy_problem", "qoc_status_string",
    "qoc_version", "qoc_set_target", "qoc_mlp_param_count", "qoc_mlp_create", "qoc_mlp_set_dataset",
    "qoc_mlp_train", "qoc_mlp_gradient", "qoc_mlp_predict", "qoc_mlp_get_params", "qoc_mlp_destroy",
    "qoc_last_error", "qoc_batch_create", "qoc_batch_set_graph", "qoc_batch_eval_grad_hess",
    "qoc_batch_eval_grad_hess_dev", "qoc_batch_destroy", "qoc_assemble_noalloc_scratch_doubles",
    "qoc_assemble_grad_hess_noalloc", "qoc_get_phase_times", "qoc_get_eig_stats",
    "qoc_set_panel_columns", "qoc_get_precision", "qoc_measure_fp64_rate",
    "qoc_batch_trust_region_solve", "qoc_trust_region_solve_bfgs", "qoc_tr_subproblem",
    "qoc_eval_grad_hess_model", "qoc_set_refine_sweeps", "qoc_selftest_bounded_wait", "qoc_set_pipeline", "qoc_set_mu_split",
    "qoc_get_tr_phase_times",
]


class TrOptions(C.Structure):
    _fields_ = [("gtol", C.c_double), ("xtol", C.c_double), ("radius0", C.c_double),
                ("radius_max", C.c_double), ("eta", C.c_double), ("max_iter", C.c_int)]


class TrReport(C.Structure):
    _fields_ = [("iters", C.c_int), ("n_eval_J", C.c_int), ("n_eval_gh", C.c_int),
                ("J", C.c_double), ("grad_norm", C.c_double), ("radius", C.c_double),
                ("stop_reason", C.c_int)]


class QocError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        detail = ""
        if status in (QOC_ECUDA, QOC_ENUMERIC, QOC_ETIMEOUT, QOC_EUNSUPPORTED):
            msg = lib().qoc_last_error().decode()
            detail = f" [{msg}]" if msg else ""
        super().__init__(f"{where}: {status_string(status)} (status {status}){detail}")


_LIB = None
_dp = C.POINTER(C.c_double)


def lib_path() -> str:
    return _build.LIB


def lib() -> C.CDLL:
    """Load libqoc.so (raises if it is missing)."""
    global _LIB
    if _LIB is None:
        path = lib_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with paper_2505_00529_gb300.build.build()")
        L = C.CDLL(path)
        L.qoc_create_problem.argtypes = [C.c_int, _dp, _dp, _dp, _dp, C.c_int, _dp, C.c_double,
                                         C.c_int, C.c_double, C.c_double, C.c_int, C.c_void_p,
                                         C.POINTER(C.c_void_p)]
        L.qoc_set_hess_method.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_eig_method.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_block_steps.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_panel_columns.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_refine_sweeps.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_pipeline.argtypes = [C.c_void_p, C.c_int]
        L.qoc_set_mu_split.argtypes = [C.c_void_p, C.c_int]
        L.qoc_get_tr_phase_times.argtypes = [C.c_void_p, _dp]
        L.qoc_selftest_bounded_wait.argtypes = [C.c_void_p, C.c_ulonglong]
        L.qoc_get_precision.argtypes = [C.c_void_p, C.POINTER(C.c_int), _dp]
        L.qoc_measure_fp64_rate.argtypes = [C.c_int, C.c_int, _dp, _dp]
        L.qoc_eval_J.argtypes = [C.c_void_p, _dp, _dp]
        L.qoc_eval_grad.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.qoc_eval_grad_hess.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp]
        L.qoc_eval_grad_hess_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.qoc_sync_status.argtypes = [C.c_void_p]
        L.qoc_trust_region_solve.argtypes = [C.c_void_p, _dp, C.POINTER(TrOptions), _dp,
                                             C.POINTER(TrReport)]
        L.qoc_trust_region_solve_bfgs.argtypes = [C.c_void_p, _dp, C.POINTER(TrOptions), _dp,
                                                  C.POINTER(TrReport)]
        L.qoc_tr_subproblem.argtypes = [C.c_int, _dp, _dp, C.c_double, C.c_int, _dp, _dp]
        L.qoc_eval_grad_hess_model.argtypes = [C.c_void_p, _dp, _dp, _dp, _dp, _dp, _dp]
        L.qoc_get_diagnostics.argtypes = [C.c_void_p, _dp, _dp, _dp]
        L.qoc_get_phase_times.argtypes = [C.c_void_p, _dp, C.c_int]
        L.qoc_get_eig_stats.argtypes = [C.c_void_p, _dp]
        L.qoc_enable_timing.argtypes = [C.c_void_p, C.c_int]
        L.qoc_read_buffer.argtypes = [C.c_void_p, C.c_int, _dp, C.c_size_t]
        L.qoc_device_bytes.argtypes = [C.c_void_p]
        L.qoc_device_bytes.restype = C.c_size_t
        L.qoc_max_basis_size.argtypes = []
        L.qoc_destroy_problem.argtypes = [C.c_void_p]
        L.qoc_destroy_problem.restype = None
        L.qoc_status_string.argtypes = [C.c_int]
        L.qoc_status_string.restype = C.c_char_p
        L.qoc_version.argtypes = []
        L.qoc_set_target.argtypes = [C.c_void_p, _dp]
        L.qoc_last_error.argtypes = []
        L.qoc_last_error.restype = C.c_char_p
        L.qoc_batch_create.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.POINTER(C.c_void_p)]
        L.qoc_batch_set_graph.argtypes = [C.c_void_p, C.c_int]
        L.qoc_batch_eval_grad_hess.argtypes = [C.c_void_p, _dp, _dp]
        L.qoc_batch_eval_grad_hess_dev.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.qoc_batch_destroy.argtypes = [C.c_void_p]
        L.qoc_batch_trust_region_solve.argtypes = [C.POINTER(C.c_void_p), C.c_int, _dp, C.POINTER(TrOptions),
                                                   _dp, C.POINTER(TrReport), C.c_void_p]
        L.qoc_batch_destroy.restype = None
        L.qoc_assemble_noalloc_scratch_doubles.argtypes = [C.c_int, C.c_int]
        L.qoc_assemble_noalloc_scratch_doubles.restype = C.c_size_t
        L.qoc_assemble_grad_hess_noalloc.argtypes = [C.c_int, C.c_int] + [C.c_void_p] * 6 + [
            C.c_double, C.c_void_p, C.c_void_p]
        _fp = C.POINTER(C.c_float)
        _ip = C.POINTER(C.c_int)
        L.qoc_mlp_param_count.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int]
        L.qoc_mlp_param_count.restype = C.c_size_t
        L.qoc_mlp_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, _fp, C.c_int, C.c_void_p,
                                     C.POINTER(C.c_void_p)]
        L.qoc_mlp_set_dataset.argtypes = [C.c_void_p, _fp, _fp, C.c_int]
        L.qoc_mlp_train.argtypes = [C.c_void_p, _ip, C.c_int, C.c_int, C.c_float, _fp]
        L.qoc_mlp_gradient.argtypes = [C.c_void_p, _fp, _fp, C.c_int, _fp, _fp]
        L.qoc_mlp_predict.argtypes = [C.c_void_p, _fp, C.c_int, _fp, C.c_int]
        L.qoc_mlp_get_params.argtypes = [C.c_void_p, _fp]
        L.qoc_mlp_destroy.argtypes = [C.c_void_p]
        L.qoc_mlp_destroy.restype = None
        _LIB = L
    return _LIB


def status_string(s: int) -> str:
    return lib().qoc_status_string(int(s)).decode()


def _check(status, where):
    if status != QOC_OK:
        raise QocError(status, where)


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _cplx(a) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(a, dtype=np.complex128))
    return a.view(np.float64)


# ---------------------------------------------------------------------------
# same names as the C ABI
# ---------------------------------------------------------------------------

def qoc_create_problem(N, H0, M, a0, a_target, K, basis, dt, steps, w_ctrl, w_term, precision,
                       cuda_stream=None):
    """Returns an opaque handle (int).  Arrays: H0, M (N,N) float; a0, a_target (N,) complex;
    basis (steps, K) float."""
    H0 = _f64(H0); M = _f64(M); B = _f64(basis)
    a0v = _cplx(a0); btv = _cplx(a_target)
    h = C.c_void_p()
    st = C.c_void_p(int(cuda_stream)) if cuda_stream else None
    _check(lib().qoc_create_problem(int(N), _ptr(H0), _ptr(M), _ptr(a0v), _ptr(btv), int(K), _ptr(B),
                                    float(dt), int(steps), float(w_ctrl), float(w_term),
                                    int(precision), st, C.byref(h)), "qoc_create_problem")
    return h.value


def qoc_destroy_problem(h):
    lib().qoc_destroy_problem(C.c_void_p(h))


def qoc_set_hess_method(h, method):
    _check(lib().qoc_set_hess_method(C.c_void_p(h), int(method)), "qoc_set_hess_method")


def qoc_set_eig_method(h, method):
    _check(lib().qoc_set_eig_method(C.c_void_p(h), int(method)), "qoc_set_eig_method")


def qoc_set_block_steps(h, steps):
    _check(lib().qoc_set_block_steps(C.c_void_p(h), int(steps)), "qoc_set_block_steps")


def qoc_set_panel_columns(h, kc):
    _check(lib().qoc_set_panel_columns(C.c_void_p(h), int(kc)), "qoc_set_panel_columns")


def qoc_get_tr_phase_times(h):
    """Device milliseconds of the last trust-region solve's phases (timing mode)."""
    out = np.zeros(3)
    _check(lib().qoc_get_tr_phase_times(C.c_void_p(h), _ptr(out)), "qoc_get_tr_phase_times")
    return {"subproblem": out[0], "eval_J": out[1], "eval_grad_hess": out[2]}


def qoc_set_pipeline(h, chunks):
    _check(lib().qoc_set_pipeline(C.c_void_p(h), int(chunks)), "qoc_set_pipeline")


def qoc_set_mu_split(h, split):
    _check(lib().qoc_set_mu_split(C.c_void_p(h), int(split)), "qoc_set_mu_split")


def qoc_set_refine_sweeps(h, sweeps):
    _check(lib().qoc_set_refine_sweeps(C.c_void_p(h), int(sweeps)), "qoc_set_refine_sweeps")


def qoc_selftest_bounded_wait(h, limit_ns):
    """The status the library reports after its bounded device wait gave up
    on a barrier that nothing completes (QOC_ETIMEOUT expected); returned,
    not raised."""
    return int(lib().qoc_selftest_bounded_wait(C.c_void_p(h), int(limit_ns)))


def qoc_get_precision(h):
    """(effective sweep precision, estimated binary32 error at the current block length)"""
    eff = C.c_int(0)
    est = C.c_double(0.0)
    _check(lib().qoc_get_precision(h, C.byref(eff), C.byref(est)), "qoc_get_precision")
    return int(eff.value), float(est.value)


def qoc_enable_timing(h, on=True):
    _check(lib().qoc_enable_timing(C.c_void_p(h), int(bool(on))), "qoc_enable_timing")


def qoc_eval_J(h, theta):
    th = _f64(theta)
    J = np.zeros(1)
    _check(lib().qoc_eval_J(C.c_void_p(h), _ptr(th), _ptr(J)), "qoc_eval_J")
    return float(J[0])


def qoc_eval_grad(h, theta):
    th = _f64(theta)
    J = np.zeros(1)
    g = np.zeros(th.size)
    _check(lib().qoc_eval_grad(C.c_void_p(h), _ptr(th), _ptr(J), _ptr(g)), "qoc_eval_grad")
    return float(J[0]), g


def qoc_eval_grad_hess(h, theta):
    th = _f64(theta)
    K = th.size
    J = np.zeros(1)
    g = np.zeros(K)
    H = np.zeros((K, K))
    _check(lib().qoc_eval_grad_hess(C.c_void_p(h), _ptr(th), _ptr(J), _ptr(g), _ptr(H)),
           "qoc_eval_grad_hess")
    return float(J[0]), g, H


def qoc_eval_grad_hess_model(h, f, jac):
    """(J, grad, hess without the model term, dJ/df) for samples f and Jacobian jac."""
    f = _f64(f).ravel()
    jac = _f64(jac)
    K = jac.shape[1]
    J = C.c_double(0.0)
    g = np.zeros(K)
    H = np.zeros((K, K))
    d = np.zeros(f.size)
    _check(lib().qoc_eval_grad_hess_model(C.c_void_p(h), _ptr(f), _ptr(jac), C.byref(J), _ptr(g), _ptr(H),
                                          _ptr(d)), "qoc_eval_grad_hess_model")
    return J.value, g, H, d


def qoc_eval_grad_hess_dev(h, theta_dev_ptr: int, out_dev_ptr: int):
    """Device pointers (e.g. torch tensor .data_ptr()); enqueues and returns."""
    _check(lib().qoc_eval_grad_hess_dev(C.c_void_p(h), C.c_void_p(int(theta_dev_ptr)),
                                        C.c_void_p(int(out_dev_ptr))), "qoc_eval_grad_hess_dev")


def qoc_sync_status(h):
    _check(lib().qoc_sync_status(C.c_void_p(h)), "qoc_sync_status")


def qoc_trust_region_solve(h, theta0, gtol=1e-10, xtol=1e-10, radius0=1.0, radius_max=1e3,
                           eta=0.1, max_iter=10000, hessian="exact"):
    """hessian="exact" (Alg. 2) or "bfgs" (Alg. 1 gradients, BFGS model)."""
    th = _f64(theta0)
    out = np.zeros_like(th)
    opt = TrOptions(gtol, xtol, radius0, radius_max, eta, int(max_iter))
    rep = TrReport()
    fn = {"exact": lib().qoc_trust_region_solve, "bfgs": lib().qoc_trust_region_solve_bfgs}[hessian]
    s = fn(C.c_void_p(h), _ptr(th), C.byref(opt), _ptr(out), C.byref(rep))
    if s not in (QOC_OK, QOC_ENOTCONV):
        raise QocError(s, "qoc_trust_region_solve" + ("" if hessian == "exact" else "_bfgs"))
    info = {k: getattr(rep, k) for k, _ in TrReport._fields_}
    info["stop"] = {0: "gtol", 1: "xtol", 2: "max_iter", 3: "no_decrease"}[rep.stop_reason]
    info["status"] = s
    return out, info


_STOP = {0: "gtol", 1: "xtol", 2: "max_iter", 3: "no_decrease", 4: "failed"}


def qoc_batch_trust_region_solve(handles, theta0s, gtol=1e-10, xtol=1e-10, radius0=1.0, radius_max=1e3,
                                 eta=0.1, max_iter=10000, cuda_stream=None):
    """Batched trust region over problem handles; theta0s: list of per-problem
    starting points.  Returns (list of theta*, list of report dicts, status)."""
    n = len(handles)
    Ks = [len(t) for t in theta0s]
    flat = np.concatenate([_f64(t).ravel() for t in theta0s])
    out = np.zeros_like(flat)
    arr = (C.c_void_p * n)(*[C.c_void_p(h) for h in handles])
    reps = (TrReport * n)()
    opt = TrOptions(gtol, xtol, radius0, radius_max, eta, int(max_iter))
    s = lib().qoc_batch_trust_region_solve(arr, n, _ptr(flat), C.byref(opt), _ptr(out), reps,
                                           C.c_void_p(cuda_stream) if cuda_stream else None)
    if s not in (QOC_OK, QOC_ENOTCONV):
        raise QocError(s, "qoc_batch_trust_region_solve")
    thetas, infos, o = [], [], 0
    for k, K in enumerate(Ks):
        thetas.append(out[o:o + K].copy())
        o += K
        info = {f: getattr(reps[k], f) for f, _ in TrReport._fields_}
        info["stop"] = _STOP[reps[k].stop_reason]
        infos.append(info)
    return thetas, infos, s


def qoc_tr_subproblem(g, H, radius, method=0):
    """(s, info) of one trust-region subproblem; info = [pred, |s|, sigma, |g|]."""
    g = _f64(g).ravel()
    H = _f64(H)
    K = g.size
    s = np.zeros(K)
    info = np.zeros(4)
    _check(lib().qoc_tr_subproblem(K, _ptr(g), _ptr(H), float(radius), int(method), _ptr(s), _ptr(info)),
           "qoc_tr_subproblem")
    return s, info


def qoc_get_diagnostics(h):
    drift = C.c_double(0.0)
    asym = C.c_double(0.0)
    ph = np.zeros(6)
    _check(lib().qoc_get_diagnostics(C.c_void_p(h), C.byref(drift), C.byref(asym), _ptr(ph)),
           "qoc_get_diagnostics")
    return {"norm_drift": drift.value, "hess_asym": asym.value,
            "phase_ms": dict(zip(["eig", "prep", "chains", "pointwise", "panels", "assembly"], ph))}


PHASES = ["control", "eig_jacobi", "eig_refine", "prep_D", "deriv_prep", "chains", "pointwise",
          "panels", "assembly", "total"]


def qoc_get_phase_times(h):
    out = np.zeros(len(PHASES))
    _check(lib().qoc_get_phase_times(C.c_void_p(h), _ptr(out), len(PHASES)), "qoc_get_phase_times")
    return dict(zip(PHASES, out))


def qoc_get_eig_stats(h):
    out = np.zeros(3)
    _check(lib().qoc_get_eig_stats(C.c_void_p(h), _ptr(out)), "qoc_get_eig_stats")
    return {"refine_updates_per_step": out[0], "cleanup_rotated_fraction": out[1],
            "final_pass_fraction": out[2]}


def qoc_read_buffer(h, which, shape, complex_=False):
    n = int(np.prod(shape)) * (2 if complex_ else 1)
    out = np.zeros(n)
    _check(lib().qoc_read_buffer(C.c_void_p(h), int(which), _ptr(out), n), "qoc_read_buffer")
    if complex_:
        return out.view(np.complex128).reshape(shape)
    return out.reshape(shape)


def qoc_set_target(h, a_target):
    bt = _cplx(a_target)
    _check(lib().qoc_set_target(C.c_void_p(h), _ptr(bt)), "qoc_set_target")


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _fptr(a):
    return a.ctypes.data_as(C.POINTER(C.c_float))


def qoc_mlp_param_count(n_in, hidden, n_hidden_layers, n_out) -> int:
    return int(lib().qoc_mlp_param_count(n_in, hidden, n_hidden_layers, n_out))


class MLP:
    """The library's warm-start network (binary32 training, bfloat16 inference)."""

    def __init__(self, n_in, hidden, n_hidden_layers, n_out, params, max_batch=256, cuda_stream=None):
        self.shape = (n_in, hidden, n_hidden_layers, n_out)
        self.np = qoc_mlp_param_count(*self.shape)
        p = _f32(params)
        if p.size != self.np:
            raise ValueError(f"expected {self.np} parameters, got {p.size}")
        h = C.c_void_p()
        st = C.c_void_p(int(cuda_stream)) if cuda_stream else None
        _check(lib().qoc_mlp_create(n_in, hidden, n_hidden_layers, n_out, _fptr(p), int(max_batch), st,
                                    C.byref(h)), "qoc_mlp_create")
        self.handle = h.value

    def set_dataset(self, X, T):
        X = _f32(X); T = _f32(T)
        _check(lib().qoc_mlp_set_dataset(C.c_void_p(self.handle), _fptr(X), _fptr(T), X.shape[0]),
               "qoc_mlp_set_dataset")

    def train(self, perms, batch, lr):
        perms = np.ascontiguousarray(np.asarray(perms, dtype=np.int32))
        epochs = perms.shape[0]
        losses = np.zeros(epochs, dtype=np.float32)
        _check(lib().qoc_mlp_train(C.c_void_p(self.handle), perms.ctypes.data_as(C.POINTER(C.c_int)),
                                   epochs, int(batch), float(lr), _fptr(losses)), "qoc_mlp_train")
        return losses

    def gradient(self, X, T):
        X = _f32(X); T = _f32(T)
        loss = np.zeros(1, dtype=np.float32)
        g = np.zeros(self.np, dtype=np.float32)
        _check(lib().qoc_mlp_gradient(C.c_void_p(self.handle), _fptr(X), _fptr(T), X.shape[0], _fptr(loss),
                                      _fptr(g)), "qoc_mlp_gradient")
        return float(loss[0]), g

    def predict(self, X, bf16=True):
        X = _f32(X)
        Y = np.zeros((X.shape[0], self.shape[3]), dtype=np.float32)
        _check(lib().qoc_mlp_predict(C.c_void_p(self.handle), _fptr(X), X.shape[0], _fptr(Y), int(bool(bf16))),
               "qoc_mlp_predict")
        return Y

    def params(self):
        out = np.zeros(self.np, dtype=np.float32)
        _check(lib().qoc_mlp_get_params(C.c_void_p(self.handle), _fptr(out)), "qoc_mlp_get_params")
        return out

    def close(self):
        if getattr(self, "handle", None):
            lib().qoc_mlp_destroy(C.c_void_p(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qoc_batch_create(handles, cuda_stream=None):
    """Batch over existing problem handles (same precision, time blocking on)."""
    arr = (C.c_void_p * len(handles))(*[C.c_void_p(h) for h in handles])
    b = C.c_void_p()
    st = C.c_void_p(int(cuda_stream)) if cuda_stream else None
    _check(lib().qoc_batch_create(arr, len(handles), st, C.byref(b)), "qoc_batch_create")
    return b.value


def qoc_batch_set_graph(b, on):
    _check(lib().qoc_batch_set_graph(C.c_void_p(b), int(bool(on))), "qoc_batch_set_graph")


def qoc_batch_eval_grad_hess(b, thetas, outs_len):
    """thetas: concatenated theta of all problems; returns the concatenated
    [J, grad, Hess] blocks (outs_len doubles)."""
    th = _f64(thetas)
    out = np.zeros(int(outs_len))
    _check(lib().qoc_batch_eval_grad_hess(C.c_void_p(b), _ptr(th), _ptr(out)), "qoc_batch_eval_grad_hess")
    return out


def qoc_batch_eval_grad_hess_dev(b, thetas_dev_ptr: int, outs_dev_ptr: int):
    _check(lib().qoc_batch_eval_grad_hess_dev(C.c_void_p(b), C.c_void_p(int(thetas_dev_ptr)),
                                              C.c_void_p(int(outs_dev_ptr))), "qoc_batch_eval_grad_hess_dev")


def qoc_batch_destroy(b):
    lib().qoc_batch_destroy(C.c_void_p(b))


QOC_NOALLOC_SCRATCH_DOUBLES = 524288


def qoc_assemble_noalloc_scratch_doubles(steps, K) -> int:
    return int(lib().qoc_assemble_noalloc_scratch_doubles(int(steps), int(K)))


def qoc_assemble_grad_hess_noalloc(steps, K, basis_dev, f_dev, g_dev, c_dev, U_dev, V_dev, w_ctrl,
                                   out_dev, cuda_stream=None):
    """Device pointers (ints); enqueues on cuda_stream and returns.  Uses the
    library's fixed device scratch array instead of allocating."""
    st = C.c_void_p(int(cuda_stream)) if cuda_stream else None
    ptrs = [C.c_void_p(int(x)) if x else None for x in (basis_dev, f_dev, g_dev, c_dev, U_dev, V_dev)]
    s = lib().qoc_assemble_grad_hess_noalloc(int(steps), int(K), *ptrs, float(w_ctrl),
                                             C.c_void_p(int(out_dev)) if out_dev else None, st)
    if s != QOC_OK:
        reason = lib().qoc_last_error().decode()
        raise QocError(s, "qoc_assemble_grad_hess_noalloc" + (f" [{reason}]" if reason and s != QOC_ECUDA else ""))


def qoc_measure_fp64_rate(ctas_per_sm=4, repeats=5):
    """(TFLOP/s, ms) of the fastest of `repeats` binary64 FMA-chain launches."""
    tf = C.c_double(0.0)
    ms = C.c_double(0.0)
    _check(lib().qoc_measure_fp64_rate(int(ctas_per_sm), int(repeats), C.byref(tf), C.byref(ms)),
           "qoc_measure_fp64_rate")
    return float(tf.value), float(ms.value)


def qoc_device_bytes(h) -> int:
    return int(lib().qoc_device_bytes(C.c_void_p(h)))


def qoc_max_basis_size() -> int:
    return int(lib().qoc_max_basis_size())


def qoc_version() -> int:
    return int(lib().qoc_version())


# ---------------------------------------------------------------------------
# convenience wrapper
# ---------------------------------------------------------------------------

class Problem:
    """Owns one qoc_problem built from a problem description with fields
    H0, M, alpha, beta, B, dt, w_f, w_t (e.g. ``inputs.Problem``)."""

    def __init__(self, prob, precision=QOC_FP64, cuda_stream=None, hess_method=None, eig_method=None,
                 block_steps=None, panel_columns=None, mu_split=None):
        self.N, self.K, self.J = prob.H0.shape[0], prob.B.shape[1], prob.B.shape[0]
        self.handle = qoc_create_problem(self.N, prob.H0, prob.M, prob.alpha, prob.beta, self.K,
                                         prob.B, prob.dt, self.J, prob.w_f, prob.w_t, precision,
                                         cuda_stream)
        if hess_method is not None:
            qoc_set_hess_method(self.handle, hess_method)
        if eig_method is not None:
            qoc_set_eig_method(self.handle, eig_method)
        if block_steps is not None:
            qoc_set_block_steps(self.handle, block_steps)
        if panel_columns is not None:
            qoc_set_panel_columns(self.handle, panel_columns)
        if mu_split is not None:
            qoc_set_mu_split(self.handle, mu_split)

    def eval_J(self, theta):
        return qoc_eval_J(self.handle, theta)

    def eval_grad(self, theta):
        return qoc_eval_grad(self.handle, theta)

    def eval_grad_hess(self, theta):
        return qoc_eval_grad_hess(self.handle, theta)

    def eval_grad_hess_model(self, f, jac):
        return qoc_eval_grad_hess_model(self.handle, f, jac)

    def trust_region_solve(self, theta0, **kw):
        return qoc_trust_region_solve(self.handle, theta0, **kw)

    def set_target(self, beta):
        qoc_set_target(self.handle, beta)

    def buffer(self, which):
        N, K, J = self.N, self.K, self.J
        spec = {
            QOC_BUF_F: ((J,), False), QOC_BUF_EIGVAL: ((J, N), False), QOC_BUF_EIGVEC: ((J, N, N), False),
            QOC_BUF_STATE: ((J + 1, N), True), QOC_BUF_COSTATE: ((J + 1, N), True),
            QOC_BUF_G: ((J,), False), QOC_BUF_C: ((J,), False), QOC_BUF_V: ((J, K), False),
            QOC_BUF_U: ((J, K), False), QOC_BUF_SJ: ((N, K), True), QOC_BUF_HESS_RAW: ((K, K), False),
        }[which]
        return qoc_read_buffer(self.handle, which, *spec)

    def diagnostics(self):
        return qoc_get_diagnostics(self.handle)

    def precision(self):
        """(effective sweep precision, estimated binary32 error) -- see qoc_get_precision"""
        return qoc_get_precision(self.handle)

    def close(self):
        if self.handle:
            qoc_destroy_problem(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Batched gradient + Hessian evaluation over several ``Problem`` objects
    (which must stay alive while the batch is used)."""

    def __init__(self, problems, cuda_stream=None, graph=True):
        self.problems = list(problems)
        self.Ks = [p.K for p in self.problems]
        self.handle = qoc_batch_create([p.handle for p in self.problems], cuda_stream)
        if not graph:
            qoc_batch_set_graph(self.handle, 0)
        self.n_theta = sum(self.Ks)
        self.n_out = sum(1 + K + K * K for K in self.Ks)

    def split(self, flat):
        res, o = [], 0
        for K in self.Ks:
            res.append((float(flat[o]), flat[o + 1:o + 1 + K].copy(),
                        flat[o + 1 + K:o + 1 + K + K * K].reshape(K, K).copy()))
            o += 1 + K + K * K
        return res

    def eval_grad_hess(self, thetas):
        """thetas: list of per-problem theta; returns a list of (J, grad, Hess)."""
        flat = np.concatenate([_f64(t).ravel() for t in thetas])
        if flat.size != self.n_theta:
            raise ValueError(f"expected {self.n_theta} coefficients in total, got {flat.size}")
        return self.split(qoc_batch_eval_grad_hess(self.handle, flat, self.n_out))

    def close(self):
        if getattr(self, "handle", None):
            qoc_batch_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
