"""The C-ABI library builds, loads and exports every entry point that
include/qoc.h declares; argument validation that needs no GPU.  CPU only:
no call here reaches a CUDA runtime function."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_2505_00529_gb300 as q
from paper_2505_00529_gb300 import _lib, build, inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return _lib.lib()


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names |= set(re.findall(r"\b(qoc_[A-Za-z_0-9]+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(L, n), n
    assert names == set(_lib.EXPORTS)


def test_exported_symbols_match_shared_object(L):
    import subprocess
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.lib_path()], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\sT\s(qoc_\w+)", out))
    assert declared_functions() <= exported


def test_host_only_entry_points(L):
    assert q.qoc_version() >= 100
    assert q.qoc_max_basis_size() >= 32
    for s in range(8):
        assert len(_lib.status_string(s)) > 0
    L.qoc_destroy_problem(None)   # NULL is a no-op


def _create(prob, **over):
    args = dict(N=prob.N, H0=prob.H0, M=prob.M, a0=prob.alpha, a_target=prob.beta, K=prob.K,
                basis=prob.B, dt=prob.dt, steps=prob.J, w_ctrl=prob.w_f, w_term=prob.w_t,
                precision=0)
    args.update(over)
    return q.qoc_create_problem(**args)


@pytest.mark.parametrize("bad", [
    dict(dt=0.0), dict(dt=-1.0), dict(dt=float("nan")), dict(w_ctrl=-1.0), dict(precision=7),
    dict(K=0), dict(steps=0), dict(N=0),
])
def test_create_rejects_bad_scalars_before_touching_the_device(L, bad):
    prob = inputs.small_problem(N=4, K=3, J=10, seed=1)
    with pytest.raises(q.QocError) as e:
        _create(prob, **bad)
    assert e.value.status == _lib.QOC_EINVAL


def test_create_rejects_nonsymmetric_and_nonfinite(L):
    prob = inputs.small_problem(N=4, K=3, J=10, seed=1)
    H = prob.H0.copy()
    H[0, 1] += 1e-6
    with pytest.raises(q.QocError) as e:
        _create(prob, H0=H)
    assert e.value.status == _lib.QOC_EINVAL
    B = prob.B.copy()
    B[3, 1] = np.inf
    with pytest.raises(q.QocError) as e:
        _create(prob, basis=B)
    assert e.value.status == _lib.QOC_EINVAL


def test_create_rejects_oversized_basis(L):
    N = q.qoc_max_basis_size() + 1
    prob = inputs.small_problem(N=N, K=2, J=3, seed=2)
    with pytest.raises(q.QocError) as e:
        _create(prob)
    assert e.value.status == _lib.QOC_EUNSUPPORTED


def test_null_pointers_rejected(L):
    h = C.c_void_p()
    s = L.qoc_create_problem(4, None, None, None, None, 2, None, 0.1, 3, 1.0, 1.0, 0, None,
                             C.byref(h))
    assert s == _lib.QOC_EINVAL
    assert L.qoc_eval_J(None, None, None) == _lib.QOC_EINVAL
    assert L.qoc_trust_region_solve(None, None, None, None, None) == _lib.QOC_EINVAL
