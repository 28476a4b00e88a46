"""Launch-shape autotuner for the sequential sweeps (batching pattern).

For one problem shape it times complete gradient + Hessian evaluations over
the candidate (block steps, panel columns per CTA) pairs with CUDA events on
the problem's stream and keeps the fastest.  Both knobs change only how the
same arithmetic is grouped into launches, except the block steps in binary32
panels, whose rounding grows like sqrt(steps): binary32 candidates stop at 4
steps per block so that the mixed results stay within 1e-6 of binary64.

Results can be cached in a JSON file keyed by (device, N, K, J, precision,
Hessian form); ``tune_batch`` tunes each distinct shape of a batch once.
"""
from __future__ import annotations

import json
import os
import statistics

import numpy as np

from . import _lib

BS_FP64 = (2, 4, 8)
BS_MIXED = (2, 4)
KC = (1, 2, 4)


def _key(device, N, K, J, precision, hess_method):
    return f"{device}|N{N}|K{K}|J{J}|p{precision}|h{hess_method}"


def candidates(N, K, J, precision):
    bss = BS_MIXED if precision == _lib.QOC_MIXED_FP32 else BS_FP64
    out = []
    for bs in bss:
        if J < 16 or J < bs:
            continue
        for kc in KC:
            if kc > K or 32 * ((N + 7) // 8) * kc > 1024:
                continue
            out.append((bs, kc))
    return out


def _time_config(P, bs, kc, theta, evals):
    """Median device time (ms) of a full evaluation with this configuration,
    from the events the library records on the problem's stream."""
    apply(P, {"block_steps": bs, "panel_columns": kc})
    P.eval_grad_hess(theta)                       # warm-up (one-time kernel set-up)
    _lib.qoc_enable_timing(P.handle, True)
    times = []
    for _ in range(evals):
        P.eval_grad_hess(theta)
        times.append(_lib.qoc_get_phase_times(P.handle)["total"])
    _lib.qoc_enable_timing(P.handle, False)
    return float(statistics.median(times))


def tune(prob, precision, hess_method=None, evals=3, cache=None, theta=None, device_name=None):
    """Fastest (block steps, panel columns) for this problem's shape.

    Returns {"block_steps", "panel_columns", "ms", "table": [(bs, kc, ms), ...],
    "cached": bool}.  `cache`: path of a JSON cache file (read and updated)."""
    hm = _lib.QOC_HESS_SECOND_ORDER_ADJOINT if hess_method is None else hess_method
    N, K, J = prob.H0.shape[0], prob.B.shape[1], prob.B.shape[0]
    if device_name is None:
        import torch
        device_name = torch.cuda.get_device_name()
    dev = device_name
    key = _key(dev, N, K, J, precision, hm)
    db = {}
    if cache and os.path.exists(cache):
        with open(cache) as fh:
            db = json.load(fh)
        if key in db:
            r = dict(db[key])
            r["cached"] = True
            return r
    # a generic evaluation point (the eigensolver's work depends on f = B theta)
    th = np.random.default_rng(K).normal(size=K) if theta is None else np.asarray(theta, dtype=float)
    table = []
    with _lib.Problem(prob, precision=precision, hess_method=hm) as P:
        cands = candidates(N, K, J, precision)
        if not cands:
            return {"block_steps": 1, "panel_columns": 0, "ms": None, "table": [], "cached": False}
        for bs, kc in cands:
            table.append((bs, kc, _time_config(P, bs, kc, th, evals)))
    best = min(table, key=lambda r: r[2])
    r = {"block_steps": best[0], "panel_columns": best[1], "ms": best[2], "table": table}
    if cache:
        db[key] = r
        tmp = cache + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(db, fh, indent=1)
        os.replace(tmp, cache)
    r["cached"] = False
    return r


def apply(P, cfg):
    """Set a tuned configuration on a live problem."""
    _lib.qoc_set_block_steps(P.handle, cfg["block_steps"])
    _lib.qoc_set_panel_columns(P.handle, cfg["panel_columns"])


def tune_batch(probs, precision, hess_method=None, evals=2, cache=None):
    """Tune each distinct (N, K, J) of a list of problems once; returns the
    per-problem configurations in order."""
    seen = {}
    out = []
    for pr in probs:
        shape = (pr.H0.shape[0], pr.B.shape[1], pr.B.shape[0])
        if shape not in seen:
            seen[shape] = tune(pr, precision, hess_method, evals=evals, cache=cache)
        out.append(seen[shape])
    return out
