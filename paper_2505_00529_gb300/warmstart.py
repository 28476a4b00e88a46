"""Learned warm start for the trust-region solve.

A multilayer perceptron (the library's own CUDA kernels, see ``MLP``) maps
a target state beta to initial control coefficients theta0.  It is trained
on optimal controls theta* that the library's trust-region solver produces
from theta = 0, and judged by the same solver: iterations and wall time from
theta0 = MLP(beta) versus theta0 = 0 on held-out targets, to the same
gradient tolerance.  theta = 0 stays the fallback.  (The paper starts its
trust region from random theta, Sec. IV-B; it has no learned component.)

Every numerical step runs in the CUDA library; this module sequences calls.
"""
from __future__ import annotations

import concurrent.futures as cf
import time

import numpy as np

from . import _lib


def features(betas: np.ndarray) -> np.ndarray:
    """[Re beta, Im beta] rows (binary32)."""
    betas = np.atleast_2d(betas)
    return np.concatenate([betas.real, betas.imag], axis=1).astype(np.float32)


def init_params(n_in, hidden, n_hidden, n_out, seed) -> np.ndarray:
    """Glorot-normal weights, zero biases, in the library's flat layout."""
    rng = np.random.default_rng(seed)
    d = [n_in] + [hidden] * n_hidden + [n_out]
    out = []
    for k in range(len(d) - 1):
        out.append(rng.normal(0.0, np.sqrt(2.0 / (d[k] + d[k + 1])), size=d[k] * d[k + 1]))
        out.append(np.zeros(d[k + 1]))
    return np.concatenate(out).astype(np.float32)


def solve_many(prob, betas, theta0s, precision=_lib.QOC_MIXED_FP32, batch=32, **tr):
    """Trust-region solves for each target, `batch` targets at a time through
    the library's batched trust region (one problem object per slot of the
    batch, re-targeted between batches).  Returns (thetas, infos, seconds)."""
    n = len(betas)
    K = prob.B.shape[1]
    thetas = np.zeros((n, K))
    infos = [None] * n
    problems = [_lib.Problem(prob, precision=precision) for _ in range(min(batch, n))]
    t0 = time.perf_counter()
    try:
        for s0 in range(0, n, batch):
            idx = list(range(s0, min(n, s0 + batch)))
            Ps = problems[:len(idx)]
            for P, i in zip(Ps, idx):
                P.set_target(betas[i])
            try:
                ths, inf, _ = _lib.qoc_batch_trust_region_solve([P.handle for P in Ps],
                                                                [theta0s[i] for i in idx], **tr)
            except _lib.QocError as e:   # recorded, not fatal: the solves of this batch count as failed
                ths = [np.full(K, np.nan)] * len(idx)
                inf = [{"iters": tr.get("max_iter", 0), "J": np.nan, "stop": f"error {e.status}"}
                       for _ in idx]
            for i, th, info in zip(idx, ths, inf):
                thetas[i] = th
                infos[i] = info
    finally:
        secs = time.perf_counter() - t0
        for P in problems:
            P.close()
    return thetas, infos, secs


def solve_sequential(prob, betas, theta0s, precision=_lib.QOC_FP64, **tr):
    """The plain method: one problem object, its exact trust region
    (qoc_trust_region_solve) run target after target.  Returns (thetas,
    infos, seconds)."""
    n = len(betas)
    K = prob.B.shape[1]
    thetas = np.zeros((n, K))
    infos = [None] * n
    t0 = time.perf_counter()
    with _lib.Problem(prob, precision=precision) as P:
        for i in range(n):
            P.set_target(betas[i])
            try:
                th, info = P.trust_region_solve(theta0s[i], **tr)
            except _lib.QocError as e:
                th, info = np.full(K, np.nan), {"iters": tr.get("max_iter", 0), "J": np.nan,
                                                 "stop": f"error {e.status}"}
            thetas[i] = th
            infos[i] = info
    return thetas, infos, time.perf_counter() - t0


GUARD_STEPS = (0.0, 0.25, 0.5, 0.75, 1.0)


def guarded_starts(prob, betas, theta_mlp, precision=_lib.QOC_MIXED_FP32, workers=4,
                   steps=GUARD_STEPS):
    """theta0 = t* MLP(beta) with t* the minimiser of J(t MLP(beta)) over
    `steps` (t = 0 included, so theta = 0 stays the fallback and the start is
    never worse in J).  Cost-only evaluations by the library; returns
    (theta0s, t*, seconds)."""
    n, K = len(betas), prob.B.shape[1]
    out = np.zeros((n, K))
    tstar = np.zeros(n)
    problems = [_lib.Problem(prob, precision=precision) for _ in range(workers)]

    def run(w):
        P = problems[w]
        for i in range(w, n, workers):
            P.set_target(betas[i])
            best, bt = None, 0.0
            for t in steps:
                try:
                    J = P.eval_J(t * theta_mlp[i])
                except _lib.QocError:
                    continue
                if best is None or J < best:
                    best, bt = J, t
            tstar[i] = bt
            out[i] = bt * theta_mlp[i]

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(run, range(workers)))
    secs = time.perf_counter() - t0
    for P in problems:
        P.close()
    return out, tstar, secs


def newton_decrement(grad, hess):
    """g^T H^-1 g when H is positive definite (Cholesky), else +inf: the
    quadratic model's predicted decrease of J (times two) to its minimiser,
    a measure of how far a start is from a local minimum in the Newton
    metric."""
    try:
        L = np.linalg.cholesky(np.asarray(hess))
    except np.linalg.LinAlgError:
        return np.inf
    y = np.linalg.solve(L, np.asarray(grad))
    return float(y @ y)


def decrement_starts(prob, betas, theta_mlp, precision=_lib.QOC_MIXED_FP32, workers=4):
    """theta0 = the one of (0, MLP(beta)) with the smaller Newton decrement
    (gradient and Hessian from the library at both), ties and two indefinite
    Hessians decided by the lower J.  Returns (theta0s, chose_mlp, seconds)."""
    n, K = len(betas), prob.B.shape[1]
    out = np.zeros((n, K))
    chose = np.zeros(n, dtype=bool)
    problems = [_lib.Problem(prob, precision=precision) for _ in range(workers)]

    def run(w):
        P = problems[w]
        for i in range(w, n, workers):
            P.set_target(betas[i])
            cand = []
            for th in (np.zeros(K), theta_mlp[i]):
                try:
                    J, g, H = P.eval_grad_hess(th)
                    cand.append((newton_decrement(g, H), J))
                except _lib.QocError:
                    cand.append((np.inf, np.inf))
            pick = 1 if (cand[1][0], cand[1][1]) <= (cand[0][0], cand[0][1]) else 0
            chose[i] = pick == 1
            out[i] = theta_mlp[i] if pick else 0.0

    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(run, range(workers)))
    secs = time.perf_counter() - t0
    for P in problems:
        P.close()
    return out, chose, secs


class WarmStart:
    """theta0 = scale * MLP([Re beta, Im beta]) + shift (outputs standardised
    on the training set)."""

    def __init__(self, N, K, hidden=256, n_hidden=3, seed=0, max_batch=256):
        self.N, self.K = N, K
        self.mlp = _lib.MLP(2 * N, hidden, n_hidden, K, init_params(2 * N, hidden, n_hidden, K, seed),
                            max_batch=max_batch)
        self.shift = np.zeros(K, dtype=np.float32)
        self.scale = np.ones(K, dtype=np.float32)

    def fit(self, betas, thetas, epochs=200, batch=128, lr=1e-3, seed=0):
        thetas = np.asarray(thetas, dtype=np.float64)
        self.shift = thetas.mean(axis=0).astype(np.float32)
        self.scale = (thetas.std(axis=0) + 1e-6).astype(np.float32)
        T = ((thetas - self.shift) / self.scale).astype(np.float32)
        X = features(betas)
        self.mlp.set_dataset(X, T)
        rng = np.random.default_rng(seed)
        perms = np.stack([rng.permutation(len(X)) for _ in range(epochs)])
        return self.mlp.train(perms, batch, lr)

    def predict(self, betas, bf16=True):
        Y = self.mlp.predict(features(betas), bf16=bf16)
        return (Y * self.scale + self.shift).astype(np.float64)

    def close(self):
        self.mlp.close()


def compare(prob, train_betas, test_betas, precision=_lib.QOC_MIXED_FP32, workers=4, epochs=200,
            batch=128, lr=1e-3, seed=0, tr_batch=32, n_plain=None, train_cache=None, **tr):
    """Full warm-start experiment: theta* for the training targets (from 0),
    train, then solve the held-out targets from 0, from the MLP, from the
    guarded start and from the decrement-chosen start; the plain binary64
    method on the first `n_plain` held-out targets (all when None).
    `train_cache`: an .npz path holding the training optima (theta*, their
    convergence flags, the seconds they took) for these targets, written
    after they are computed and read instead of recomputing them."""
    import os
    K = prob.B.shape[1]
    N = prob.H0.shape[0]
    cached = None
    if train_cache and os.path.exists(train_cache):
        z = np.load(train_cache)
        if z["betas"].shape == train_betas.shape and np.array_equal(z["betas"], train_betas):
            cached = z
    if cached is not None:
        th_train, ok, t_data = cached["theta"], cached["ok"], float(cached["seconds"])
    else:
        th_train, info_train, t_data = solve_many(prob, train_betas, np.zeros((len(train_betas), K)),
                                                  precision, tr_batch, **tr)
        ok = np.array([i["stop"] in ("gtol", "xtol") and np.all(np.isfinite(t))
                       for i, t in zip(info_train, th_train)])
        if train_cache:
            np.savez(train_cache, betas=train_betas, theta=th_train, ok=ok, seconds=t_data)
    ws = WarmStart(N, K, seed=seed)
    t0 = time.perf_counter()
    losses = ws.fit(train_betas[ok], th_train[ok], epochs=epochs, batch=batch, lr=lr, seed=seed)
    t_train = time.perf_counter() - t0
    theta0 = ws.predict(test_betas)
    _, info_zero, t_zero = solve_many(prob, test_betas, np.zeros((len(test_betas), K)), precision, tr_batch, **tr)
    _, info_mlp, t_mlp = solve_many(prob, test_betas, theta0, precision, tr_batch, **tr)
    theta_g, tstar, t_guard_eval = guarded_starts(prob, test_betas, theta0, precision, workers)
    _, info_g, t_g = solve_many(prob, test_betas, theta_g, precision, tr_batch, **tr)
    theta_d, chose, t_dec_eval = decrement_starts(prob, test_betas, theta0, precision, workers)
    _, info_d, t_d = solve_many(prob, test_betas, theta_d, precision, tr_batch, **tr)
    ws.close()
    # the plain method on (a prefix of) the same targets: binary64, one problem
    # at a time, from theta = 0; the combined form timed on the same prefix
    npl = len(test_betas) if n_plain is None else min(n_plain, len(test_betas))
    _, info_plain, t_plain = solve_sequential(prob, test_betas[:npl], np.zeros((npl, K)),
                                              _lib.QOC_FP64, **tr)
    _, info_comb, t_comb = solve_many(prob, test_betas[:npl], theta0[:npl], precision, tr_batch, **tr)
    conv = lambda i: i["stop"] in ("gtol", "xtol")
    good = np.array([conv(a) and conv(b) and conv(c) and conv(d)
                     for a, b, c, d in zip(info_zero, info_mlp, info_g, info_d)])
    itd = np.array([i["iters"] for i in info_d])[good]
    Jd = np.array([i["J"] for i in info_d])[good]
    ghd = np.array([i.get("n_eval_gh", 0) for i in info_d])[good]
    gh0 = np.array([i.get("n_eval_gh", 0) for i in info_zero])[good]
    gh1 = np.array([i.get("n_eval_gh", 0) for i in info_mlp])[good]
    it0 = np.array([i["iters"] for i in info_zero])[good]
    it1 = np.array([i["iters"] for i in info_mlp])[good]
    itg = np.array([i["iters"] for i in info_g])[good]
    J0 = np.array([i["J"] for i in info_zero])[good]
    J1 = np.array([i["J"] for i in info_mlp])[good]
    Jg = np.array([i["J"] for i in info_g])[good]
    return {
        "n_train": int(ok.sum()), "n_train_failed": int((~ok).sum()), "n_test": len(test_betas),
        "n_test_compared": int(good.sum()), "dataset_seconds": t_data,
        "train_seconds": t_train, "final_train_loss": float(losses[-1]),
        "iters_zero_mean": float(it0.mean()), "iters_mlp_mean": float(it1.mean()),
        "iters_zero_median": float(np.median(it0)), "iters_mlp_median": float(np.median(it1)),
        "iters_ratio_mean": float(np.mean(it0 / np.maximum(it1, 1))),
        "frac_mlp_fewer_iters": float(np.mean(it1 < it0)), "frac_mlp_more_iters": float(np.mean(it1 > it0)),
        "hess_evals_zero_mean": float(gh0.mean()), "hess_evals_mlp_mean": float(gh1.mean()),
        "wall_ratio_zero_over_mlp": t_zero / t_mlp,
        "wall_zero_s": t_zero, "wall_mlp_s": t_mlp,
        "J_zero_mean": float(J0.mean()), "J_mlp_mean": float(J1.mean()),
        "frac_mlp_not_worse_J": float(np.mean(J1 <= J0 * (1 + 1e-6))),
        "converged_zero": float(np.mean([i["stop"] in ("gtol", "xtol") for i in info_zero])),
        "converged_mlp": float(np.mean([i["stop"] in ("gtol", "xtol") for i in info_mlp])),
        "combined_vs_plain_fp64": {
            "form": "batched trust region (batches of %d), %s, theta0 from the network" % (
                tr_batch, "mixed precision" if precision == _lib.QOC_MIXED_FP32 else "binary64"),
            "plain": "binary64, one problem at a time, theta0 = 0",
            "targets": npl,
            "wall_combined_s": t_comb, "wall_plain_s": t_plain, "speedup": t_plain / t_comb,
            "iters_combined_mean": float(np.mean([i["iters"] for i in info_comb])),
            "iters_plain_mean": float(np.mean([i["iters"] for i in info_plain])),
            "converged_combined": float(np.mean([conv(i) for i in info_comb])),
            "converged_plain": float(np.mean([conv(i) for i in info_plain])),
            "frac_combined_not_worse_J": float(np.mean([
                a["J"] <= b["J"] * (1 + 1e-6) for a, b in zip(info_comb, info_plain)
                if conv(a) and conv(b)])),
        },
        "decrement": {
            "rule": "theta0 = the one of 0 and MLP(beta) with the smaller Newton decrement g^T H^-1 g "
                    "(H positive definite; else +inf), ties by J",
            "chose_mlp_fraction": float(chose.mean()),
            "iters_mean": float(itd.mean()), "iters_median": float(np.median(itd)),
            "frac_fewer_iters": float(np.mean(itd < it0)), "frac_more_iters": float(np.mean(itd > it0)),
            "hess_evals_mean": float(ghd.mean()),
            "wall_s": t_d + t_dec_eval, "choice_eval_s": t_dec_eval,
            "J_mean": float(Jd.mean()), "frac_not_worse_J": float(np.mean(Jd <= J0 * (1 + 1e-6))),
            "converged": float(np.mean([conv(i) for i in info_d])),
        },
        "guarded": {
            "rule": "theta0 = t* MLP(beta), t* = argmin J(t MLP(beta)) over t in "
                    + ", ".join(f"{t:g}" for t in GUARD_STEPS),
            "t_star_mean": float(tstar.mean()), "t_star_zero_fraction": float(np.mean(tstar == 0.0)),
            "iters_mean": float(itg.mean()), "iters_median": float(np.median(itg)),
            "iters_ratio_mean": float(np.mean(it0 / np.maximum(itg, 1))),
            "frac_fewer_iters": float(np.mean(itg < it0)), "frac_more_iters": float(np.mean(itg > it0)),
            "wall_s": t_g + t_guard_eval, "guard_eval_s": t_guard_eval,
            "J_mean": float(Jg.mean()), "frac_not_worse_J": float(np.mean(Jg <= J0 * (1 + 1e-6))),
            "converged": float(np.mean([conv(i) for i in info_g])),
        },
    }
