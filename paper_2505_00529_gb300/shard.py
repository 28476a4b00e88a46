"""Independent problems spread over ranks (one process per GPU).

The problems of a batch share nothing, so the only exchange between ranks is
a final gather of each problem's results to rank 0: no collective touches
the evaluation itself.  Problems are assigned by estimated work so that the
ranks finish together: largest first, each to the rank with the least work
so far (longest-processing-time order), ties to the lowest rank.

The work estimate is the method's per-step algorithmic count (Alg. 2 per
time step: eigendecomposition 9 N^3, M~ = W^T M W 4 N^3, the second-
derivative term 8 N^3, the forward and backward panels 8 N^2 (K + 1) each)
times the number of steps.

Every numerical step runs in the CUDA library (``Batch``,
``qoc_batch_trust_region_solve``); this module only partitions, sequences
and gathers.
"""
from __future__ import annotations

import numpy as np


def estimated_flops(N: int, K: int, J: int) -> float:
    """Algorithmic flops of one gradient + Hessian evaluation."""
    return float(J) * (21.0 * N ** 3 + 16.0 * N ** 2 * (K + 1))


def partition(shapes, world: int):
    """Assign problems (a list of (N, K, J)) to `world` ranks.  Returns a
    list of index lists, one per rank, each in ascending index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    cost = [estimated_flops(*s) for s in shapes]
    order = sorted(range(len(shapes)), key=lambda i: (-cost[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(i)
        load[r] += cost[i]
    return [sorted(p) for p in parts]


def gather_results(local, indices, n_total, rank, world, dist=None):
    """Rank 0 receives every rank's (index, result) pairs and returns the
    results in global order; other ranks return None.  Without a process
    group (`dist` None, world 1) the local results are returned in order."""
    pairs = list(zip(indices, local))
    if dist is None or world == 1:
        gathered = [pairs]
    else:
        gathered = [None] * world if rank == 0 else None
        dist.gather_object(pairs, gathered, dst=0)
        if rank != 0:
            return None
    out = [None] * n_total
    for part in gathered:
        for i, r in part:
            out[i] = r
    missing = [i for i, r in enumerate(out) if r is None]
    if missing:
        raise RuntimeError(f"no result for problems {missing[:8]}")
    return out


def evaluate_sharded(probs, thetas, rank, world, dist=None, precision=None, evaluate=None,
                     cuda_stream=None):
    """Gradient + Hessian of every problem, this rank's share evaluated as
    one library batch (``evaluate(probs, thetas)`` replaces it, e.g. for a
    host-only run), then gathered to rank 0 as (J, grad, Hess) tuples in the
    original order.  Returns (results or None, this rank's indices)."""
    mine = partition([(p.H0.shape[0], p.B.shape[1], p.B.shape[0]) for p in probs], world)[rank]
    my_probs = [probs[i] for i in mine]
    my_thetas = [thetas[i] for i in mine]
    if evaluate is not None:
        local = evaluate(my_probs, my_thetas) if mine else []
    else:
        local = _evaluate_batch(my_probs, my_thetas, precision, cuda_stream) if mine else []
    return gather_results(local, mine, len(probs), rank, world, dist), mine


def _evaluate_batch(probs, thetas, precision, cuda_stream):
    from . import _lib
    prec = _lib.QOC_MIXED_FP32 if precision is None else precision
    Ps = [_lib.Problem(p, precision=prec) for p in probs]
    try:
        with _lib.Batch(Ps, cuda_stream=cuda_stream) as b:
            res = b.eval_grad_hess(thetas)
        return [(float(J), np.asarray(g), np.asarray(H)) for J, g, H in res]
    finally:
        for P in Ps:
            P.close()


def solve_sharded(probs, theta0s, rank, world, dist=None, precision=None, solve=None, **tr):
    """Trust-region solves of every problem, this rank's share through the
    library's batched trust region (``solve(probs, theta0s)`` replaces it),
    gathered to rank 0 as (theta*, report) pairs in the original order."""
    mine = partition([(p.H0.shape[0], p.B.shape[1], p.B.shape[0]) for p in probs], world)[rank]
    my_probs = [probs[i] for i in mine]
    my_t0 = [theta0s[i] for i in mine]
    if solve is not None:
        local = solve(my_probs, my_t0) if mine else []
    elif mine:
        from . import _lib
        prec = _lib.QOC_MIXED_FP32 if precision is None else precision
        Ps = [_lib.Problem(p, precision=prec) for p in my_probs]
        try:
            ths, infos, _ = _lib.qoc_batch_trust_region_solve([P.handle for P in Ps], my_t0, **tr)
        finally:
            for P in Ps:
                P.close()
        local = list(zip(ths, infos))
    else:
        local = []
    return gather_results(local, mine, len(probs), rank, world, dist), mine
