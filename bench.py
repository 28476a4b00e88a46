#!/usr/bin/env python
"""Gradient+Hessian evaluations per second of the discrete quantum-optimal-
control cost on GB300 (second-order adjoint method, Alg. 2), on the N=32,
K=64 (sine/cosine), J=4000 workload: CI-shaped synthetic H0 (diagonal
energies U[-10,0], band-8 couplings N(0,0.1^2)), dense M N(0,0.3^2), T=20.

One step = one full evaluation (J, grad, K x K Hessian) at a fixed seeded
theta, inputs resident in device memory.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on the host)

A single problem is a dependent chain of J steps and does not shard: with
N > 1 processes (torchrun) every rank runs an independent replica and the
value is the total over ranks (weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grad+Hessian evals/s and TR solves/s vs plain FP64 on GB300 at rel err ≤1e-6"
UNIT = "evals/s"
WORKLOAD = {"workload": "synthetic CI-shaped single problem, N=32 basis, K=64 sine/cosine "
                        "coefficients, J=4000 steps, T=20 (dt=0.005)",
            "N": 32, "K": 64, "J": 4000}
# library kernel launches per gradient + Hessian evaluation on the time-blocked path:
# control, binary32 Jacobi, binary64 refinement, 3 preparation parts (D, P~, X'),
# 2 block products, state chain + fill, terminal, costate chain + fill, drift,
# 3 pointwise parts (p^, y^/g, c), 3 block-source launches (Q, W/Gamma, backward),
# tangent and second-order adjoint panels, 2 panel contractions, grad, hess partial,
# hess final
LAUNCHES_PER_EVAL = 27
# DRAM bytes of one k_eig_refine launch on this workload (ncu capture of the
# current kernel: 32.93 MB read, 0 written; algorithmic: W read once, 32.8 MB)
REFINE_TRAFFIC_BYTES = 32.93e6
FP64_PEAK_TFLOPS = 1.26    # 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (measured 1.20 at 1.99 GHz)
FP32_PEAK_TFLOPS = 80.5    # 152 SMs x 128 FMA/clk x 2 flop x 2.07 GHz (measured 70 at 1.99 GHz)


def env_int(k, d):
    try:
        return int(os.environ.get(k, d))
    except ValueError:
        return d


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest x over the ranks of the process group `dist` (x itself
    without one): every rank times its own replica and the job is as slow as
    its slowest rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, ms):
    """Evaluations per second of the whole job: each of the `world` ranks
    finishes one evaluation per step of `ms` milliseconds (the slowest rank's)."""
    return world * 1000.0 / ms


# --------------------------------------------------------------------------
# CPU oracle timing (a deliberately slow reference: spawned process, 1 thread)
# --------------------------------------------------------------------------
ORACLE_SNIPPET = r"""
import sys, time, json
sys.path.insert(0, %r)
import numpy as np
from paper_2505_00529_gb300 import inputs
from oracle import qoc_oracle as orc
p = inputs.config_problem(2)
js = %d
p.B = p.B[:js]          # first js steps of the same problem (same dt)
th = inputs.eval_theta(p.K, 0)
t0 = time.perf_counter()
r = orc.evaluate(p, th, order=2)
dt = time.perf_counter() - t0
print(json.dumps({"seconds": dt, "steps": js}))
"""


def time_oracle(sample_steps: int) -> dict:
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET % (ROOT, sample_steps)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    J = WORKLOAD["J"]
    # the oracle's cost is linear in the number of steps: scale the sample to one full evaluation
    per_eval = d["seconds"] * J / d["steps"]
    return {"value": 1.0 / per_eval, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one oracle evaluation over the first {sample_steps} of the {J} steps "
                      f"({d['seconds']:.2f} s), scaled by {J}/{sample_steps}"}


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    per = []
    sample = args.ref_sample_steps
    for _ in range(args.warmup):
        time_oracle(max(8, sample // 8))
    for _ in range(args.steps):
        per.append(1.0 / time_oracle(sample)["value"])
    ms = 1000.0 * statistics.mean(per)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": dict(WORKLOAD, precision="fp64 (CPU oracle)"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: one oracle evaluation over the first {sample} "
                                       f"of {WORKLOAD['J']} steps, scaled to the full problem"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index, path):
        self.path = path
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        try:
            self.fh.close()
        except Exception:
            pass

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx = float(f[2])
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except FileNotFoundError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def refine_flops(N, J, updates_per_step, rotated_fraction, final_fraction):
    """Binary64 flops of one k_eig_refine launch: per step, u Ogita-Aishima
    updates with two binary64 N^3 products each (H W, and the W^T H W and W^T W
    triangles); the third product, W E, is binary64 only in an update that
    ends the refinement early (the others form it in binary32, not counted);
    the final residual pass (2 N^3 FMA) on the steps that take it (fraction p;
    the others finish early), and W V (N^3 FMA) when the clean-up rotated
    (fraction r); 2 flops per FMA."""
    fma = (2.0 * updates_per_step + (1.0 - final_fraction) + 2.0 * final_fraction
           + rotated_fraction) * N ** 3
    return 2.0 * fma * J


def run_ours(args):
    import numpy as np
    import torch

    rank, world, local = env_int("RANK", 0), env_int("WORLD_SIZE", 1), env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs
    build.build()

    prob = inputs.config_problem(2)
    N, K, J = prob.N, prob.K, prob.J
    theta = inputs.eval_theta(K, 0)
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)     # a real (non-default) stream the library runs on
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > L2 (129 MB)

    from paper_2505_00529_gb300 import autotune
    tuned = {}

    def measure(precision, steps, warmup, timing=True):
        if not args.no_autotune and precision not in tuned:
            tuned[precision] = autotune.tune(prob, precision, evals=3, theta=theta)
        P = q.Problem(prob, precision=precision, cuda_stream=stream.cuda_stream)
        if precision in tuned:
            autotune.apply(P, tuned[precision])
        if timing:
            q.qoc_enable_timing(P.handle, True)
        th = torch.tensor(theta, dtype=torch.float64, device=dev)
        out = torch.zeros(1 + K + K * K, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            q.qoc_eval_grad_hess_dev(P.handle, th.data_ptr(), out.data_ptr())
        q.qoc_sync_status(P.handle)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        phases = []
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(steps):
            flush.fill_(float(k))                         # evict L2 between timed steps
            ev[k][0].record(stream)
            q.qoc_eval_grad_hess_dev(P.handle, th.data_ptr(), out.data_ptr())
            ev[k][1].record(stream)
            if timing:
                q.qoc_sync_status(P.handle)
                ph = q.qoc_get_diagnostics(P.handle)["phase_ms"]
                ph.update({"k_" + k: v for k, v in q.qoc_get_phase_times(P.handle).items()})
                ph.update(q.qoc_get_eig_stats(P.handle))
                phases.append(ph)
        torch.cuda.synchronize()
        q.qoc_sync_status(P.handle)
        ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in ev), dist, dev)
        res = out.cpu().numpy().copy()
        return P, ms, phases, res

    # ---- headline: device-resident evaluations ----
    clk_dir = tempfile.mkdtemp(prefix="qoc_clocks_")
    clk = ClockSampler(local, os.path.join(clk_dir, f"clocks_rank{rank}.csv"))
    with clk:
        P, ms, phases, res = measure(prec, args.steps, args.warmup, timing=True)
    clocks = clk.summary()
    value = whole_job_rate(world, ms)

    # ---- end to end through the host API (theta from host, results back to host) ----
    e2e_times = []
    for k in range(args.warmup + args.steps):
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.eval_grad_hess(theta)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_ms = max_over_ranks(1000.0 * statistics.mean(e2e_times), dist, dev)
    P.close()

    # ---- plain FP64 GPU method on the same workload ----
    fp64 = None
    if prec != q.QOC_FP64 and not args.no_fp64:
        P64, ms64, _, res64 = measure(q.QOC_FP64, max(2, args.steps // 4), 1, timing=False)
        P64.close()
        hess_rel = float(np.linalg.norm(res[1 + K:] - res64[1 + K:]) / np.linalg.norm(res64[1 + K:]))
        grad_rel = float(np.linalg.norm(res[1:1 + K] - res64[1:1 + K]) / np.linalg.norm(res64[1:1 + K]))
        fp64 = {"value": whole_job_rate(world, ms64), "unit": UNIT, "ms_per_step": ms64,
                "speedup_mixed_over_fp64": ms64 / ms,
                "mixed_vs_fp64_rel_err": {"J": abs(res[0] - res64[0]) / abs(res64[0]),
                                          "grad": grad_rel, "hess": hess_rel}}

    # ---- trust-region solves (from theta = 0, same problem) ----
    tr = None
    if not args.no_tr:
        with q.Problem(prob, precision=prec, cuda_stream=stream.cuda_stream) as PT:
            t0 = time.perf_counter()
            th_star, info = PT.trust_region_solve(np.zeros(K), gtol=1e-6, xtol=1e-10, max_iter=500)
            t1 = time.perf_counter()
        tr_s = max_over_ranks(t1 - t0, dist, dev)
        tr = {"value": world / tr_s, "unit": "TR solves/s", "iters": info["iters"],
              "n_eval_gh": info["n_eval_gh"], "n_eval_J": info["n_eval_J"], "J": info["J"],
              "grad_norm": info["grad_norm"], "stop": info["stop"], "gtol": 1e-6}

    # ---- roofline of the dominant kernel (k_eig_refine: timed by events around its launch) ----
    ph_mean = {k: statistics.mean(p[k] for p in phases) for k in phases[0]} if phases else {}
    roof = None
    if ph_mean:
        u, rot = ph_mean["refine_updates_per_step"], ph_mean["cleanup_rotated_fraction"]
        fin = ph_mean["final_pass_fraction"]
        t_ref = ph_mean["k_eig_refine"]
        flops = refine_flops(N, J, u, rot, fin)
        ach = flops / (t_ref * 1e-3) / 1e12
        roof = {"bound": "alu", "kernel": "k_eig_refine", "achieved": ach, "peak": FP64_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": ach / FP64_PEAK_TFLOPS,
                "traffic": REFINE_TRAFFIC_BYTES if (N, J) == (32, 4000) else None,
                "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one k_eig_refine "
                                  "launch (ncu capture of this workload)",
                "peak_source": "binary64 FMA rate from unit counts x max SM clock (152 SMs x 2 DFMA/clk "
                               "x 2 x 2.07 GHz); MEASURED_PEAKS.json has no binary64 figure",
                "algorithmic": f"(2u + 1 + p + r) N^3 binary64 FMA per step, u = {u:.3f} updates/step, "
                               f"p = {fin:.3f} final-pass fraction, r = {rot:.3f} clean-up rotated "
                               f"fraction, N={N}, J={J}",
                "kernel_ms": t_ref,
                "phase_ms": {k: v for k, v in ph_mean.items() if not k.startswith("k_") and k in
                             ("eig", "prep", "chains", "pointwise", "panels", "assembly")},
                "kernel_phase_ms": {k[2:]: v for k, v in ph_mean.items() if k.startswith("k_")}}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = time_oracle(args.ref_sample_steps)
        except Exception as e:  # reported, never silently dropped
            cpu = {"error": str(e)[-300:]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 panels + f64" if prec == q.QOC_MIXED_FP32 else "f64",
                "data": "synthetic",
                "config": dict(WORKLOAD, precision=args.precision, l2="flushed between timed steps",
                               parallelism=f"replicas x{world}" if world > 1 else "single problem",
                               launch=({"block_steps": tuned[prec]["block_steps"],
                                        "panel_columns": tuned[prec]["panel_columns"],
                                        "autotune_table_ms": tuned[prec]["table"]}
                                       if prec in tuned else "library defaults")),
                "e2e": {"value": whole_job_rate(world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": 8 * K, "d2h_bytes_per_step": 8 * (1 + K + K * K)},
                "gpu_launches": LAUNCHES_PER_EVAL * args.steps,
                "clocks": clocks, "roofline": roof, "cpu_baseline": cpu,
                "fp64_plain": fp64, "tr_solve": tr}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_warm_start(args):
    """Learned warm start on the N=32 system (H0, M of the bench workload),
    horizon shortened to T=5 (J=1000, dt=0.005) with a K=64 Fourier basis:
    theta* from the library's trust region on random unit targets, MLP
    2N -> 256^3 -> K trained by the library's kernels, then held-out targets
    solved from theta=0, from the MLP's theta0, and from the guarded start
    t* MLP(beta) (t* minimising J over t in {0, 1/4, 1/2, 3/4, 1}) to the
    same tolerance."""
    import numpy as np
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs, warmstart
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    build.build()
    base = inputs.config_problem(4)
    J = 1000
    prob = inputs.Problem(base.H0, base.M, base.alpha, base.beta,
                          inputs.sine_cosine_basis(J, base.dt, 64), base.dt, base.dt, 1.0, "warm-start")
    train = inputs.random_targets(4000, prob.N, args.ws_train)
    test = inputs.random_targets(4001, prob.N, args.ws_test)
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    t0 = time.perf_counter()
    r = warmstart.compare(prob, train, test, precision=prec, workers=args.ws_workers, epochs=args.ws_epochs,
                          batch=128, lr=1e-3, seed=0, gtol=args.ws_gtol, xtol=1e-12, max_iter=500)
    r["total_seconds"] = time.perf_counter() - t0
    line = {"metric": "trust-region iterations and wall time on held-out targets: learned warm start vs theta=0",
            "value": r["wall_ratio_zero_over_mlp"],
            "unit": "wall-time ratio of the held-out solves, theta=0 / MLP start (same final tolerance)",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f32 panels + f64" if prec else "f64",
            "data": "synthetic",
            "config": {"workload": f"N=32 system, K=64 Fourier basis, T=5, J={J}; {args.ws_train} training / "
                                   f"{args.ws_test} held-out random unit targets; MLP 64-256-256-256-64 GELU, "
                                   f"{args.ws_epochs} epochs Adam, bfloat16 inference", "gtol": args.ws_gtol},
            "warm_start": r}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """Batching pattern: the batched-workload recipe (N from {8,...,128} step
    8, K from {16,32,64,128}, J from {2000,4000,8000}, per-problem seeds).
    Problems are created chunk by chunk within a device-memory budget; each
    chunk is one batch (per-problem phase streams, one launch per sequential
    sweep over the chunk, CUDA graph replay), timed with CUDA events; the
    same problems evaluated one after another give the comparison."""
    import numpy as np
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    build.build()
    dev = torch.device("cuda", local)
    nmax = q.qoc_max_basis_size()
    probs, i = [], 0
    while len(probs) < args.batch_size:
        pr = inputs.config_problem(3, i)
        i += 1
        if pr.N <= nmax:
            probs.append(pr)
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    thetas = [inputs.eval_theta(pr.K, 7 + k) for k, pr in enumerate(probs)]
    cfgs, tune_s = None, None
    if not args.no_autotune:
        from paper_2505_00529_gb300 import autotune
        t0 = time.perf_counter()
        cfgs = autotune.tune_batch(probs, prec, evals=2)
        tune_s = time.perf_counter() - t0
    budget = args.batch_mem_gb * (1 << 30)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for k in range(steps):
            flush.fill_(float(k))
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            ts.append((e0, e1))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(c) for a, c in ts)

    def wall(fn, steps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for k in range(steps):
            flush.fill_(float(k))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            ts.append(1000.0 * (time.perf_counter() - t0))
        return statistics.mean(ts)

    total_b = total_s = 0.0
    chunks, worst, peak_bytes, k0 = [], 0.0, 0, 0
    while k0 < len(probs):
        Ps, used = [], 0
        while k0 + len(Ps) < len(probs):
            P = q.Problem(probs[k0 + len(Ps)], precision=prec)
            nb = q.qoc_device_bytes(P.handle)
            if Ps and used + nb > budget:
                P.close()
                break
            if cfgs is not None:
                from paper_2505_00529_gb300 import autotune
                autotune.apply(P, cfgs[k0 + len(Ps)])
            Ps.append(P)
            used += nb
        idx = list(range(k0, k0 + len(Ps)))
        b = q.Batch(Ps, cuda_stream=stream.cuda_stream)
        th = torch.tensor(np.concatenate([thetas[k] for k in idx]), dtype=torch.float64, device=dev)
        out = torch.zeros(b.n_out, dtype=torch.float64, device=dev)
        ms_b = timed(lambda: q.qoc_batch_eval_grad_hess_dev(b.handle, th.data_ptr(), out.data_ptr()),
                     args.steps, args.warmup)
        for P in Ps:
            q.qoc_sync_status(P.handle)
        th_i = [torch.tensor(thetas[k], dtype=torch.float64, device=dev) for k in idx]
        out_i = [torch.zeros(1 + probs[k].K ** 2 + probs[k].K, dtype=torch.float64, device=dev) for k in idx]

        def sequential():
            for P, t, o in zip(Ps, th_i, out_i):
                q.qoc_eval_grad_hess_dev(P.handle, t.data_ptr(), o.data_ptr())
                q.qoc_sync_status(P.handle)
        ms_s = wall(sequential, 1)
        res = b.split(out.cpu().numpy())
        for j in range(0, len(Ps), max(1, len(Ps) // 4)):   # batched results = per-problem ones
            Jk, gk, Hk = Ps[j].eval_grad_hess(thetas[idx[j]])
            worst = max(worst, float(np.linalg.norm(res[j][2] - Hk) / np.linalg.norm(Hk)))
        chunks.append({"problems": len(Ps), "device_gb": round(used / 2 ** 30, 1), "batched_ms": ms_b,
                       "sequential_ms": ms_s})
        total_b += ms_b
        total_s += ms_s
        peak_bytes = max(peak_bytes, used)
        b.close()
        for P in Ps:
            P.close()
        del out, th
        k0 += len(Ps)
    shapes = [(pr.N, pr.K, pr.J) for pr in probs]
    line = {"metric": "batched grad+Hessian evaluations/s over uneven problems",
            "value": len(probs) * 1000.0 / total_b, "unit": "problem evals/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_b, "higher_is_better": True,
            "dtype": "f32 panels + f64" if prec == q.QOC_MIXED_FP32 else "f64", "data": "synthetic",
            "config": {"workload": f"{len(probs)} uneven problems from the batched-workload recipe",
                       "N_range": [min(x[0] for x in shapes), max(x[0] for x in shapes)],
                       "K_values": sorted({x[1] for x in shapes}), "J_values": sorted({x[2] for x in shapes}),
                       "total_steps": sum(x[2] for x in shapes), "l2": "flushed between timed steps",
                       "graph": True, "autotuned": tune_s is not None, "autotune_seconds": tune_s,
                       "memory_budget_gb": args.batch_mem_gb},
            "chunks": chunks, "sequential_ms": total_s, "speedup_over_sequential": total_s / total_b,
            "batched_vs_individual_hess_rel_max": worst, "peak_chunk_device_gb": round(peak_bytes / 2 ** 30, 1)}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--ref-sample-steps", type=int, default=400)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-tr", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="library default launch shapes")
    ap.add_argument("--warm-start", action="store_true", help="run the learned warm-start experiment")
    ap.add_argument("--batch", action="store_true", help="run the batched uneven-problem measurement")
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--batch-mem-gb", type=float, default=160.0,
                    help="device memory per batch chunk (problems are created chunk by chunk)")
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-test", type=int, default=200)
    ap.add_argument("--ws-epochs", type=int, default=300)
    ap.add_argument("--ws-workers", type=int, default=8)
    ap.add_argument("--ws-gtol", type=float, default=1e-5)
    args = ap.parse_args()
    if args.warm_start:
        return run_warm_start(args)
    if args.batch:
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
