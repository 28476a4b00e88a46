#!/usr/bin/env python
"""Gradient+Hessian evaluations per second of the discrete quantum-optimal-
control cost on GB300 (second-order adjoint method, Alg. 2), on the N=32,
K=64 (sine/cosine), J=4000 workload: CI-shaped synthetic H0 (diagonal
energies U[-10,0], band-8 couplings N(0,0.1^2)), dense M N(0,0.3^2), T=20.

One step = one full evaluation (J, grad, K x K Hessian) at a fixed seeded
theta, inputs resident in device memory.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64] [--no-extra]
  python bench.py --impl reference ...   (the FP64 CPU oracle, timed on the host)
  python bench.py --fp64-peak            (binary64 peak: FMA chains and cuBLAS DGEMM)
  python bench.py --profile ...          (the workload's evaluations only, for ncu)
  python bench.py --batch / --warm-start (the batched and warm-start measurements)
  python bench.py --scaling              (wall time vs J on the maximal model, Fig. 1)
  python bench.py --tr-ratios            (Alg. 1 + BFGS vs Alg. 2 trust regions, Tables I/II)

Besides the headline, the line carries the plain binary64 GPU method on the
same workload, trust-region solves, the binary64-bound kernels against the
binary64 FMA rate measured in the same run, the CPU oracle (one whole
evaluation on one core), and the other workloads (small single, largest
single, a batch of the uneven recipe) measured the same way.

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
# the `config` both arms print (the workload, and how the timed steps treat
# the cache); what differs between the arms goes under `run`
CONFIG = dict(WORKLOAD, l2="GPU arm: L2 flushed between timed steps (reference arm: host CPU)")
# library kernel launches per gradient + Hessian evaluation on the time-blocked path:
# control, binary32 Jacobi, binary64 refinement, 3 preparation parts (D, P~, X'),
# 2 block products, state chain + fill, terminal, costate chain + fill, drift,
# 3 pointwise parts (p^, y^/g, c), 3 block-source launches (Q, W/Gamma, backward),
# tangent and second-order adjoint panels, 2 panel contractions, grad, Hessian
# chunk partials, chunk sum, symmetrisation, asymmetry (ncu launch list: 29)
LAUNCHES_PER_EVAL = 29
# DRAM bytes (read + written) of a kernel's launches in one evaluation on a
# workload, from an ncu capture of the current kernel: (kernel, N, J) -> bytes.
# k_prep: P part 33.88 MB read + 39.58 MB written, X part 99.44 + 29.17 MB.
# (k_eig_refine read 32.95 MB, W of every step once, before it took its steps
# in the start's order; it has changed since, so it reports none.)
TRAFFIC_BYTES = {("k_prep", 32, 4000): 202.07e6}


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
p.B = p.B[:js]          # js = J: the whole workload; fewer: its first js steps (warm-up only)
th = inputs.eval_theta(p.K, 0)
t0 = time.perf_counter()
r = orc.evaluate(p, th, order=2)
dt = time.perf_counter() - t0
print(json.dumps({"seconds": dt, "steps": js}))
"""


def time_oracle(steps: int = WORKLOAD["J"]) -> dict:
    """One oracle evaluation (J, gradient, Hessian) of the bench workload on
    one host core, timed whole: `steps` = J is the full workload."""
    env = dict(os.environ, OPENBLAS_NUM_THREADS="1", OMP_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-c", ORACLE_SNIPPET % (ROOT, steps)],
                       capture_output=True, text=True, env=env, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": 1.0 / d["seconds"], "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": d["seconds"],
            "sample": f"one whole oracle evaluation of the workload ({d['steps']} steps, "
                      f"{d['seconds']:.2f} s), nothing extrapolated"}


def run_reference(args):
    rank = env_int("RANK", 0)
    if rank != 0:
        return 0
    for _ in range(args.warmup):            # untimed: short samples that load numpy and warm the caches
        time_oracle(100)
    per = [time_oracle()["seconds"] for _ in range(args.steps)]
    ms = 1000.0 * statistics.mean(per)
    value = 1000.0 / ms
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": CONFIG, "run": {"precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: one whole oracle evaluation of the {WORKLOAD['J']}-step "
                                       f"workload (J, gradient, Hessian), timed whole; warm-up steps "
                                       f"evaluate its first 100 steps"},
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
        q.qoc_set_pipeline(P.handle, args.pipeline)
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
            q.qoc_enable_timing(PT.handle, True)
            t0 = time.perf_counter()
            th_star, info = PT.trust_region_solve(np.zeros(K), gtol=1e-6, xtol=1e-10, max_iter=500)
            t1 = time.perf_counter()
            trph = q.qoc_get_tr_phase_times(PT.handle)
        tr_s = max_over_ranks(t1 - t0, dist, dev)
        trph["host_and_sync"] = 1e3 * (t1 - t0) - sum(trph.values())
        tr = {"value": world / tr_s, "unit": "TR solves/s", "iters": info["iters"],
              "n_eval_gh": info["n_eval_gh"], "n_eval_J": info["n_eval_J"], "J": info["J"],
              "grad_norm": info["grad_norm"], "stop": info["stop"], "gtol": 1e-6,
              "phase_ms": trph,
              "phase_how": "device time by CUDA events around each phase of the solve (timing mode); "
                           "host_and_sync = wall time minus their sum"}

    # ---- batched trust-region solves: 32 random targets of the same system, from theta = 0 ----
    trb = None
    if not args.no_tr:
        betas = inputs.random_targets(4100, N, 32)
        Ps = [q.Problem(prob, precision=prec, cuda_stream=stream.cuda_stream) for _ in betas]
        try:
            for P, bt in zip(Ps, betas):
                P.set_target(bt)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            _, infos, _st = q.qoc_batch_trust_region_solve([P.handle for P in Ps], [np.zeros(K)] * len(Ps),
                                                           gtol=1e-6, xtol=1e-10, max_iter=500,
                                                           cuda_stream=stream.cuda_stream)
            t1 = time.perf_counter()
        finally:
            for P in Ps:
                P.close()
        trb_s = max_over_ranks(t1 - t0, dist, dev)
        trb = {"value": world * len(betas) / trb_s, "unit": "TR solves/s", "problems": len(betas),
               "seconds": trb_s, "iters_mean": float(np.mean([i["iters"] for i in infos])),
               "iters_max": int(max(i["iters"] for i in infos)),
               "stops": {s_: sum(i["stop"] == s_ for i in infos) for s_ in ("gtol", "xtol", "max_iter",
                                                                            "no_decrease", "failed")},
               "how": "qoc_batch_trust_region_solve over 32 random targets of the workload's system, "
                      "theta0 = 0, gtol 1e-6; every trial point evaluated with its gradient and Hessian"}

    # ---- roofline: the binary64-bound kernels against the measured binary64 rate ----
    fp64_tf, fp64_ms = q.qoc_measure_fp64_rate(4, 5)
    ph_mean = {k: statistics.mean(p[k] for p in phases) for k in phases[0]} if phases else {}
    roof = None
    if ph_mean:
        roof = roofline(N, J, ph_mean, fp64_tf)

    extra = {}
    if not args.no_extra:
        extra = run_extra_workloads(q, inputs, stream, flush, dev, dist)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        try:
            cpu = time_oracle()
        except Exception as e:  # reported, never silently dropped
            cpu = {"error": str(e)[-300:]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f32 panels + f64" if prec == q.QOC_MIXED_FP32 else "f64",
                "data": "synthetic",
                "config": CONFIG,
                "run": dict(precision=args.precision,
                               parallelism=f"replicas x{world}" if world > 1 else "single problem",
                               pipeline_chunks=args.pipeline if args.pipeline >= 0 else "library choice (off)",
                               hessian=("second-order adjoint, unsplit (the qoc_set_mu_split built-in "
                                        "choice for binary32 sweeps)" if prec == q.QOC_MIXED_FP32 else
                                        "second-order adjoint, terminal part in closed form (the "
                                        "qoc_set_mu_split built-in choice for binary64 sweeps)"),
                               launch=({"block_steps": tuned[prec]["block_steps"],
                                        "panel_columns": tuned[prec]["panel_columns"],
                                        "autotune_table_ms": tuned[prec]["table"]}
                                       if prec in tuned else "library defaults")),
                "e2e": {"value": whole_job_rate(world, e2e_ms), "unit": UNIT, "ms_per_step": e2e_ms,
                        "h2d_bytes_per_step": 8 * K, "d2h_bytes_per_step": 8 * (1 + K + K * K)},
                "gpu_launches": LAUNCHES_PER_EVAL * args.steps,
                "clocks": clocks, "roofline": roof, "cpu_baseline": cpu,
                "fp64_plain": fp64, "tr_solve": tr, "tr_solve_batched": trb,
                "fp64_fma_peak": {"tflops": fp64_tf, "ms": fp64_ms, "how": "qoc_measure_fp64_rate: "
                                  "independent binary64 FMA chains, 4 CTAs x 256 threads per SM, best of 5"},
                "eig_stats": {k: ph_mean[k] for k in ("refine_updates_per_step", "cleanup_rotated_fraction",
                                                      "final_pass_fraction") if k in ph_mean},
                "other_workloads": extra}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


# algorithmic binary64 flops per time step (the per-step counts of the method:
# eigendecomposition 9 N^3, the textbook count of the symmetric QR with
# vectors; M~ = W^T M W 4 N^3 and the second-derivative term X' 8 N^3)
def eig_flops_per_step(N):
    return 9.0 * N ** 3


def prep_flops_per_step(N):
    return 12.0 * N ** 3


def roofline(N, J, ph, fp64_tf):
    """Achieved binary64 rate of the binary64-bound kernels: algorithmic flops
    per launch (per-step count x J steps) / the kernel's duration, measured by
    CUDA events around its launch on the problem's stream, against the binary64
    FMA rate measured in this run.  The dominant one (longest) is the line's
    roofline; the others are listed with it."""
    rows = {
        "k_prep": (prep_flops_per_step(N) * J, ph["k_deriv_prep"],
                   "M~ = W^T M W (4 N^3) and X' (8 N^3) per step"),
        "k_eig_refine": (eig_flops_per_step(N) * J, ph["k_eig_refine"],
                         "the whole eigendecomposition's 9 N^3 per step, credited to the refinement kernel"),
        "eig (binary32 Jacobi start + k_eig_refine)": (eig_flops_per_step(N) * J, ph["k_eig_jacobi"] + ph["k_eig_refine"],
                                                "9 N^3 per step over both eigensolver kernels"),
    }
    kern = {}
    for name, (fl, t, how) in rows.items():
        ach = fl / (t * 1e-3) / 1e12
        kern[name] = {"achieved": ach, "frac": ach / fp64_tf, "kernel_ms": t, "algorithmic_gflop": fl / 1e9,
                      "count": how}
    dom = max(("k_prep", "k_eig_refine"), key=lambda k: kern[k]["kernel_ms"])
    d = kern[dom]
    return {"bound": "alu", "kernel": dom, "achieved": d["achieved"], "peak": fp64_tf, "unit": "TFLOP/s",
            "frac": d["frac"], "traffic": TRAFFIC_BYTES.get((dom, N, J)),
            "traffic_source": "dram__bytes_read.sum + dram__bytes_write.sum of one launch (ncu capture of "
                              "this workload, current kernel)" if TRAFFIC_BYTES.get((dom, N, J)) else None,
            "peak_source": "binary64 FMA rate measured in this run (qoc_measure_fp64_rate); "
                           "MEASURED_PEAKS.json has no binary64 figure",
            "algorithmic": f"{d['algorithmic_gflop']:.3f} GFLOP per launch: {d['count']}, N={N}, J={J}",
            "note": "for problems on binary32 sweeps with N <= 32 the binary64 N^3 products run on the "
                    "tensor pipe by error-free splitting (six 8-bit slices per entry, bf16 mma with exact "
                    "binary32 accumulation), so the effective binary64 rate can exceed the binary64 "
                    "pipe's FMA peak",
            "kernel_ms": d["kernel_ms"], "kernels": kern,
            "phase_ms": {k: v for k, v in ph.items() if not k.startswith("k_") and k in
                         ("eig", "prep", "chains", "pointwise", "panels", "assembly")},
            "kernel_phase_ms": {k[2:]: v for k, v in ph.items() if k.startswith("k_")}}


def _timed_evals(q, P, K, th, out, stream, flush, steps, warmup):
    """Mean device time (ms) of `steps` gradient + Hessian evaluations of P."""
    import torch
    for _ in range(warmup):
        q.qoc_eval_grad_hess_dev(P.handle, th.data_ptr(), out.data_ptr())
    q.qoc_sync_status(P.handle)
    ev = []
    for k in range(steps):
        flush.fill_(float(k))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        q.qoc_eval_grad_hess_dev(P.handle, th.data_ptr(), out.data_ptr())
        e1.record(stream)
        ev.append((e0, e1))
    torch.cuda.synchronize()
    q.qoc_sync_status(P.handle)
    return statistics.mean(a.elapsed_time(b) for a, b in ev)


def run_extra_workloads(q, inputs, stream, flush, dev, dist):
    """The other single-problem workloads and a batch of the uneven recipe,
    device-resident, each timed with CUDA events (L2 flushed in between):
    small single (N=4, K=8, J=1000) in both precisions, largest single
    (N=256, K=128, J=10^4) one evaluation in mixed precision (the policy's
    sweep precision reported), and the first 32 problems of the batched
    recipe as one batch against the same problems one by one."""
    import numpy as np
    import torch
    res = {}
    p1 = inputs.config_problem(1)
    th1 = torch.tensor(inputs.eval_theta(p1.K, 0), dtype=torch.float64, device=dev)
    o1 = torch.zeros(1 + p1.K + p1.K ** 2, dtype=torch.float64, device=dev)
    r1 = {}
    for name, prec in (("fp64", q.QOC_FP64), ("mixed", q.QOC_MIXED_FP32)):
        with q.Problem(p1, precision=prec, cuda_stream=stream.cuda_stream) as P:
            t = max_over_ranks(_timed_evals(q, P, p1.K, th1, o1, stream, flush, 20, 3), dist, dev)
            r1[name] = {"evals_per_s": 1000.0 / t, "ms": t, "sweep_precision": P.precision()[0]}
    res["small single N=4 K=8 J=1000"] = r1
    p5 = inputs.config_problem(5)
    th5 = torch.tensor(inputs.eval_theta(p5.K, 5), dtype=torch.float64, device=dev)
    o5 = torch.zeros(1 + p5.K + p5.K ** 2, dtype=torch.float64, device=dev)
    with q.Problem(p5, precision=q.QOC_MIXED_FP32, cuda_stream=stream.cuda_stream) as P:
        eff, est = P.precision()
        t = max_over_ranks(_timed_evals(q, P, p5.K, th5, o5, stream, flush, 1, 0), dist, dev)
    res["largest single N=256 K=128 J=10000"] = {
        "precision": "mixed", "sweep_precision": "fp64" if eff == q.QOC_FP64 else "fp32",
        "binary32_error_estimate": est, "evals_per_s": 1000.0 / t, "ms": t}
    probs = [inputs.config_problem(3, i) for i in range(32)]
    Ps = [q.Problem(p, precision=q.QOC_MIXED_FP32) for p in probs]
    try:
        with q.Batch(Ps, cuda_stream=stream.cuda_stream) as b:
            thetas = [inputs.eval_theta(p.K, 7 + k) for k, p in enumerate(probs)]
            th = torch.tensor(np.concatenate(thetas), dtype=torch.float64, device=dev)
            out = torch.zeros(b.n_out, dtype=torch.float64, device=dev)
            q.qoc_batch_eval_grad_hess_dev(b.handle, th.data_ptr(), out.data_ptr())   # eager + graph capture
            torch.cuda.synchronize()
            ev = []
            for k in range(2):
                flush.fill_(float(k))
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                q.qoc_batch_eval_grad_hess_dev(b.handle, th.data_ptr(), out.data_ptr())
                e1.record(stream)
                ev.append((e0, e1))
            torch.cuda.synchronize()
            for P in Ps:
                q.qoc_sync_status(P.handle)
            tb = max_over_ranks(statistics.mean(a.elapsed_time(c) for a, c in ev), dist, dev)
            ths = [torch.tensor(t_, dtype=torch.float64, device=dev) for t_ in thetas]
            outs = [torch.zeros(1 + p.K + p.K ** 2, dtype=torch.float64, device=dev) for p in probs]
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for P, t_, o_ in zip(Ps, ths, outs):
                q.qoc_eval_grad_hess_dev(P.handle, t_.data_ptr(), o_.data_ptr())
            e1.record(stream)
            torch.cuda.synchronize()
            ts = max_over_ranks(e0.elapsed_time(e1), dist, dev)
        res["batched recipe, first 32 problems"] = {
            "problem_evals_per_s": 32 * 1000.0 / tb, "batched_ms": tb, "one_by_one_ms": ts,
            "speedup_over_one_by_one": ts / tb, "binary64_sweep_problems":
                sum(P.precision()[0] == q.QOC_FP64 for P in Ps),
            "N": [p.N for p in probs], "K": [p.K for p in probs], "J": [p.J for p in probs]}
    finally:
        for P in Ps:
            P.close()
    return res


def run_fp64_peak(args):
    """Binary64 peak of this GPU: the library's FMA-chain kernel and cuBLAS
    DGEMM (torch.matmul in float64, 8192^3), with the SM clocks sampled."""
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build
    local = env_int("LOCAL_RANK", 0)
    torch.cuda.set_device(local)
    build.build()
    clk = ClockSampler(local, os.path.join(tempfile.mkdtemp(prefix="qoc_clocks_"), "clocks.csv"))
    with clk:
        fma = [q.qoc_measure_fp64_rate(c, 5) for c in (1, 2, 4, 8)]
        n = 8192
        a = torch.randn(n, n, dtype=torch.float64, device="cuda")
        b = torch.randn(n, n, dtype=torch.float64, device="cuda")
        torch.matmul(a, b)
        torch.cuda.synchronize()
        best = None
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            best = t if best is None else min(best, t)
    dgemm = 2.0 * n ** 3 / (best * 1e-3) / 1e12
    print(json.dumps({"metric": "binary64 peak", "fma_chain_tflops": {str(c): f[0] for c, f in zip((1, 2, 4, 8), fma)},
                      "cublas_dgemm_tflops": dgemm, "dgemm_ms": best, "n": n, "clocks": clk.summary()}), flush=True)
    return 0


# the paper's OLS slopes of log2 wall time against log2 J (Sec. IV-A), context only
PAPER_SLOPES = {"alg1": {4: 0.9082, 16: 0.9067, 64: 0.9999, 144: 1.001},
                "alg2": {4: 0.9871, 16: 0.9938, 64: 0.9975, 144: 1.006}}


def run_scaling(args):
    """Wall-time scaling in J (Sec. IV-A, Fig. 1): the maximal model (K = J),
    N in {4, 16, 64, 144}, J = 2^2 .. 2^10; per (N, J) `scaling_runs` timed
    evaluations of Alg. 1 (J and gradient) and Alg. 2 (J, gradient, Hessian)
    at the same theta ~ N(0, 1), through the host API (theta in, results out,
    as a caller of the library sees them), mean and standard deviation; then
    the OLS slope of log2(mean time) against log2(J) per N and algorithm."""
    import numpy as np
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    build.build()
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    Ns = [int(x) for x in args.scaling_n.split(",")]
    kappas = list(range(2, 11))
    rows, slopes = [], {}
    for N in Ns:
        t1, t2 = [], []
        for kap in kappas:
            J = 2 ** kap
            prob = inputs.scaling_problem(N, J, seed=100 * N + kap)
            theta = inputs.eval_theta(J, 7 * N + kap)
            with q.Problem(prob, precision=prec) as P:
                for _ in range(3):
                    P.eval_grad(theta)
                    P.eval_grad_hess(theta)
                a1, a2 = [], []
                for _ in range(args.scaling_runs):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    P.eval_grad(theta)
                    a1.append(1000.0 * (time.perf_counter() - t0))
                    t0 = time.perf_counter()
                    P.eval_grad_hess(theta)
                    a2.append(1000.0 * (time.perf_counter() - t0))
                sweep = P.precision()[0]
            rows.append({"N": N, "J": J, "alg1_ms": statistics.mean(a1), "alg1_sd": statistics.pstdev(a1),
                         "alg2_ms": statistics.mean(a2), "alg2_sd": statistics.pstdev(a2),
                         "sweep_precision": "fp64" if sweep == q.QOC_FP64 else "fp32"})
            t1.append(statistics.mean(a1))
            t2.append(statistics.mean(a2))
        x = np.log2([2.0 ** k for k in kappas])
        slopes[N] = {"alg1": float(np.polyfit(x, np.log2(t1), 1)[0]),
                     "alg2": float(np.polyfit(x, np.log2(t2), 1)[0]),
                     "alg2_over_alg1_at_J1024": t2[-1] / t1[-1]}
    print(json.dumps({"metric": "wall time vs J, maximal model (log-log OLS slope)", "unit": "ms",
                      "precision": args.precision, "runs_per_point": args.scaling_runs,
                      "config": {"workload": "maximal model K=J, alpha=e_1, beta=e_N, diagonal H0 U[-2,0], "
                                             "symmetric M N(0,0.5^2), dt=0.1, theta ~ N(0,1), host API"},
                      "slopes": slopes, "paper_slopes_A100_context": PAPER_SLOPES, "points": rows}),
          flush=True)
    return 0


def run_tr_ratios(args):
    """Gradient-only (Alg. 1 + BFGS) against exact-Hessian (Alg. 2) trust
    regions, the comparison of Sec. IV-B (Tables I and II) on synthetic
    stand-ins for its molecular systems: N in {4, 16} (the sizes of the
    STO-3G and 6-31G full-CI problems), the maximal model with J = 200 steps
    of dt = 0.1 (K = J = 200), rho = 1e6 (w_f = 1/2, w_t = rho/2),
    alpha = e_1, beta = e_N, tolerances delta = epsilon = 1e-10, at most 10^4
    iterations.  Each trial draws theta0 ~ N(0, 1) and solves from it with
    both methods; per-trial ratios Alg1/Alg2 of iterations, wall time, final
    cost, final |grad| and target violation |a_J - beta| are summarised by
    their mean and (0.05, 0.95) quantiles as in Table II."""
    import numpy as np
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    build.build()
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    J, rho = 200, 1e6
    out = {}
    for N in (4, 16):
        base = inputs.scaling_problem(N, J, seed=7000 + N)
        prob = inputs.Problem(base.H0, base.M, base.alpha, base.beta, base.B, base.dt, 0.5, rho / 2,
                              name=f"tables_N{N}")
        rows = []
        with q.Problem(prob, precision=prec) as P:
            for t in range(args.tr_trials):
                th0 = np.random.default_rng(500 + t).normal(size=J)
                rec = {}
                for alg, hess in (("alg1", "bfgs"), ("alg2", "exact")):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    th, info = P.trust_region_solve(th0, gtol=1e-10, xtol=1e-10, max_iter=10000, hessian=hess)
                    wall = time.perf_counter() - t0
                    viol = np.sqrt(max(info["J"] - 0.5 * float(th @ th), 0.0) / (rho / 2))
                    rec[alg] = {"iters": info["iters"], "wall_s": wall, "cost": info["J"],
                                "grad": info["grad_norm"], "viol": viol, "stop": info["stop"]}
                rows.append(rec)
        summ = {}
        for key in ("iters", "wall_s", "cost", "grad", "viol"):
            a1 = np.array([r["alg1"][key] for r in rows], float)
            a2 = np.array([r["alg2"][key] for r in rows], float)
            ratio = a1 / np.maximum(a2, 1e-300)
            summ[key] = {"alg1_mean": float(a1.mean()), "alg2_mean": float(a2.mean()),
                         "ratio_mean": float(ratio.mean()),
                         "ratio_q05": float(np.quantile(ratio, 0.05)), "ratio_q95": float(np.quantile(ratio, 0.95))}
        summ["stops"] = {alg: {s_: sum(r[alg]["stop"] == s_ for r in rows) for s_ in ("gtol", "xtol", "max_iter",
                                                                                 "no_decrease")}
                         for alg in ("alg1", "alg2")}
        out[f"N={N}"] = summ
    print(json.dumps({"metric": "per-trial ratios Alg1 (BFGS) / Alg2 (exact Hessian) of trust-region solves",
                      "trials": args.tr_trials, "precision": args.precision,
                      "config": {"workload": "maximal model J=K=200, dt=0.1, rho=1e6, alpha=e_1, beta=e_N, "
                                             "diagonal H0 U[-2,0], symmetric M N(0,0.5^2), tol 1e-10"},
                      "results": out}), flush=True)
    return 0


def run_profile(args):
    """The bench workload only (for ncu): `warmup` + `steps` evaluations of the
    N=32, K=64, J=4000 problem at library defaults, no extras, no output line."""
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    build.build()
    prob = inputs.config_problem(2)
    theta = inputs.eval_theta(prob.K, 0)
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    with q.Problem(prob, precision=prec) as P:
        for _ in range(args.warmup + args.steps):
            P.eval_grad_hess(theta)
    return 0


def run_warm_start(args):
    """Learned warm start on the N=32 system (H0, M of the bench workload,
    dt=0.005) with a K=64 Fourier basis over J = --ws-steps steps (4000:
    T=20, the bench workload itself): theta* from the library's trust region
    on random unit targets, MLP 2N -> 256^3 -> K trained by the library's
    kernels, then held-out targets solved from theta=0, from the MLP's
    theta0, from the guarded start t* MLP(beta) (t* minimising J over t in
    {0, 1/4, 1/2, 3/4, 1}) and from the decrement-chosen start (0 or
    MLP(beta), the smaller Newton decrement) to the same tolerance; the plain
    binary64 method on the first --ws-plain held-out targets."""
    import numpy as np
    import torch
    import paper_2505_00529_gb300 as q
    from paper_2505_00529_gb300 import build, inputs, warmstart
    torch.cuda.set_device(env_int("LOCAL_RANK", 0))
    build.build()
    base = inputs.config_problem(4)
    J = args.ws_steps
    prob = base if J == base.J else inputs.Problem(base.H0, base.M, base.alpha, base.beta,
                                                   inputs.sine_cosine_basis(J, base.dt, 64), base.dt,
                                                   base.dt, 1.0, "warm-start")
    train = inputs.random_targets(4000, prob.N, args.ws_train)
    test = inputs.random_targets(4001, prob.N, args.ws_test)
    prec = q.QOC_MIXED_FP32 if args.precision == "mixed" else q.QOC_FP64
    t0 = time.perf_counter()
    r = warmstart.compare(prob, train, test, precision=prec, workers=args.ws_workers, epochs=args.ws_epochs,
                          batch=128, lr=1e-3, seed=0, n_plain=args.ws_plain, train_cache=args.ws_cache,
                          gtol=args.ws_gtol, xtol=1e-12, max_iter=500)
    r["total_seconds"] = time.perf_counter() - t0
    line = {"metric": "trust-region iterations and wall time on held-out targets: learned warm start vs theta=0",
            "value": r["wall_ratio_zero_over_mlp"],
            "unit": "wall-time ratio of the held-out solves, theta=0 / MLP start (same final tolerance)",
            "higher_is_better": True, "n_gpus": 1, "dtype": "f32 panels + f64" if prec else "f64",
            "data": "synthetic",
            "config": {"workload": f"N=32 system, K=64 Fourier basis, T={J * base.dt:g}, J={J}; "
                                   f"{args.ws_train} training / "
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-tr", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="library default launch shapes")
    ap.add_argument("--pipeline", type=int, default=-1,
                    help="forward-pipeline chunks of the timed problem (0 off, -1 library choice)")
    ap.add_argument("--no-extra", action="store_true", help="skip the other workloads")
    ap.add_argument("--fp64-peak", action="store_true", help="measure the binary64 peak and exit")
    ap.add_argument("--profile", action="store_true", help="evaluations of the bench workload only (for ncu)")
    ap.add_argument("--scaling", action="store_true", help="wall time vs J on the maximal model (Fig. 1)")
    ap.add_argument("--tr-ratios", action="store_true", help="Alg. 1 + BFGS vs Alg. 2 trust regions (Tables I/II)")
    ap.add_argument("--tr-trials", type=int, default=10)
    ap.add_argument("--scaling-runs", type=int, default=20)
    ap.add_argument("--scaling-n", default="4,16,64,144")
    ap.add_argument("--warm-start", action="store_true", help="run the learned warm-start experiment")
    ap.add_argument("--batch", action="store_true", help="run the batched uneven-problem measurement")
    ap.add_argument("--batch-size", type=int, default=256)
    ap.add_argument("--batch-mem-gb", type=float, default=160.0,
                    help="device memory per batch chunk (problems are created chunk by chunk)")
    ap.add_argument("--ws-steps", type=int, default=4000, help="time steps J of the warm-start system")
    ap.add_argument("--ws-plain", type=int, default=200,
                    help="held-out targets also solved by the plain binary64 method")
    ap.add_argument("--ws-cache", default=None, help=".npz file caching the training optima")
    ap.add_argument("--ws-train", type=int, default=2000)
    ap.add_argument("--ws-test", type=int, default=200)
    ap.add_argument("--ws-epochs", type=int, default=300)
    ap.add_argument("--ws-workers", type=int, default=8)
    ap.add_argument("--ws-gtol", type=float, default=1e-5)
    args = ap.parse_args()
    if args.fp64_peak:
        return run_fp64_peak(args)
    if args.profile:
        return run_profile(args)
    if args.scaling:
        return run_scaling(args)
    if args.tr_ratios:
        return run_tr_ratios(args)
    if args.warm_start:
        return run_warm_start(args)
    if args.batch:
        return run_batch(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
