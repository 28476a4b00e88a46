"""Writes largest_N256_K128_J200.npz: the binary64 oracle's evaluation of the
largest single-problem system (N = 256 basis, K = 128 sine coefficients,
dt = 0.004, CI-shaped H0 with band-32 couplings, dense M) on its first 200
time steps, at theta = eval_theta(128, 5).

The oracle needs a few seconds per step at N = 256, far too long to rerun
inside the GPU tests, so its result is stored once.  Only `oracle/` and the
seeded input generators are called here; nothing comes from the CUDA path.

Stored (all float64): J, grad (K), hess (K x K, symmetrised), hess_raw,
g, c (200 each), U, V (200 x K), and for the sampled steps
STEP_SAMPLE = 0, 10, ..., 200 the states a_j and costates lambda_j
(interleaved re/im, 21 x 2N) and for steps 0, 10, ..., 190 the eigenvalues.

    python tests/golden/make_largest_N256.py
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2505_00529_gb300 import inputs  # noqa: E402
from oracle import qoc_oracle as orc       # noqa: E402

STEPS = 200
OUT = os.path.join(HERE, "largest_N256_K128_J200.npz")


def problem():
    full = inputs.config_problem(5)
    return inputs.Problem(full.H0, full.M, full.alpha, full.beta, full.B[:STEPS], full.dt, full.w_f,
                          full.w_t, name="largest-200"), inputs.eval_theta(full.K, 5)


def interleave(z):
    z = np.asarray(z)
    out = np.empty(z.shape[:-1] + (2 * z.shape[-1],))
    out[..., 0::2] = z.real
    out[..., 1::2] = z.imag
    return out


def main():
    prob, theta = problem()
    t0 = time.perf_counter()
    r = orc.evaluate(prob, theta, order=2, keep=True)
    rows = np.arange(0, STEPS + 1, 10)
    np.savez_compressed(
        OUT, J=r["J"], grad=r["grad"], hess=r["hess"], hess_raw=r["hess_raw"], g=r["g"], c=r["c"],
        U=r["U"], V=r["V"], step_sample=rows, a=interleave(r["a"][rows]), lam=interleave(r["lam"][rows]),
        eig_steps=rows[:-1], eig=r["eig"][rows[:-1]], theta=theta)
    print(f"wrote {OUT} in {time.perf_counter() - t0:.0f} s")


if __name__ == "__main__":
    main()
