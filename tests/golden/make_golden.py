"""Write the stored expected values under tests/golden/ from the oracle only.

    python tests/golden/make_golden.py

* kernel_ridge_oracle_iters.json -- the oracle's own RandRAND-PCG solve of
  the kernel ridge workload (n = 20000, d = 8, k = 500, mu = 1e-3, 4 right-hand
  sides, bf16-rounded Gaussian Omega, rtol 1e-6): inner iterations per column
  and the float64 relative residuals; used to scale the CPU reference timing.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import randrand as O  # noqa: E402
from workloads import generators as W  # noqa: E402


def kernel_ridge_iters():
    n, k, mu, m, seed = 20000, 500, 1e-3, 4, 0x52522
    X = W.mixture_points(n, 8, 10, seed=seed)
    B = W.gaussian_rhs(n, m, seed)
    t0 = time.time()
    op = O.GaussKernelOp(X, materialize=True)
    bd = O.build(op, mu, k, "gaussian", seed, omega_precision="bf16")
    Xs, infos = O.solve(bd, B, rtol=1e-6)
    res = O.true_rel_residual(op, mu, Xs, B)
    return {"workload": "gaussian_kernel_ridge", "n": n, "k": k, "mu": mu, "nrhs": m,
            "seed": seed, "rtol": 1e-6,
            "inner_iters": [i.inner_iters for i in infos],
            "outer_iters": [i.outer_iters for i in infos],
            "inner_iters_max": max(i.inner_iters for i in infos),
            "rel_residual": [float(r) for r in res], "tau": bd.tau, "normE": bd.normE,
            "lam_max": bd.lam_max, "oracle_seconds": time.time() - t0}


if __name__ == "__main__":
    json.dump(kernel_ridge_iters(), open(os.path.join(HERE, "kernel_ridge_oracle_iters.json"), "w"),
              indent=1)
    print("written")
