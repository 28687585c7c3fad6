"""Writes cond_sigma.json: the noise level of the ill-conditioned SE workload.

Workload: n = 16384 points X ~ N(0, 1) in d = 16 (seed 0), SE kernel with
alpha = 1, rho = 4.  The noise variance is chosen so the covariance has
condition number about 1e5:  sigma^2 = lambda_max(K^f) / 1e5, with
lambda_max of the noise-free matrix K^f from 30 power iterations.

K^f is built by the CPU oracle (oracle.se_cov); the power iteration is plain
NumPy.  Nothing here touches the GPU library.  Run from the repository root:
    python tests/golden/make_cond_sigma.py
"""
import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1907_01063_gb300 import workloads as W  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "cond_sigma.json")


def lambda_max(n, d, alpha, rho, seed, iters=30):
    X = W.gp_inputs(n, d, seed)
    Kf = O.se_cov(X, alpha, rho, 0.0, 0.0, full=True)
    v = np.ones(n) / math.sqrt(n)
    lam = 0.0
    for _ in range(iters):
        w = Kf @ v
        lam = float(v @ w)
        v = w / np.linalg.norm(w)
    return lam


def main():
    n, d, alpha, rho, seed, target = 16384, 16, 1.0, 4.0, 0, 1e5
    t0 = time.time()
    lam = lambda_max(n, d, alpha, rho, seed)
    sigma2 = lam / target
    rec = {"n": n, "d": d, "alpha": alpha, "rho": rho, "seed": seed, "power_iters": 30,
           "lambda_max": lam, "target_cond": target, "sigma2": sigma2, "sigma": math.sqrt(sigma2),
           "cond_upper_bound": (lam + sigma2) / sigma2,
           "note": "lambda_min(K) >= sigma^2, so cond(K) <= (lambda_max + sigma^2) / sigma^2"}
    with open(OUT, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), f"({time.time() - t0:.1f} s)")


if __name__ == "__main__":
    main()
