"""Writes the noise levels of the ill-conditioned SE workloads.

cond_sigma.json: n = 16384 points X ~ N(0, 1) in d = 16 (seed 0), SE kernel
with alpha = 1, rho = 4, noise variance sigma^2 = lambda_max(K^f) / 1e5, so the
covariance has condition number about 1e5 (the benchmark's workload).

cond_sigma_n4096_1e6.json: the same recipe at n = 4096 with target 1e6, the
edge of the conditioning range the FP64 parity bar is stated for.  At this
size the record also holds the condition number itself, from the extreme
eigenvalues of the oracle's K (a LAPACK eigenvalue routine; descriptive only).

lambda_max of the noise-free matrix K^f comes from 30 power iterations.  K^f
and K are built by the CPU oracle (oracle.se_cov); the power iteration is
plain NumPy.  Nothing here touches the GPU library.  Run from the repository
root:
    python tests/golden/make_cond_sigma.py [n4096]
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


def record(n, d, alpha, rho, seed, target, exact_cond=False):
    lam = lambda_max(n, d, alpha, rho, seed)
    sigma2 = lam / target
    rec = {"n": n, "d": d, "alpha": alpha, "rho": rho, "seed": seed, "power_iters": 30,
           "lambda_max": lam, "target_cond": target, "sigma2": sigma2, "sigma": math.sqrt(sigma2),
           "cond_upper_bound": (lam + sigma2) / sigma2,
           "note": "lambda_min(K) >= sigma^2, so cond(K) <= (lambda_max + sigma^2) / sigma^2"}
    if exact_cond:
        K = O.se_cov(W.gp_inputs(n, d, seed), alpha, rho, math.sqrt(sigma2), 0.0, full=True)
        ev = np.linalg.eigvalsh(K)
        rec["lambda_min_K"] = float(ev[0])
        rec["lambda_max_K"] = float(ev[-1])
        rec["cond"] = float(ev[-1] / ev[0])
    return rec


def main(which):
    t0 = time.time()
    if which == "n4096":
        rec = record(4096, 16, 1.0, 4.0, 0, 1e6, exact_cond=True)
        out = os.path.join(os.path.dirname(OUT), "cond_sigma_n4096_1e6.json")
    else:
        rec = record(16384, 16, 1.0, 4.0, 0, 1e5)
        out = OUT
    with open(out, "w") as f:
        json.dump(rec, f, indent=1)
    print(json.dumps(rec), f"({time.time() - t0:.1f} s)")


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else "n16384")
