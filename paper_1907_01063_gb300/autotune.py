"""Autotuner for the library's tuning knobs.

Times the candidate values of each knob on the device at hand and keeps the
fastest; results are cached per device name and workload shape in a JSON
file (``GPCHOL_TUNE_CACHE``, default ``~/.cache/gpchol/tune.json``) so later
runs apply them without timing again.

Knobs:
  * batch_block: block size inside the batched per-GP pass (32 or 64), timed
    on a batch of GPs with the caller's size mix, separately per precision.
  * fp64_block: block size of the FP64 blocked factorisation and adjoint
    (64, 96 or 128), timed on chol + adjoint at a stand-in order.
The mixed path's block is fixed to its 128-wide slice chunk.
"""
from __future__ import annotations

import json
import os
import time

import numpy as np
import torch

import paper_1907_01063_gb300 as gp
from paper_1907_01063_gb300 import workloads as W

_DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "gpchol", "tune.json")


def _cache_path() -> str:
    return os.environ.get("GPCHOL_TUNE_CACHE", _DEFAULT_CACHE)


def _load() -> dict:
    try:
        with open(_cache_path()) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(db: dict):
    path = _cache_path()
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + f".{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(db, f, indent=1)
        os.replace(tmp, path)
    except OSError:
        pass  # a read-only home only costs re-tuning


def _device_key() -> str:
    return torch.cuda.get_device_name().replace(" ", "_")


def _time(fn, reps: int = 2) -> float:
    fn()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def tune_batch_block(batch: "gp.Batch", X, y, hyp, force: bool = False) -> dict:
    """Pick the batched block size for this batch's size mix and precision; applies it."""
    key = f"{_device_key()}/batch/{batch.precision}/{batch.batch}x{batch.nmax}/sum{batch.total_rows}"
    db = _load()
    if key in db and not force:
        gp.set_tuning(gp.GPC_TUNE_BATCH_BLOCK, db[key]["best"])
        return db[key]
    times = {}
    for b in (32, 64):
        gp.set_tuning(gp.GPC_TUNE_BATCH_BLOCK, b)
        times[b] = _time(lambda: gp.batched_gp_lml_grad(batch, X, y, hyp))
    best = min(times, key=times.get)
    gp.set_tuning(gp.GPC_TUNE_BATCH_BLOCK, best)
    rec = {"best": best, "ms": {str(k): v for k, v in times.items()}, "when": time.time()}
    db[key] = rec
    _store(db)
    return rec


def tune_fp64_block(n: int = 4096, force: bool = False) -> dict:
    """Pick the FP64 factorisation block size (timed on chol + adjoint at order n); applies it."""
    key = f"{_device_key()}/fp64_block/{n}"
    db = _load()
    if key in db and not force:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, db[key]["best"])
        return db[key]
    L0 = W.known_factor(n, seed=0)
    Ld = torch.as_tensor(L0, device="cuda")
    K = Ld @ Ld.T
    Lbar = torch.as_tensor(W.random_lower(n, seed=1), device="cuda")
    times = {}
    for b in (64, 96, 128):
        gp.set_tuning(gp.GPC_TUNE_BLOCK, b)
        ws = gp.workspace(n, "fp64")
        L = torch.empty_like(K)

        def run():
            gp.chol(K, out=L, ws=ws, check=False)
            gp.chol_adjoint(L, Lbar, ws=ws)

        times[b] = _time(run)
    best = min(times, key=times.get)
    gp.set_tuning(gp.GPC_TUNE_BLOCK, best)
    rec = {"best": best, "ms": {str(k): v for k, v in times.items()}, "when": time.time()}
    db[key] = rec
    _store(db)
    return rec


def apply_cached() -> dict:
    """Apply every cached choice for this device without timing anything."""
    db = _load()
    dev = _device_key()
    applied = {}
    for key, rec in db.items():
        if not key.startswith(dev + "/"):
            continue
        if "/fp64_block/" in key:
            gp.set_tuning(gp.GPC_TUNE_BLOCK, rec["best"])
            applied["fp64_block"] = rec["best"]
    return applied


if __name__ == "__main__":
    print(tune_fp64_block(force=True))
    sizes = W.batch_sizes(512, 64, 1024, seed=0)
    b = gp.Batch(sizes)
    rows = int(np.sum(sizes))
    X = torch.randn(rows, 4, dtype=torch.float64, device="cuda")
    y = torch.randn(rows, dtype=torch.float64, device="cuda")
    hyp = torch.tensor([[1.0, 1.0, 0.1]] * len(sizes), dtype=torch.float64)
    print(tune_batch_block(b, X, y, hyp, force=True))
    bm = gp.Batch(sizes, precision="mixed")
    print(tune_batch_block(bm, X, y, hyp, force=True))
