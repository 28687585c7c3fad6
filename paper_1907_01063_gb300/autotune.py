"""Autotuner for the library's tuning knobs.

Times the candidate values of each knob on the device at hand and keeps the
fastest; results are cached per device name and workload shape in a JSON
file (``GPCHOL_TUNE_CACHE``, default ``~/.cache/gpchol/tune.json``) so later
runs apply them without timing again.

Offline (``tune_*``: dedicated timing runs, cached) and online
(``OnlineTuner``: the caller's own repeated calls are the timing runs).

Knobs:
  * batch_block: block size inside the batched per-GP pass (32 or 64), timed
    on a batch of GPs with the caller's size mix, separately per precision.
  * fp64_block: block size of the FP64 blocked factorisation and adjoint
    (64, 96 or 128), timed on chol + adjoint at a stand-in order.
  * the mixed schedule (tune_mixed): the update depth D -- the tcgen05
    trailing and background products take K = 128 D per read-modify-write of
    their double-float output tiles (D in 1, 2, 4, 6, 8) -- and the SMs the
    background products leave to the FP64 chain in the factorisation (2, 4,
    8) and in the adjoint (8, 16, 24); the slice chunk (the K tile of one
    exponent group) stays 128.
  * the FP64 schedule (tune_fp64): the block size above together with the
    minimum K per split of the split-K products (the K tile of a partial
    product: 32, 64, 128) and the output tile of the FP64 products (single
    products up to a size limit take 32 x 32 tiles, the rest 64 x 64; the
    limit is searched over 256, 0 (always 64 x 64), 128 and 512).
Schedules with several knobs are searched coordinate by coordinate
(coordinate_search): each knob in turn over its candidates with the others
held at their best so far.  Cache keys carry the device, the precision and the
order rounded up to a power of two between 1024 and 16384 (n_bucket).
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

        times[b] = _time(run, reps=1 if n >= 8192 else 2)  # one FP64 pass at n = 16384 is seconds
    best = min(times, key=times.get)
    gp.set_tuning(gp.GPC_TUNE_BLOCK, best)
    rec = {"best": best, "ms": {str(k): v for k, v in times.items()}, "when": time.time()}
    db[key] = rec
    _store(db)
    return rec


def n_bucket(n: int) -> int:
    """The order a tuning result is keyed and timed at: n rounded up to a power
    of two, clamped to [1024, 16384]."""
    b = 1024
    while b < n and b < 16384:
        b *= 2
    return b


def coordinate_search(knobs, measure, start=None) -> dict:
    """Coordinate search over knob values.

    knobs: list of (name, candidates); measure(config: dict) -> ms.  Starting
    from ``start`` (default: every knob's first candidate), each knob in turn
    is set to each of its candidates with the other knobs fixed at their best
    so far, and keeps the fastest (ties: the earlier candidate).  Returns
    {"best": config, "ms": {description: ms}} with every configuration timed."""
    best = dict(start) if start else {name: cands[0] for name, cands in knobs}
    times = {}

    def key(cfg):
        return ",".join(f"{k}={cfg[k]}" for k, _ in knobs)

    for name, cands in knobs:
        scores = []
        for c in cands:
            cfg = dict(best, **{name: c})
            k = key(cfg)
            if k not in times:
                times[k] = float(measure(cfg))
            scores.append((times[k], c))
        best[name] = min(scores, key=lambda sc: sc[0])[1]
    return {"best": best, "ms": times}


_MIXED_KNOBS = [("mixed_defer", (6, 1, 2, 4, 8)), ("mixed_free_sms", (2, 4, 8)),
                ("mixed_adj_free_sms", (16, 8, 24))]
_FP64_KNOBS = [("fp64_block", (128, 64, 96)), ("splitk_min", (32, 64, 128)),
               ("f64_small_tile", (256, 0, 128, 512))]
_KNOB_IDS = {"mixed_defer": gp.GPC_TUNE_MIXED_DEFER, "mixed_free_sms": gp.GPC_TUNE_MIXED_FREE_SMS,
             "mixed_adj_free_sms": gp.GPC_TUNE_MIXED_ADJ_FREE_SMS, "fp64_block": gp.GPC_TUNE_BLOCK,
             "splitk_min": gp.GPC_TUNE_SPLITK_MIN, "f64_small_tile": gp.GPC_TUNE_F64_SMALL_TILE}


def _apply(cfg: dict):
    for name, value in cfg.items():
        gp.set_tuning(_KNOB_IDS[name], int(value))


def _chol_adjoint_stand_in(n: int):
    """An SE covariance of order n (built by the library) and a random lower L-bar."""
    X = torch.as_tensor(W.gp_inputs(n, 16, seed=0), device="cuda")
    K = gp.se_cov(X, 1.0, 4.0, 0.3, 1e-6)
    g = torch.Generator(device="cuda").manual_seed(1)
    return K, torch.tril(torch.randn(n, n, dtype=torch.float64, device="cuda", generator=g))


def _tune_schedule(kind: str, precision: str, knobs, n: int, force: bool) -> dict:
    nb = n_bucket(n)
    key = f"{_device_key()}/{kind}/{nb}"
    db = _load()
    if key in db and not force:
        _apply(db[key]["best"])
        return db[key]
    K, Lbar = _chol_adjoint_stand_in(nb)
    saved = {name: gp.get_tuning(_KNOB_IDS[name]) for name, _ in knobs}
    ws_cache = {}

    def measure(cfg):
        _apply(cfg)
        size = gp.workspace_size(nb, precision)
        if size not in ws_cache:
            ws_cache.clear()
            torch.cuda.empty_cache()
            ws_cache[size] = gp.workspace(nb, precision)
        ws = ws_cache[size]
        L = torch.empty_like(K)

        def run():
            gp.chol(K, precision, out=L, ws=ws, check=False)
            gp.chol_adjoint(L, Lbar, precision=precision, ws=ws)

        return _time(run)

    try:
        res = coordinate_search(knobs, measure, start=saved)
    finally:
        _apply(saved)
    _apply(res["best"])
    rec = {"best": res["best"], "ms": res["ms"], "n": nb, "when": time.time()}
    db[key] = rec
    _store(db)
    return rec


def tune_mixed(n: int = 16384, force: bool = False) -> dict:
    """Tune the mixed schedule (update depth D, free SMs of the factorisation
    and of the adjoint) on chol + adjoint at n_bucket(n); applies the result."""
    return _tune_schedule("mixed", "mixed", _MIXED_KNOBS, n, force)


def tune_fp64(n: int = 4096, force: bool = False) -> dict:
    """Tune the FP64 schedule (block size, split-K minimum K per split) on
    chol + adjoint at n_bucket(n); applies the result."""
    return _tune_schedule("fp64", "fp64", _FP64_KNOBS, n, force)


class _EventTimer:
    """CUDA-event pairs on the current stream; read back only when asked."""

    def start(self):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        return (e0, e1)

    def stop(self, token):
        token[1].record()

    def elapsed_ms(self, token) -> float:
        token[1].synchronize()
        return token[0].elapsed_time(token[1])


class OnlineTuner:
    """Online tuning across repeated calls (Section 5): an MCMC or optimisation
    loop calls the same primitive with the same input sizes every iteration, so
    the calls themselves serve as the timing runs.

    For each key (the caller's description of the call and its sizes) the
    first ``len(candidates) * reps`` calls run with the candidate values of
    ``knob`` in turn, each bracketed by a timer pair on the caller's stream
    (no synchronisation while exploring).  At the next call the times are read
    back once, the candidate with the smallest mean is kept (ties: the earlier
    candidate), and every later call of that key runs with it untimed.  The
    knob is set before each call and restored right after it is enqueued (the
    library reads it at enqueue time), so other code sees no change.

    ``setter``/``getter`` default to ``gp.set_tuning``/``gp.get_tuning`` and
    ``timer`` to CUDA events; tests pass fakes.  A knob that changes workspace
    sizes (the FP64 block does) needs ``fn`` to size its own workspace.
    """

    def __init__(self, knob: int, candidates, reps: int = 1, timer=None, setter=None, getter=None):
        if not candidates or reps < 1:
            raise ValueError("need at least one candidate and one repetition")
        self.knob = knob
        self.candidates = list(candidates)
        self.reps = int(reps)
        self._timer = timer if timer is not None else _EventTimer()
        self._set = setter if setter is not None else gp.set_tuning
        self._get = getter if getter is not None else gp.get_tuning
        self._state = {}  # key -> {"samples": [(candidate index, token)], "best": value or None, "ms": {}}

    def _schedule(self, i: int) -> int:
        return i // self.reps

    def _decide(self, st: dict):
        sums, counts = {}, {}
        for ci, tok in st["samples"]:
            ms = self._timer.elapsed_ms(tok)
            sums[ci] = sums.get(ci, 0.0) + ms
            counts[ci] = counts.get(ci, 0) + 1
        means = {ci: sums[ci] / counts[ci] for ci in sums}
        best = min(sorted(means), key=lambda ci: means[ci])
        st["best"] = self.candidates[best]
        st["ms"] = {self.candidates[ci]: m for ci, m in means.items()}
        st["samples"] = []

    def __call__(self, key, fn):
        st = self._state.setdefault(key, {"samples": [], "best": None, "ms": {}, "calls": 0})
        explore = len(self.candidates) * self.reps
        if st["best"] is None and st["calls"] >= explore:
            self._decide(st)
        old = self._get(self.knob)
        if st["best"] is not None:
            value, tok = st["best"], None
        else:
            ci = self._schedule(st["calls"])
            value = self.candidates[ci]
        try:
            self._set(self.knob, value)
            if st["best"] is None:
                tok = self._timer.start()
                out = fn()
                self._timer.stop(tok)
                st["samples"].append((ci, tok))
            else:
                out = fn()
        finally:
            self._set(self.knob, old)
        st["calls"] += 1
        return out

    def best(self, key):
        """The value chosen for key (None while still exploring)."""
        st = self._state.get(key)
        if st is None:
            return None
        if st["best"] is None and st["calls"] >= len(self.candidates) * self.reps:
            self._decide(st)
        return st["best"]

    def times(self, key) -> dict:
        """Mean milliseconds per candidate for key, once decided."""
        self.best(key)
        return dict(self._state.get(key, {}).get("ms", {}))


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
        elif "/mixed/" in key or "/fp64/" in key:
            _apply(rec["best"])
            applied.update(rec["best"])
    return applied


if __name__ == "__main__":
    print(tune_fp64_block(force=True))
    print(tune_mixed(16384, force=True))
    sizes = W.batch_sizes(512, 64, 1024, seed=0)
    b = gp.Batch(sizes)
    rows = int(np.sum(sizes))
    X = torch.randn(rows, 4, dtype=torch.float64, device="cuda")
    y = torch.randn(rows, dtype=torch.float64, device="cuda")
    hyp = torch.tensor([[1.0, 1.0, 0.1]] * len(sizes), dtype=torch.float64)
    print(tune_batch_block(b, X, y, hyp, force=True))
    bm = gp.Batch(sizes, precision="mixed")
    print(tune_batch_block(bm, X, y, hyp, force=True))
