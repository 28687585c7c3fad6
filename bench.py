#!/usr/bin/env python
"""Benchmark of the GP-likelihood hot path on GB300.

One step = one full pass of the path on resident inputs: squared-exponential
covariance K (n x n) from X (n x d), Cholesky factor L, the two triangular
solves, log det and log marginal likelihood, the upstream adjoint Lbar, the
blocked Cholesky adjoint Kbar, and the hyperparameter gradient.  The metric is
chol+adjoint GFLOP/s: (n^3/3 + the adjoint's counted flops) per step divided
by the step's device time (the covariance, solves and gradient kernels are
inside the timed step but add no counted flops).

Workload (default): n = 16384, d = 16, X ~ N(0, 1), alpha = 1, rho = 4 and
sigma^2 = lambda_max(K^f) / 1e5 (condition number about 1e5), targets from an
approximate GP draw.  K, L and Kbar are 2 GiB each, far larger than L2, so no
L2 flush is needed between steps.

The same JSON line also carries:
  * the FP64 path's step beside the mixed headline (mixed_vs_fp64);
  * the batched workload: 512 GPs per GPU, one persistent launch, dealt to the ranks by n^3;
  * `tri`: the triangular inverse and the triangular solve's reverse mode at the same n;
  * `gemm_glm`: the FP64 GEMM and its reverse mode, and the fused Bernoulli-logit GLM likelihood;
  * `mixed_product_alone`: the split-BF16 tcgen05 product by itself at K = 128, 768 and 1024
    (the kernel's own fraction of the sustained BF16 peak, beside the step-averaged `roofline`);
  * the oracle (`cpu_baseline`) and the multi-core CPU baseline (`cpu_parallel_baseline`) on a
    leading block of the workload;
  * `fp64_vs_oracle` and `mixed_vs_oracle`: each path's L, Kbar, alpha, log det, LML and
    gradient against the oracle's pass on the whole workload, computed after every timed
    leg (--no-oracle-parity skips it).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank runs an independent replica on its own GPU
(replicas only: one dense factorisation is not sharded).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "chol+adjoint GFLOP/s and % tensor peak at n=16384; mixed vs FP64 at LML rel err ≤1e-8"
COND_FILE = os.path.join(ROOT, "tests", "golden", "cond_sigma.json")


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--d", type=int, default=16)
    p.add_argument("--precision", choices=["fp64", "mixed", "both"], default="both",
                   help="both: time the FP64 and the mixed path; the headline is the mixed path")
    p.add_argument("--block", type=int, default=0, help="block size b (0: library default)")
    p.add_argument("--e2e-steps", type=int, default=2)
    p.add_argument("--trace-steps", type=int, default=2,
                   help="steps repeated with per-launch events for the roofline")
    p.add_argument("--cpu-sample", type=int, default=3072,
                   help="order of the leading block the oracle factors for cpu_baseline")
    p.add_argument("--ref-sample", type=int, default=2048,
                   help="order of the leading block one reference step factors")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-oracle-parity", action="store_true",
                   help="skip the comparison of both paths' results with the oracle's pass at the full size "
                        "(about two minutes of host work after every timed leg)")
    p.add_argument("--no-batched", action="store_true", help="skip the batched-GP workload")
    p.add_argument("--batch", type=int, default=512)
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--no-graph", action="store_true", help="time direct launches instead of a CUDA graph replay")
    p.add_argument("--no-tri", action="store_true", help="skip the triangular inverse / solve-adjoint leg")
    p.add_argument("--tri-m", type=int, default=1024, help="right-hand-side columns of the solve-adjoint leg")
    p.add_argument("--tri-reps", type=int, default=2)
    p.add_argument("--no-gemm-glm", action="store_true", help="skip the GEMM and GLM legs")
    p.add_argument("--no-product-alone", action="store_true",
                   help="skip timing the split-BF16 product by itself")
    p.add_argument("--glm-n", type=int, default=1 << 20)
    p.add_argument("--glm-k", type=int, default=512)
    return p.parse_args()


# ---------------------------------------------------------------- flop counts
def chol_flops(n: int) -> float:
    return n ** 3 / 3.0


def adjoint_flops(n: int, b: int) -> float:
    """Counted flops of the blocked adjoint sweep: panel solve m b^2, GEMM 2mnk,
    lower-only Cbar^T C m b^2, diagonal-block work (4/3) b^3, Rbar update
    2 b j (m + b)."""
    total = 0.0
    k = n
    while k > 0:
        j = max(0, k - b)
        nb = k - j
        m = n - k
        total += m * nb * nb          # Cbar <- Cbar D^{-1}
        total += 2.0 * m * j * nb     # Bbar -= Cbar R
        total += m * nb * nb          # Dbar -= Cbar^T C (lower)
        total += 4.0 / 3.0 * nb ** 3  # diagonal block
        total += 2.0 * nb * j * (m + nb)  # Rbar -= Cbar^T B + Dbar R
        k -= b
    return total


# ---------------------------------------------------------------- workload
def workload(n: int, d: int):
    from paper_1907_01063_gb300 import workloads as W
    alpha, rho = 1.0, 4.0
    sigma = None
    if os.path.exists(COND_FILE):
        rec = json.load(open(COND_FILE))
        if rec.get("n") == n and rec.get("d") == d:
            sigma = rec["sigma"]
    if sigma is None:
        # Other sizes: the same recipe's lambda_max scales about linearly in n.
        rec = json.load(open(COND_FILE))
        sigma = math.sqrt(rec["lambda_max"] * n / rec["n"] / rec["target_cond"])
    X = W.gp_inputs(n, d, seed=0)
    y = W.gp_targets(X, alpha, rho, sigma, seed=1)
    return X, y, (alpha, rho, sigma), 0.0


def describe(n, d, hyp, b, precision, cuda_graph=None):
    out = {"workload": f"GP LML + gradient, SE kernel, n={n}, d={d}, cond~1e5 ({precision})",
           "n": n, "d": d, "alpha": hyp[0], "rho": hyp[1], "sigma": round(hyp[2], 6),
           "block": b, "precision": precision,
           "l2": "inputs larger than L2 (K, L, Kbar are 8 n^2 bytes each)",
           "parallelism": "replicas"}
    if cuda_graph is not None:
        out["timed"] = "one step captured in a CUDA graph, replayed per step" if cuda_graph else "direct launches"
    return out


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(self.index)],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle timing
def oracle_sample(ns: int, d: int, hyp):
    """Unblocked oracle chol + adjoint on the leading ns x ns block (its own
    SE covariance of the first ns points); returns (seconds, counted flops)."""
    from oracle import oracle as O
    from paper_1907_01063_gb300 import workloads as W
    X = W.gp_inputs(ns, d, seed=0)
    K = O.se_cov(X, hyp[0], hyp[1], hyp[2], 0.0)
    Lbar = W.random_lower(ns, seed=2)
    t0 = time.perf_counter()
    L = O.chol(K)
    O.chol_adjoint(L, Lbar)
    dt = time.perf_counter() - t0
    return dt, chol_flops(ns) + 2.0 * ns ** 3 / 3.0


def cpu_baseline(ns: int, d: int, hyp):
    dt, fl = oracle_sample(ns, d, hyp)
    return {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": (f"single-threaded unblocked FP64 oracle: Cholesky-Banachiewicz + unblocked "
                       f"reverse-mode adjoint of the leading {ns}x{ns} block of the workload "
                       f"(flops n^3/3 + 2n^3/3), {dt:.1f} s on {os.cpu_count()} host cores available")}


def cpu_parallel_baseline(ns: int, d: int, hyp):
    """The same unblocked chol + reverse mode in column order with OpenMP over
    the rows of each column, on all host cores, on the same leading ns x ns
    block.  Reported beside the oracle; unavailable (not an error) where its
    OpenMP build failed."""
    try:
        from oracle import oracle as O
        from paper_1907_01063_gb300 import workloads as W
        threads = O.cpu_threads()
        X = W.gp_inputs(ns, d, seed=0)
        K = O.se_cov(X, hyp[0], hyp[1], hyp[2], 0.0)
        Lbar = W.random_lower(ns, seed=2)
        t0 = time.perf_counter()
        L = O.cpu_chol(K)
        O.cpu_chol_adjoint(L, Lbar)
        dt = time.perf_counter() - t0
    except Exception as exc:  # noqa: BLE001 - reported in the JSON line instead
        return {"unavailable": f"{type(exc).__name__}: {exc}"}
    fl = chol_flops(ns) + 2.0 * ns ** 3 / 3.0
    return {"value": fl / dt / 1e9, "unit": "GFLOP/s", "cores": threads, "kind": "multi-core CPU baseline",
            "sample": (f"unblocked FP64 Cholesky + reverse mode in column order, OpenMP over the rows of each "
                       f"column, leading {ns}x{ns} block of the workload (flops n^3/3 + 2n^3/3), {dt:.2f} s")}


def oracle_parity_legs(results, X, y, hyp, jitter):
    """Each path's L, K-bar, alpha, log det, LML value and hyperparameter
    gradient against the oracle's pass on the same workload (the oracle's
    O(n^3) steps by the multi-core routines whose factor is bitwise the
    oracle's; tests/test_cpu_baseline.py).  Run after every timed leg."""
    import numpy as np
    from oracle import oracle as O
    t0 = time.perf_counter()
    ref = O.gp_lml_and_grad_multicore(X, y, hyp[0], hyp[1], hyp[2], jitter)
    dt = time.perf_counter() - t0

    def frob(a, b):
        return float(np.linalg.norm(a - b) / np.linalg.norm(b))

    out = {}
    for prec, res in results.items():
        h = res.pop("host", None)
        if h is None:
            continue
        out[f"{prec}_vs_oracle"] = {
            "L_rel_frob": frob(h["L"], ref["L"]), "Kbar_rel_frob": frob(h["Kbar"], ref["Kbar"]),
            "alpha_rel": frob(h["alpha"], ref["alpha"]),
            "logdet_rel_err": abs(h["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
            "lml_rel_err": abs(h["value"] - ref["value"]) / abs(ref["value"]),
            "grad_rel_err": frob(h["grad"], ref["grad"]),
            "oracle": (f"oracle pass on the host ({O.cpu_threads()} threads for the two O(n^3) steps, "
                       f"{dt:.0f} s)")}
        out[f"{prec}_vs_oracle"]["meets_lml_1e-8"] = out[f"{prec}_vs_oracle"]["lml_rel_err"] <= 1e-8
    return out


# ---------------------------------------------------------------- distributed
def make_sync(world, device):
    """Barrier and max-over-ranks around the timed regions: NCCL between GPU
    ranks in the benchmark, gloo between CPU ranks in the tests."""
    import torch
    import torch.distributed as dist

    def barrier():
        if device.type == "cuda":
            torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    def max_over_ranks(v):
        if world == 1:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    return barrier, max_over_ranks


def whole_job_rate(world, steps, units_per_step, t_ms):
    """Units per second over all ranks: every rank processes its own copy of
    the workload (replicas), and the slowest rank's time counts."""
    return world * steps * units_per_step / (t_ms / 1e3)


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    if rank != 0:
        return
    n, d = args.n, args.d
    _, _, hyp, _ = workload(n, d)
    ns = args.ref_sample
    for _ in range(args.warmup):
        oracle_sample(ns, d, hyp)
    times, flops = [], 0.0
    for _ in range(args.steps):
        dt, fl = oracle_sample(ns, d, hyp)
        times.append(dt)
        flops += fl
    total = sum(times)
    value = flops / total / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": describe(n, d, hyp, 0, "fp64"),
        "cpu_baseline": {"value": value, "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                         "sample": (f"each step: single-threaded unblocked FP64 oracle chol + "
                                    f"adjoint of the leading {ns}x{ns} block of the workload")},
        "e2e": {"value": value, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def batched_sizes(batch: int, seed: int = 0) -> list[int]:
    from paper_1907_01063_gb300 import workloads as W
    return [int(v) for v in W.batch_sizes(batch, 64, 1024, seed=seed)]


def batched_workload(batch: int, d: int = 4, seed: int = 0, sigma: float = 0.1, indices=None):
    """A batch of GPs with n_i ~ U{64..1024}, X ~ N(0, 1) in d = 4, rho_i ~ U(0.2, 2),
    alpha = 1, sigma = 0.1; targets from an approximate GP draw.  Every GP has its
    own seeds, so ``indices`` (a rank's share) generates just those GPs."""
    from paper_1907_01063_gb300 import workloads as W
    import numpy as np
    sizes_all = batched_sizes(batch, seed)
    rho_all = W.batch_lengthscales(batch, 0.2, 2.0, seed=seed + 1)
    idx = list(range(batch)) if indices is None else list(indices)
    Xs, ys = [], []
    for i in idx:
        X = W.gp_inputs(sizes_all[i], d, seed=1000 + i)
        Xs.append(X)
        ys.append(W.gp_targets(X, 1.0, float(rho_all[i]), sigma, seed=2000 + i, features=256))
    hyp = np.stack([np.ones(len(idx)), rho_all[idx], np.full(len(idx), sigma)], axis=1)
    return [sizes_all[i] for i in idx], np.concatenate(Xs), np.concatenate(ys), hyp


def run_batched(args, gp, dev, stream, barrier, max_over_ranks, world, rank, tuned, prec):
    """The batched workload, sharded: with N ranks the job is N x batch GPs, dealt
    to the ranks by cost (shard.partition_by_cost), so each rank has about one
    batch of work (weak scaling); per-GP results are gathered once after the
    timed region.  With one rank the shard is the whole batch."""
    import torch
    from paper_1907_01063_gb300 import shard
    total = args.batch * world
    sizes_all = batched_sizes(total)
    mine = shard.partition_by_cost(sizes_all, world)[rank]
    sizes, X, y, hyp = batched_workload(total, indices=mine)
    b = gp.Batch(sizes, device=dev, precision=prec)
    Xd = torch.as_tensor(X, device=dev).contiguous()
    yd = torch.as_tensor(y, device=dev).contiguous()
    hd = torch.as_tensor(hyp, device=dev).contiguous()
    if not args.no_autotune:
        from paper_1907_01063_gb300 import autotune
        tuned[f"batch_block_{prec}"] = autotune.tune_batch_block(b, Xd, yd, hd)["best"]
    nb = gp.get_tuning(gp.GPC_TUNE_BATCH_BLOCK)
    flops_all = sum(chol_flops(n) + adjoint_flops(n, nb) for n in sizes_all)
    # one persistent launch per step, captured once in a CUDA graph and replayed
    gp.batched_gp_lml_grad(b, Xd, yd, hd)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gp.batched_gp_lml_grad(b, Xd, yd, hd)
    for _ in range(args.warmup):
        graph.replay()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        graph.replay()
    e1.record(stream)
    barrier()
    t_ms = max_over_ranks(e0.elapsed_time(e1))
    values, _ = shard.gather_results(mine, b.value, b.grad3, total, world, device=dev)
    info_ok = torch.tensor([float((b.info[:, 1] == 0).all().item())], dtype=torch.float64, device=dev)
    all_ok = max_over_ranks(-info_ok.item()) <= -1.0  # every rank's GPs finished
    rate = args.steps / (t_ms / 1e3)
    return {"workload": f"{total} GPs ({args.batch} per GPU, dealt by n^3), n_i ~ U{{64..1024}}, d=4, SE kernel, "
                        f"rho_i ~ U(0.2,2), sigma=0.1 ({prec})",
            "value": rate * flops_all / 1e9, "unit": "GFLOP/s",
            "gp_per_s": rate * total, "ms_per_step": t_ms / args.steps,
            "flops_per_step": flops_all, "gps": total, "gps_this_rank": len(mine),
            "sum_n": int(sum(sizes_all)), "max_n": int(max(sizes_all)),
            "cuda_graph": True, "kernels_per_step": 2, "block": nb, "sharding": "by n^3, no collective in the step",
            "all_ok": bool(all_ok),
            "value_checksum": float(values.double().sum().item()),
            "_values": values.cpu().numpy()}


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import torch.distributed as dist

    import paper_1907_01063_gb300 as gp

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    if args.block:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, args.block)
    n, d = args.n, args.d
    X, y, hyp, jitter = workload(n, d)
    a, r, s = hyp
    precisions = ["fp64", "mixed"] if args.precision == "both" else [args.precision]

    Xd = torch.as_tensor(X, device=dev)
    yd = torch.as_tensor(y, device=dev)
    K = torch.empty(n, n, dtype=torch.float64, device=dev)
    L = torch.empty_like(K)
    Kbar = torch.empty_like(K)
    ws = gp.workspace(n, "mixed" if "mixed" in precisions else "fp64", dev)
    hws = torch.empty(gp.se_hyper_grad_workspace_size(n), dtype=torch.uint8, device=dev)
    info = gp.new_info(dev)
    g3 = torch.empty(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    barrier, max_over_ranks = make_sync(world, dev)
    oracle_parity = not args.no_oracle_parity and rank == 0 and n <= 16384

    def run(prec):
        b = gp.get_tuning(gp.GPC_TUNE_BLOCK) if prec == "fp64" else 128
        step_flops = chol_flops(n) + adjoint_flops(n, b)

        def step(Xs, ys):
            gp.se_cov(Xs, a, r, s, jitter, out=K, precision=prec)
            res = gp.gp_lml(K, ys, prec, L=L, ws=ws, info=info, check=False)
            gp.gp_lml_grad(L, res["alpha"], 1.0, prec, out=Kbar, ws=ws)
            gp.se_hyper_grad(Xs, a, r, s, Kbar, ws=hws, out=g3, precision=prec)
            return res

        for _ in range(args.warmup):
            res = step(Xd, yd)
        barrier()
        gp.check_info(info, f"warm-up step ({prec})")
        launches0 = gp.launch_count()
        res = step(Xd, yd)
        launches_per_step = gp.launch_count() - launches0
        # One step captured once in a CUDA graph and replayed: the same kernels
        # with the same arguments, without the per-launch gaps of ~4000 small
        # launches (the library enqueues everything on the caller's stream and
        # joins its auxiliary stream back with events, so it captures whole).
        graph = None
        if not args.no_graph:
            try:
                side = torch.cuda.Stream()
                side.wait_stream(torch.cuda.current_stream())
                with torch.cuda.stream(side):
                    step(Xd, yd)
                torch.cuda.current_stream().wait_stream(side)
                torch.cuda.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph):
                    res = step(Xd, yd)
                graph.replay()
                torch.cuda.synchronize()
            except RuntimeError as exc:  # capture refused: time direct launches instead
                print(f"bench: CUDA graph capture failed ({exc}); timing direct launches", file=sys.stderr)
                graph = None
                res = step(Xd, yd)
        clocks = ClockSampler(local)
        clocks.start()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        for _ in range(args.steps):
            if graph is not None:
                graph.replay()
            else:
                res = step(Xd, yd)
        ev1.record(stream)
        barrier()
        launches = launches_per_step * args.steps
        t_ms = max_over_ranks(ev0.elapsed_time(ev1))
        # per-launch device times for the roofline: the same steps again with an
        # event pair around every launch (kept out of the region above because
        # ~3000 event pairs per mixed step add a few percent to its time)
        trace_steps = max(1, min(args.trace_steps, args.steps))
        gp.trace_enable(True)
        barrier()
        ev0.record(stream)
        for _ in range(trace_steps):
            step(Xd, yd)
        ev1.record(stream)
        barrier()
        traced_ms = ev0.elapsed_time(ev1) / trace_steps
        trace = gp.trace_summary()
        gp.trace_enable(False)
        clk = clocks.stop()
        st = info.tolist()
        if st[1] not in (gp.GPC_OK, gp.GPC_ERR_NO_CONVERGENCE):
            gp.check_info(info, f"timed step ({prec})")
        out = {"prec": prec, "block": b, "step_flops": step_flops, "t_ms": t_ms, "launches": launches,
               "cuda_graph": graph is not None,
               "trace": trace, "trace_steps": trace_steps, "traced_ms_per_step": traced_ms, "clocks": clk, "value": whole_job_rate(world, args.steps, step_flops, t_ms) / 1e9,
               "lml": res["value"].item(), "logdet": res["logdet"].item(), "grad": g3.tolist(),
               "refine_status": st[1]}
        # end to end: pinned host inputs in, scalars out, every step
        Xh = torch.as_tensor(X).pin_memory()
        yh = torch.as_tensor(y).pin_memory()
        out_h = torch.empty(4, dtype=torch.float64).pin_memory()
        Xe, ye = torch.empty_like(Xd), torch.empty_like(yd)
        e2e_steps = max(1, args.e2e_steps)
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(e2e_steps):
            Xe.copy_(Xh, non_blocking=True)
            ye.copy_(yh, non_blocking=True)
            res_e = step(Xe, ye)
            out_h[0:1].copy_(res_e["value"].reshape(1), non_blocking=True)
            out_h[1:4].copy_(g3, non_blocking=True)
        e1.record(stream)
        barrier()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1))
        out["e2e"] = {"value": whole_job_rate(world, e2e_steps, step_flops, e2e_ms) / 1e9, "unit": "GFLOP/s",
                      "h2d_bytes_per_step": Xh.numel() * 8 + yh.numel() * 8, "d2h_bytes_per_step": 32,
                      "ms_per_step": e2e_ms / e2e_steps}
        if oracle_parity:
            # the last step's outputs (same inputs every step), kept on the host
            # for the comparison with the oracle after every timed leg
            torch.cuda.synchronize()
            out["host"] = {"L": L.cpu().numpy(), "Kbar": Kbar.cpu().numpy(), "alpha": res_e["alpha"].cpu().numpy(),
                           "logdet": res_e["logdet"].item(), "value": res_e["value"].item(),
                           "grad": g3.cpu().numpy()}
        return out

    tuned = {}
    if not args.no_autotune:
        from paper_1907_01063_gb300 import autotune
        # FP64 schedule (block size, split-K minimum, small-product tile limit),
        # timed on chol + adjoint at the workload's order capped at 8192 (one
        # FP64 pass at 16384 takes seconds); the choice is applied
        rec64 = autotune.tune_fp64(min(n, 8192))
        tuned["fp64_block"] = rec64["best"]["fp64_block"]
        tuned["fp64_schedule"] = dict(rec64["best"], timed_at_n=rec64["n"])
        tuned["fp64_schedule_ms"] = rec64["ms"]
        if "mixed" in precisions:
            rec = autotune.tune_mixed(n)
            tuned["mixed_schedule"] = dict(rec["best"], timed_at_n=rec["n"],
                                           product_k_tile=128 * rec["best"]["mixed_defer"])
            tuned["mixed_schedule_ms"] = rec["ms"]
        # the tuned schedule may need a larger workspace (the group depths enter its size)
        need = gp.workspace_size(n, "mixed" if "mixed" in precisions else "fp64")
        if ws.numel() < need:
            del ws
            torch.cuda.empty_cache()
            ws = gp.workspace(n, "mixed" if "mixed" in precisions else "fp64", dev)

    results = {p_: run(p_) for p_ in precisions}

    def run_tri():
        """Section 3.2 at the headline size: the lower-triangular inverse of the
        step's Cholesky factor, and the reverse mode of C = L^{-1} B for an
        n x m right-hand side (Bbar = L^{-T} Cbar, Lbar = -tril(Bbar C^T)) from
        the kept inverse.  Inputs are resident and 2 GiB each (no L2 flush)."""
        m, reps = args.tri_m, max(1, args.tri_reps)
        prec0 = precisions[-1]
        gp.se_cov(Xd, a, r, s, jitter, out=K, precision=prec0)
        gp.chol(K, prec0, out=L, ws=ws, info=info)
        Linv, Lbar = Kbar, K
        g = torch.Generator(device="cpu")
        g.manual_seed(5)
        B = torch.randn(n, m, generator=g, dtype=torch.float64).to(dev)
        Cbar = torch.randn(n, m, generator=g, dtype=torch.float64).to(dev)
        C = torch.empty(n, m, dtype=torch.float64, device=dev)
        Bbar = torch.empty_like(C)

        def inverse():
            gp.tri_inverse(L, out=Linv)

        def adjoint():
            gp.tri_solve_adjoint(Linv, C, Cbar, Bbar=Bbar, Lbar=Lbar)

        gp.tri_solve(L, B, Linv=Linv, out=C)  # warm-up of the inverse, and C
        adjoint()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(fn):
            l0 = gp.launch_count()
            barrier()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            barrier()
            return max_over_ranks(e0.elapsed_time(e1)) / reps, (gp.launch_count() - l0) // reps

        inv_ms, inv_launches = timed(inverse)
        adj_ms, adj_launches = timed(adjoint)
        gp.trace_enable(True)
        inverse()
        torch.cuda.synchronize()
        trace = gp.trace_summary()
        gp.trace_enable(False)
        gm = trace.get("gemm_f64", {})
        inv_flops, adj_flops = n ** 3 / 3.0, 2.0 * n * n * m
        return {"n": n, "m": m, "reps": reps, "factor_precision": prec0,
                "inverse": {"ms": inv_ms, "gflops": inv_flops / (inv_ms / 1e3) / 1e9,
                            "flops": inv_flops, "launches": inv_launches,
                            "kernel_ms": {k: round(v["ms"], 3) for k, v in trace.items() if v["launches"]},
                            "gemm_f64_gflops": (gm["flops"] / (gm["ms"] / 1e3) / 1e9) if gm.get("ms") else None},
                "solve_adjoint": {"ms": adj_ms, "gflops": adj_flops / (adj_ms / 1e3) / 1e9,
                                  "flops": adj_flops, "launches": adj_launches}}

    def run_gemm_glm():
        """Section 3.1 and 3.4 legs: FP64 GEMM C = A B and its reverse mode on
        square 4096 matrices, a large-k product (128 x 128 output, k = 2^20,
        split over k), and the fused Bernoulli-logit GLM likelihood with its
        gradient on the logistic-regression toy data (one pass over X)."""
        from paper_1907_01063_gb300 import workloads as W
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def timed(fn, reps):
            fn()
            l0 = gp.launch_count()
            barrier()
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            barrier()
            return max_over_ranks(e0.elapsed_time(e1)) / reps, (gp.launch_count() - l0) // reps

        g = torch.Generator(device=dev)
        g.manual_seed(7)
        gws = gp.gemm_workspace(dev)
        out = {}
        s_ = 4096
        A = torch.randn(s_, s_, generator=g, dtype=torch.float64, device=dev)
        B = torch.randn(s_, s_, generator=g, dtype=torch.float64, device=dev)
        C = torch.empty_like(A)
        ms, la = timed(lambda: gp.gemm(A, B, out=C, ws=gws), 3)
        fl = 2.0 * s_ ** 3
        out["gemm_4096"] = {"ms": ms, "gflops": fl / (ms / 1e3) / 1e9, "frac_of_fp64_peak": None, "launches": la}
        ms, la = timed(lambda: gp.gemm_adjoint(A, B, C, ws=gws), 2)
        out["gemm_adjoint_4096"] = {"ms": ms, "gflops": 2 * fl / (ms / 1e3) / 1e9, "launches": la}
        del A, B, C
        kk = 1 << 20
        A = torch.randn(128, kk, generator=g, dtype=torch.float64, device=dev)
        B = torch.randn(kk, 128, generator=g, dtype=torch.float64, device=dev)
        C = torch.empty(128, 128, dtype=torch.float64, device=dev)
        ms, la = timed(lambda: gp.gemm(A, B, out=C, ws=gws), 3)
        out["gemm_128x128_k1M_splitk"] = {"ms": ms, "gflops": 2.0 * 128 * 128 * kk / (ms / 1e3) / 1e9, "launches": la}
        del A, B, C
        n_, k_ = args.glm_n, args.glm_k
        X, y = W.glm_data(n_, k_, "bernoulli_logit", seed=0)
        Xd, yd = torch.as_tensor(X, device=dev), torch.as_tensor(y, device=dev)
        del X, y
        beta = torch.zeros(k_, dtype=torch.float64, device=dev)
        beta[0], beta[1] = 3.0, -2.0
        gl_ws = gp.glm_workspace(k_, dev)
        r = gp.glm("bernoulli_logit", Xd, yd, 1.0, beta)
        ms, la = timed(lambda: gp.glm("bernoulli_logit", Xd, yd, 1.0, beta, ws=gl_ws), 20)
        byts = 8.0 * (n_ * k_ + 2 * n_ + 2 * k_)
        hbm = peaks.get("hbm_gbs", 6800.0)
        gp.trace_enable(True)
        gp.glm("bernoulli_logit", Xd, yd, 1.0, beta)
        torch.cuda.synchronize()
        tr = gp.trace_summary()
        gp.trace_enable(False)
        kern_ms = tr["glm"]["ms"]
        out["glm_bernoulli_logit"] = {
            "n": n_, "k": k_, "ms": ms, "launches": la, "bytes": byts, "gbs": byts / (ms / 1e3) / 1e9,
            "frac_of_hbm": byts / (ms / 1e3) / 1e9 / hbm, "glm_kernel_ms": kern_ms,
            "glm_kernel_frac_of_hbm": byts / (kern_ms / 1e3) / 1e9 / hbm if kern_ms else None,
            "lp": r["lp"].item(), "peak_source": "of measured: MEASURED_PEAKS hbm_gbs",
            "l2": "X is 8 n k bytes, larger than L2"}
        return out

    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}

    def run_product_isolated():
        """The split-BF16 tcgen05 product alone (no other kernel running), on an
        8192 x 8192 double-float output at three K depths: K = 128 reads and
        writes the output once per 128-wide chunk (the depth of the adjoint's
        B-bar updates), K = 768 is the factorisation's deferred depth.  Kernel
        time from the library's per-launch events; flops 30 M N K (15 slice
        products per FP64 multiply-add)."""
        g = torch.Generator(device=dev)
        g.manual_seed(11)
        out = {}
        sust = peaks.get("bf16_tflops_sustained")
        burst = peaks.get("bf16_tflops")
        for kk in (128, 768, 1024):
            A = torch.randn(8192, kk, generator=g, dtype=torch.float64, device=dev)
            B = torch.randn(8192, kk, generator=g, dtype=torch.float64, device=dev)
            gp.test_ozaki_gemm(A, B)
            torch.cuda.synchronize()
            gp.trace_enable(True)
            for _ in range(3):
                gp.test_ozaki_gemm(A, B)
            torch.cuda.synchronize()
            tr = gp.trace_summary()["gemm_mixed"]
            gp.trace_enable(False)
            tf = tr["flops"] / (tr["ms"] * 1e-3) / 1e12
            out[f"8192x8192xK{kk}"] = {"kernel_ms": tr["ms"] / tr["launches"], "tflops": tf,
                                         "frac_of_burst_bf16": tf / burst if burst else None,
                                         "frac_of_sustained_bf16": tf / sust if sust else None}
            del A, B
        out["peak_source"] = "of measured: bf16_tflops (burst) and bf16_tflops_sustained"
        return out

    product_alone = None
    if "mixed" in precisions and not args.no_product_alone and rank == 0:
        product_alone = run_product_isolated()
    extra = None
    if not args.no_gemm_glm:
        torch.cuda.nvtx.range_push("gemm_glm")
        extra = run_gemm_glm()
        torch.cuda.nvtx.range_pop()

    tri = None
    if not args.no_tri:
        torch.cuda.nvtx.range_push("tri")  # lets a profiler select this leg's launches
        tri = run_tri()
        torch.cuda.nvtx.range_pop()

    batched = None
    if not args.no_batched:
        batched = {}
        for bp in precisions:
            batched[bp] = run_batched(args, gp, dev, stream, barrier, max_over_ranks, world, rank, tuned, bp)
        vals = {bp: r.pop("_values") for bp, r in batched.items()}
        if "fp64" in vals and "mixed" in vals:
            import numpy as np
            batched["mixed"]["max_rel_value_diff_vs_fp64"] = float(
                np.max(np.abs(vals["mixed"] - vals["fp64"]) / np.maximum(1.0, np.abs(vals["fp64"]))))

    fp64_peak = gp.fp64_peak_gflops(dev)
    nominal_fp64 = peaks.get("bf16_tflops", 1900.0) * 1e3 * 1.25 / 2250.0

    # DRAM bytes per launch of the split product averaged over a step: no capture
    # of the current schedule (deferred K = 128 D updates) takes DRAM counters over
    # every launch of a full-size step, so the field is null; one launch's DRAM
    # traffic against its work is in profiles/ozaki_gemm_kernel_k128_vs_k768_n8192.md.
    ozaki_traffic = {}

    def roofline(res):
        trace = {k: dict(v, ms=v["ms"] / res["trace_steps"], flops=v["flops"] / res["trace_steps"],
                         bytes=v["bytes"] / res["trace_steps"], launches=v["launches"] / res["trace_steps"])
                 for k, v in res["trace"].items()}
        dom_name, dom = max(((k, v) for k, v in trace.items() if v["launches"]), key=lambda kv: kv[1]["ms"])
        avg = dom["ms"] / max(dom["launches"], 1)
        if dom_name == "gemm_mixed":
            peak = peaks.get("bf16_tflops_sustained", 1695.9)
            achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e12 if dom["ms"] else 0.0
            return {"kernel": "ozaki_gemm_kernel (tcgen05 BF16 slice products, 15 per FP64 product)",
                    "bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak, "traffic": ozaki_traffic.get(n), "launches_per_step": dom["launches"],
                    "avg_launch_ms": avg, "peak_source": "of measured: MEASURED_PEAKS bf16_tflops_sustained",
                    "traffic_note": "null: no per-launch DRAM capture of the current schedule at this size",
                    "fp64_equivalent_gflops": dom["flops"] / 15.0 / (dom["ms"] / 1e3) / 1e9}
        if dom_name in ("gemm_f64", "diag", "trsm"):
            achieved = dom["flops"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] else 0.0
            names = {"gemm_f64": "gemm_f64_kernel (FP64 mma.sync m16n8k16)",
                     "diag": "diagonal-block kernels (potrf_diag, trtri_batched)",
                     "trsm": "trsm_quad_kernel (FP64 panel solves)"}
            return {"kernel": names[dom_name],
                    "bound": "tensor" if dom_name == "gemm_f64" else "alu", "achieved": achieved, "peak": fp64_peak, "unit": "GFLOP/s",
                    "frac": achieved / fp64_peak, "traffic": None, "launches_per_step": dom["launches"],
                    "avg_launch_ms": avg,
                    "peak_source": "of measured: FP64 DMMA m16n8k16 issue rate measured in this run (gpc_fp64_peak)",
                    "peak_nominal_ratio": nominal_fp64}
        achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] else 0.0
        peak = peaks.get("hbm_gbs", 6800.0)
        return {"kernel": dom_name, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "launches_per_step": dom["launches"], "avg_launch_ms": avg,
                "peak_source": "of measured: MEASURED_PEAKS hbm_gbs"}

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    cpu = cpu_par = None
    if not args.no_cpu_baseline and world == 1:
        cpu = cpu_baseline(args.cpu_sample, d, hyp)
        cpu_par = cpu_parallel_baseline(args.cpu_sample, d, hyp)
    head = results["mixed"] if "mixed" in results else results["fp64"]
    prec = head["prec"]

    def kernel_ms(res):
        return {k: round(v["ms"] / res["trace_steps"], 3) for k, v in res["trace"].items() if v["launches"]}

    def summary(res):
        return {"value": res["value"], "unit": "GFLOP/s", "ms_per_step": res["t_ms"] / args.steps,
                "gpu_launches": res["launches"], "roofline": roofline(res), "e2e": res["e2e"],
                "lml": res["lml"], "logdet": res["logdet"], "grad": res["grad"], "clocks": res["clocks"],
                "kernel_ms_per_step": kernel_ms(res), "traced_ms_per_step": res["traced_ms_per_step"]}

    line = {
        "metric": METRIC, "value": head["value"], "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["t_ms"] / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16x5+f64" if prec == "mixed" else "f64", "data": "synthetic",
        "config": describe(n, d, hyp, head["block"], prec, head["cuda_graph"]),
        "e2e": head["e2e"],
        "gpu_launches": head["launches"],
        "roofline": roofline(head),
        "cpu_baseline": cpu,
        "cpu_parallel_baseline": cpu_par,
        "clocks": head["clocks"],
        "flops_per_step": head["step_flops"],
        "kernel_ms_per_step": kernel_ms(head),
        "traced_ms_per_step": head["traced_ms_per_step"],
    }
    if batched is not None:
        line["batched"] = batched
    if extra is not None:
        for key in ("gemm_4096", "gemm_adjoint_4096", "gemm_128x128_k1M_splitk"):
            extra[key]["frac_of_fp64_peak"] = extra[key]["gflops"] / fp64_peak
        gl = extra["glm_bernoulli_logit"]
        if gl["glm_kernel_ms"]:
            # two FP64 multiply-adds per element of X (eta, then X^T d): on GB300 the
            # FP64 pipe, not HBM, bounds the kernel
            gl["fp64_gflops"] = 4.0 * gl["n"] * gl["k"] / (gl["glm_kernel_ms"] / 1e3) / 1e9
            gl["frac_of_fp64_peak"] = gl["fp64_gflops"] / fp64_peak
            gl["bound"] = "alu (FP64)"
        line["gemm_glm"] = extra
    if product_alone is not None:
        line["mixed_product_alone"] = product_alone
    if tri is not None:
        for leg in ("inverse", "solve_adjoint"):
            tri[leg]["frac_of_fp64_peak"] = tri[leg]["gflops"] / fp64_peak
        tri["peak_source"] = "of measured: FP64 DMMA m16n8k16 issue rate measured in this run (gpc_fp64_peak)"
        line["tri"] = tri
    if tuned:
        line["tuned"] = tuned
    if "fp64" in results and "mixed" in results:
        f, m = results["fp64"], results["mixed"]
        gf, gm = f["grad"], m["grad"]
        line["fp64"] = summary(f)
        line["mixed"] = summary(m)
        line["mixed_vs_fp64"] = {
            "speedup": m["value"] / f["value"],
            "lml_rel_err": abs(m["lml"] - f["lml"]) / abs(f["lml"]),
            "logdet_rel_err": abs(m["logdet"] - f["logdet"]) / abs(f["logdet"]),
            "grad_rel_err": math.sqrt(sum((x - y_) ** 2 for x, y_ in zip(gm, gf)) / sum(y_ ** 2 for y_ in gf)),
            "meets_lml_1e-8": abs(m["lml"] - f["lml"]) / abs(f["lml"]) <= 1e-8,
            "refine_status": m["refine_status"],
        }
    else:
        line.update({"lml": head["lml"], "grad": head["grad"]})
    if oracle_parity:
        line.update(oracle_parity_legs(results, X, y, hyp, jitter))
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
