"""Sharding a batch of independent GPs over ranks (one GPU per rank).

A batch of GPs needs no exchange while it runs: each rank factors and
differentiates its own GPs in one persistent launch.  The GPs are dealt out
by cost, largest first, each to the rank with the least work so far
(longest-processing-time-first), cost n_i^3 (the factorisation plus the
adjoint are about n^3 flops); the per-GP results (value and the three
hyperparameter derivatives) are gathered once after the work.

Host-side logic only; the device work is ``batched_gp_lml_grad`` on each
rank's ``Batch``.
"""
from __future__ import annotations

import numpy as np


def partition_by_cost(sizes, world: int) -> list[list[int]]:
    """GP indices per rank, each list ascending.  Deterministic: ties in size
    keep index order, ties in load go to the lower rank."""
    if world < 1:
        raise ValueError("world must be >= 1")
    sizes = [int(v) for v in sizes]
    order = sorted(range(len(sizes)), key=lambda i: (-sizes[i], i))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(sizes[i]) ** 3
    return [sorted(p) for p in parts]


def row_offsets(sizes) -> np.ndarray:
    """First row of each GP in the packed X / y arrays (and the total at the end)."""
    return np.concatenate([[0], np.cumsum(np.asarray(sizes, dtype=np.int64))])


def take(indices, sizes, X: np.ndarray, y: np.ndarray, hyp: np.ndarray):
    """The packed arrays of the GPs in ``indices`` (in that order):
    (sizes, X rows, y, hyp rows)."""
    off = row_offsets(sizes)
    idx = list(indices)
    sub_sizes = [int(sizes[i]) for i in idx]
    rows = np.concatenate([np.arange(off[i], off[i + 1]) for i in idx]) if idx else np.zeros(0, dtype=np.int64)
    return sub_sizes, X[rows], y[rows], hyp[idx]


def gather_results(indices, value, grad3, total: int, world: int, device=None):
    """All ranks' per-GP results in global order: (value[total], grad3[total, 3]).

    ``indices`` are this rank's GP indices, ``value`` (len) and ``grad3``
    (len x 3) its results in that order.  One all_gather of an
    (index, value, g_alpha, g_rho, g_sigma) row per GP, padded to the largest
    share; with world == 1 nothing is communicated."""
    import torch
    import torch.distributed as dist

    value = torch.as_tensor(value, dtype=torch.float64, device=device).reshape(-1)
    grad3 = torch.as_tensor(grad3, dtype=torch.float64, device=device).reshape(-1, 3)
    idx = torch.as_tensor(list(indices), dtype=torch.float64, device=value.device).reshape(-1)
    rows = torch.cat([idx[:, None], value[:, None], grad3], dim=1)
    if world > 1:
        cnt = torch.tensor([rows.shape[0]], dtype=torch.int64, device=value.device)
        counts = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(counts, cnt)
        width = int(max(int(c.item()) for c in counts))
        pad = torch.full((width, 5), -1.0, dtype=torch.float64, device=value.device)
        pad[: rows.shape[0]] = rows
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad)
        rows = torch.cat(parts, dim=0)
    rows = rows[rows[:, 0] >= 0]
    out_v = torch.full((total,), float("nan"), dtype=torch.float64, device=value.device)
    out_g = torch.full((total, 3), float("nan"), dtype=torch.float64, device=value.device)
    pos = rows[:, 0].long()
    out_v[pos] = rows[:, 1]
    out_g[pos] = rows[:, 2:]
    return out_v, out_g
