"""Sharding a batch of GPs over ranks: the partition by cost, the slicing of
the packed arrays, and the one gather after the work, on CPU ranks (gloo,
world size 2).  The per-rank compute is the oracle standing in for the
device's batched launch, so the gathered results can be compared with a
single-process pass over the whole batch."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import oracle as O
from paper_1907_01063_gb300 import shard
from paper_1907_01063_gb300 import workloads as W


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_every_gp_once_and_balances_cost():
    sizes = [int(v) for v in W.batch_sizes(1024, 64, 1024, seed=0)]
    for world in (1, 2, 3, 8):
        parts = shard.partition_by_cost(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(float(sizes[i]) ** 3 for i in p) for p in parts]
        # longest-processing-time-first: the spread is at most the largest single cost
        assert max(loads) - min(loads) <= max(float(v) ** 3 for v in sizes)
        assert parts == shard.partition_by_cost(sizes, world)  # deterministic
    assert shard.partition_by_cost(sizes, 1) == [list(range(len(sizes)))]
    with pytest.raises(ValueError):
        shard.partition_by_cost(sizes, 0)


def test_partition_by_hand():
    # costs 27, 8, 8, 1 over two ranks: 3 -> r0; 2 -> r1; 2 -> r1 (8 < 27); 1 -> r1 (16 < 27)
    assert shard.partition_by_cost([3, 2, 2, 1], 2) == [[0], [1, 2, 3]]


def test_take_slices_the_packed_arrays():
    sizes = [3, 1, 4, 2]
    X = np.arange(10 * 2, dtype=float).reshape(10, 2)
    y = np.arange(10, dtype=float)
    hyp = np.arange(4 * 3, dtype=float).reshape(4, 3)
    s, Xs, ys, hs = shard.take([2, 0], sizes, X, y, hyp)
    assert s == [4, 3]
    assert np.array_equal(ys, np.array([4.0, 5, 6, 7, 0, 1, 2]))
    assert np.array_equal(Xs, X[[4, 5, 6, 7, 0, 1, 2]])
    assert np.array_equal(hs, hyp[[2, 0]])


def _problem(count=12, d=2):
    sizes = [int(v) for v in W.batch_sizes(count, 5, 40, seed=3)]
    rho = W.batch_lengthscales(count, 0.5, 2.0, seed=4)
    Xs, ys = [], []
    for i, n in enumerate(sizes):
        X = W.gp_inputs(n, d, seed=100 + i)
        Xs.append(X)
        ys.append(W.gp_targets(X, 1.0, float(rho[i]), 0.3, seed=200 + i, features=64))
    hyp = np.stack([np.ones(count), rho, np.full(count, 0.3)], axis=1)
    return sizes, np.concatenate(Xs), np.concatenate(ys), hyp


def _oracle_pass(sizes, X, y, hyp):
    off = shard.row_offsets(sizes)
    vals, grads = [], []
    for i in range(len(sizes)):
        r = O.gp_lml_and_grad(X[off[i]:off[i + 1]], y[off[i]:off[i + 1]], *hyp[i])
        vals.append(r["value"])
        grads.append(r["grad"])
    return np.array(vals), np.array(grads).reshape(-1, 3)


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes, X, y, hyp = _problem()
        mine = shard.partition_by_cost(sizes, world)[rank]
        s, Xs, ys, hs = shard.take(mine, sizes, X, y, hyp)
        v, g = _oracle_pass(s, Xs, ys, hs)
        allv, allg = shard.gather_results(mine, v, g, len(sizes), world)
        out[rank] = (mine, allv.numpy(), allg.numpy())
    finally:
        dist.destroy_process_group()


def test_two_ranks_gather_equals_one_pass():
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, free_port(), out), nprocs=world, join=True)
        res = dict(out)
    sizes, X, y, hyp = _problem()
    v0, g0 = _oracle_pass(sizes, X, y, hyp)
    assert sorted(res[0][0] + res[1][0]) == list(range(len(sizes)))
    assert res[0][0] and res[1][0]  # both ranks had work
    for r in range(world):
        assert np.array_equal(res[r][1], v0)  # same arithmetic per GP: bitwise equal
        assert np.array_equal(res[r][2], g0)


def test_gather_with_one_rank_needs_no_process_group():
    v, g = shard.gather_results([2, 0], [5.0, 7.0], [[1, 2, 3], [4, 5, 6]], 3, 1)
    assert v[0].item() == 7.0 and v[2].item() == 5.0 and torch.isnan(v[1])
    assert g[2].tolist() == [1.0, 2.0, 3.0]


def test_bench_batched_workload_by_index_equals_slicing_the_whole():
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    total = 10
    sizes, X, y, hyp = bench.batched_workload(total)
    assert sizes == bench.batched_sizes(total)
    for world in (2, 3):
        for rank, part in enumerate(shard.partition_by_cost(sizes, world)):
            s, Xs, ys, hs = bench.batched_workload(total, indices=part)
            s2, X2, y2, h2 = shard.take(part, sizes, X, y, hyp)
            assert s == s2
            assert np.array_equal(Xs, X2) and np.array_equal(ys, y2) and np.array_equal(hs, h2)
