"""Batched GPs in one persistent launch, against the CPU oracle per GP."""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


# Mixed path: split-BF16 products with double-float accumulation and FP64
# refinement of alpha; the value and gradient stay within 1e-9 / 1e-7
# (relative) of the FP64 oracle on these conditioning levels (sigma = 0.1, so
# cond(K) is at most about n / sigma^2 ~ 1e5).
MIXED_VALUE_TOL, MIXED_GRAD_TOL = 1e-9, 1e-7


def make_batch(sizes, d=4, seed=0, sigma=0.1):
    rho = W.batch_lengthscales(len(sizes), 0.2, 2.0, seed=seed + 1)
    Xs, ys, hyps = [], [], []
    for i, n in enumerate(sizes):
        X = W.gp_inputs(n, d, seed=1000 + i)
        y = W.gp_targets(X, 1.0, float(rho[i]), sigma, seed=2000 + i)
        Xs.append(X)
        ys.append(y)
        hyps.append((1.0, float(rho[i]), sigma))
    return Xs, ys, np.array(hyps)


def run_batch(sizes, Xs, ys, hyps, block=None, precision="fp64"):
    b = gp.Batch(sizes, precision=precision)
    X = torch.as_tensor(np.concatenate(Xs), device="cuda").contiguous()
    y = torch.as_tensor(np.concatenate(ys), device="cuda").contiguous()
    old = gp.get_tuning(gp.GPC_TUNE_BATCH_BLOCK)
    try:
        if block:
            gp.set_tuning(gp.GPC_TUNE_BATCH_BLOCK, block)
        v, g, info = gp.batched_gp_lml_grad(b, X, y, torch.as_tensor(hyps))
        torch.cuda.synchronize()
    finally:
        gp.set_tuning(gp.GPC_TUNE_BATCH_BLOCK, old)
    return b, v.cpu().numpy(), g.cpu().numpy(), info.cpu().numpy()


SIZES = [1, 5, 33, 64, 65, 100, 128, 129, 200, 257, 63, 3]


@pytest.mark.parametrize("block", [32, 64])
def test_batched_matches_oracle(block):
    Xs, ys, hyps = make_batch(SIZES, seed=block)
    b, v, g, info = run_batch(SIZES, Xs, ys, hyps, block)
    assert np.all(info[:, 1] == gp.GPC_OK)
    for i, n in enumerate(SIZES):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        assert abs(v[i] - ref["value"]) <= 1e-10 * max(1.0, abs(ref["value"])), (i, n)
        assert np.linalg.norm(g[i] - ref["grad"]) <= 1e-8 * np.linalg.norm(ref["grad"]), (i, n)
        if n in (65, 257):
            L = b.factor(i).cpu().numpy()
            assert np.linalg.norm(L - ref["L"]) <= 1e-10 * np.linalg.norm(ref["L"])


def test_batched_equals_single_gp_path():
    sizes = [300, 77, 513]
    Xs, ys, hyps = make_batch(sizes, seed=5)
    _, v, g, info = run_batch(sizes, Xs, ys, hyps)
    for i, n in enumerate(sizes):
        X = torch.as_tensor(Xs[i], device="cuda")
        h = torch.tensor(hyps[i], dtype=torch.float64, requires_grad=True)
        val = gp.gp_lml_value(X, torch.as_tensor(ys[i], device="cuda"), h, 0.0)
        val.backward()
        assert abs(v[i] - val.item()) <= 1e-11 * abs(val.item())
        assert np.linalg.norm(g[i] - h.grad.numpy()) <= 1e-9 * np.linalg.norm(h.grad.numpy())


def test_batched_failure_is_isolated():
    # one GP with a NaN noise level has a NaN diagonal: only it fails
    sizes = [40, 50, 60]
    Xs, ys, hyps = make_batch(sizes, seed=9)
    hyps[1, 2] = np.nan
    _, v, g, info = run_batch(sizes, Xs, ys, hyps)
    assert info[1, 1] in (gp.GPC_ERR_NOT_PD, gp.GPC_ERR_NAN)
    assert np.isnan(v[1])
    for i in (0, 2):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        assert info[i, 1] == gp.GPC_OK
        assert abs(v[i] - ref["value"]) <= 1e-10 * abs(ref["value"])


def test_batched_rejects_sizes_above_nmax_on_device():
    sizes = [10, 20]
    Xs, ys, hyps = make_batch(sizes, seed=3)
    b = gp.Batch(sizes)
    X = torch.as_tensor(np.concatenate(Xs), device="cuda").contiguous()
    y = torch.as_tensor(np.concatenate(ys), device="cuda").contiguous()
    hyp = torch.as_tensor(hyps, device="cuda").contiguous()
    st = gp.capi.gpc_batched_gp_lml_grad(2, 10, b.n.data_ptr(), b.offK.data_ptr(), b.rowX.data_ptr(), 4,
                                         X.data_ptr(), y.data_ptr(), hyp.data_ptr(), 0, b.K.data_ptr(),
                                         b.value.data_ptr(), b.grad3.data_ptr(), b.info.data_ptr(),
                                         b.ws.data_ptr(), b.ws.numel(), torch.cuda.current_stream().cuda_stream)
    assert st == gp.GPC_OK
    info = b.info.cpu().numpy()
    assert info[0, 1] == gp.GPC_OK and info[1, 1] == gp.GPC_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_config5_sample(precision):
    # the batch workload's size mix (n ~ U{64..1024}, d = 4, rho ~ U(0.2, 2)),
    # checked against the oracle on its three smallest and three largest
    # members (the largest take the most blocks of the per-GP sweep)
    sizes = list(W.batch_sizes(64, 64, 1024, seed=0))
    Xs, ys, hyps = make_batch(sizes, seed=0)
    _, v, g, info = run_batch(sizes, Xs, ys, hyps, precision=precision)
    assert np.all(info[:, 1] == gp.GPC_OK)
    vtol, gtol = (1e-10, 1e-8) if precision == "fp64" else (MIXED_VALUE_TOL, MIXED_GRAD_TOL)
    order = np.argsort(sizes)
    assert sizes[order[-1]] > 900
    for i in list(order[:3]) + list(order[-3:]):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        assert abs(v[i] - ref["value"]) <= vtol * max(1.0, abs(ref["value"])), (i, sizes[i])
        assert np.linalg.norm(g[i] - ref["grad"]) <= gtol * np.linalg.norm(ref["grad"]), (i, sizes[i])


def test_batched_graph_replay_matches_direct_call():
    sizes = [90, 17, 150, 64]
    Xs, ys, hyps = make_batch(sizes, seed=11)
    b = gp.Batch(sizes)
    X = torch.as_tensor(np.concatenate(Xs), device="cuda").contiguous()
    y = torch.as_tensor(np.concatenate(ys), device="cuda").contiguous()
    hyp = torch.as_tensor(hyps, device="cuda").contiguous()
    gp.batched_gp_lml_grad(b, X, y, hyp)
    torch.cuda.synchronize()
    v0, g0 = b.value.clone(), b.grad3.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gp.batched_gp_lml_grad(b, X, y, hyp)
    b.value.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.value, v0) and torch.equal(b.grad3, g0)


# ---------------------------------------------------------------- mixed path
# (tolerances MIXED_VALUE_TOL, MIXED_GRAD_TOL are defined at the top)


@pytest.mark.parametrize("block", [32, 64])
def test_batched_mixed_matches_oracle(block):
    Xs, ys, hyps = make_batch(SIZES, seed=block + 1)
    b, v, g, info = run_batch(SIZES, Xs, ys, hyps, block, precision="mixed")
    assert np.all(info[:, 1] == gp.GPC_OK)
    worst_v = worst_g = 0.0
    for i, n in enumerate(SIZES):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        ev = abs(v[i] - ref["value"]) / max(1.0, abs(ref["value"]))
        eg = np.linalg.norm(g[i] - ref["grad"]) / np.linalg.norm(ref["grad"])
        worst_v, worst_g = max(worst_v, ev), max(worst_g, eg)
        assert ev <= MIXED_VALUE_TOL, (i, n, ev)
        assert eg <= MIXED_GRAD_TOL, (i, n, eg)
        if n in (65, 257):
            L = b.factor(i).cpu().numpy()
            assert np.linalg.norm(L - ref["L"]) <= 1e-9 * np.linalg.norm(ref["L"])
            assert not np.any(np.triu(L, 1))
    print(f"batched mixed block {block}: value {worst_v:.3e} grad {worst_g:.3e}")


def test_batched_mixed_full_batch_against_fp64_and_oracle():
    # the full batch workload (512 GPs, n ~ U{64..1024}, d = 4) through both
    # precisions in the launch configuration the benchmark times; the oracle
    # checks the smallest and the largest members
    sizes = list(W.batch_sizes(512, 64, 1024, seed=0))
    Xs, ys, hyps = make_batch(sizes, seed=0)
    _, vf, gf, inf = run_batch(sizes, Xs, ys, hyps)
    _, vm, gm, inm = run_batch(sizes, Xs, ys, hyps, precision="mixed")
    assert np.all(inf[:, 1] == gp.GPC_OK) and np.all(inm[:, 1] == gp.GPC_OK)
    ev = np.abs(vm - vf) / np.maximum(1.0, np.abs(vf))
    eg = np.linalg.norm(gm - gf, axis=1) / np.linalg.norm(gf, axis=1)
    print(f"batched mixed vs fp64 (512 GPs): value {ev.max():.3e} grad {eg.max():.3e}")
    assert ev.max() <= MIXED_VALUE_TOL and eg.max() <= MIXED_GRAD_TOL
    order = np.argsort(sizes)
    for i in (order[0], order[-1]):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        assert abs(vf[i] - ref["value"]) <= 1e-10 * max(1.0, abs(ref["value"]))
        assert abs(vm[i] - ref["value"]) <= MIXED_VALUE_TOL * max(1.0, abs(ref["value"]))
        assert np.linalg.norm(gm[i] - ref["grad"]) <= MIXED_GRAD_TOL * np.linalg.norm(ref["grad"])


def test_batched_mixed_failure_is_isolated():
    sizes = [40, 50, 60]
    Xs, ys, hyps = make_batch(sizes, seed=9)
    hyps[1, 2] = np.nan
    _, v, g, info = run_batch(sizes, Xs, ys, hyps, precision="mixed")
    assert info[1, 1] in (gp.GPC_ERR_NOT_PD, gp.GPC_ERR_NAN)
    assert np.isnan(v[1])
    for i in (0, 2):
        ref = O.gp_lml_and_grad(Xs[i], ys[i], *hyps[i], 0.0)
        assert info[i, 1] == gp.GPC_OK
        assert abs(v[i] - ref["value"]) <= MIXED_VALUE_TOL * abs(ref["value"])


def test_batched_mixed_graph_replay_is_deterministic():
    sizes = [90, 17, 150, 64, 300]
    Xs, ys, hyps = make_batch(sizes, seed=12)
    b = gp.Batch(sizes, precision="mixed")
    X = torch.as_tensor(np.concatenate(Xs), device="cuda").contiguous()
    y = torch.as_tensor(np.concatenate(ys), device="cuda").contiguous()
    hyp = torch.as_tensor(hyps, device="cuda").contiguous()
    gp.batched_gp_lml_grad(b, X, y, hyp)
    torch.cuda.synchronize()
    v0, g0 = b.value.clone(), b.grad3.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        gp.batched_gp_lml_grad(b, X, y, hyp)
    b.value.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(b.value, v0) and torch.equal(b.grad3, g0)


def test_batched_fp64_workspace_refuses_mixed_run():
    sizes = [10, 20]
    b = gp.Batch(sizes)
    X = torch.zeros(30, 4, dtype=torch.float64, device="cuda")
    y = torch.zeros(30, dtype=torch.float64, device="cuda")
    with pytest.raises(gp.GpcholError):
        gp.batched_gp_lml_grad(b, X, y, torch.ones(2, 3, dtype=torch.float64), precision="mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batched_refuses_short_workspace(precision):
    import ctypes
    sizes = [10, 20]
    b = gp.Batch(sizes, precision=precision)
    X = torch.zeros(30, 4, dtype=torch.float64, device="cuda")
    y = torch.zeros(30, dtype=torch.float64, device="cuda")
    hyp = torch.ones(2, 3, dtype=torch.float64, device="cuda")
    code = gp.precision_code(precision)
    st = gp.capi.gpc_batched_gp_lml_grad(b.batch, b.nmax, b.n.data_ptr(), b.offK.data_ptr(), b.rowX.data_ptr(), 4,
                                         X.data_ptr(), y.data_ptr(), hyp.data_ptr(), code, b.K.data_ptr(),
                                         b.value.data_ptr(), b.grad3.data_ptr(), b.info.data_ptr(), b.ws.data_ptr(),
                                         b.ws.numel() - 1, None)
    assert st == gp.GPC_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sharded_batch_matches_whole_batch(precision):
    """The GPs of a batch run as three shards dealt by cost (one launch each,
    one after another on this GPU) give the whole batch's results."""
    from paper_1907_01063_gb300 import shard
    sizes = [int(v) for v in W.batch_sizes(24, 16, 300, seed=5)]
    Xs, ys, hyps = make_batch(sizes, seed=7)
    _, v0, g0, info0 = run_batch(sizes, Xs, ys, hyps, precision=precision)
    assert np.all(info0[:, 1] == gp.GPC_OK)
    v, g = np.full(len(sizes), np.nan), np.full((len(sizes), 3), np.nan)
    for part in shard.partition_by_cost(sizes, 3):
        _, vp, gp_, info = run_batch([sizes[i] for i in part], [Xs[i] for i in part], [ys[i] for i in part],
                                     hyps[part], precision=precision)
        assert np.all(info[:, 1] == gp.GPC_OK)
        vv, gg = shard.gather_results(part, vp, gp_, len(sizes), 1)
        keep = ~np.isnan(vv.numpy())
        v[keep], g[keep] = vv.numpy()[keep], gg.numpy()[keep]
    assert np.all(np.abs(v - v0) <= 1e-13 * np.maximum(1.0, np.abs(v0)))
    assert np.all(np.abs(g - g0) <= 1e-11 * np.maximum(1.0, np.abs(g0)))
