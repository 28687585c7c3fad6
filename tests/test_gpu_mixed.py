"""Mixed-precision path: split-BF16 tensor-core products against exact values
and the FP64 oracle, through the C ABI.

The product's error model: each K chunk is exact in its three high-order
slice groups (integer sums below 2^24) and rounded only 2^-32 below them;
the 40-bit split and the dropped slice pairs leave about 2^-38 relative to
max|a| max|b| per chunk; accumulation is in double-float (about 2^-48).  Tolerances below are stated
against that model (with a safety factor), or as exact equality where the
operands have few enough significant bits for every step to be exact.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def int_operand(rows, k, bits, seed):
    g = np.random.default_rng(seed)
    return g.integers(-(2 ** bits - 1), 2 ** bits, size=(rows, k)).astype(np.int64)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (5, 7, 16), (128, 64, 128), (130, 70, 128), (257, 129, 100)])
def test_ozaki_exact_on_16_bit_operands(M, N, K):
    # 16-bit integer operands scaled by 2^-16: two slices hold them exactly, all
    # partial sums stay below 2^24, so the product must be exact.
    a = int_operand(M, K, 16, 1)
    b = int_operand(N, K, 16, 2)
    exact = (a @ b.T)  # |entries| < K 2^32 < 2^40: exact in int64 and in float64
    C = gp.test_ozaki_gemm(dev(a * 2.0 ** -16), dev(b * 2.0 ** -16)).cpu().numpy()
    assert np.array_equal(C, exact.astype(np.float64) * 2.0 ** -32)


@pytest.mark.parametrize("M,N,K", [(1, 1, 1), (64, 64, 64), (129, 65, 33), (300, 200, 96), (128, 128, 128),
                                   (200, 130, 129), (300, 257, 513), (128, 1000, 4096)])
def test_ozaki_accuracy_random(M, N, K):
    g = np.random.default_rng(M + N + K)
    A = g.standard_normal((M, K))
    B = g.standard_normal((N, K))
    ref = A @ B.T
    C = gp.test_ozaki_gemm(dev(A), dev(B)).cpu().numpy()
    bound = np.abs(A) @ np.abs(B).T
    err = np.abs(C - ref)
    assert np.all(err <= 2.0 ** -35 * bound + 1e-300), float(np.max(err / bound))


def test_ozaki_wide_dynamic_range():
    g = np.random.default_rng(7)
    # per-row scales of both operands are absorbed by the per-(row, chunk) exponents
    A = g.standard_normal((130, 256)) * np.exp(g.uniform(-20, 20, size=(130, 1)))
    B = g.standard_normal((90, 256)) * np.exp(g.uniform(-20, 20, size=(90, 1)))
    ref = A @ B.T
    C = gp.test_ozaki_gemm(dev(A), dev(B)).cpu().numpy()
    bound = np.abs(A) @ np.abs(B).T
    assert np.all(np.abs(C - ref) <= 2.0 ** -34 * bound)


def se_problem(n, d=3, seed=0, jitter=1e-6, rho=1.0, sigma=0.3):
    X = W.gp_inputs(n, d, seed)
    return X, O.se_cov(X, 1.0, rho, sigma, jitter)


MIXED_SIZES = [1, 2, 17, 64, 65, 96, 127, 128, 129, 191, 200, 257, 300, 513]


@pytest.mark.parametrize("n", MIXED_SIZES)
def test_chol_mixed_close_to_oracle(n):
    _, K = se_problem(n, seed=n)
    L = gp.chol(dev(K), precision="mixed").cpu().numpy()
    Lo = O.chol(K)
    assert np.all(np.triu(L, 1) == 0)
    assert rel(L, Lo) <= 1e-9
    ld, ldo = 2 * np.log(np.diag(L)).sum(), 2 * np.log(np.diag(Lo)).sum()
    assert abs(ld - ldo) <= 1e-11 * max(1.0, abs(ldo))


def test_chol_mixed_known_factor_and_in_place():
    n = 700
    L0 = W.known_factor(n, seed=3)
    K = dev(L0) @ dev(L0).T
    L = gp.chol(K.clone(), precision="mixed").cpu().numpy()
    assert rel(L, L0) <= 1e-9
    Kc = K.clone()
    gp.chol(Kc, precision="mixed", out=Kc)
    assert np.array_equal(Kc.cpu().numpy(), L)


def test_chol_mixed_not_pd():
    _, K = se_problem(300, seed=1)
    K = K.copy()
    K[200, 200] = -1.0
    info = gp.new_info()
    gp.chol(dev(K), precision="mixed", info=info, check=False)
    assert info.tolist() == [200, gp.GPC_ERR_NOT_PD]


@pytest.mark.parametrize("n", MIXED_SIZES)
def test_adjoint_mixed_close_to_oracle(n):
    _, K = se_problem(n, seed=20 + n, jitter=1e-4)
    Lo = O.chol(K)
    Lbar = W.random_lower(n, seed=n)
    G = gp.chol_adjoint(dev(Lo), dev(Lbar), precision="mixed").cpu().numpy()
    Go = O.chol_adjoint(Lo, Lbar)
    assert np.all(np.triu(G, 1) == 0)
    assert rel(G, Go) <= 1e-9


def cond_problem(n, d=4, seed=0, cond=1e5):
    """SE covariance with sigma^2 = lambda_max / cond (an ill-conditioned GP)."""
    X = W.gp_inputs(n, d, seed)
    Kf = O.se_cov(X, 1.0, 2.0, 0.0, 0.0, full=True)
    lam = np.linalg.eigvalsh(Kf)[-1]
    sigma = float(np.sqrt(lam / cond))
    y = W.gp_targets(X, 1.0, 2.0, sigma, seed=seed + 1)
    return X, y, (1.0, 2.0, sigma)


@pytest.mark.parametrize("n", [256, 1000])
def test_gp_lml_mixed_with_refinement(n):
    X, y, (a, r, s) = cond_problem(n)
    ref = O.gp_lml_and_grad(X, y, a, r, s, 0.0)
    K = gp.se_cov(dev(X), a, r, s, 0.0)
    res = gp.gp_lml(K, dev(y), precision="mixed", check=False)
    pivot, status = res["info"].tolist()
    assert status == gp.GPC_OK, gp.status_string(status)
    assert abs(res["value"].item() - ref["value"]) <= 1e-10 * abs(ref["value"])
    assert abs(res["logdet"].item() - ref["logdet"]) <= 1e-10 * abs(ref["logdet"])
    # the refined solve reaches FP64 accuracy for this conditioning
    assert rel(res["alpha"].cpu().numpy(), ref["alpha"]) <= 1e-9
    Kbar = gp.gp_lml_grad(res["L"], res["alpha"], 1.0, precision="mixed").cpu().numpy()
    assert rel(Kbar, ref["Kbar"]) <= 1e-8
    g = gp.se_hyper_grad(dev(X), a, r, s, dev(Kbar)).cpu().numpy()
    # the hyperparameter gradient sums K-bar against dK with cancellation; at
    # condition 1e5 FP64 rounding alone moves it by ~1e-9 relative
    assert rel(g, ref["grad"]) <= 1e-7


def test_gp_lml_mixed_rejects_in_place():
    X, y, (a, r, s) = cond_problem(64)
    K = gp.se_cov(dev(X), a, r, s, 0.0)
    with pytest.raises(gp.GpcholError):
        gp.gp_lml(K, dev(y), precision="mixed", L=K)


@pytest.mark.parametrize("n,d,rho", [(1, 1, 1.0), (33, 16, 4.0), (257, 3, 0.3), (300, 7, 1.3), (130, 2, 0.05)])
def test_se_cov_mixed_double_float(n, d, rho):
    # r^2 and exp in double-float: about 2^-46 per entry against the FP64 oracle;
    # rho = 0.05 sends many entries past r^2 / (2 rho^2) = 80 (the FP64 fallback)
    X = W.gp_inputs(n, d, seed=n + d)
    Ko = O.se_cov(X, 1.3, rho, 0.2, 1e-8, full=True)
    K = gp.se_cov(dev(X), 1.3, rho, 0.2, 1e-8, full=True, precision="mixed").cpu().numpy()
    # an absolute error of ~2^-46 t in the exponent t = r^2 / (2 rho^2) moves
    # e^{-t} by ~2^-46 t relative (the same growth FP64 has at 2^-53)
    off = ~np.eye(n, dtype=bool)
    t = np.ones_like(Ko)
    with np.errstate(divide="ignore"):
        t[off] = np.maximum(1.0, -np.log(Ko[off] / 1.3 ** 2))
    t[~np.isfinite(t)] = 1.0  # FP64 underflow to zero: the absolute term covers it
    assert np.all(np.abs(K - Ko) <= 2e-13 * t * np.abs(Ko) + 1e-300)
    assert np.array_equal(np.diag(K), np.diag(Ko))


def test_hyper_grad_mixed_close_to_oracle_and_deterministic():
    n, d = 513, 4
    X = W.gp_inputs(n, d, seed=5)
    Kbar = np.tril(W.random_lower(n, seed=6))
    ref = O.se_hyper_grad(X, 1.1, 0.7, 0.3, Kbar)
    g1 = gp.se_hyper_grad(dev(X), 1.1, 0.7, 0.3, dev(Kbar), precision="mixed")
    g2 = gp.se_hyper_grad(dev(X), 1.1, 0.7, 0.3, dev(Kbar), precision="mixed")
    assert torch.equal(g1, g2)
    # relative to the sum of absolute terms (Kbar has mixed signs)
    absref = O.se_hyper_grad(X, 1.1, 0.7, 0.3, np.abs(Kbar))
    assert np.all(np.abs(g1.cpu().numpy() - ref) <= 1e-12 * np.abs(absref))


def test_gp_step_mixed_covariance_end_to_end():
    X, y, (a, r, s) = cond_problem(1000)
    ref = O.gp_lml_and_grad(X, y, a, r, s, 0.0)
    K = gp.se_cov(dev(X), a, r, s, 0.0, precision="mixed")
    res = gp.gp_lml(K, dev(y), precision="mixed", check=False)
    assert res["info"].tolist()[1] == gp.GPC_OK
    assert abs(res["value"].item() - ref["value"]) <= 1e-10 * abs(ref["value"])
    Kbar = gp.gp_lml_grad(res["L"], res["alpha"], 1.0, precision="mixed")
    g = gp.se_hyper_grad(dev(X), a, r, s, Kbar, precision="mixed").cpu().numpy()
    assert rel(g, ref["grad"]) <= 1e-7


def test_gp_step_captures_in_a_cuda_graph():
    # the whole step (covariance, mixed factorisation with the auxiliary
    # stream's lookahead, refinement, adjoint, gradient) captures into one
    # graph whose replay reproduces the direct launches bit for bit
    n = 777
    X, y, (a, r, s) = cond_problem(n)
    Xd, yd = dev(X), dev(y)
    K = torch.empty(n, n, dtype=torch.float64, device="cuda")
    L, Kbar = torch.empty_like(K), torch.empty_like(K)
    ws = gp.workspace(n, "mixed", torch.device("cuda"))
    hws = torch.empty(gp.se_hyper_grad_workspace_size(n), dtype=torch.uint8, device="cuda")
    info = gp.new_info(torch.device("cuda"))
    g3 = torch.empty(3, dtype=torch.float64, device="cuda")
    val = torch.empty(1, dtype=torch.float64, device="cuda")

    def step():
        gp.se_cov(Xd, a, r, s, 0.0, out=K, precision="mixed")
        res = gp.gp_lml(K, yd, "mixed", L=L, ws=ws, info=info, check=False)
        gp.gp_lml_grad(L, res["alpha"], 1.0, "mixed", out=Kbar, ws=ws)
        gp.se_hyper_grad(Xd, a, r, s, Kbar, ws=hws, out=g3, precision="mixed")
        val.copy_(res["value"].reshape(1))

    step()
    torch.cuda.synchronize()
    v0, g0, L0 = val.clone(), g3.clone(), L.clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        step()
    torch.cuda.current_stream().wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step()
    val.zero_()
    g3.zero_()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert info.tolist()[1] == gp.GPC_OK
    assert torch.equal(val, v0) and torch.equal(g3, g0) and torch.equal(L, L0)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 127, 128, 129, 191, 300])
def test_gp_lml_mixed_edge_sizes(n):
    # the double-float solves at their edges: one sub-block (n <= 64), a
    # one-row last sub-block (65, 129), block boundaries of the factorisation
    # (128) and ragged tails; alpha after refinement, the value and log det
    # against the oracle's pass
    X, y, (a, r, s) = cond_problem(n, cond=1e4)
    ref = O.gp_lml_and_grad(X, y, a, r, s, 0.0)
    K = gp.se_cov(dev(X), a, r, s, 0.0)
    res = gp.gp_lml(K, dev(y), precision="mixed", check=False)
    assert res["info"].tolist()[1] == gp.GPC_OK
    assert abs(res["value"].item() - ref["value"]) <= 1e-10 * max(abs(ref["value"]), 1.0)
    assert abs(res["logdet"].item() - ref["logdet"]) <= 1e-10 * max(abs(ref["logdet"]), 1.0)
    assert rel(res["alpha"].cpu().numpy(), ref["alpha"]) <= 1e-10
