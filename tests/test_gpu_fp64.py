"""FP64 parity of the CUDA path against the CPU oracle, through the C ABI.

Tolerance: relative Frobenius error <= 1e-10 for L, Kbar and the solves (the
stated bar for jittered SE matrices with condition number <= 1e6), and the
same relative bound on scalars.  Sizes span several 64-wide GEMM tiles and
128-wide factorisation blocks with ragged tails.
"""

import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def se_problem(n, d=3, seed=0, jitter=1e-6, rho=1.0, sigma=0.3):
    X = W.gp_inputs(n, d, seed)
    return X, O.se_cov(X, 1.0, rho, sigma, jitter)


SIZES = [1, 2, 3, 15, 16, 17, 63, 64, 65, 127, 128, 129, 200, 257, 300, 513]


@pytest.mark.parametrize("n", SIZES)
def test_chol_matches_oracle(n):
    _, K = se_problem(n, seed=n)
    L = gp.chol(dev(K)).cpu().numpy()
    Lo = O.chol(K)
    assert rel(L, Lo) <= TOL
    assert np.all(np.triu(L, 1) == 0)


@pytest.mark.parametrize("block", [16, 32, 64, 128])
def test_chol_block_sizes(block):
    old = gp.get_tuning(gp.GPC_TUNE_BLOCK)
    try:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, block)
        _, K = se_problem(333, seed=2)
        L = gp.chol(dev(K)).cpu().numpy()
        assert rel(L, O.chol(K)) <= TOL
        Lbar = W.random_lower(333, seed=3)
        G = gp.chol_adjoint(dev(L), dev(Lbar)).cpu().numpy()
        assert rel(G, O.chol_adjoint(L, Lbar)) <= TOL
        # the likelihood's solves use the factorisation's block inverses at this block size
        y = W.gp_inputs(333, 1, seed=4)[:, 0]
        ref = O.gp_lml(K, y)
        res = gp.gp_lml(dev(K), dev(y))
        assert rel(res["alpha"].cpu().numpy(), ref["alpha"]) <= TOL
        assert abs(res["value"].item() - ref["value"]) <= TOL * abs(ref["value"])
    finally:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, old)


@pytest.mark.parametrize("tile_limit", [0, 256, 4096])
def test_small_product_tile_limit(tile_limit):
    # The FP64 products take 32 x 32 output tiles up to a tuned size limit
    # (0: never, 4096: every product of this size); the factor, the adjoint
    # and a plain GEMM must match the oracle with either tile.
    old = gp.get_tuning(gp.GPC_TUNE_F64_SMALL_TILE)
    try:
        gp.set_tuning(gp.GPC_TUNE_F64_SMALL_TILE, tile_limit)
        _, K = se_problem(451, seed=6)
        L = gp.chol(dev(K)).cpu().numpy()
        assert rel(L, O.chol(K)) <= TOL
        Lbar = W.random_lower(451, seed=7)
        G = gp.chol_adjoint(dev(L), dev(Lbar)).cpu().numpy()
        assert rel(G, O.chol_adjoint(L, Lbar)) <= TOL
        A = W.gp_inputs(97, 203, seed=8)
        B = W.gp_inputs(203, 45, seed=9)
        assert rel(gp.gemm(dev(A), dev(B)).cpu().numpy(), O.gemm(A, B)) <= 1e-12
    finally:
        gp.set_tuning(gp.GPC_TUNE_F64_SMALL_TILE, old)


def test_chol_in_place_padded_ld_and_upper_ignored():
    n = 250
    _, K = se_problem(n, seed=5)
    buf = torch.full((n, n + 7), 99.0, dtype=torch.float64, device="cuda")
    Kv = buf[:, :n]
    Kv.copy_(dev(np.tril(K) + np.triu(np.full((n, n), 7.0), 1)))
    out = gp.chol(Kv, out=Kv)
    assert out.data_ptr() == Kv.data_ptr()
    L = Kv.cpu().numpy()
    assert rel(L, O.chol(K)) <= TOL
    assert np.all(buf[:, n:].cpu().numpy() == 99.0), "padding columns were touched"


def test_chol_known_factor_4096():
    n = 4096
    L0 = W.known_factor(n, seed=0)
    K = dev(L0) @ dev(L0).T
    L = gp.chol(K).cpu().numpy()
    # forward error ~ cond(L0) * u; cond(L0) is modest for this recipe
    assert rel(L, L0) <= TOL
    ld = 2.0 * np.log(np.diag(L)).sum()
    assert abs(ld - 2.0 * np.log(np.diag(L0)).sum()) <= 1e-12 * abs(ld)


def test_chol_paper_toeplitz():
    n = 1000
    A = W.toeplitz_spd(n)
    L = gp.chol(dev(A)).cpu().numpy()
    assert rel(L, O.chol(A)) <= TOL


@pytest.mark.parametrize("n,bad", [(5, 2), (200, 150), (300, 0), (129, 128)])
def test_chol_not_pd_reports_first_pivot(n, bad):
    _, K = se_problem(n, seed=1)
    K = K.copy()
    K[bad, bad] = -1.0
    _, info_o = O.chol_info(K)
    info = gp.new_info()
    gp.chol(dev(K), info=info, check=False)
    pivot, status = info.tolist()
    assert pivot == info_o == bad
    assert status == gp.GPC_ERR_NOT_PD
    with pytest.raises(gp.NotPositiveDefinite):
        gp.chol(dev(K))


def test_chol_nan_pivot():
    _, K = se_problem(70, seed=1)
    K = K.copy()
    K[40, 40] = np.nan
    info = gp.new_info()
    gp.chol(dev(K), info=info, check=False)
    assert info.tolist() == [40, gp.GPC_ERR_NAN]


@pytest.mark.parametrize("n", SIZES)
def test_adjoint_matches_oracle(n):
    _, K = se_problem(n, seed=10 + n, jitter=1e-4)
    Lo = O.chol(K)
    Lbar = W.random_lower(n, seed=n)
    G = gp.chol_adjoint(dev(Lo), dev(Lbar)).cpu().numpy()
    Go = O.chol_adjoint(Lo, Lbar)
    assert rel(G, Go) <= TOL
    assert np.all(np.triu(G, 1) == 0)


def test_adjoint_in_place_and_symmetric_out():
    n = 200
    _, K = se_problem(n, seed=4, jitter=1e-4)
    Lo = O.chol(K)
    Lbar = W.random_lower(n, seed=9)
    Go = O.chol_adjoint(Lo, Lbar)
    A = dev(Lbar + np.triu(np.ones((n, n)), 1))  # upper part of Lbar is ignored
    gp.chol_adjoint(dev(Lo), A, out=A)
    assert rel(A.cpu().numpy(), Go) <= TOL
    S = gp.chol_adjoint(dev(Lo), dev(Lbar), symmetric_out=True).cpu().numpy()
    ref = np.tril(Go, -1) / 2
    ref = ref + ref.T + np.diag(np.diag(Go))
    assert rel(S, ref) <= TOL


@pytest.mark.parametrize("n,d", [(1, 1), (5, 2), (33, 16), (257, 2), (300, 7)])
def test_se_cov_matches_oracle(n, d):
    X = W.gp_inputs(n, d, seed=n)
    for full in (False, True):
        K = gp.se_cov(dev(X), 1.3, 0.8, 0.2, 1e-8, full=full).cpu().numpy()
        Ko = O.se_cov(X, 1.3, 0.8, 0.2, 1e-8, full=full)
        assert rel(K, Ko) <= 1e-13


@pytest.mark.parametrize("n", [1, 63, 64, 65, 300, 1000])
def test_trsv_matches_oracle(n):
    L0 = W.known_factor(n, seed=n)
    x = W.gp_inputs(n, 1, seed=1)[:, 0]
    for trans in (False, True):
        xd = dev(x)
        gp.trsv(dev(L0), xd, trans=trans)
        assert rel(xd.cpu().numpy(), O.trsv(L0, x, trans)) <= TOL


def config1():
    n, d = 256, 2
    X = W.gp_inputs(n, d, seed=0)
    y = W.gp_targets(X, 1.0, 0.5, 0.1, seed=1)
    return X, y, (1.0, 0.5, 0.1), 1e-8


def test_gp_lml_config1():
    X, y, (a, r, s), jit = config1()
    ref = O.gp_lml_and_grad(X, y, a, r, s, jit)
    K = gp.se_cov(dev(X), a, r, s, jit)
    res = gp.gp_lml(K, dev(y))
    assert rel(res["L"].cpu().numpy(), ref["L"]) <= TOL
    assert rel(res["alpha"].cpu().numpy(), ref["alpha"]) <= 1e-9
    assert abs(res["logdet"].item() - ref["logdet"]) <= TOL * abs(ref["logdet"])
    assert abs(res["value"].item() - ref["value"]) <= TOL * abs(ref["value"])
    Kbar = gp.gp_lml_grad(res["L"], res["alpha"]).cpu().numpy()
    assert rel(Kbar, ref["Kbar"]) <= 1e-9
    g = gp.se_hyper_grad(dev(X), a, r, s, dev(Kbar)).cpu().numpy()
    assert rel(g, ref["grad"]) <= 1e-9


def test_autograd_gp_lml_matches_oracle():
    X, y, hyp, jit = config1()
    h = torch.tensor(hyp, dtype=torch.float64, requires_grad=True)
    v = gp.gp_lml_value(dev(X), dev(y), h, jit)
    v.backward()
    ref = O.gp_lml_and_grad(X, y, *hyp, jit)
    assert abs(v.item() - ref["value"]) <= TOL * abs(ref["value"])
    assert rel(h.grad.numpy(), ref["grad"]) <= 1e-9


def test_autograd_chol_matches_oracle():
    n = 150
    _, K = se_problem(n, seed=3, jitter=1e-3)
    Wt = W.random_lower(n, seed=4)
    Kt = dev(K).requires_grad_(True)
    L = gp.Chol.apply(Kt)
    (L * dev(Wt)).sum().backward()
    ref = O.chol_adjoint(O.chol(K), Wt)
    assert rel(Kt.grad.cpu().numpy(), ref) <= TOL


def test_hyper_grad_deterministic():
    X, y, (a, r, s), jit = config1()
    Kbar = dev(W.random_lower(256, seed=2))
    g1 = gp.se_hyper_grad(dev(X), a, r, s, Kbar)
    g2 = gp.se_hyper_grad(dev(X), a, r, s, Kbar)
    assert torch.equal(g1, g2)


def test_zero_size_calls():
    e = torch.empty(0, 0, dtype=torch.float64, device="cuda")
    assert gp.chol(e).shape == (0, 0)
    assert gp.chol_adjoint(e, e).shape == (0, 0)
