"""GEMM with its reverse mode (Section 3.1) and the fused GLM likelihoods
(Section 3.4) against the oracle, through the C ABI.

Tolerance: relative 1e-12 (FP64 sums in a different order than the oracle's
left-to-right loops: about sqrt(k) u).  GEMM shapes span several 64 x 64
tiles with ragged edges, an empty k, and k much larger than m and n (the
split-k case).  GLM sizes span several row blocks, k not a multiple of 32 or
256, k above 1024, and n = 0 and k = 0.  The largest GLM case is the bench's
workload (n = 2^20, k = 512), computed whole by the oracle.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-12


def rel(a, b):
    a, b = np.asarray(a, dtype=np.float64), np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


GEMM_SHAPES = [(1, 1, 1), (17, 33, 65), (64, 64, 64), (130, 70, 300), (65, 129, 0), (64, 64, 70000),
               (3, 5, 20000)]


@pytest.mark.parametrize("m,n,k", GEMM_SHAPES)
@pytest.mark.parametrize("split", [False, True])
def test_gemm_matches_oracle(m, n, k, split):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A, B = rng.standard_normal((m, k)), rng.standard_normal((k, n))
    ws = gp.gemm_workspace("cuda") if split else None
    C = gp.gemm(dev(A), dev(B), ws=ws).cpu().numpy()
    ref = O.gemm(A, B)
    if k == 0:
        assert np.array_equal(C, np.zeros((m, n)))
    else:
        assert rel(C, ref) <= TOL


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (17, 33, 65), (130, 70, 300), (64, 3, 20000)])
def test_gemm_adjoint_matches_oracle(m, n, k):
    rng = np.random.default_rng(m + n + k)
    A, B, Cb = rng.standard_normal((m, k)), rng.standard_normal((k, n)), rng.standard_normal((m, n))
    Ab0, Bb0 = O.gemm_adjoint(A, B, Cb)
    Ab, Bb = gp.gemm_adjoint(dev(A), dev(B), dev(Cb), ws=gp.gemm_workspace("cuda"))
    assert rel(Ab.cpu().numpy(), Ab0) <= TOL
    assert rel(Bb.cpu().numpy(), Bb0) <= TOL


def test_autograd_matmul_matches_oracle():
    rng = np.random.default_rng(9)
    A, B, Wt = rng.standard_normal((70, 90)), rng.standard_normal((90, 40)), rng.standard_normal((70, 40))
    At, Bt = dev(A).requires_grad_(True), dev(B).requires_grad_(True)
    (gp.MatMul.apply(At, Bt) * dev(Wt)).sum().backward()
    Ab0, Bb0 = O.gemm_adjoint(A, B, Wt)
    assert rel(At.grad.cpu().numpy(), Ab0) <= TOL
    assert rel(Bt.grad.cpu().numpy(), Bb0) <= TOL


FAMILIES = ["normal_id", "bernoulli_logit", "poisson_log", "neg_binomial_2_log"]
GLM_SIZES = [(0, 5), (1, 1), (7, 0), (100, 3), (1000, 64), (3000, 300), (2000, 1025), (50, 5000)]


def glm_case(family, n, k, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    beta = rng.standard_normal(k) / max(1.0, np.sqrt(k))
    alpha = 0.2
    eta = alpha + X @ beta
    mu = np.exp(np.clip(eta, -5, 5))
    phi = 0.7  # the dispersion check_glm passes as sigma
    y = {"normal_id": eta + rng.standard_normal(n),
         "bernoulli_logit": (rng.random(n) < 0.5).astype(float),
         "poisson_log": rng.poisson(mu).astype(float),
         "neg_binomial_2_log": rng.negative_binomial(phi, phi / (phi + mu)).astype(float)}[family]
    return X, y, alpha, beta


def check_glm(family, X, y, alpha, beta, sigma=0.7, tol=TOL):
    r0 = O.glm(family, X, y, alpha, beta, sigma)
    r = gp.glm(family, dev(X), dev(y), alpha, dev(beta), sigma)
    lp, da, ds = r["lp"].item(), r["dalpha"].item(), r["dsigma"].item()
    db = r["dbeta"].cpu().numpy()
    assert abs(lp - r0["lp"]) <= tol * max(1.0, abs(r0["lp"])), (lp, r0["lp"])
    assert abs(da - r0["dalpha"]) <= tol * max(1.0, np.abs(r0["dbeta"]).max(initial=0.0), abs(r0["dalpha"]))
    if X.shape[1]:
        assert rel(db, r0["dbeta"]) <= tol * 10, rel(db, r0["dbeta"])
    assert abs(ds - r0["dsigma"]) <= tol * max(1.0, abs(r0["dsigma"]))
    return r


@pytest.mark.parametrize("family", FAMILIES)
@pytest.mark.parametrize("n,k", GLM_SIZES)
def test_glm_matches_oracle(family, n, k):
    X, y, alpha, beta = glm_case(family, n, k, seed=n + 3 * k)
    check_glm(family, X, y, alpha, beta)


def test_glm_bernoulli_extreme_eta():
    X = np.array([[1.0], [-1.0], [1.0], [-1.0]])
    y = np.array([1.0, 0.0, 0.0, 1.0])
    r = check_glm("bernoulli_logit", X, y, 0.0, np.array([800.0]))
    assert np.isfinite(r["lp"].item())


def test_glm_is_bitwise_reproducible():
    X, y = W.glm_data(50000, 200, "bernoulli_logit", seed=2)
    beta = np.linspace(-0.5, 0.5, 200)
    Xd, yd, bd = dev(X), dev(y), dev(beta)
    a = gp.glm("bernoulli_logit", Xd, yd, 0.1, bd)
    b = gp.glm("bernoulli_logit", Xd, yd, 0.1, bd)
    assert a["lp"].item() == b["lp"].item()
    assert torch.equal(a["dbeta"], b["dbeta"])


def test_autograd_glm_matches_oracle():
    X, y = W.glm_data(3000, 40, "normal_id", seed=4)
    beta = np.linspace(-1.0, 1.0, 40)
    al = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    bt = dev(beta).requires_grad_(True)
    sg = torch.tensor(1.3, dtype=torch.float64, requires_grad=True)
    lp = gp.glm_lpmf("normal_id", dev(X), dev(y), al, bt, sg)
    lp.backward()
    r0 = O.glm("normal_id", X, y, 0.3, beta, 1.3)
    assert abs(lp.item() - r0["lp"]) <= TOL * abs(r0["lp"])
    assert abs(al.grad.item() - r0["dalpha"]) <= 1e-10 * max(1.0, abs(r0["dalpha"]))
    assert rel(bt.grad.cpu().numpy(), r0["dbeta"]) <= 1e-11
    assert abs(sg.grad.item() - r0["dsigma"]) <= 1e-10 * max(1.0, abs(r0["dsigma"]))


def test_glm_bench_workload_whole():
    """The bench's workload (logistic regression toy data, n = 2^20, k = 512),
    computed whole by the oracle."""
    n, k = 1 << 20, 512
    X, y = W.glm_data(n, k, "bernoulli_logit", seed=0)
    beta = np.zeros(k)
    beta[0], beta[1] = 3.0, -2.0
    check_glm("bernoulli_logit", X, y, 1.0, beta)


@pytest.mark.parametrize("phi", [0.013, 0.7, 3.0, 9.99, 10.0, 57.5, 2500.0])
def test_neg_binomial_dispersion_derivative_and_digamma(phi):
    # one observation per call, no covariates: dsigma = psi(y + phi) - psi(phi)
    # + log phi - log(mu + phi) + 1 - (y + phi)/(mu + phi), so the device
    # digamma is compared with the oracle's over small and large arguments
    for y0 in (0.0, 1.0, 3.0, 9.0, 42.0, 1000.0, 123456.0):
        X = np.zeros((1, 0))
        y = np.array([y0])
        check_glm("neg_binomial_2_log", X, y, 0.3, np.zeros(0), sigma=phi)


def ordinal_case(n, k, C, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    beta = rng.standard_normal(k) / max(1.0, np.sqrt(k))
    cuts = np.sort(rng.standard_normal(C - 1)) * 1.5
    eta = X @ beta
    s = 1.0 / (1.0 + np.exp(-(eta[:, None] - cuts[None, :])))  # P(y > m)
    u = rng.random(n)
    y = np.sum(u[:, None] < s, axis=1).astype(float)
    return X, y, beta, cuts


ORD_SIZES = [(0, 3, 3), (1, 1, 2), (7, 0, 4), (100, 3, 4), (1000, 64, 5), (3000, 300, 16), (2000, 1025, 3),
             (50, 5000, 2)]


@pytest.mark.parametrize("n,k,C", ORD_SIZES)
def test_glm_ordinal_matches_oracle(n, k, C):
    X, y, beta, cuts = ordinal_case(n, k, C, seed=n + k + C)
    r0 = O.glm_ordinal(X, y, beta, cuts)
    r = gp.glm_ordinal(dev(X), dev(y), dev(beta), dev(cuts))
    assert abs(r["lp"].item() - r0["lp"]) <= TOL * max(1.0, abs(r0["lp"]))
    if k:
        assert rel(r["dbeta"].cpu().numpy(), r0["dbeta"]) <= 10 * TOL
    assert np.allclose(r["dcuts"].cpu().numpy(), r0["dcuts"], rtol=10 * TOL,
                       atol=10 * TOL * max(1.0, np.abs(r0["dcuts"]).max(initial=0.0)))


def categorical_case(n, k, C, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    beta = rng.standard_normal((k, C)) / max(1.0, np.sqrt(k))
    alpha = rng.standard_normal(C) * 0.5
    eta = alpha[None, :] + X @ beta
    p = np.exp(eta - eta.max(axis=1, keepdims=True))
    p /= p.sum(axis=1, keepdims=True)
    u = rng.random(n)
    y = np.minimum(np.sum(u[:, None] > np.cumsum(p, axis=1), axis=1), C - 1).astype(float)
    return X, y, alpha, beta


CAT_SIZES = [(0, 3, 3), (1, 1, 2), (7, 0, 4), (100, 3, 4), (1000, 64, 5), (3000, 300, 16), (2000, 500, 8),
             (50, 4096, 2)]


@pytest.mark.parametrize("n,k,C", CAT_SIZES)
def test_glm_categorical_matches_oracle(n, k, C):
    X, y, alpha, beta = categorical_case(n, k, C, seed=3 * n + k + C)
    r0 = O.glm_categorical(X, y, alpha, beta)
    r = gp.glm_categorical(dev(X), dev(y), dev(alpha), dev(beta))
    assert abs(r["lp"].item() - r0["lp"]) <= TOL * max(1.0, abs(r0["lp"]))
    da = r["dalpha"].cpu().numpy()
    assert np.allclose(da, r0["dalpha"], rtol=10 * TOL, atol=10 * TOL * max(1.0, np.abs(r0["dalpha"]).max(initial=0.0)))
    if k:
        assert rel(r["dbeta"].cpu().numpy(), r0["dbeta"]) <= 10 * TOL


def test_glm_class_labels_outside_the_support_give_nan():
    X = np.ones((3, 2))
    yo = np.array([0.0, 5.0, 1.0])  # 5 is not a class of C = 3
    r = gp.glm_ordinal(dev(X), dev(yo), dev(np.array([0.1, 0.2])), dev(np.array([-0.5, 0.5])))
    assert np.isnan(r["lp"].item())
    yc = np.array([0.0, -1.0, 1.0])
    r = gp.glm_categorical(dev(X), dev(yc), dev(np.zeros(3)), dev(np.ones((2, 3))))
    assert np.isnan(r["lp"].item())


def test_glm_categorical_is_bitwise_reproducible():
    X, y, alpha, beta = categorical_case(40000, 100, 6, seed=9)
    a = gp.glm_categorical(dev(X), dev(y), dev(alpha), dev(beta))
    b = gp.glm_categorical(dev(X), dev(y), dev(alpha), dev(beta))
    assert a["lp"].item() == b["lp"].item() and torch.equal(a["dbeta"], b["dbeta"])
