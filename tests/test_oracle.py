"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

Nothing here compares the oracle with itself: each test uses a closed form, a
hand-computed value, a library routine for a special case (LAPACK through
NumPy/SciPy), central finite differences, or an independent derivation.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.spatial.distance
import scipy.stats

from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

U = np.finfo(np.float64).eps / 2


def rel_fro(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def spd_se(n, d=3, seed=0, jitter=1e-6):
    X = W.gp_inputs(n, d, seed)
    return X, O.se_cov(X, 1.0, 1.0, 0.3, jitter)


# ---------------------------------------------------------------- chol
def test_chol_1x1():
    assert O.chol([[4.0]])[0, 0] == 2.0
    assert O.chol([[2.0]])[0, 0] == math.sqrt(2.0)


def test_chol_2x2_by_hand():
    # [[4,2],[2,5]] = [[2,0],[1,2]] [[2,1],[0,2]]
    L = O.chol(np.array([[4.0, 2.0], [2.0, 5.0]]))
    assert np.array_equal(L, np.array([[2.0, 0.0], [1.0, 2.0]]))


def test_chol_3x3_by_hand():
    # L = [[1,0,0],[2,3,0],[4,5,6]] -> K = L L^T
    L0 = np.array([[1.0, 0, 0], [2, 3, 0], [4, 5, 6]])
    K = np.array([[1.0, 2, 4], [2, 13, 23], [4, 23, 77]])
    assert np.array_equal(O.chol(K), L0)


def test_chol_identity_and_diagonal():
    assert np.array_equal(O.chol(np.eye(7)), np.eye(7))
    d = np.array([1.0, 4.0, 9.0, 0.25, 16.0])
    assert np.array_equal(O.chol(np.diag(d)), np.diag(np.sqrt(d)))


@pytest.mark.parametrize("n", [1, 5, 37, 64, 129])
def test_chol_known_factor(n):
    L0 = W.known_factor(n, seed=n)
    K = L0 @ L0.T
    L = O.chol(K)
    # forward error bound ~ cond(L0) * n * u
    assert rel_fro(L, L0) < 1e3 * n * U * np.linalg.cond(L0)
    assert np.all(np.triu(L, 1) == 0)
    # log det from the factor's diagonal
    ld = 2.0 * np.log(np.diag(L)).sum()
    assert abs(ld - 2.0 * np.log(np.diag(L0)).sum()) < 1e-12 * max(1.0, abs(ld))


@pytest.mark.parametrize("n", [2, 50, 150])
def test_chol_reconstruction(n):
    _, K = spd_se(n)
    L = O.chol(K)
    assert rel_fro(L @ L.T, np.tril(K) + np.tril(K, -1).T) < 4 * n * U


def test_chol_toeplitz_matches_lapack():
    A = W.toeplitz_spd(60)
    L = O.chol(A)
    assert rel_fro(L, np.linalg.cholesky(A)) < 1e-14


def test_chol_reads_lower_only():
    _, K = spd_se(30)
    K2 = np.tril(K) + np.triu(np.full_like(K, 123.0), 1)
    assert np.array_equal(O.chol(K2), O.chol(np.tril(K) + np.tril(K, -1).T))


def test_chol_failing_pivot():
    _, info = O.chol_info(np.diag([1.0, -1.0, 1.0]))
    assert info == 1
    _, info = O.chol_info(np.array([[1.0, 2.0], [2.0, 1.0]]))  # s = 1 - 4 < 0
    assert info == 1
    K = np.eye(4)
    K[2, 2] = np.nan
    _, info = O.chol_info(K)
    assert info == 2
    _, info = O.chol_info(np.zeros((3, 3)))
    assert info == 0
    with pytest.raises(O.NotPositiveDefinite):
        O.chol(np.diag([1.0, 0.0]))


# ---------------------------------------------------------------- adjoint
def chol_fd_grad(K, Wt, h_rel=1e-6):
    """Central differences of f(K) = sum(W o chol(K)) over the lower entries."""
    n = K.shape[0]
    G = np.zeros_like(K)
    for i in range(n):
        for j in range(i + 1):
            h = h_rel * max(1.0, abs(K[i, j]))
            Kp = K.copy()
            Km = K.copy()
            Kp[i, j] += h
            Km[i, j] -= h
            G[i, j] = ((Wt * O.chol(Kp)).sum() - (Wt * O.chol(Km)).sum()) / (2 * h)
    return G


def test_adjoint_1x1():
    L = O.chol([[9.0]])
    assert O.chol_adjoint(L, [[6.0]])[0, 0] == 6.0 / (2 * 3.0)


@pytest.mark.parametrize("n", [2, 3, 5, 8, 13, 16])
def test_adjoint_finite_differences(n):
    _, K = spd_se(n, seed=n, jitter=1e-2)
    Wt = W.random_lower(n, seed=100 + n)
    L = O.chol(K)
    G = O.chol_adjoint(L, Wt)
    Gfd = chol_fd_grad(K, Wt)
    assert rel_fro(G, Gfd) < 1e-6
    assert np.all(np.triu(G, 1) == 0)


def test_adjoint_diagonal_matrix_closed_form():
    d = np.array([4.0, 9.0, 0.25, 2.0])
    L = np.diag(np.sqrt(d))
    Lbar = W.random_lower(4, seed=3)
    G = O.chol_adjoint(L, Lbar)
    ref = np.zeros((4, 4))
    for i in range(4):
        for j in range(i):
            ref[i, j] = Lbar[i, j] / L[j, j]
        ref[i, i] = Lbar[i, i] / (2 * L[i, i])
    assert rel_fro(G, ref) < 1e-15


@pytest.mark.parametrize("n", [1, 7, 64, 100])
def test_adjoint_unblocked_equals_symbolic(n):
    _, K = spd_se(n, seed=7, jitter=1e-3)
    L = O.chol(K)
    Lbar = W.random_lower(n, seed=8)
    a = O.chol_adjoint(L, Lbar)
    s = O.chol_adjoint_symbolic(L, Lbar)
    assert rel_fro(a, s) < 1e-10


def blocked_adjoint_reading(L, Lbar, b):
    """The block sweep of Section 3.3 (reverse mode) as read for this library.

    Slices are half-open; k runs N, N-b, ... > 0 and j = max(0, k - b).  The
    garbled last statement is read as "halve the diagonal of D_adj, then zero
    its strict upper triangle".  This test-only NumPy version checks the
    reading against the unblocked definition; it is not used anywhere else.
    """
    N = L.shape[0]
    A = np.tril(Lbar).copy()
    k = N
    while k > 0:
        j = max(0, k - b)
        R, D, B, C = L[j:k, 0:j], L[j:k, j:k], L[k:N, 0:j], L[k:N, j:k]
        Dinv = np.linalg.inv(D)
        Cb = A[k:N, j:k] @ Dinv
        A[k:N, j:k] = Cb
        A[k:N, 0:j] -= Cb @ R
        Db = A[j:k, j:k] - Cb.T @ C
        P = D.T @ np.tril(Db)
        M = np.tril(P) + np.tril(P, -1).T
        Db = Dinv.T @ M @ Dinv
        Db = 0.5 * (Db + Db.T)
        A[j:k, 0:j] -= Cb.T @ B + Db @ R
        Db = np.tril(Db)
        Db[np.arange(k - j), np.arange(k - j)] *= 0.5
        A[j:k, j:k] = Db
        k -= b
    return A


@pytest.mark.parametrize("n,b", [(11, 3), (20, 8), (33, 16), (16, 16), (5, 8)])
def test_blocked_sweep_reading_matches_oracle(n, b):
    _, K = spd_se(n, seed=n + b, jitter=1e-3)
    L = O.chol(K)
    Lbar = W.random_lower(n, seed=5)
    ref = O.chol_adjoint(L, Lbar)
    assert rel_fro(blocked_adjoint_reading(L, Lbar, b), ref) < 1e-11


# ---------------------------------------------------------------- covariance
def test_se_cov_two_points_by_hand():
    K = O.se_cov(np.array([[0.0], [1.0]]), 2.0, 1.0, 0.5, 0.0, full=True)
    assert K[0, 0] == 4.25 and K[1, 1] == 4.25
    assert abs(K[1, 0] - 4.0 * math.exp(-0.5)) < 1e-15
    assert K[0, 1] == K[1, 0]


def test_se_cov_matches_cdist():
    X = W.gp_inputs(50, 3, seed=2)
    K = O.se_cov(X, 1.3, 0.7, 0.2, 1e-8, full=True)
    D2 = scipy.spatial.distance.cdist(X, X, "sqeuclidean")
    ref = 1.3 ** 2 * np.exp(-D2 / (2 * 0.7 ** 2)) + np.eye(50) * (0.2 ** 2 + 1e-8)
    assert rel_fro(K, ref) < 1e-14
    Kl = O.se_cov(X, 1.3, 0.7, 0.2, 1e-8, full=False)
    assert np.all(np.triu(Kl, 1) == 0) and np.array_equal(np.tril(Kl), np.tril(K))


# ---------------------------------------------------------------- solves, LML
def test_trsv_matches_lapack():
    L0 = W.known_factor(40, seed=1)
    x = W.gp_inputs(40, 1, seed=2)[:, 0]
    for trans in (False, True):
        ref = scipy.linalg.solve_triangular(L0, x, lower=True, trans=1 if trans else 0)
        assert rel_fro(O.trsv(L0, x, trans), ref) < 1e-13


@pytest.mark.parametrize("n", [1, 3, 40, 200])
def test_lml_matches_scipy_logpdf(n):
    X = W.gp_inputs(n, 2, seed=n)
    y = W.gp_targets(X, 1.0, 0.5, 0.1, seed=n + 1)
    K = O.se_cov(X, 1.0, 0.5, 0.1, 1e-8, full=True)
    r = O.gp_lml(K, y)
    ref = scipy.stats.multivariate_normal(mean=np.zeros(n), cov=K).logpdf(y)
    assert abs(r["value"] - ref) < 1e-9 * max(1.0, abs(ref))
    sign, ld = np.linalg.slogdet(K)
    assert sign > 0 and abs(r["logdet"] - ld) < 1e-10 * max(1.0, abs(ld))
    assert rel_fro(r["alpha"], np.linalg.solve(K, y)) < 1e-8


def test_lml_lbar_finite_differences():
    n = 6
    _, K = spd_se(n, seed=4, jitter=1e-2)
    y = W.gp_inputs(n, 1, seed=9)[:, 0]
    r = O.gp_lml(K, y)
    L = r["L"]

    def value_of_L(Lm):
        z = scipy.linalg.solve_triangular(Lm, y, lower=True)
        return -0.5 * z @ z - np.log(np.diag(Lm)).sum()

    G = np.zeros((n, n))
    h = 1e-6
    for i in range(n):
        for j in range(i + 1):
            Lp, Lm = L.copy(), L.copy()
            Lp[i, j] += h
            Lm[i, j] -= h
            G[i, j] = (value_of_L(Lp) - value_of_L(Lm)) / (2 * h)
    Lbar = O.lml_lbar(L, r["alpha"], r["z"], 1.0)
    assert rel_fro(Lbar, G) < 1e-7
    assert rel_fro(O.lml_lbar(L, r["alpha"], r["z"], -2.5), -2.5 * G) < 1e-7


@pytest.mark.parametrize("n", [1, 10, 120])
def test_lml_kbar_closed_form(n):
    X = W.gp_inputs(n, 2, seed=3)
    y = W.gp_targets(X, 1.0, 0.5, 0.1, seed=4)
    K = O.se_cov(X, 1.0, 0.5, 0.1, 1e-8, full=True)
    r = O.gp_lml(K, y)
    Kbar = O.chol_adjoint(r["L"], O.lml_lbar(r["L"], r["alpha"], r["z"]))
    a = np.linalg.solve(K, y)
    Kinv = np.linalg.inv(K)
    G = np.outer(a, a) - Kinv          # off-diagonal: d value / d K_ij (pair i,j)
    ref = np.tril(G, -1) + np.diag(0.5 * np.diag(G))
    assert rel_fro(Kbar, ref) < 1e-8


def test_hyper_grad_finite_differences():
    n = 40
    X = W.gp_inputs(n, 3, seed=11)
    hyp = np.array([1.2, 0.9, 0.3])
    y = W.gp_targets(X, *hyp, seed=12)

    def value(h):
        return O.gp_lml(O.se_cov(X, h[0], h[1], h[2], 1e-8), y)["value"]

    r = O.gp_lml_and_grad(X, y, *hyp, jitter=1e-8)
    fd = np.zeros(3)
    for t in range(3):
        e = np.zeros(3)
        e[t] = 1e-6
        fd[t] = (value(hyp + e) - value(hyp - e)) / 2e-6
    assert np.allclose(r["grad"], fd, rtol=1e-6, atol=1e-6)


def test_hyper_grad_sigma_only_on_diagonal():
    n = 5
    X = W.gp_inputs(n, 2, seed=1)
    Kbar = np.tril(np.ones((n, n)))
    g = O.se_hyper_grad(X, 1.0, 1.0, 0.25, Kbar)
    assert abs(g[2] - n * 2 * 0.25) < 1e-15


# ---------------------------------------------------------------- triangular inverse and solve
def rand_lower(n, seed, diag=2.0):
    rng = np.random.default_rng(seed)
    return np.tril(rng.standard_normal((n, n)) / math.sqrt(n)) + np.diag(diag + rng.random(n))


def test_tri_inverse_bidiagonal_exact():
    # unit lower bidiagonal with -1 below the diagonal: the inverse is the
    # lower triangle of ones, and the inverse of that is the bidiagonal again
    n = 9
    E = np.eye(n) - np.eye(n, k=-1)
    ones = np.tril(np.ones((n, n)))
    assert np.array_equal(O.tri_inverse(E), ones)
    assert np.array_equal(O.tri_inverse(ones), E)


def test_tri_inverse_2x2_by_hand():
    # [[a, 0], [c, b]]^{-1} = [[1/a, 0], [-c/(a b), 1/b]]
    X = O.tri_inverse(np.array([[2.0, 0.0], [3.0, 4.0]]))
    assert np.array_equal(X, np.array([[0.5, 0.0], [-0.375, 0.25]]))


def test_tri_inverse_exact_rational():
    # exact rational inverse of an integer lower-triangular matrix with unequal
    # diagonal entries (sympy), brute force on a tiny case
    sympy = pytest.importorskip("sympy")
    rng = np.random.default_rng(3)
    n = 6
    L = np.tril(rng.integers(-4, 5, (n, n)).astype(float), -1) + np.diag([1.0, 2, 3, 5, 7, 11])
    Xs = sympy.Matrix(L.astype(int).tolist()).inv()
    ref = np.array(Xs.tolist(), dtype=float)
    assert np.abs(O.tri_inverse(L) - ref).max() <= 1e-14 * np.abs(ref).max()


@pytest.mark.parametrize("n", [1, 17, 130])
def test_tri_inverse_matches_lapack(n):
    L = rand_lower(n, seed=n)
    ref, info = scipy.linalg.lapack.dtrtri(L, lower=1)
    assert info == 0
    assert rel_fro(O.tri_inverse(L), np.tril(ref)) <= 1e-14


def test_tri_inverse_reads_lower_only():
    L = rand_lower(12, seed=5)
    J = L + np.triu(np.full((12, 12), 7.0), 1)
    assert np.array_equal(O.tri_inverse(J), O.tri_inverse(L))
    assert np.array_equal(np.triu(O.tri_inverse(J), 1), np.zeros((12, 12)))


def test_tri_solve_first_differences_exact():
    # L = lower ones: L^{-1} B takes first differences of the rows of B
    n, m = 11, 4
    rng = np.random.default_rng(0)
    B = rng.integers(-50, 50, (n, m)).astype(float)
    ref = B - np.vstack([np.zeros((1, m)), B[:-1]])
    assert np.array_equal(O.tri_solve(np.tril(np.ones((n, n))), B), ref)


@pytest.mark.parametrize("n,m", [(1, 1), (33, 5), (150, 17)])
def test_tri_solve_matches_lapack(n, m):
    L = rand_lower(n, seed=7)
    B = np.random.default_rng(8).standard_normal((n, m))
    ref = scipy.linalg.solve_triangular(L, B, lower=True)
    assert rel_fro(O.tri_solve(L, B), ref) <= 1e-14


def test_tri_solve_adjoint_1x1():
    # c = b / l: bbar = cbar / l, lbar = -cbar b / l^2
    Bb, Lb = O.tri_solve_adjoint([[4.0]], [[3.0 / 4.0]], [[2.0]])
    assert Bb[0, 0] == 0.5 and Lb[0, 0] == -2.0 * 3.0 / 16.0


@pytest.mark.parametrize("n,m", [(5, 3), (8, 1)])
def test_tri_solve_adjoint_finite_differences(n, m):
    # f(L, B) = sum(W * L^{-1} B): central differences in every lower entry of L
    # and every entry of B, with LAPACK's solve for f
    rng = np.random.default_rng(n + m)
    L = rand_lower(n, seed=n)
    B = rng.standard_normal((n, m))
    Wt = rng.standard_normal((n, m))

    def f(Lm, Bm):
        return float(np.sum(Wt * scipy.linalg.solve_triangular(Lm, Bm, lower=True)))

    C = O.tri_solve(L, B)
    Bb, Lb = O.tri_solve_adjoint(L, C, Wt)
    h = 1e-6
    for i in range(n):
        for j in range(i + 1):
            Lp, Lm = L.copy(), L.copy()
            Lp[i, j] += h
            Lm[i, j] -= h
            fd = (f(Lp, B) - f(Lm, B)) / (2 * h)
            assert abs(Lb[i, j] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, j)
    for i in range(n):
        for j in range(m):
            Bp, Bm = B.copy(), B.copy()
            Bp[i, j] += h
            Bm[i, j] -= h
            fd = (f(L, Bp) - f(L, Bm)) / (2 * h)
            assert abs(Bb[i, j] - fd) <= 1e-7 * max(1.0, abs(fd)), (i, j)
    assert np.array_equal(np.triu(Lb, 1), np.zeros((n, n)))


# ---------------------------------------------------------------- GEMM and its reverse mode
def test_gemm_exact_integers_and_numpy():
    rng = np.random.default_rng(1)
    A = rng.integers(-9, 10, (7, 5)).astype(float)
    B = rng.integers(-9, 10, (5, 3)).astype(float)
    assert np.array_equal(O.gemm(A, B), A @ B)  # small integers: every sum is exact
    A, B = rng.standard_normal((33, 65)), rng.standard_normal((65, 17))
    assert rel_fro(O.gemm(A, B), A @ B) <= 1e-15


def test_gemm_adjoint_finite_differences():
    # f(A, B) = sum(W * A B) is bilinear: central differences are exact up to rounding
    rng = np.random.default_rng(2)
    A, B, Wt = rng.standard_normal((4, 3)), rng.standard_normal((3, 5)), rng.standard_normal((4, 5))
    Ab, Bb = O.gemm_adjoint(A, B, Wt)
    h = 1e-3
    for M, G in ((A, Ab), (B, Bb)):
        for idx in np.ndindex(M.shape):
            old = M[idx]
            M[idx] = old + h
            fp = float(np.sum(Wt * (A @ B)))
            M[idx] = old - h
            fm = float(np.sum(Wt * (A @ B)))
            M[idx] = old
            assert abs(G[idx] - (fp - fm) / (2 * h)) <= 1e-10 * max(1.0, abs(G[idx])), idx


# ---------------------------------------------------------------- GLM likelihoods
def glm_data(n=60, k=5, seed=0):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, k))
    beta = rng.standard_normal(k) / 2
    return rng, X, beta, 0.3


def test_glm_bernoulli_logit_matches_scipy():
    import scipy.special as sp
    rng, X, beta, alpha = glm_data()
    eta = alpha + X @ beta
    y = (rng.random(len(eta)) < sp.expit(eta)).astype(float)
    r = O.glm("bernoulli_logit", X, y, alpha, beta)
    assert abs(r["lp"] - scipy.stats.bernoulli.logpmf(y, sp.expit(eta)).sum()) <= 1e-12 * abs(r["lp"])
    assert np.abs(r["dbeta"] - X.T @ (y - sp.expit(eta))).max() <= 1e-12
    assert r["dsigma"] == 0.0


def test_glm_bernoulli_zero_coefficients_closed_form():
    # beta = 0, alpha = 0: every p_i = 1/2, lp = -n log 2, d_i = y_i - 1/2
    rng, X, beta, _ = glm_data(n=40, k=3)
    y = (rng.random(40) < 0.5).astype(float)
    r = O.glm("bernoulli_logit", X, y, 0.0, np.zeros(3))
    assert abs(r["lp"] + 40 * math.log(2.0)) <= 1e-13 * 40
    assert abs(r["dalpha"] - float(np.sum(y - 0.5))) <= 1e-13
    assert np.abs(r["dbeta"] - X.T @ (y - 0.5)).max() <= 1e-13


def test_glm_bernoulli_extreme_eta_stays_finite():
    # eta = +-800: softplus(eta) = max(eta, 0) + log1p(exp(-|eta|)) without overflow
    X = np.array([[1.0], [-1.0], [1.0], [-1.0]])
    y = np.array([1.0, 0.0, 0.0, 1.0])
    r = O.glm("bernoulli_logit", X, y, 0.0, np.array([800.0]))
    # the two well-predicted rows contribute ~0, the two mispredicted ones -800 each
    assert abs(r["lp"] + 1600.0) <= 1e-9
    assert r["dbeta"][0] == -2.0 and r["dalpha"] == 0.0


def test_glm_poisson_and_normal_match_scipy():
    rng, X, beta, alpha = glm_data(seed=3)
    eta = alpha + X @ beta
    yp = rng.poisson(np.exp(eta)).astype(float)
    r = O.glm("poisson_log", X, yp, alpha, beta)
    assert abs(r["lp"] - scipy.stats.poisson.logpmf(yp, np.exp(eta)).sum()) <= 1e-12 * abs(r["lp"])
    assert np.abs(r["dbeta"] - X.T @ (yp - np.exp(eta))).max() <= 1e-11
    sigma = 0.7
    yn = eta + sigma * rng.standard_normal(len(eta))
    r = O.glm("normal_id", X, yn, alpha, beta, sigma)
    assert abs(r["lp"] - scipy.stats.norm.logpdf(yn, eta, sigma).sum()) <= 1e-12 * abs(r["lp"])


@pytest.mark.parametrize("family", ["normal_id", "bernoulli_logit", "poisson_log"])
def test_glm_gradient_finite_differences(family):
    rng, X, beta, alpha = glm_data(n=30, k=4, seed=4)
    eta = alpha + X @ beta
    y = {"normal_id": eta + rng.standard_normal(30),
         "bernoulli_logit": (rng.random(30) < 0.5).astype(float),
         "poisson_log": rng.poisson(np.exp(eta)).astype(float)}[family]
    sigma = 0.8
    r = O.glm(family, X, y, alpha, beta, sigma)

    def f(a, b, s):
        return O.glm(family, X, y, a, b, s)["lp"]

    h = 1e-6
    assert abs(r["dalpha"] - (f(alpha + h, beta, sigma) - f(alpha - h, beta, sigma)) / (2 * h)) <= 1e-6
    for j in range(4):
        e = np.zeros(4)
        e[j] = h
        fd = (f(alpha, beta + e, sigma) - f(alpha, beta - e, sigma)) / (2 * h)
        assert abs(r["dbeta"][j] - fd) <= 1e-6 * max(1.0, abs(fd)), j
    if family == "normal_id":
        fd = (f(alpha, beta, sigma + h) - f(alpha, beta, sigma - h)) / (2 * h)
        assert abs(r["dsigma"] - fd) <= 1e-6 * max(1.0, abs(fd))


# ---------------------------------------------------------------- the other GLMs of Section 3.4
def test_digamma_matches_scipy():
    import scipy.special as sp
    for x in [1e-4, 0.3, 1.0, 1.4616321449683623, 2.5, 7.0, 11.999, 12.0, 40.0, 1e5]:
        ref = sp.digamma(x)
        assert abs(O.psi(x) - ref) <= 1e-14 * max(1.0, abs(ref)), x


def test_glm_negative_binomial_matches_scipy():
    rng, X, beta, alpha = glm_data(seed=6)
    eta = alpha + X @ beta
    phi = 2.5
    mu = np.exp(eta)
    y = rng.negative_binomial(phi, phi / (mu + phi)).astype(float)
    r = O.glm("neg_binomial_2_log", X, y, alpha, beta, phi)
    ref = scipy.stats.nbinom.logpmf(y, phi, phi / (mu + phi)).sum()
    assert abs(r["lp"] - ref) <= 1e-12 * abs(ref)


def test_glm_negative_binomial_gradient_finite_differences():
    rng, X, beta, alpha = glm_data(n=30, k=3, seed=7)
    mu = np.exp(alpha + X @ beta)
    phi = 1.7
    y = rng.negative_binomial(phi, phi / (mu + phi)).astype(float)
    r = O.glm("neg_binomial_2_log", X, y, alpha, beta, phi)

    def f(a, b, p):
        return O.glm("neg_binomial_2_log", X, y, a, b, p)["lp"]

    h = 1e-6
    assert abs(r["dalpha"] - (f(alpha + h, beta, phi) - f(alpha - h, beta, phi)) / (2 * h)) <= 1e-6
    for j in range(3):
        e = np.zeros(3)
        e[j] = h
        fd = (f(alpha, beta + e, phi) - f(alpha, beta - e, phi)) / (2 * h)
        assert abs(r["dbeta"][j] - fd) <= 1e-6 * max(1.0, abs(fd))
    fd = (f(alpha, beta, phi + h) - f(alpha, beta, phi - h)) / (2 * h)
    assert abs(r["dsigma"] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_glm_categorical_matches_log_softmax_and_normalises():
    import scipy.special as sp
    rng = np.random.default_rng(8)
    n, k, C = 40, 3, 4
    X = rng.standard_normal((n, k))
    alpha, beta = rng.standard_normal(C), rng.standard_normal((k, C))
    y = rng.integers(0, C, n).astype(float)
    r = O.glm_categorical(X, y, alpha, beta)
    ls = sp.log_softmax(alpha + X @ beta, axis=1)
    assert abs(r["lp"] - ls[np.arange(n), y.astype(int)].sum()) <= 1e-12 * abs(r["lp"])
    # one observation: the class probabilities sum to one
    tot = sum(np.exp(O.glm_categorical(X[:1], [c], alpha, beta)["lp"]) for c in range(C))
    assert abs(tot - 1.0) <= 1e-14


def test_glm_categorical_two_classes_is_bernoulli_logit():
    rng, X, beta, alpha = glm_data(seed=9)
    y = (rng.random(len(X)) < 0.5).astype(float)
    rb = O.glm("bernoulli_logit", X, y, alpha, beta)
    rc = O.glm_categorical(X, y, [0.0, alpha], np.stack([np.zeros_like(beta), beta], axis=1))
    assert abs(rc["lp"] - rb["lp"]) <= 1e-12 * abs(rb["lp"])
    assert np.abs(rc["dbeta"][:, 1] - rb["dbeta"]).max() <= 1e-12
    assert abs(rc["dalpha"][1] - rb["dalpha"]) <= 1e-12


def test_glm_categorical_gradient_finite_differences():
    rng = np.random.default_rng(10)
    n, k, C = 25, 2, 3
    X = rng.standard_normal((n, k))
    alpha, beta = rng.standard_normal(C), rng.standard_normal((k, C))
    y = rng.integers(0, C, n).astype(float)
    r = O.glm_categorical(X, y, alpha, beta)
    h = 1e-6
    for c in range(C):
        e = np.zeros(C)
        e[c] = h
        fd = (O.glm_categorical(X, y, alpha + e, beta)["lp"] - O.glm_categorical(X, y, alpha - e, beta)["lp"]) / (2 * h)
        assert abs(r["dalpha"][c] - fd) <= 1e-6
        for j in range(k):
            E = np.zeros((k, C))
            E[j, c] = h
            fd = (O.glm_categorical(X, y, alpha, beta + E)["lp"] - O.glm_categorical(X, y, alpha, beta - E)["lp"]) / (2 * h)
            assert abs(r["dbeta"][j, c] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_glm_ordinal_normalises_and_two_classes_is_bernoulli_logit():
    rng, X, beta, alpha = glm_data(n=50, k=3, seed=11)
    cuts = np.array([-1.0, 0.2, 1.5])
    for i in range(5):
        tot = sum(np.exp(O.glm_ordinal(X[i:i + 1], [c], beta, cuts)["lp"]) for c in range(4))
        assert abs(tot - 1.0) <= 1e-14
    y = (rng.random(50) < 0.5).astype(float)
    ro = O.glm_ordinal(X, y, beta, [0.7])
    rb = O.glm("bernoulli_logit", X, y, -0.7, beta)
    assert abs(ro["lp"] - rb["lp"]) <= 1e-12 * abs(rb["lp"])
    assert np.abs(ro["dbeta"] - rb["dbeta"]).max() <= 1e-12
    assert abs(ro["dcuts"][0] + rb["dalpha"]) <= 1e-12


def test_glm_ordinal_gradient_finite_differences():
    rng = np.random.default_rng(12)
    n, k = 30, 2
    X = rng.standard_normal((n, k))
    beta, cuts = np.array([0.8, -0.5]), np.array([-1.2, -0.1, 0.9, 2.0])
    y = rng.integers(0, 5, n).astype(float)
    r = O.glm_ordinal(X, y, beta, cuts)
    h = 1e-6
    for j in range(k):
        e = np.zeros(k)
        e[j] = h
        fd = (O.glm_ordinal(X, y, beta + e, cuts)["lp"] - O.glm_ordinal(X, y, beta - e, cuts)["lp"]) / (2 * h)
        assert abs(r["dbeta"][j] - fd) <= 1e-6 * max(1.0, abs(fd))
    for m in range(4):
        e = np.zeros(4)
        e[m] = h
        fd = (O.glm_ordinal(X, y, beta, cuts + e)["lp"] - O.glm_ordinal(X, y, beta, cuts - e)["lp"]) / (2 * h)
        assert abs(r["dcuts"][m] - fd) <= 1e-6 * max(1.0, abs(fd))
