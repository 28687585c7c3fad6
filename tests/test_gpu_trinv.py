"""Triangular inverse, solve and solve adjoint (Section 3.2) against the oracle,
through the C ABI.

The matrices are Cholesky factors of jittered SE covariances (what a GP
prediction or a triangular-solve gradient inverts), so the condition numbers
are those of the method's workloads.  Sizes span several 128-wide diagonal
blocks and doubling levels with ragged last pairs (n not a power-of-two
multiple of 128).  Tolerance: relative Frobenius error <= 1e-10 (the FP64 bar
of the factorisation path); the strict upper triangle and any ld padding are
checked exactly.  At n = 16384 (the benchmark's size) sampled columns of the
inverse, of the solve and of the adjoint come from the oracle one column at a
time.
"""
import json
import os

import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10
HERE = os.path.dirname(os.path.abspath(__file__))


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def factor(n, seed=0, d=3, sigma=0.3):
    X = W.gp_inputs(n, d, seed)
    return O.chol(O.se_cov(X, 1.0, 1.0, sigma, 1e-6))


SIZES = [1, 2, 17, 64, 65, 127, 128, 129, 200, 255, 256, 257, 300, 383, 385, 513, 640, 1000, 1025]


@pytest.mark.parametrize("n", SIZES)
def test_tri_inverse_matches_oracle(n):
    L = factor(n, seed=n)
    ref = O.tri_inverse(L)
    X = gp.tri_inverse(dev(L)).cpu().numpy()
    print(f"n={n}: Linv {rel(X, ref):.3e}")
    assert rel(X, ref) <= TOL
    assert np.array_equal(np.triu(X, 1), np.zeros((n, n)))


@pytest.mark.parametrize("n", [65, 300, 1000])
def test_tri_inverse_padded_ld_in_place_and_upper_ignored(n):
    L = factor(n, seed=1)
    ref = O.tri_inverse(L)
    ld = n + 5
    # out of place into a padded buffer: the padding columns are not touched
    buf = torch.full((n, ld), float("nan"), dtype=torch.float64, device="cuda")
    gp.tri_inverse(dev(L), out=buf[:, :n])
    out = buf.cpu().numpy()
    assert rel(out[:, :n], ref) <= TOL
    assert np.isnan(out[:, n:]).all()
    # in place, with junk in the strict upper triangle of the input
    Lj = L + np.triu(np.full((n, n), 7.0), 1)
    big = torch.full((n, ld), -3.0, dtype=torch.float64, device="cuda")
    big[:, :n] = dev(Lj)
    Lv = big[:, :n]
    gp.tri_inverse(Lv, out=Lv)
    got = big.cpu().numpy()
    assert rel(got[:, :n], ref) <= TOL
    assert np.array_equal(np.triu(got[:, :n], 1), np.zeros((n, n)))
    assert (got[:, n:] == -3.0).all()


@pytest.mark.parametrize("n,m", [(1, 1), (65, 3), (129, 64), (300, 100), (513, 1), (1000, 130)])
def test_tri_solve_matches_oracle(n, m):
    L = factor(n, seed=2)
    B = np.random.default_rng(n + m).standard_normal((n, m))
    ref = O.tri_solve(L, B)
    C, X = gp.tri_solve(dev(L), dev(B))
    print(f"n={n} m={m}: C {rel(C.cpu().numpy(), ref):.3e}")
    assert rel(C.cpu().numpy(), ref) <= TOL
    assert rel(X.cpu().numpy(), O.tri_inverse(L)) <= TOL


@pytest.mark.parametrize("n,m", [(1, 1), (65, 3), (129, 64), (300, 100), (1000, 130)])
def test_tri_solve_adjoint_matches_oracle(n, m):
    L = factor(n, seed=3)
    rng = np.random.default_rng(n * m)
    B = rng.standard_normal((n, m))
    Cbar = rng.standard_normal((n, m))
    C0 = O.tri_solve(L, B)
    Bb0, Lb0 = O.tri_solve_adjoint(L, C0, Cbar)
    C, X = gp.tri_solve(dev(L), dev(B))
    Bb, Lb = gp.tri_solve_adjoint(X, C, dev(Cbar))
    Bb, Lb = Bb.cpu().numpy(), Lb.cpu().numpy()
    print(f"n={n} m={m}: Bbar {rel(Bb, Bb0):.3e} Lbar {rel(Lb, Lb0):.3e}")
    assert rel(Bb, Bb0) <= TOL
    assert rel(Lb, Lb0) <= TOL
    assert np.array_equal(np.triu(Lb, 1), np.zeros((n, n)))


def test_tri_solve_adjoint_overwrites_outputs():
    # outputs filled with NaN beforehand: nothing of their old contents is read
    n, m = 257, 9
    L = factor(n, seed=4)
    rng = np.random.default_rng(5)
    B, Cbar = rng.standard_normal((n, m)), rng.standard_normal((n, m))
    Bb0, Lb0 = O.tri_solve_adjoint(L, O.tri_solve(L, B), Cbar)
    C, X = gp.tri_solve(dev(L), dev(B))
    Bb = torch.full((n, m), float("nan"), dtype=torch.float64, device="cuda")
    Lb = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    gp.tri_solve_adjoint(X, C, dev(Cbar), Bbar=Bb, Lbar=Lb)
    Bb, Lb = Bb.cpu().numpy(), Lb.cpu().numpy()
    assert rel(Bb, Bb0) <= TOL
    assert rel(Lb, Lb0) <= TOL
    assert np.array_equal(np.triu(Lb, 1), np.zeros((n, n)))


def test_autograd_tri_solve_matches_oracle():
    n, m = 200, 7
    L = factor(n, seed=6)
    rng = np.random.default_rng(7)
    B, Wt = rng.standard_normal((n, m)), rng.standard_normal((n, m))
    Lt = dev(L).requires_grad_(True)
    Bt = dev(B).requires_grad_(True)
    f = (gp.mdivide_left_tri_low(Lt, Bt) * dev(Wt)).sum()
    f.backward()
    Bb0, Lb0 = O.tri_solve_adjoint(L, O.tri_solve(L, B), Wt)
    assert abs(f.item() - float(np.sum(Wt * O.tri_solve(L, B)))) <= 1e-12 * max(1.0, abs(f.item()))
    assert rel(Bt.grad.cpu().numpy(), Bb0) <= TOL
    assert rel(Lt.grad.cpu().numpy(), Lb0) <= TOL
    # a vector right-hand side
    b = dev(B[:, 0]).requires_grad_(True)
    Lt.grad = None
    c = gp.mdivide_left_tri_low(Lt, b)
    assert c.shape == (n,)
    (c * dev(Wt[:, 0])).sum().backward()
    bb0, lb0 = O.tri_solve_adjoint(L, O.tri_solve(L, B[:, :1]), Wt[:, :1])
    assert rel(b.grad.cpu().numpy(), bb0[:, 0]) <= TOL
    assert rel(Lt.grad.cpu().numpy(), lb0) <= TOL


def test_zero_width_right_hand_side():
    n = 130
    L = factor(n, seed=8)
    C, X = gp.tri_solve(dev(L), torch.empty(n, 0, dtype=torch.float64, device="cuda"))
    assert C.shape == (n, 0)
    assert rel(X.cpu().numpy(), O.tri_inverse(L)) <= TOL
    Bb, Lb = gp.tri_solve_adjoint(X, C, torch.empty(n, 0, dtype=torch.float64, device="cuda"))
    assert (Lb.cpu().numpy() == 0.0).all()


def test_fullsize_16384_sampled_columns():
    """n = 16384: sampled columns of L^{-1}, of L^{-1} B and of the adjoint from
    the oracle, one column at a time, for the seeded known factor (diag U(1, 2),
    strictly lower N(0, 1/n)); and, for the factor of the benchmark's SE
    covariance (d = 16, condition ~1e5), the residual L x_j = e_j of sampled
    columns (a property that holds at any size)."""
    n = 16384
    Lh = W.known_factor(n, seed=0)
    L = dev(Lh)
    cols = [0, 4095, 8191, 12345, n - 1]
    E = np.zeros((n, len(cols)))
    E[cols, range(len(cols))] = 1.0
    ref_cols = O.tri_solve(Lh, E)  # column j of L^{-1}
    Linv = torch.empty_like(L)
    gp.tri_inverse(L, out=Linv)
    got = Linv[:, cols].cpu().numpy()
    errs = [rel(got[:, t], ref_cols[:, t]) for t in range(len(cols))]
    print(f"n={n}: sampled Linv columns {max(errs):.3e}")
    assert max(errs) <= TOL
    assert int(torch.count_nonzero(Linv.triu(1))) == 0
    # a two-column solve and its adjoint
    rng = np.random.default_rng(11)
    B, Cbar = rng.standard_normal((n, 2)), rng.standard_normal((n, 2))
    C, Xs = gp.tri_solve(L, dev(B), Linv=Linv)
    C0 = O.tri_solve(Lh, B)
    assert rel(C.cpu().numpy(), C0) <= TOL
    Bb, Lb = gp.tri_solve_adjoint(Xs, C, dev(Cbar))
    Bb0 = np.stack([O.trsv(Lh, Cbar[:, t], trans=True) for t in range(2)], axis=1)
    assert rel(Bb.cpu().numpy(), Bb0) <= TOL
    rows = [0, 1, 777, 8192, n - 1]
    Lb_rows = Lb[rows].cpu().numpy()
    for t, r in enumerate(rows):
        ref = -(Bb0[r] @ C0[: r + 1].T)  # Lbar_rj = -sum_t Bbar_rt C_jt for j <= r
        assert rel(Lb_rows[t, : r + 1], ref) <= TOL
        assert (Lb_rows[t, r + 1:] == 0.0).all()
    del L, Linv, Lb, C, Xs, Bb
    torch.cuda.empty_cache()

    rec = json.load(open(os.path.join(HERE, "golden", "cond_sigma.json")))
    assert rec["n"] == n
    K = gp.se_cov(dev(W.gp_inputs(n, rec["d"], seed=0)), rec["alpha"], rec["rho"], rec["sigma"], 0.0)
    Lse = gp.chol(K, out=K)
    Xse = gp.tri_inverse(Lse)
    Lh = Lse.cpu().numpy()
    Xc = Xse[:, cols].cpu().numpy()
    for t, j in enumerate(cols):
        r = Lh @ Xc[:, t]
        r[j] -= 1.0
        bound = 1e-13 * np.linalg.norm(Lh[j:, j:], 1) * np.linalg.norm(Xc[:, t], 1)
        assert np.linalg.norm(r, 1) <= bound, (j, np.linalg.norm(r, 1), bound)
    del K, Lse, Xse
    torch.cuda.empty_cache()
