"""The multi-core CPU baseline (unblocked Cholesky and its reverse mode in
column order, OpenMP over the rows of each column) against the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W


@pytest.mark.parametrize("n", [1, 2, 7, 130, 300])
def test_cpu_baseline_matches_oracle(n):
    L0 = W.known_factor(n, seed=n)
    K = L0 @ L0.T
    Lbar = W.random_lower(n, seed=1)
    L = O.chol(K)
    assert np.linalg.norm(O.cpu_chol(K) - L) <= 1e-13 * np.linalg.norm(L)
    Kb = O.chol_adjoint(L, Lbar)
    assert np.linalg.norm(O.cpu_chol_adjoint(L, Lbar) - Kb) <= 1e-12 * np.linalg.norm(Kb)


@pytest.mark.parametrize("n", [1, 5, 63, 257, 1024])
def test_cpu_baseline_factor_is_bitwise_the_oracles(n):
    # the stand-in for the oracle's O(n^3) steps at full size: the same
    # recurrence, the same operations in the same order for every entry
    X = W.gp_inputs(n, 16, seed=n)
    K = O.se_cov(X, 1.0, 4.0, 0.05, 0.0)
    L = O.chol(K)
    assert np.array_equal(O.cpu_chol(K), L)
    Lbar = W.random_lower(n, seed=n + 1)
    Kb = O.chol_adjoint(L, Lbar)
    assert np.linalg.norm(O.cpu_chol_adjoint(L, Lbar) - Kb) <= 1e-13 * np.linalg.norm(Kb)


def test_multicore_pass_equals_oracle_pass():
    n = 300
    X = W.gp_inputs(n, 2, seed=0)
    y = W.gp_targets(X, 1.0, 0.5, 0.1, seed=1)
    a = O.gp_lml_and_grad(X, y, 1.0, 0.5, 0.1, 1e-8)
    b = O.gp_lml_and_grad_multicore(X, y, 1.0, 0.5, 0.1, 1e-8)
    assert np.array_equal(a["L"], b["L"]) and np.array_equal(a["K"], b["K"])
    assert a["value"] == b["value"] and a["logdet"] == b["logdet"]
    assert np.array_equal(a["alpha"], b["alpha"])
    assert np.linalg.norm(b["Kbar"] - a["Kbar"]) <= 1e-13 * np.linalg.norm(a["Kbar"])
    assert np.linalg.norm(b["grad"] - a["grad"]) <= 1e-12 * np.linalg.norm(a["grad"])


def test_cpu_baseline_reports_the_failing_pivot():
    K = np.eye(5)
    K[3, 3] = -1.0
    with pytest.raises(O.NotPositiveDefinite) as e:
        O.cpu_chol(K)
    assert e.value.info == 3
    assert O.cpu_threads() >= 1
