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


def test_cpu_baseline_reports_the_failing_pivot():
    K = np.eye(5)
    K[3, 3] = -1.0
    with pytest.raises(O.NotPositiveDefinite) as e:
        O.cpu_chol(K)
    assert e.value.info == 3
    assert O.cpu_threads() >= 1
