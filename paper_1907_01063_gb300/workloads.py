"""Seeded synthetic inputs for the Cholesky / GP-likelihood workloads.

This module only draws random numbers and lays them out; it holds none of the
arithmetic of the method (no covariance, factorisation, solve or adjoint), so
both the GPU tests and the CPU oracle can take their inputs from it.  All
draws come from ``torch.Generator`` on the CPU and are returned as float64
NumPy arrays.

Recipes
-------
* GP inputs: X ~ N(0, 1), n x d.
* GP targets: an approximate draw from a zero-mean GP with the
  squared-exponential covariance, by random Fourier features
  (Rahimi & Recht 2007): f(x) = alpha sqrt(2/D) sum_r cos(w_r . x + b_r),
  w_r ~ N(0, I / rho^2), b_r ~ U(0, 2 pi), plus sigma eps, eps ~ N(0, 1).
* Known factor: L0 lower, diagonal ~ U(1, 2), strictly lower ~ N(0, 1/n).
* The paper's Toeplitz SPD test matrix (Section 3.3, speedup measurements):
  A_ij = n - |i - j| off the diagonal, A_ii = n^2.
* Random adjoints: W ~ N(0, 1) in the lower triangle.
* Batches of GPs: n_i ~ U{lo..hi} inclusive, rho_i ~ U(rho_lo, rho_hi).
* The paper's 1-D GP regression data (Section 4.2): x ~ U(-10, 10),
  y ~ N(f(x), 1/10) with f(x) = x + x^2 - x^3 + 100 sin(2x) shifted and scaled
  to mean 0 and variance 1 (the sample's own mean and variance stand in for
  the unstated constants).
"""
from __future__ import annotations

import math

import numpy as np
import torch


def _gen(seed: int) -> torch.Generator:
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    return g


def gp_inputs(n: int, d: int, seed: int = 0) -> np.ndarray:
    """X ~ N(0, 1) with shape (n, d)."""
    return torch.randn(n, d, generator=_gen(seed), dtype=torch.float64).numpy()


def gp_targets(X: np.ndarray, alpha: float, rho: float, sigma: float, seed: int = 1,
               features: int = 512) -> np.ndarray:
    """Approximate GP draw at the rows of X (random Fourier features) plus noise."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    g = _gen(seed)
    w = torch.randn(d, features, generator=g, dtype=torch.float64).numpy() / rho
    b = torch.rand(features, generator=g, dtype=torch.float64).numpy() * (2.0 * math.pi)
    eps = torch.randn(n, generator=g, dtype=torch.float64).numpy()
    f = alpha * math.sqrt(2.0 / features) * np.cos(X @ w + b).sum(axis=1)
    return f + sigma * eps


def known_factor(n: int, seed: int = 0) -> np.ndarray:
    """Lower-triangular L0 with diag ~ U(1, 2) and strictly-lower ~ N(0, 1/n)."""
    g = _gen(seed)
    off = torch.randn(n, n, generator=g, dtype=torch.float64).numpy() / math.sqrt(max(n, 1))
    diag = 1.0 + torch.rand(n, generator=g, dtype=torch.float64).numpy()
    L0 = np.tril(off, -1)
    L0[np.arange(n), np.arange(n)] = diag
    return L0


def toeplitz_spd(n: int) -> np.ndarray:
    """A_ij = n - |i - j| (i != j), A_ii = n^2."""
    i = np.arange(n)
    A = (n - np.abs(i[:, None] - i[None, :])).astype(np.float64)
    A[i, i] = float(n) * float(n)
    return A


def random_lower(n: int, seed: int = 0) -> np.ndarray:
    """W ~ N(0, 1) in the lower triangle, zero above."""
    W = torch.randn(n, n, generator=_gen(seed), dtype=torch.float64).numpy()
    return np.tril(W)


def batch_sizes(batch: int, lo: int, hi: int, seed: int = 0) -> np.ndarray:
    """n_i ~ U{lo..hi} inclusive, int64."""
    return torch.randint(lo, hi + 1, (batch,), generator=_gen(seed)).numpy().astype(np.int64)


def batch_lengthscales(batch: int, lo: float, hi: float, seed: int = 1) -> np.ndarray:
    """rho_i ~ U(lo, hi)."""
    return lo + (hi - lo) * torch.rand(batch, generator=_gen(seed), dtype=torch.float64).numpy()


def paper_gp_1d(n: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """The 1-D regression data of Section 4.2 as (x with shape (n, 1), y)."""
    g = _gen(seed)
    x = -10.0 + 20.0 * torch.rand(n, generator=g, dtype=torch.float64).numpy()
    f = x + x ** 2 - x ** 3 + 100.0 * np.sin(2.0 * x)
    f = (f - f.mean()) / max(f.std(), 1e-300)
    y = f + math.sqrt(0.1) * torch.randn(n, generator=g, dtype=torch.float64).numpy()
    return x[:, None], y


def glm_data(n: int, k: int, family: str = "bernoulli_logit", seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """Toy GLM data after the logistic-regression experiment of Section 4.1:
    X ~ N(0, 1) (n x k, k >= 2), latent mu_i = 3 X_i1 - 2 X_i2 + 1 (the other
    columns are noise); y_i ~ Bernoulli(1 / (1 + e^-mu_i)).  The Poisson-log
    and normal-identity variants use the same X with y_i ~ Poisson(e^(mu_i / 4))
    and y_i ~ N(mu_i, 1)."""
    g = _gen(seed)
    X = torch.randn(n, k, generator=g, dtype=torch.float64).numpy()
    mu = 3.0 * X[:, 0] - 2.0 * X[:, 1] + 1.0 if k >= 2 else np.ones(n)
    u = torch.rand(n, generator=g, dtype=torch.float64).numpy()
    if family == "bernoulli_logit":
        y = (u < 1.0 / (1.0 + np.exp(-mu))).astype(np.float64)
    elif family == "poisson_log":
        y = torch.poisson(torch.as_tensor(np.exp(mu / 4.0)), generator=g).numpy().astype(np.float64)
    else:
        y = mu + torch.randn(n, generator=g, dtype=torch.float64).numpy()
    return X, y

