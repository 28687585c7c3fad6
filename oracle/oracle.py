"""NumPy/ctypes front end of the plain FP64 CPU oracle (``gpchol_oracle.c``) and
of the multi-core CPU baseline (``cpu_baseline.c``, timed by the benchmark).

This is test infrastructure: only the tests, the smoke check and the
benchmark's CPU-baseline leg import it.  It shares nothing with the GPU
library.  Every function takes and returns float64 NumPy arrays (row-major);
the arithmetic lives in the C file, compiled with ``-O2 -ffp-contract=off``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpchol_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "libgpchol_oracle.so")
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build``; returns the library path."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC))
    if force or stale:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_CPU_SRC = os.path.join(_HERE, "cpu_baseline.c")
_CPU_LIB_PATH = os.path.join(_HERE, "_build", "libgpchol_cpu_baseline.so")
_cpu_lib = None


def build_cpu_baseline(force: bool = False) -> str:
    """Compile the multi-core CPU baseline (OpenMP) into ``oracle/_build``."""
    os.makedirs(os.path.dirname(_CPU_LIB_PATH), exist_ok=True)
    stale = (not os.path.exists(_CPU_LIB_PATH)
             or os.path.getmtime(_CPU_LIB_PATH) < os.path.getmtime(_CPU_SRC))
    if force or stale:
        tmp = _CPU_LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-std=c11",
                               "-shared", "-fPIC", "-o", tmp, _CPU_SRC, "-lm"])
        os.replace(tmp, _CPU_LIB_PATH)
    return _CPU_LIB_PATH


def _load_cpu():
    global _cpu_lib
    if _cpu_lib is None:
        lib = ctypes.CDLL(build_cpu_baseline())
        i = ctypes.c_int
        lib.cpu_baseline_threads.argtypes = []
        lib.cpu_baseline_threads.restype = i
        lib.cpu_baseline_chol.argtypes = [i, _D, _D]
        lib.cpu_baseline_chol.restype = i
        lib.cpu_baseline_chol_adjoint.argtypes = [i, _D, _D, _D]
        lib.cpu_baseline_chol_adjoint.restype = i
        _cpu_lib = lib
    return _cpu_lib


def cpu_threads() -> int:
    """Threads the multi-core CPU baseline uses."""
    return int(_load_cpu().cpu_baseline_threads())


def cpu_chol(K) -> np.ndarray:
    """Multi-core CPU baseline Cholesky (column order, rows of a column in parallel)."""
    K = _mat(K)
    n = K.shape[0]
    L = np.zeros_like(K)
    info = _load_cpu().cpu_baseline_chol(n, _p(K), _p(L))
    if info >= 0:
        raise NotPositiveDefinite(info)
    return L


def cpu_chol_adjoint(L, Lbar) -> np.ndarray:
    """Multi-core CPU baseline reverse mode of cpu_chol."""
    L, Lbar = _mat(L), _mat(Lbar)
    Kbar = np.zeros_like(L)
    if _load_cpu().cpu_baseline_chol_adjoint(L.shape[0], _p(L), _p(Lbar), _p(Kbar)) != 0:
        raise MemoryError("scratch allocation failed")
    return Kbar


def _load():
    global _lib
    if _lib is None:
        # GPCHOL_ORACLE_LIB lets the mutation test load a deliberately broken copy.
        lib = ctypes.CDLL(os.environ.get("GPCHOL_ORACLE_LIB") or build())
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_chol.argtypes = [i, _D, i, _D, i]
        lib.oracle_chol.restype = i
        lib.oracle_chol_adjoint.argtypes = [i, _D, i, _D, i, _D, i]
        lib.oracle_chol_adjoint.restype = i
        lib.oracle_chol_adjoint_symbolic.argtypes = [i, _D, i, _D, i, _D, i]
        lib.oracle_chol_adjoint_symbolic.restype = i
        lib.oracle_trsv.argtypes = [i, _D, i, _D, i]
        lib.oracle_trsv.restype = None
        lib.oracle_se_cov.argtypes = [i, i, _D, i, d, d, d, d, _D, i, i]
        lib.oracle_se_cov.restype = None
        lib.oracle_gp_lml.argtypes = [i, _D, i, _D, _D, i, _D, _D, _D, _D]
        lib.oracle_gp_lml.restype = i
        lib.oracle_gp_lml_factored.argtypes = [i, _D, i, _D, _D, _D, _D, _D]
        lib.oracle_gp_lml_factored.restype = i
        lib.oracle_lml_lbar.argtypes = [i, _D, i, _D, _D, d, _D, i]
        lib.oracle_lml_lbar.restype = None
        lib.oracle_se_hyper_grad.argtypes = [i, i, _D, i, d, d, d, _D, i, _D]
        lib.oracle_se_hyper_grad.restype = None
        lib.oracle_tri_inverse.argtypes = [i, _D, i, _D, i]
        lib.oracle_tri_inverse.restype = None
        lib.oracle_tri_solve.argtypes = [i, i, _D, i, _D, i, _D, i]
        lib.oracle_tri_solve.restype = None
        lib.oracle_tri_solve_adjoint.argtypes = [i, i, _D, i, _D, i, _D, i, _D, i, _D, i]
        lib.oracle_tri_solve_adjoint.restype = None
        lib.oracle_gemm.argtypes = [i, i, i, _D, i, _D, i, _D, i]
        lib.oracle_gemm.restype = None
        lib.oracle_gemm_adjoint.argtypes = [i, i, i, _D, i, _D, i, _D, i, _D, i, _D, i]
        lib.oracle_gemm_adjoint.restype = None
        lib.oracle_glm.argtypes = [i, i, i, _D, i, _D, d, _D, d, _D, _D, _D, _D]
        lib.oracle_glm.restype = i
        lib.oracle_psi.argtypes = [d]
        lib.oracle_psi.restype = d
        lib.oracle_glm_categorical.argtypes = [i, i, i, _D, i, _D, _D, _D, _D, _D, _D]
        lib.oracle_glm_categorical.restype = i
        lib.oracle_glm_ordinal.argtypes = [i, i, i, _D, i, _D, _D, _D, _D, _D, _D]
        lib.oracle_glm_ordinal.restype = None
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_D)


def _mat(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[0] != a.shape[1]:
        raise ValueError("expected a square matrix")
    return a


class NotPositiveDefinite(ValueError):
    def __init__(self, info: int):
        super().__init__(f"matrix is not positive definite (pivot {info})")
        self.info = info


def chol(K) -> np.ndarray:
    """Lower Cholesky factor (Cholesky-Banachiewicz); raises on a failing pivot."""
    K = _mat(K)
    n = K.shape[0]
    L = np.zeros_like(K)
    info = _load().oracle_chol(n, _p(K), n, _p(L), n)
    if info >= 0:
        raise NotPositiveDefinite(info)
    return L


def chol_info(K) -> tuple[np.ndarray, int]:
    """As ``chol`` but returns (partial L, info) with info = -1 on success."""
    K = _mat(K)
    n = K.shape[0]
    L = np.zeros_like(K)
    info = _load().oracle_chol(n, _p(K), n, _p(L), n)
    return L, int(info)


def chol_adjoint(L, Lbar) -> np.ndarray:
    """Unblocked reverse mode of ``chol``: Kbar (lower) from L and Lbar."""
    L, Lbar = _mat(L), _mat(Lbar)
    n = L.shape[0]
    Kbar = np.zeros_like(L)
    if _load().oracle_chol_adjoint(n, _p(L), n, _p(Lbar), n, _p(Kbar), n) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return Kbar


def chol_adjoint_symbolic(L, Lbar) -> np.ndarray:
    """Symbolic adjoint L^{-T} Phi(L^T Lbar) L^{-1}, folded to the lower convention."""
    L, Lbar = _mat(L), _mat(Lbar)
    n = L.shape[0]
    Kbar = np.zeros_like(L)
    if _load().oracle_chol_adjoint_symbolic(n, _p(L), n, _p(Lbar), n, _p(Kbar), n) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return Kbar


def trsv(L, x, trans: bool = False) -> np.ndarray:
    """L^{-1} x (trans False) or L^{-T} x (trans True) by substitution."""
    L = _mat(L)
    out = np.array(x, dtype=np.float64, copy=True)
    _load().oracle_trsv(L.shape[0], _p(L), L.shape[0], _p(out), 1 if trans else 0)
    return out


def tri_inverse(L) -> np.ndarray:
    """L^{-1} of a lower-triangular L, column by column from L X = I."""
    L = _mat(L)
    n = L.shape[0]
    X = np.zeros_like(L)
    _load().oracle_tri_inverse(n, _p(L), n, _p(X), n)
    return X


def _rect(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1:
        a = a.reshape(-1, 1).copy()
    if a.ndim != 2:
        raise ValueError("expected a matrix or a vector")
    return a


def tri_solve(L, B) -> np.ndarray:
    """C = L^{-1} B (L lower, B n x m) by forward substitution."""
    L = _mat(L)
    B = _rect(B)
    n, m = B.shape
    if n != L.shape[0]:
        raise ValueError("shape mismatch")
    C = np.zeros_like(B)
    _load().oracle_tri_solve(n, m, _p(L), n, _p(B), m, _p(C), m)
    return C


def tri_solve_adjoint(L, C, Cbar):
    """(Bbar, Lbar) of C = L^{-1} B given Cbar: L^{-T} Cbar and -tril(Bbar C^T)."""
    L = _mat(L)
    C, Cbar = _rect(C), _rect(Cbar)
    n, m = C.shape
    if Cbar.shape != C.shape or n != L.shape[0]:
        raise ValueError("shape mismatch")
    Bbar = np.zeros_like(C)
    Lbar = np.zeros_like(L)
    _load().oracle_tri_solve_adjoint(n, m, _p(L), n, _p(C), m, _p(Cbar), m, _p(Bbar), m, _p(Lbar), n)
    return Bbar, Lbar


def gemm(A, B) -> np.ndarray:
    """C = A B by the plain triple loop."""
    A, B = _rect(A), _rect(B)
    m, k = A.shape
    if B.shape[0] != k:
        raise ValueError("shape mismatch")
    n = B.shape[1]
    C = np.zeros((m, n))
    _load().oracle_gemm(m, n, k, _p(A), k, _p(B), n, _p(C), n)
    return C


def gemm_adjoint(A, B, Cbar):
    """(Abar, Bbar) = (Cbar B^T, A^T Cbar) for C = A B."""
    A, B, Cbar = _rect(A), _rect(B), _rect(Cbar)
    m, k = A.shape
    n = B.shape[1]
    if B.shape[0] != k or Cbar.shape != (m, n):
        raise ValueError("shape mismatch")
    Abar, Bbar = np.zeros((m, k)), np.zeros((k, n))
    _load().oracle_gemm_adjoint(m, n, k, _p(A), k, _p(B), n, _p(Cbar), n, _p(Abar), k, _p(Bbar), n)
    return Abar, Bbar


GLM_FAMILIES = {"normal_id": 0, "bernoulli_logit": 1, "poisson_log": 2, "neg_binomial_2_log": 3}


def psi(x: float) -> float:
    """Digamma (recurrence to x >= 12, then the asymptotic series)."""
    return float(_load().oracle_psi(float(x)))


def glm(family: str, X, y, alpha: float, beta, sigma: float = 1.0) -> dict:
    """GLM log likelihood and gradient: dict(lp, dalpha, dbeta, dsigma); for the
    negative binomial, sigma is the dispersion phi and dsigma is d lp / d phi."""
    X = _rect(X)
    n, k = X.shape
    y = np.ascontiguousarray(y, dtype=np.float64)
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    if y.shape != (n,) or beta.shape != (k,):
        raise ValueError("shape mismatch")
    lp, da, ds = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    db = np.zeros(k)
    if _load().oracle_glm(GLM_FAMILIES[family], n, k, _p(X), k, _p(y), float(alpha), _p(beta), float(sigma),
                          ctypes.byref(lp), ctypes.byref(da), _p(db), ctypes.byref(ds)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return {"lp": lp.value, "dalpha": da.value, "dbeta": db, "dsigma": ds.value}


def glm_categorical(X, y, alpha, beta) -> dict:
    """Categorical-logit GLM: y in {0..C-1}, alpha (C), beta (k x C); dict(lp, dalpha, dbeta)."""
    X = _rect(X)
    n, k = X.shape
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    C = alpha.shape[0]
    beta = np.ascontiguousarray(beta, dtype=np.float64).reshape(k, C)
    y = np.ascontiguousarray(y, dtype=np.float64)
    if y.shape != (n,):
        raise ValueError("shape mismatch")
    lp = ctypes.c_double()
    da, db = np.zeros(C), np.zeros((k, C))
    if _load().oracle_glm_categorical(n, k, C, _p(X), k, _p(y), _p(alpha), _p(beta), ctypes.byref(lp), _p(da),
                                      _p(db)) != 0:
        raise MemoryError("oracle scratch allocation failed")
    return {"lp": lp.value, "dalpha": da, "dbeta": db}


def glm_ordinal(X, y, beta, cuts) -> dict:
    """Ordinal-logit GLM: y in {0..C-1}, increasing cuts (C-1), beta (k); dict(lp, dbeta, dcuts)."""
    X = _rect(X)
    n, k = X.shape
    beta = np.ascontiguousarray(beta, dtype=np.float64)
    cuts = np.ascontiguousarray(cuts, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    C = cuts.shape[0] + 1
    lp = ctypes.c_double()
    db, dc = np.zeros(k), np.zeros(C - 1)
    _load().oracle_glm_ordinal(n, k, C, _p(X), k, _p(y), _p(beta), _p(cuts), ctypes.byref(lp), _p(db), _p(dc))
    return {"lp": lp.value, "dbeta": db, "dcuts": dc}


def se_cov(X, alpha: float, rho: float, sigma: float, jitter: float = 0.0,
           full: bool = False) -> np.ndarray:
    """Squared-exponential covariance of the rows of X (n x d)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, d = X.shape
    K = np.zeros((n, n))
    _load().oracle_se_cov(n, d, _p(X), d, alpha, rho, sigma, jitter, _p(K), n, 1 if full else 0)
    return K


def gp_lml(K, y):
    """Returns dict(L, z, alpha, logdet, value) for y ~ N(0, K)."""
    K = _mat(K)
    n = K.shape[0]
    y = np.ascontiguousarray(y, dtype=np.float64)
    L = np.zeros_like(K)
    z = np.zeros(n)
    a = np.zeros(n)
    ld = ctypes.c_double()
    val = ctypes.c_double()
    info = _load().oracle_gp_lml(n, _p(K), n, _p(y), _p(L), n, _p(z), _p(a),
                                 ctypes.byref(ld), ctypes.byref(val))
    if info == -2:
        raise MemoryError("oracle scratch allocation failed")
    if info >= 0:
        raise NotPositiveDefinite(info)
    return {"L": L, "z": z, "alpha": a, "logdet": ld.value, "value": val.value}


def gp_lml_factored(L, y):
    """The steps of gp_lml after the factorisation, for a given factor L:
    dict(z, alpha, logdet, value)."""
    L = _mat(L)
    n = L.shape[0]
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.zeros(n)
    a = np.zeros(n)
    ld = ctypes.c_double()
    val = ctypes.c_double()
    if _load().oracle_gp_lml_factored(n, _p(L), n, _p(y), _p(z), _p(a), ctypes.byref(ld),
                                      ctypes.byref(val)) == -2:
        raise MemoryError("oracle scratch allocation failed")
    return {"z": z, "alpha": a, "logdet": ld.value, "value": val.value}


def lml_lbar(L, alpha, z, gbar: float = 1.0) -> np.ndarray:
    """Upstream Lbar = gbar (tril(alpha z^T) - diag(1/L_ii))."""
    L = _mat(L)
    n = L.shape[0]
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    Lbar = np.zeros_like(L)
    _load().oracle_lml_lbar(n, _p(L), n, _p(alpha), _p(z), gbar, _p(Lbar), n)
    return Lbar


def se_hyper_grad(X, alpha: float, rho: float, sigma: float, Kbar) -> np.ndarray:
    """(d/d alpha, d/d rho, d/d sigma) of f given Kbar = df/dK (lower convention)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    Kbar = _mat(Kbar)
    n, d = X.shape
    g = np.zeros(3)
    _load().oracle_se_hyper_grad(n, d, _p(X), d, alpha, rho, sigma, _p(Kbar), n, _p(g))
    return g


def gp_lml_and_grad(X, y, alpha: float, rho: float, sigma: float, jitter: float = 0.0):
    """Full oracle pass: K, chol, LML, Lbar, Kbar and hyperparameter gradient."""
    K = se_cov(X, alpha, rho, sigma, jitter)
    r = gp_lml(K, y)
    Lbar = lml_lbar(r["L"], r["alpha"], r["z"], 1.0)
    Kbar = chol_adjoint(r["L"], Lbar)
    g = se_hyper_grad(X, alpha, rho, sigma, Kbar)
    r.update({"K": K, "Lbar": Lbar, "Kbar": Kbar, "grad": g})
    return r


def gp_lml_and_grad_multicore(X, y, alpha: float, rho: float, sigma: float, jitter: float = 0.0):
    """The pass of gp_lml_and_grad with its two O(n^3) steps taken by the
    multi-core unblocked routines of cpu_baseline.c, for sizes the
    single-threaded oracle cannot finish in test time (n = 16384: about two
    minutes on 16 cores instead of half an hour).  cpu_chol runs the oracle's
    recurrence with the same operations in the same order for every entry, so
    its factor is bitwise equal to chol's; cpu_chol_adjoint runs the same
    statements with the rows of a column summed in another order (within
    1e-13 of chol_adjoint).  tests/test_cpu_baseline.py checks both.  Every
    other step is the oracle's own."""
    K = se_cov(X, alpha, rho, sigma, jitter)
    L = cpu_chol(K)
    r = gp_lml_factored(L, y)
    Lbar = lml_lbar(L, r["alpha"], r["z"], 1.0)
    Kbar = cpu_chol_adjoint(L, Lbar)
    del Lbar
    g = se_hyper_grad(X, alpha, rho, sigma, Kbar)
    r.update({"K": K, "L": L, "Kbar": Kbar, "grad": g})
    return r
