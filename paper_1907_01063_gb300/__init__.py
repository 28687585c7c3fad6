"""GB300 (sm_103a) Cholesky, Cholesky adjoint and Gaussian-process likelihood.

Python binding of libgpchol.so (C ABI in include/gpchol.h).  The binding only
marshals arguments: every step runs in the library's CUDA kernels on the
current torch stream.  PyTorch supplies device memory and streams.

Two layers:
  * ``capi`` -- the C entry points with their C names (``capi.gpc_chol`` ...),
    taking raw integers for pointers and streams;
  * tensor functions with the same names minus the prefix (``chol``,
    ``chol_adjoint``, ``gp_lml``, ``tri_solve``, ``gemm``, ``glm`` ...) and the
    autograd functions ``Chol``, ``GPLml``, ``TriSolve``, ``MatMul`` and ``GLMLpmf``.
There is no CPU fallback: without the compiled library every call raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

GPC_OK = 0
GPC_ERR_INVALID_ARG = 1
GPC_ERR_NOT_PD = 2
GPC_ERR_NAN = 3
GPC_ERR_CUDA = 4
GPC_ERR_TIMEOUT = 5
GPC_ERR_NO_CONVERGENCE = 6
GPC_FP64 = 0
GPC_MIXED = 1
GPC_TUNE_BLOCK = 0
GPC_TUNE_SLICES = 1
GPC_TUNE_SPLITK_MIN = 2
GPC_TUNE_BATCH_BLOCK = 3
GPC_TUNE_MIXED_DEFER = 4
GPC_TUNE_MIXED_FREE_SMS = 5
GPC_TUNE_MIXED_CTA_ITEMS = 6
GPC_TUNE_MIXED_PRIORITY = 7
GPC_TUNE_MIXED_ADJ_FREE_SMS = 8
GPC_TUNE_F64_SMALL_TILE = 9

PRECISIONS = {"fp64": GPC_FP64, "mixed": GPC_MIXED, GPC_FP64: GPC_FP64, GPC_MIXED: GPC_MIXED}

_c_int, _c_double, _c_size, _c_vp = ctypes.c_int, ctypes.c_double, ctypes.c_size_t, ctypes.c_void_p

# name -> (argtypes, restype)
_SIGNATURES = {
    "gpc_status_string": ([_c_int], ctypes.c_char_p),
    "gpc_get_error": ([ctypes.POINTER(_c_int), _c_int, _c_vp], _c_int),
    "gpc_test_set_fault": ([_c_int, ctypes.c_longlong], _c_int),
    "gpc_test_recip_rsqrt": ([_c_int, _c_vp, _c_vp, _c_vp], _c_int),
    "gpc_test_split_f64": ([_c_int, _c_vp, _c_vp, _c_vp, _c_vp], _c_int),
    "gpc_version": ([], _c_int),
    "gpc_workspace_size": ([_c_int, _c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_set_tuning": ([_c_int, _c_int], _c_int),
    "gpc_get_tuning": ([_c_int, ctypes.POINTER(_c_int)], _c_int),
    "gpc_se_cov": ([_c_int, _c_int, _c_vp, _c_int, _c_double, _c_double, _c_double, _c_double,
                    _c_vp, _c_int, _c_int, _c_int, _c_vp], _c_int),
    "gpc_chol": ([_c_int, _c_vp, _c_int, _c_vp, _c_int, _c_int, _c_vp, _c_size, _c_vp, _c_vp], _c_int),
    "gpc_chol_adjoint": ([_c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_int, _c_int,
                          _c_vp, _c_size, _c_vp], _c_int),
    "gpc_trsv": ([_c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_trsv_noalloc": ([_c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp], _c_int),
    "gpc_tri_inverse": ([_c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp], _c_int),
    "gpc_gemm_workspace_size": ([ctypes.POINTER(_c_size)], _c_int),
    "gpc_gemm": ([_c_int, _c_int, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_size, _c_vp],
                 _c_int),
    "gpc_gemm_adjoint": ([_c_int, _c_int, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int,
                          _c_vp, _c_int, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_glm_workspace_size": ([_c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_glm": ([_c_int, ctypes.c_longlong, _c_int, _c_vp, ctypes.c_longlong, _c_vp, _c_double, _c_vp, _c_double,
                 _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_glm_ordinal": ([ctypes.c_longlong, _c_int, _c_int, _c_vp, ctypes.c_longlong, _c_vp, _c_vp, _c_vp, _c_vp,
                         _c_vp, _c_vp, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_glm_categorical_workspace_size": ([_c_int, _c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_glm_categorical": ([ctypes.c_longlong, _c_int, _c_int, _c_vp, ctypes.c_longlong, _c_vp, _c_vp, _c_vp,
                             _c_vp, _c_vp, _c_vp, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_tri_solve": ([_c_int, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp],
                      _c_int),
    "gpc_tri_solve_adjoint": ([_c_int, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int, _c_vp, _c_int,
                               _c_vp, _c_int, _c_vp], _c_int),
    "gpc_gp_lml": ([_c_int, _c_vp, _c_int, _c_vp, _c_vp, _c_int, _c_int, _c_vp, _c_vp, _c_vp,
                    _c_vp, _c_size, _c_vp, _c_vp], _c_int),
    "gpc_gp_lml_grad": ([_c_int, _c_vp, _c_int, _c_vp, _c_double, _c_vp, _c_int, _c_int, _c_vp,
                         _c_size, _c_vp], _c_int),
    "gpc_se_hyper_grad": ([_c_int, _c_int, _c_vp, _c_int, _c_double, _c_double, _c_double, _c_vp,
                           _c_int, _c_vp, _c_int, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_se_hyper_grad_workspace_size": ([_c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_test_ozaki_workspace_size": ([_c_int, _c_int, _c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_test_ozaki_gemm": ([_c_int, _c_int, _c_int, _c_vp, _c_vp, _c_vp, _c_vp, _c_size, _c_vp, _c_vp], _c_int),
    "gpc_batched_workspace_size": ([_c_int, _c_int, _c_int, ctypes.POINTER(_c_size)], _c_int),
    "gpc_batched_gp_lml_grad": ([_c_int, _c_int, _c_vp, _c_vp, _c_vp, _c_int, _c_vp, _c_vp, _c_vp, _c_int,
                                 _c_vp, _c_vp, _c_vp, _c_vp, _c_vp, _c_size, _c_vp], _c_int),
    "gpc_launch_count": ([ctypes.POINTER(ctypes.c_longlong)], _c_int),
    "gpc_fp64_peak": ([_c_vp, _c_size, ctypes.POINTER(_c_double), _c_vp], _c_int),
    "gpc_trace_enable": ([_c_int], _c_int),
    "gpc_trace_summary": ([_c_int, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_c_double),
                           ctypes.POINTER(_c_double), ctypes.POINTER(_c_double)], _c_int),
    "gpc_trace_timeline": ([ctypes.c_longlong, ctypes.POINTER(_c_int), ctypes.POINTER(_c_int),
                            ctypes.POINTER(ctypes.c_ulonglong), ctypes.POINTER(ctypes.c_float),
                            ctypes.POINTER(ctypes.c_float), ctypes.POINTER(_c_double),
                            ctypes.POINTER(ctypes.c_longlong)], _c_int),
    "gpc_trace_name": ([_c_int, ctypes.c_char_p, _c_size], _c_int),
}

TRACE_CLASSES = {"gemm_f64": 0, "diag": 1, "trsv": 2, "se_cov": 3, "hyper_grad": 4, "elementwise": 5,
                 "gemm_mixed": 6, "split": 7, "trsm": 8, "glm": 9}
GLM_FAMILIES = {"normal_id": 0, "bernoulli_logit": 1, "poisson_log": 2, "neg_binomial_2_log": 3}
GPC_GLM_MAX_CLASSES = 16
GPC_GLM_MAX_KC = 8192
GPC_GLM_MAX_K = 12288


class GpcholError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {status_string(status)}")
        self.status = status


class NotPositiveDefinite(GpcholError):
    def __init__(self, status: int, pivot: int):
        super().__init__(status, f"factorisation failed at pivot {pivot}")
        self.pivot = pivot


class _CApi:
    """The C entry points, loaded on first use."""

    def __init__(self):
        self._lib = None

    def load(self):
        if self._lib is None:
            path = library_path()
            lib = ctypes.CDLL(path)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = res
            self._lib = lib
        return self._lib

    def __getattr__(self, name):
        if name.startswith("gpc_"):
            return getattr(self.load(), name)
        raise AttributeError(name)


capi = _CApi()


def library_path(build_if_missing: bool = True) -> str:
    """Path of the compiled library, building it with nvcc when missing."""
    if os.path.exists(_build.LIB):
        return _build.LIB
    if not build_if_missing:
        raise FileNotFoundError(f"{_build.LIB} is missing; run paper_1907_01063_gb300.build.build()")
    return _build.build()


def status_string(status: int) -> str:
    return capi.gpc_status_string(int(status)).decode()


def _check(status: int, what: str):
    if status != GPC_OK:
        raise GpcholError(status, what)


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _square(t: torch.Tensor, name: str) -> int:
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.shape[0] == t.shape[1]):
        raise ValueError(f"{name} must be a square float64 CUDA tensor")
    if t.shape[0] > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (stride(1) == 1)")
    return int(t.stride(0)) if t.shape[0] > 0 else 1


def _vector(t: torch.Tensor, n: int, name: str):
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 1 and t.shape[0] == n
            and (n == 0 or t.stride(0) == 1)):
        raise ValueError(f"{name} must be a contiguous float64 CUDA vector of length {n}")


def precision_code(precision) -> int:
    try:
        return PRECISIONS[precision]
    except KeyError:
        raise ValueError(f"unknown precision {precision!r}") from None


def get_error(clear: bool = False) -> int:
    """The library error word of the current device after synchronising the
    current stream: GPC_OK, or GPC_ERR_TIMEOUT if a bounded device wait gave
    up since the last clear.  clear=True resets it."""
    v = ctypes.c_int()
    _check(capi.gpc_get_error(ctypes.byref(v), 1 if clear else 0, _stream()), "gpc_get_error")
    return v.value


GPC_TEST_WAIT_NS = 0
GPC_TEST_TRSV_WITHHOLD = 1
GPC_TEST_OZAKI_NO_LOADS = 2


def set_test_fault(key: int, value: int):
    """Fault-injection knob of the test hooks (gpc_test_set_fault)."""
    _check(capi.gpc_test_set_fault(int(key), int(value)), "gpc_test_set_fault")


def set_tuning(key: int, value: int):
    _check(capi.gpc_set_tuning(key, int(value)), "gpc_set_tuning")


def get_tuning(key: int) -> int:
    v = ctypes.c_int()
    _check(capi.gpc_get_tuning(key, ctypes.byref(v)), "gpc_get_tuning")
    return v.value


def workspace_size(n: int, precision="fp64") -> int:
    b = ctypes.c_size_t()
    _check(capi.gpc_workspace_size(int(n), precision_code(precision), ctypes.byref(b)),
           "gpc_workspace_size")
    return b.value


def workspace(n: int, precision="fp64", device=None) -> torch.Tensor:
    """A byte tensor large enough for any call at order <= n."""
    return torch.empty(workspace_size(n, precision), dtype=torch.uint8,
                       device=device if device is not None else "cuda")


def new_info(device=None) -> torch.Tensor:
    return torch.full((2,), -1, dtype=torch.int32, device=device if device is not None else "cuda")


def check_info(info: torch.Tensor, what: str = "factorisation"):
    """Synchronises on info (2 device ints) and raises on a device-side failure."""
    pivot, status = (int(v) for v in info.tolist())
    if status in (GPC_ERR_NOT_PD, GPC_ERR_NAN):
        raise NotPositiveDefinite(status, pivot)
    if status != GPC_OK:
        raise GpcholError(status, what)


def _ws_for(n: int, precision, ws: torch.Tensor | None, device) -> torch.Tensor:
    need = workspace_size(n, precision)
    if ws is None:
        return torch.empty(need, dtype=torch.uint8, device=device)
    if ws.numel() * ws.element_size() < need or not ws.is_cuda:
        raise ValueError(f"workspace too small: need {need} bytes")
    return ws


def launch_count() -> int:
    """Running total of kernels this library has launched in this process."""
    v = ctypes.c_longlong()
    _check(capi.gpc_launch_count(ctypes.byref(v)), "gpc_launch_count")
    return v.value


def fp64_peak_gflops(device=None) -> float:
    """Measured FP64 tensor (mma.sync m16n8k16) throughput of the device, GFLOP/s."""
    ws = torch.empty(4 << 20, dtype=torch.uint8, device=device if device is not None else "cuda")
    v = ctypes.c_double()
    _check(capi.gpc_fp64_peak(ws.data_ptr(), ws.numel(), ctypes.byref(v), _stream()), "gpc_fp64_peak")
    return v.value


def trace_enable(on: bool = True, timeline: bool = False):
    """Start (clearing totals) or stop per-launch CUDA-event timing; with
    timeline=True every launch's start and duration is kept as well."""
    _check(capi.gpc_trace_enable((2 if timeline else 1) if on else 0), "gpc_trace_enable")


def trace_timeline() -> list:
    """Recorded launches in order: class, kernel, stream, start and duration (ms), flops."""
    count = ctypes.c_longlong()
    _check(capi.gpc_trace_timeline(0, None, None, None, None, None, None, ctypes.byref(count)),
           "gpc_trace_timeline")
    n = count.value
    cls = (ctypes.c_int * max(n, 1))()
    name = (ctypes.c_int * max(n, 1))()
    stream = (ctypes.c_ulonglong * max(n, 1))()
    start = (ctypes.c_float * max(n, 1))()
    dur = (ctypes.c_float * max(n, 1))()
    flops = (ctypes.c_double * max(n, 1))()
    _check(capi.gpc_trace_timeline(n, cls, name, stream, start, dur, flops, ctypes.byref(count)),
           "gpc_trace_timeline")
    classes = {v: k for k, v in TRACE_CLASSES.items()}
    names = {}
    buf = ctypes.create_string_buffer(256)
    out = []
    for i in range(min(n, count.value)):
        if name[i] not in names:
            _check(capi.gpc_trace_name(name[i], buf, 256), "gpc_trace_name")
            names[name[i]] = buf.value.decode()
        out.append({"class": classes.get(cls[i], str(cls[i])), "kernel": names[name[i]], "stream": stream[i],
                    "start_ms": start[i], "dur_ms": dur[i], "flops": flops[i]})
    return out


def trace_summary() -> dict:
    """Per kernel class: launches, device ms, algorithmic flops and bytes."""
    out = {}
    for name, cls in TRACE_CLASSES.items():
        n, ms, fl, by = ctypes.c_longlong(), ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _check(capi.gpc_trace_summary(cls, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(fl),
                                      ctypes.byref(by)), "gpc_trace_summary")
        out[name] = {"launches": n.value, "ms": ms.value, "flops": fl.value, "bytes": by.value}
    return out


# ---------------------------------------------------------------- tensor API
def se_cov(X: torch.Tensor, alpha: float, rho: float, sigma: float, jitter: float = 0.0,
           full: bool = False, out: torch.Tensor | None = None, precision="fp64") -> torch.Tensor:
    """Squared-exponential covariance of the rows of X (lower triangle, or full);
    precision "mixed" evaluates r^2 and the exponential in double-float."""
    if not (X.is_cuda and X.dtype == torch.float64 and X.dim() == 2 and X.stride(1) == 1):
        raise ValueError("X must be a row-major float64 CUDA matrix")
    n, d = X.shape
    K = out if out is not None else torch.zeros(n, n, dtype=torch.float64, device=X.device)
    ldk = _square(K, "K")
    _check(capi.gpc_se_cov(n, d, _ptr(X), max(int(X.stride(0)), d), float(alpha), float(rho),
                           float(sigma), float(jitter), _ptr(K), ldk, 1 if full else 0,
                           precision_code(precision), _stream()),
           "gpc_se_cov")
    return K


def chol(K: torch.Tensor, precision="fp64", out: torch.Tensor | None = None,
         ws: torch.Tensor | None = None, info: torch.Tensor | None = None,
         check: bool = True) -> torch.Tensor:
    """Lower Cholesky factor of the SPD matrix whose lower triangle is in K."""
    n = K.shape[0]
    ldk = _square(K, "K")
    L = out if out is not None else torch.empty_like(K)
    ldl = _square(L, "L")
    wsb = _ws_for(n, precision, ws, K.device)
    inf = info if info is not None else new_info(K.device)
    _check(capi.gpc_chol(n, _ptr(K), ldk, _ptr(L), ldl, precision_code(precision), _ptr(wsb),
                         wsb.numel(), _ptr(inf), _stream()), "gpc_chol")
    if check:
        check_info(inf, "gpc_chol")
    return L


def chol_adjoint(L: torch.Tensor, Lbar: torch.Tensor, precision="fp64", symmetric_out: bool = False,
                 out: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Kbar from L and Lbar (reverse mode of chol); lower convention unless symmetric_out."""
    n = L.shape[0]
    ldl = _square(L, "L")
    ldlb = _square(Lbar, "Lbar")
    Kbar = out if out is not None else torch.empty_like(Lbar)
    ldkb = _square(Kbar, "Kbar")
    wsb = _ws_for(n, precision, ws, L.device)
    _check(capi.gpc_chol_adjoint(n, _ptr(L), ldl, _ptr(Lbar), ldlb, _ptr(Kbar), ldkb,
                                 precision_code(precision), 1 if symmetric_out else 0, _ptr(wsb),
                                 wsb.numel(), _stream()), "gpc_chol_adjoint")
    return Kbar


def trsv(L: torch.Tensor, x: torch.Tensor, trans: bool = False,
         ws: torch.Tensor | None = None) -> torch.Tensor:
    """x <- L^{-1} x (or L^{-T} x), in place; returns x."""
    n = L.shape[0]
    ldl = _square(L, "L")
    _vector(x, n, "x")
    wsb = _ws_for(n, "fp64", ws, L.device)
    _check(capi.gpc_trsv(n, _ptr(L), ldl, _ptr(x), 1 if trans else 0, _ptr(wsb), wsb.numel(),
                         _stream()), "gpc_trsv")
    return x


def _rect(t: torch.Tensor, n: int, name: str) -> tuple[int, int]:
    """(m, ld) of an n x m row-major float64 CUDA matrix."""
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2 and t.shape[0] == n):
        raise ValueError(f"{name} must be a float64 CUDA matrix with {n} rows")
    m = int(t.shape[1])
    if n > 0 and m > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (stride(1) == 1)")
    return m, (int(t.stride(0)) if n > 0 and m > 0 else max(m, 1))


def tri_inverse(L: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
    """L^{-1} of the lower triangle of L (zero strict upper); out may be L itself."""
    n = L.shape[0]
    ldl = _square(L, "L")
    X = out if out is not None else torch.empty_like(L)
    ldx = _square(X, "Linv")
    _check(capi.gpc_tri_inverse(n, _ptr(L), ldl, _ptr(X), ldx, _stream()), "gpc_tri_inverse")
    return X


def tri_solve(L: torch.Tensor, B: torch.Tensor, Linv: torch.Tensor | None = None,
              out: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """(C, Linv) with C = L^{-1} B through the inverse, as one product."""
    n = L.shape[0]
    ldl = _square(L, "L")
    m, ldb = _rect(B, n, "B")
    X = Linv if Linv is not None else torch.empty_like(L)
    ldx = _square(X, "Linv")
    C = out if out is not None else torch.empty(n, m, dtype=torch.float64, device=B.device)
    _, ldc = _rect(C, n, "C")
    _check(capi.gpc_tri_solve(n, m, _ptr(L), ldl, _ptr(B), ldb, _ptr(X), ldx, _ptr(C), ldc, _stream()),
           "gpc_tri_solve")
    return C, X


def tri_solve_adjoint(Linv: torch.Tensor, C: torch.Tensor, Cbar: torch.Tensor,
                      Bbar: torch.Tensor | None = None,
                      Lbar: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """(Bbar, Lbar) of C = L^{-1} B: L^{-T} Cbar and -tril(Bbar C^T)."""
    n = Linv.shape[0]
    ldx = _square(Linv, "Linv")
    m, ldc = _rect(C, n, "C")
    mb, ldcb = _rect(Cbar, n, "Cbar")
    if mb != m:
        raise ValueError("C and Cbar must have the same shape")
    Bb = Bbar if Bbar is not None else torch.empty_like(C, memory_format=torch.contiguous_format)
    _, ldbb = _rect(Bb, n, "Bbar")
    Lb = Lbar if Lbar is not None else torch.empty_like(Linv)
    ldlb = _square(Lb, "Lbar")
    _check(capi.gpc_tri_solve_adjoint(n, m, _ptr(Linv), ldx, _ptr(C), ldc, _ptr(Cbar), ldcb, _ptr(Bb), ldbb,
                                      _ptr(Lb), ldlb, _stream()),
           "gpc_tri_solve_adjoint")
    return Bb, Lb


def gemm_workspace(device=None) -> torch.Tensor:
    """Scratch that lets gemm / gemm_adjoint split long k ranges over CTAs."""
    b = ctypes.c_size_t()
    _check(capi.gpc_gemm_workspace_size(ctypes.byref(b)), "gpc_gemm_workspace_size")
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def _rows(t: torch.Tensor, name: str) -> tuple[int, int, int]:
    """(rows, cols, ld) of a row-major float64 CUDA matrix."""
    if not (t.is_cuda and t.dtype == torch.float64 and t.dim() == 2):
        raise ValueError(f"{name} must be a float64 CUDA matrix")
    r, c = int(t.shape[0]), int(t.shape[1])
    if r > 0 and c > 0 and t.stride(1) != 1:
        raise ValueError(f"{name} must be row-major (stride(1) == 1)")
    return r, c, (int(t.stride(0)) if r > 0 and c > 0 else max(c, 1))


def gemm(A: torch.Tensor, B: torch.Tensor, out: torch.Tensor | None = None,
         ws: torch.Tensor | None = None) -> torch.Tensor:
    """C = A B on the FP64 tensor path (ws: optional split-k scratch)."""
    m, k, lda = _rows(A, "A")
    k2, n, ldb = _rows(B, "B")
    if k2 != k:
        raise ValueError("inner dimensions differ")
    C = out if out is not None else torch.empty(m, n, dtype=torch.float64, device=A.device)
    _, _, ldc = _rows(C, "C")
    _check(capi.gpc_gemm(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(C), ldc, _ptr(ws),
                         0 if ws is None else ws.numel(), _stream()), "gpc_gemm")
    return C


def gemm_adjoint(A: torch.Tensor, B: torch.Tensor, Cbar: torch.Tensor,
                 ws: torch.Tensor | None = None) -> tuple[torch.Tensor, torch.Tensor]:
    """(Abar, Bbar) = (Cbar B^T, A^T Cbar) for C = A B."""
    m, k, lda = _rows(A, "A")
    _, n, ldb = _rows(B, "B")
    _, _, ldcb = _rows(Cbar, "Cbar")
    if tuple(Cbar.shape) != (m, n) or B.shape[0] != k:
        raise ValueError("shape mismatch")
    Abar = torch.empty(m, k, dtype=torch.float64, device=A.device)
    Bbar = torch.empty(k, n, dtype=torch.float64, device=A.device)
    _check(capi.gpc_gemm_adjoint(m, n, k, _ptr(A), lda, _ptr(B), ldb, _ptr(Cbar), ldcb, _ptr(Abar), max(k, 1),
                                 _ptr(Bbar), max(n, 1), _ptr(ws), 0 if ws is None else ws.numel(), _stream()),
           "gpc_gemm_adjoint")
    return Abar, Bbar


def glm_workspace(k: int, device=None) -> torch.Tensor:
    """Scratch for glm with k covariates (per-CTA partial gradient rows)."""
    b = ctypes.c_size_t()
    _check(capi.gpc_glm_workspace_size(int(k), ctypes.byref(b)), "gpc_glm_workspace_size")
    return torch.empty(b.value, dtype=torch.uint8, device=device)


def glm(family: str, X: torch.Tensor, y: torch.Tensor, alpha: float, beta: torch.Tensor, sigma: float = 1.0,
        ws: torch.Tensor | None = None) -> dict:
    """Fused GLM log likelihood and gradient: dict(lp, dalpha, dbeta, dsigma) of device tensors."""
    n, k, ldx = _rows(X, "X")
    _vector(y, n, "y")
    _vector(beta, k, "beta")
    dev = X.device
    if ws is None:
        ws = glm_workspace(k, dev)
    out = torch.empty(3, dtype=torch.float64, device=dev)
    dbeta = torch.empty(k, dtype=torch.float64, device=dev)
    _check(capi.gpc_glm(GLM_FAMILIES[family], n, k, _ptr(X), ldx, _ptr(y), float(alpha), _ptr(beta), float(sigma),
                        out.data_ptr(), out.data_ptr() + 8, _ptr(dbeta), out.data_ptr() + 16, _ptr(ws), ws.numel(),
                        _stream()), "gpc_glm")
    return {"lp": out[0], "dalpha": out[1], "dbeta": dbeta, "dsigma": out[2]}


def glm_ordinal(X: torch.Tensor, y: torch.Tensor, beta: torch.Tensor, cuts: torch.Tensor,
                ws: torch.Tensor | None = None) -> dict:
    """Ordinal-logit GLM: y in {0..C-1}, increasing cuts (C-1); dict(lp, dbeta, dcuts) of device tensors."""
    n, k, ldx = _rows(X, "X")
    _vector(y, n, "y")
    _vector(beta, k, "beta")
    C = int(cuts.shape[0]) + 1
    _vector(cuts, C - 1, "cuts")
    dev = X.device
    if ws is None:
        ws = glm_workspace(k, dev)
    lp = torch.empty((), dtype=torch.float64, device=dev)
    dbeta = torch.empty(k, dtype=torch.float64, device=dev)
    dcuts = torch.empty(C - 1, dtype=torch.float64, device=dev)
    _check(capi.gpc_glm_ordinal(n, k, C, _ptr(X), ldx, _ptr(y), _ptr(beta), _ptr(cuts), lp.data_ptr(), _ptr(dbeta),
                                dcuts.data_ptr(), _ptr(ws), ws.numel(), _stream()), "gpc_glm_ordinal")
    return {"lp": lp, "dbeta": dbeta, "dcuts": dcuts}


def glm_categorical(X: torch.Tensor, y: torch.Tensor, alpha: torch.Tensor, beta: torch.Tensor,
                    ws: torch.Tensor | None = None) -> dict:
    """Categorical-logit GLM: y in {0..C-1}, alpha (C), beta (k x C); dict(lp, dalpha, dbeta) of device tensors."""
    n, k, ldx = _rows(X, "X")
    _vector(y, n, "y")
    C = int(alpha.shape[0])
    _vector(alpha, C, "alpha")
    if not (beta.is_cuda and beta.dtype == torch.float64 and tuple(beta.shape) == (k, C) and beta.is_contiguous()):
        raise ValueError(f"beta must be a contiguous float64 CUDA matrix of shape ({k}, {C})")
    dev = X.device
    if ws is None:
        b = ctypes.c_size_t()
        _check(capi.gpc_glm_categorical_workspace_size(k, C, ctypes.byref(b)), "gpc_glm_categorical_workspace_size")
        ws = torch.empty(b.value, dtype=torch.uint8, device=dev)
    lp = torch.empty((), dtype=torch.float64, device=dev)
    dalpha = torch.empty(C, dtype=torch.float64, device=dev)
    dbeta = torch.empty(k, C, dtype=torch.float64, device=dev)
    _check(capi.gpc_glm_categorical(n, k, C, _ptr(X), ldx, _ptr(y), _ptr(alpha), _ptr(beta), lp.data_ptr(),
                                    dalpha.data_ptr(), _ptr(dbeta), _ptr(ws), ws.numel(), _stream()),
           "gpc_glm_categorical")
    return {"lp": lp, "dalpha": dalpha, "dbeta": dbeta}


def gp_lml(K: torch.Tensor, y: torch.Tensor, precision="fp64", L: torch.Tensor | None = None,
           ws: torch.Tensor | None = None, info: torch.Tensor | None = None, check: bool = True):
    """Log marginal likelihood of y ~ N(0, K): returns dict(L, alpha, logdet, value).

    logdet and value are 0-d device tensors (no host synchronisation unless
    ``check`` reads the info flags).
    """
    n = K.shape[0]
    ldk = _square(K, "K")
    _vector(y, n, "y")
    Lt = L if L is not None else torch.empty_like(K)
    ldl = _square(Lt, "L")
    alpha = torch.empty(n, dtype=torch.float64, device=K.device)
    scal = torch.empty(2, dtype=torch.float64, device=K.device)
    wsb = _ws_for(n, precision, ws, K.device)
    inf = info if info is not None else new_info(K.device)
    _check(capi.gpc_gp_lml(n, _ptr(K), ldk, _ptr(y), _ptr(Lt), ldl, precision_code(precision),
                           scal.data_ptr(), _ptr(alpha), scal.data_ptr() + 8, _ptr(wsb), wsb.numel(),
                           _ptr(inf), _stream()), "gpc_gp_lml")
    if check:
        check_info(inf, "gpc_gp_lml")
    return {"L": Lt, "alpha": alpha, "logdet": scal[0], "value": scal[1], "info": inf}


def gp_lml_grad(L: torch.Tensor, alpha: torch.Tensor, gbar: float = 1.0, precision="fp64",
                out: torch.Tensor | None = None, ws: torch.Tensor | None = None) -> torch.Tensor:
    """Kbar = gbar * d value / dK (lower convention) through the Cholesky adjoint."""
    n = L.shape[0]
    ldl = _square(L, "L")
    _vector(alpha, n, "alpha")
    Kbar = out if out is not None else torch.empty_like(L)
    ldkb = _square(Kbar, "Kbar")
    wsb = _ws_for(n, precision, ws, L.device)
    _check(capi.gpc_gp_lml_grad(n, _ptr(L), ldl, _ptr(alpha), float(gbar), _ptr(Kbar), ldkb,
                                precision_code(precision), _ptr(wsb), wsb.numel(), _stream()),
           "gpc_gp_lml_grad")
    return Kbar


def se_hyper_grad_workspace_size(n: int) -> int:
    b = ctypes.c_size_t()
    _check(capi.gpc_se_hyper_grad_workspace_size(int(n), ctypes.byref(b)),
           "gpc_se_hyper_grad_workspace_size")
    return b.value


def se_hyper_grad(X: torch.Tensor, alpha: float, rho: float, sigma: float, Kbar: torch.Tensor,
                  ws: torch.Tensor | None = None, out: torch.Tensor | None = None,
                  precision="fp64") -> torch.Tensor:
    """(d/d alpha, d/d rho, d/d sigma) as a 3-vector on the device."""
    n, d = X.shape
    ldkb = _square(Kbar, "Kbar")
    g = out if out is not None else torch.empty(3, dtype=torch.float64, device=X.device)
    need = se_hyper_grad_workspace_size(n)
    wsb = ws if ws is not None else torch.empty(need, dtype=torch.uint8, device=X.device)
    _check(capi.gpc_se_hyper_grad(n, d, _ptr(X), max(int(X.stride(0)), d), float(alpha), float(rho),
                                  float(sigma), _ptr(Kbar), ldkb, _ptr(g), precision_code(precision),
                                  _ptr(wsb), wsb.numel() * wsb.element_size(), _stream()),
           "gpc_se_hyper_grad")
    return g


def test_ozaki_gemm(A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    """A @ B.T through the mixed path's split-BF16 tensor-core product (test hook)."""
    M, K = A.shape
    N, K2 = B.shape
    if K != K2 or not (A.is_contiguous() and B.is_contiguous()):
        raise ValueError("A (M x K) and B (N x K) must be contiguous with equal K")
    nb = ctypes.c_size_t()
    _check(capi.gpc_test_ozaki_workspace_size(M, N, K, ctypes.byref(nb)), "gpc_test_ozaki_workspace_size")
    ws = torch.empty(nb.value, dtype=torch.uint8, device=A.device)
    C = torch.empty(M, N, dtype=torch.float64, device=A.device)
    err = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(capi.gpc_test_ozaki_gemm(M, N, K, A.data_ptr(), B.data_ptr(), C.data_ptr(), ws.data_ptr(),
                                    ws.numel(), err.data_ptr(), _stream()), "gpc_test_ozaki_gemm")
    if int(err.item()) != 0:
        raise GpcholError(int(err.item()), "gpc_test_ozaki_gemm")
    return C


class Batch:
    """Device layout of a batch of GPs for batched_gp_lml_grad.

    sizes: host sequence of n_i; the covariance/factor of GP i occupies
    n_i^2 doubles of K at offK[i]; its inputs are rows rowX[i] .. of X and y.
    precision: "fp64" or "mixed"; the workspace is sized for it, and a batch
    made for "fp64" cannot run the mixed path (its workspace is smaller).
    """

    def __init__(self, sizes, device=None, precision="fp64"):
        device = device if device is not None else "cuda"
        self.precision = precision
        self.sizes = [int(v) for v in sizes]
        self.batch = len(self.sizes)
        self.nmax = max(self.sizes) if self.sizes else 1
        offk, rowx, ok, rx = [], [], 0, 0
        for v in self.sizes:
            offk.append(ok)
            rowx.append(rx)
            ok += v * v
            rx += v
        self.total_k, self.total_rows = ok, rx
        self.n = torch.tensor(self.sizes, dtype=torch.int32, device=device)
        self.offK = torch.tensor(offk, dtype=torch.int64, device=device)
        self.rowX = torch.tensor(rowx, dtype=torch.int64, device=device)
        self.K = torch.empty(max(ok, 1), dtype=torch.float64, device=device)
        self.value = torch.empty(self.batch, dtype=torch.float64, device=device)
        self.grad3 = torch.empty(self.batch, 3, dtype=torch.float64, device=device)
        self.info = torch.empty(self.batch, 2, dtype=torch.int32, device=device)
        nbytes = ctypes.c_size_t()
        _check(capi.gpc_batched_workspace_size(self.batch, self.nmax, precision_code(precision),
                                                 ctypes.byref(nbytes)),
               "gpc_batched_workspace_size")
        self.ws = torch.empty(nbytes.value, dtype=torch.uint8, device=device)

    def factor(self, i):
        """Cholesky factor of GP i (a view into K)."""
        o = int(self.offK[i].item())
        v = self.sizes[i]
        return self.K[o:o + v * v].view(v, v)


def batched_gp_lml_grad(batch: Batch, X: torch.Tensor, y: torch.Tensor, hyp: torch.Tensor,
                        precision=None):
    """Log marginal likelihood and (alpha, rho, sigma) gradient of every GP in
    the batch in one launch; returns (value [batch], grad3 [batch, 3], info [batch, 2]).
    precision defaults to the batch's own."""
    precision = batch.precision if precision is None else precision
    if not (X.is_cuda and X.dtype == torch.float64 and X.dim() == 2 and X.is_contiguous()):
        raise ValueError("X must be a contiguous float64 CUDA matrix")
    if X.shape[0] != batch.total_rows or y.numel() != batch.total_rows:
        raise ValueError("X and y must hold sum(n_i) rows")
    hyp = hyp.to(device=X.device, dtype=torch.float64).contiguous()
    if hyp.numel() != 3 * batch.batch:
        raise ValueError("hyp must have shape (batch, 3)")
    _check(capi.gpc_batched_gp_lml_grad(batch.batch, batch.nmax, batch.n.data_ptr(), batch.offK.data_ptr(),
                                        batch.rowX.data_ptr(), X.shape[1], X.data_ptr(), y.data_ptr(),
                                        hyp.data_ptr(), precision_code(precision), batch.K.data_ptr(),
                                        batch.value.data_ptr(), batch.grad3.data_ptr(), batch.info.data_ptr(),
                                        batch.ws.data_ptr(), batch.ws.numel(), _stream()),
           "gpc_batched_gp_lml_grad")
    return batch.value, batch.grad3, batch.info


# ---------------------------------------------------------------- autograd
class Chol(torch.autograd.Function):
    """L = chol(K) with the blocked adjoint as backward.

    The gradient returned for K is the lower-convention Kbar: entry (i, j),
    i >= j, is d f / d K_ij over the entries chol reads; the upper triangle of
    K does not influence L and gets zero gradient.
    """

    @staticmethod
    def forward(ctx, K, precision="fp64"):
        L = chol(K.detach(), precision)
        ctx.precision = precision
        ctx.save_for_backward(L)
        return L

    @staticmethod
    def backward(ctx, Lbar):
        (L,) = ctx.saved_tensors
        Lbar = torch.tril(Lbar.contiguous())
        return chol_adjoint(L, Lbar, ctx.precision), None


class GPLml(torch.autograd.Function):
    """Log marginal likelihood of y under an SE-kernel GP, differentiable in
    (alpha, rho, sigma); K is rebuilt on the device and only L and alpha are
    kept for the backward pass."""

    @staticmethod
    def forward(ctx, X, y, hyp, jitter=0.0, precision="fp64"):
        a, r, s = (float(v) for v in hyp.detach().cpu().tolist())
        K = se_cov(X, a, r, s, jitter, precision=precision)
        res = gp_lml(K, y, precision, L=K if precision_code(precision) == GPC_FP64 else None)
        ctx.save_for_backward(X, res["L"], res["alpha"])
        ctx.hyp = (a, r, s)
        ctx.hyp_device = hyp.device
        ctx.precision = precision
        return res["value"].clone()

    @staticmethod
    def backward(ctx, gvalue):
        X, L, alpha = ctx.saved_tensors
        a, r, s = ctx.hyp
        Kbar = gp_lml_grad(L, alpha, 1.0, ctx.precision)
        g = se_hyper_grad(X, a, r, s, Kbar, precision=ctx.precision)
        return None, None, (g * gvalue).to(ctx.hyp_device), None, None


class TriSolve(torch.autograd.Function):
    """C = L^{-1} B with the lower triangle of L; backward gives
    Bbar = L^{-T} Cbar and Lbar = -tril(Bbar C^T) from the kept inverse.
    A 1-D B is treated as one column."""

    @staticmethod
    def forward(ctx, L, B):
        vec = B.dim() == 1
        Bm = B.detach().reshape(-1, 1) if vec else B.detach()
        if Bm.shape[1] > 0 and Bm.stride(1) != 1:
            Bm = Bm.contiguous()
        C, X = tri_solve(L.detach(), Bm)
        ctx.vec = vec
        ctx.save_for_backward(X, C)
        return C.reshape(-1) if vec else C

    @staticmethod
    def backward(ctx, Cbar):
        X, C = ctx.saved_tensors
        Cb = Cbar.reshape(-1, 1) if ctx.vec else Cbar
        Bb, Lb = tri_solve_adjoint(X, C, Cb.contiguous())
        return Lb, (Bb.reshape(-1) if ctx.vec else Bb)


def mdivide_left_tri_low(L, B):
    """Differentiable L^{-1} B for lower-triangular L (upper triangle ignored)."""
    return TriSolve.apply(L, B)


class MatMul(torch.autograd.Function):
    """C = A B with the GEMM reverse mode (Abar = Cbar B^T, Bbar = A^T Cbar) as backward."""

    @staticmethod
    def forward(ctx, A, B):
        A_, B_ = A.detach().contiguous(), B.detach().contiguous()
        ctx.save_for_backward(A_, B_)
        return gemm(A_, B_)

    @staticmethod
    def backward(ctx, Cbar):
        A, B = ctx.saved_tensors
        return gemm_adjoint(A, B, Cbar.contiguous())


class GLMLpmf(torch.autograd.Function):
    """GLM log likelihood of y given X, differentiable in alpha, beta and sigma
    (the gradient comes from the same fused kernel as the value)."""

    @staticmethod
    def forward(ctx, X, y, alpha, beta, sigma, family):
        r = glm(family, X.detach(), y.detach(), float(alpha), beta.detach().contiguous(), float(sigma))
        ctx.save_for_backward(r["dalpha"].reshape(1), r["dbeta"], r["dsigma"].reshape(1))
        ctx.devs = (alpha.device, sigma.device)
        return r["lp"].clone()

    @staticmethod
    def backward(ctx, g):
        da, db, ds = ctx.saved_tensors
        return (None, None, (g * da[0]).to(ctx.devs[0]), g * db, (g * ds[0]).to(ctx.devs[1]), None)


def glm_lpmf(family: str, X, y, alpha, beta, sigma=None):
    """Differentiable GLM log likelihood; alpha and sigma are 0-d tensors (sigma only for normal_id)."""
    if sigma is None:
        sigma = torch.ones((), dtype=torch.float64)
    return GLMLpmf.apply(X, y, alpha, beta, sigma, family)


def gp_lml_value(X, y, hyp, jitter=0.0, precision="fp64"):
    """Differentiable log marginal likelihood; hyp = tensor([alpha, rho, sigma])."""
    return GPLml.apply(X, y, hyp, jitter, precision)
