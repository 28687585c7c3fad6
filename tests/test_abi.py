"""The C-ABI library loads and exports every symbol include/gpchol.h declares.

Runs without a GPU: only host-side entry points are called (status strings,
version, workspace sizing, tuning, and argument checks that return before any
CUDA call).
"""
import ctypes
import os
import re

import pytest

import paper_1907_01063_gb300 as gp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = "".join(open(os.path.join(ROOT, "include", f)).read()
                  for f in sorted(os.listdir(os.path.join(ROOT, "include"))) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gpc_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("gpc_chol", "gpc_chol_adjoint", "gpc_gp_lml", "gpc_gp_lml_grad", "gpc_trsv",
                     "gpc_se_cov", "gpc_se_hyper_grad", "gpc_workspace_size"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(gp.library_path())
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(gp._SIGNATURES)


def test_host_only_calls():
    assert gp.capi.gpc_version() >= 100
    assert "not positive definite" in gp.status_string(gp.GPC_ERR_NOT_PD)
    assert gp.status_string(12345) == "unknown gpchol status"
    assert gp.workspace_size(0) > 0
    assert gp.workspace_size(4096) < gp.workspace_size(8192)


def test_tuning_roundtrip_and_validation():
    old = gp.get_tuning(gp.GPC_TUNE_BLOCK)
    try:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, 64)
        assert gp.get_tuning(gp.GPC_TUNE_BLOCK) == 64
        for bad in (0, 8, 100, 256):
            with pytest.raises(gp.GpcholError):
                gp.set_tuning(gp.GPC_TUNE_BLOCK, bad)
        with pytest.raises(gp.GpcholError):
            gp.set_tuning(99, 1)
        # the slice count is fixed by the split kernels: readable, settable only to itself
        assert gp.get_tuning(gp.GPC_TUNE_SLICES) == 5
        gp.set_tuning(gp.GPC_TUNE_SLICES, 5)
        for bad in (3, 4, 6):
            with pytest.raises(gp.GpcholError):
                gp.set_tuning(gp.GPC_TUNE_SLICES, bad)
    finally:
        gp.set_tuning(gp.GPC_TUNE_BLOCK, old)


def test_argument_checks_return_before_any_launch():
    c = gp.capi
    bad = gp.GPC_ERR_INVALID_ARG
    fake = 0x1000  # never dereferenced: every call below fails validation first
    size = ctypes.c_size_t()
    assert c.gpc_workspace_size(-1, 0, ctypes.byref(size)) == bad
    assert c.gpc_workspace_size(10, 7, ctypes.byref(size)) == bad
    # negative n, ld < n, null pointers, unknown precision, tiny workspace
    assert c.gpc_chol(-1, fake, 1, fake, 1, 0, fake, 1 << 30, fake, None) == bad
    assert c.gpc_chol(10, fake, 9, fake, 10, 0, fake, 1 << 30, fake, None) == bad
    assert c.gpc_chol(10, None, 10, fake, 10, 0, fake, 1 << 30, fake, None) == bad
    assert c.gpc_chol(10, fake, 10, fake, 10, 5, fake, 1 << 30, fake, None) == bad
    assert c.gpc_chol(10, fake, 10, fake + 8, 10, 0, fake, 1 << 30, fake, None) == bad  # overlap
    assert c.gpc_chol(10, fake, 10, fake, 11, 0, fake, 1 << 30, fake, None) == bad  # in place, ld differs
    assert c.gpc_chol(10, fake, 10, fake, 10, 0, fake, 16, fake, None) == bad
    assert c.gpc_chol(10, fake, 10, 0x100000, 10, 0, fake, 1 << 30, None, None) == bad  # no info
    assert c.gpc_chol_adjoint(10, fake, 10, 0x100000, 10, 0x100000, 10, 0, 0, fake, 16, None) == bad
    assert c.gpc_chol_adjoint(10, fake, 10, 0x100000, 10, fake, 10, 0, 0, fake, 1 << 30, None) == bad
    assert c.gpc_trsv(10, None, 10, fake, 0, fake, 1 << 20, None) == bad
    assert c.gpc_se_cov(10, 0, fake, 1, 1.0, 1.0, 0.1, 0.0, fake, 10, 0, 0, None) == bad
    assert c.gpc_se_cov(10, 2, fake, 2, 1.0, 0.0, 0.1, 0.0, fake, 10, 0, 0, None) == bad
    assert c.gpc_se_cov(10, 2, fake, 2, 1.0, -1.0, 0.1, 0.0, fake, 10, 0, 0, None) == bad
    assert c.gpc_gp_lml(10, fake, 10, fake, 0x100000, 10, 0, None, fake, fake, fake, 1 << 30,
                        fake, None) == bad
    assert c.gpc_se_hyper_grad(10, 2, fake, 2, 1.0, 1.0, 0.1, fake, 10, None, 0, fake, 1 << 20, None) == bad
    # zero-size calls that need no device work
    assert c.gpc_chol_adjoint(0, None, 0, None, 0, None, 0, 0, 0, None, 0, None) == gp.GPC_OK
    assert c.gpc_trsv(0, None, 0, None, 0, None, 0, None) == gp.GPC_OK
    assert c.gpc_se_cov(0, 1, None, 1, 1.0, 1.0, 0.1, 0.0, None, 0, 0, 0, None) == gp.GPC_OK
    assert c.gpc_se_cov(10, 2, fake, 2, 1.0, 1.0, 0.1, 0.0, fake, 10, 0, 7, None) == bad  # precision


def test_triangular_argument_checks_return_before_any_launch():
    c = gp.capi
    bad = gp.GPC_ERR_INVALID_ARG
    fake, far, farther = 0x1000, 0x100000, 0x200000  # never dereferenced
    assert c.gpc_tri_inverse(-1, fake, 1, far, 1, None) == bad
    assert c.gpc_tri_inverse(10, None, 10, far, 10, None) == bad
    assert c.gpc_tri_inverse(10, fake, 9, far, 10, None) == bad
    assert c.gpc_tri_inverse(10, fake, 10, fake + 8, 10, None) == bad  # partial overlap
    assert c.gpc_tri_inverse(10, fake, 10, fake, 11, None) == bad  # in place, ld differs
    assert c.gpc_tri_solve(10, -1, fake, 10, far, 3, farther, 10, 0x300000, 3, None) == bad
    assert c.gpc_tri_solve(10, 3, fake, 10, far, 2, farther, 10, 0x300000, 3, None) == bad  # ldb < m
    assert c.gpc_tri_solve(10, 3, fake, 10, far, 3, farther, 10, far, 3, None) == bad  # C == B
    assert c.gpc_tri_solve(10, 3, fake, 10, far, 3, far, 10, 0x300000, 3, None) == bad  # B inside Linv
    assert c.gpc_tri_solve(10, 3, fake, 10, None, 3, farther, 10, 0x300000, 3, None) == bad
    assert c.gpc_tri_solve_adjoint(10, 3, fake, 10, far, 3, farther, 3, far, 3, 0x300000, 10,
                                   None) == bad  # Bbar == C
    assert c.gpc_tri_solve_adjoint(10, 3, fake, 10, far, 3, farther, 3, 0x300000, 3, fake, 10,
                                   None) == bad  # Lbar == Linv
    assert c.gpc_tri_solve_adjoint(10, 3, fake, 10, far, 3, farther, 3, 0x300000, 3, 0x400000, 9,
                                   None) == bad  # ldlb < n
    # zero-size calls need no device work
    assert c.gpc_tri_inverse(0, None, 0, None, 0, None) == gp.GPC_OK
    assert c.gpc_tri_solve(0, 5, None, 0, None, 0, None, 0, None, 0, None) == gp.GPC_OK
    assert c.gpc_tri_solve_adjoint(0, 5, None, 0, None, 0, None, 0, None, 0, None, 0, None) == gp.GPC_OK


def test_gemm_and_glm_argument_checks_return_before_any_launch():
    c = gp.capi
    bad = gp.GPC_ERR_INVALID_ARG
    fake, far, farther = 0x1000, 0x100000, 0x200000  # never dereferenced
    size = ctypes.c_size_t()
    assert c.gpc_gemm_workspace_size(ctypes.byref(size)) == gp.GPC_OK and size.value > 0
    assert c.gpc_gemm(-1, 2, 2, fake, 2, far, 2, farther, 2, None, 0, None) == bad
    assert c.gpc_gemm(4, 3, 2, fake, 1, far, 3, farther, 3, None, 0, None) == bad  # lda < k
    assert c.gpc_gemm(4, 3, 2, fake, 2, far, 3, fake, 3, None, 0, None) == bad  # C overlaps A
    assert c.gpc_gemm(4, 3, 2, fake, 2, far, 3, farther, 3, 0x300000, 16, None) == bad  # short workspace
    assert c.gpc_gemm(4, 3, 2, None, 2, far, 3, farther, 3, None, 0, None) == bad
    assert c.gpc_gemm(0, 3, 2, None, 2, None, 3, None, 3, None, 0, None) == gp.GPC_OK
    assert c.gpc_gemm_adjoint(4, 3, 2, fake, 2, far, 3, farther, 3, fake, 2, 0x300000, 3, None, 0,
                              None) == bad  # Abar == A
    assert c.gpc_gemm_adjoint(4, 3, 2, fake, 2, far, 3, farther, 3, 0x300000, 2, 0x300000, 3, None, 0,
                              None) == bad  # Abar overlaps Bbar
    assert c.gpc_glm_workspace_size(-1, ctypes.byref(size)) == bad
    assert c.gpc_glm_workspace_size(gp.GPC_GLM_MAX_K + 1 if hasattr(gp, "GPC_GLM_MAX_K") else 12289,
                                    ctypes.byref(size)) == bad
    assert c.gpc_glm_workspace_size(100, ctypes.byref(size)) == gp.GPC_OK
    ws = size.value
    out = 0x400000
    assert c.gpc_glm(7, 10, 3, fake, 3, far, 0.0, farther, 1.0, out, out + 8, out + 32, out + 16, 0x500000, ws,
                     None) == bad  # family
    assert c.gpc_glm(0, 10, 3, fake, 3, far, 0.0, farther, 0.0, out, out + 8, out + 32, out + 16, 0x500000, ws,
                     None) == bad  # sigma <= 0 for the normal family
    assert c.gpc_glm(1, 10, 3, fake, 2, far, 0.0, farther, 1.0, out, out + 8, out + 32, out + 16, 0x500000, ws,
                     None) == bad  # ldx < k
    assert c.gpc_glm(1, 10, 3, fake, 3, far, 0.0, farther, 1.0, out, out + 8, out + 32, out + 16, 0x500000, 8,
                     None) == bad  # short workspace
    assert c.gpc_glm(1, 10, 3, fake, 3, None, 0.0, farther, 1.0, out, out + 8, out + 32, out + 16, 0x500000, ws,
                     None) == bad  # no y


def test_error_word_and_fault_knobs_host_checks():
    c = gp.capi
    bad = gp.GPC_ERR_INVALID_ARG
    assert c.gpc_get_error(None, 0, None) == bad  # null status: rejected before any CUDA call
    assert c.gpc_test_set_fault(99, 0) == bad
    assert c.gpc_test_set_fault(gp.GPC_TEST_WAIT_NS, -1) == bad
    assert c.gpc_test_set_fault(gp.GPC_TEST_WAIT_NS, 10 ** 11) == bad
    assert c.gpc_test_set_fault(gp.GPC_TEST_TRSV_WITHHOLD, -2) == bad
    assert c.gpc_test_set_fault(gp.GPC_TEST_OZAKI_NO_LOADS, 2) == bad
    # valid settings are host-side only; restore the defaults
    for key, value, default in ((gp.GPC_TEST_WAIT_NS, 1000, 0), (gp.GPC_TEST_TRSV_WITHHOLD, 3, -1),
                                (gp.GPC_TEST_OZAKI_NO_LOADS, 1, 0)):
        assert c.gpc_test_set_fault(key, value) == gp.GPC_OK
        assert c.gpc_test_set_fault(key, default) == gp.GPC_OK


def test_mixed_schedule_knobs_roundtrip_and_validation():
    knobs = {gp.GPC_TUNE_MIXED_DEFER: ((1, 8), (0, 9)), gp.GPC_TUNE_MIXED_FREE_SMS: ((0, 32), (-1, 33)),
             gp.GPC_TUNE_MIXED_CTA_ITEMS: ((0, 1024), (-1, 1025)), gp.GPC_TUNE_MIXED_PRIORITY: ((0, 1), (-1, 2)),
             gp.GPC_TUNE_F64_SMALL_TILE: ((0, 4096), (-1, 4097))}
    for key, (good, bad) in knobs.items():
        old = gp.get_tuning(key)
        try:
            for v in good:
                gp.set_tuning(key, v)
                assert gp.get_tuning(key) == v
            for v in bad:
                with pytest.raises(gp.GpcholError):
                    gp.set_tuning(key, v)
        finally:
            gp.set_tuning(key, old)
    # the deferral depth enters the mixed workspace size (its group slice buffers)
    old = gp.get_tuning(gp.GPC_TUNE_MIXED_DEFER)
    try:
        gp.set_tuning(gp.GPC_TUNE_MIXED_DEFER, 1)
        small = gp.workspace_size(8192, "mixed")
        gp.set_tuning(gp.GPC_TUNE_MIXED_DEFER, 8)
        assert gp.workspace_size(8192, "mixed") >= small
    finally:
        gp.set_tuning(gp.GPC_TUNE_MIXED_DEFER, old)


def test_glm_family_argument_checks():
    c = gp.capi
    bad = gp.GPC_ERR_INVALID_ARG
    fake = 0x1000
    size = ctypes.c_size_t()
    assert c.gpc_glm_categorical_workspace_size(10, 1, ctypes.byref(size)) == bad       # C < 2
    assert c.gpc_glm_categorical_workspace_size(10, 17, ctypes.byref(size)) == bad      # C > max
    assert c.gpc_glm_categorical_workspace_size(4096, 3, ctypes.byref(size)) == bad     # k C > max
    assert c.gpc_glm_categorical_workspace_size(100, 3, ctypes.byref(size)) == gp.GPC_OK and size.value > 0
    # ordinal: C range, missing cuts, short workspace -- all before any launch
    assert c.gpc_glm_ordinal(10, 2, 1, fake, 2, fake, fake, fake, fake, fake, fake, fake, 1 << 30, None) == bad
    assert c.gpc_glm_ordinal(10, 2, 3, fake, 2, fake, fake, None, fake, fake, fake, fake, 1 << 30, None) == bad
    assert c.gpc_glm_ordinal(10, 2, 3, fake, 2, fake, fake, fake, fake, fake, fake, fake, 8, None) == bad
    assert c.gpc_glm_categorical(-1, 2, 3, fake, 2, fake, fake, fake, fake, fake, fake, fake, 1 << 30, None) == bad
    assert c.gpc_glm_categorical(10, 2, 3, fake, 1, fake, fake, fake, fake, fake, fake, fake, 1 << 30, None) == bad
    # the negative binomial needs a positive dispersion
    assert c.gpc_glm(3, 10, 2, fake, 2, fake, 0.0, fake, 0.0, fake, fake, fake, fake, fake, 1 << 30, None) == bad
