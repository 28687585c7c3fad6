"""gpc_trsv_noalloc: the triangular solve for callers that cannot allocate.

Some callers cannot give the library device memory for scratch -- code that
runs under a device-memory budget owned by a framework's pool, or loops that
must not call cudaMalloc/cudaFree because cudaFree can synchronise the device.
For them the solve keeps its small scratch (ticket counter and ready flags) in
a fixed array inside the library.  This test calls that entry point through
the C ABI and checks it against gpc_trsv, the entry point that takes a
caller workspace, on two calls in a row (the shared array must be cleared
between calls), against the oracle (padded leading dimension, n = 4096),
checks that a timed-out wait shows in the library error word, and checks the
size limit.  The file name makes pytest
collect it last.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu
TOL = 1e-10
MAX_N = 262144


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def reference_solve(L, x, trans):
    out = x.clone()
    gp.trsv(L, out, trans=trans)
    return out


@pytest.mark.parametrize("n", [1, 64, 300, 1000])
def test_noalloc_matches_workspace_entry_point_twice(n):
    L = torch.as_tensor(W.known_factor(n, seed=n), device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call, trans in enumerate((0, 1)):  # two calls in a row share the scratch array
        x0 = torch.as_tensor(W.gp_inputs(n, 1, seed=10 + call)[:, 0], device="cuda")
        ref = reference_solve(L, x0, bool(trans)).cpu().numpy()
        x = x0.clone()
        st = gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x.data_ptr(), trans, stream)
        assert st == gp.GPC_OK
        got = x.cpu().numpy()
        assert rel(got, ref) <= TOL
    # the same solve again on the same inputs: identical result
    x1 = x0.clone()
    x2 = x0.clone()
    assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x1.data_ptr(), 1, stream) == gp.GPC_OK
    assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x2.data_ptr(), 1, stream) == gp.GPC_OK
    assert rel(x2.cpu().numpy(), x1.cpu().numpy()) <= TOL


@pytest.mark.parametrize("n,ldl", [(300, 333), (1000, 1024)])
def test_noalloc_padded_leading_dimension(n, ldl):
    Lh = W.known_factor(n, seed=3)
    Lp = np.full((n, ldl), np.nan)  # padding columns never read
    Lp[:, :n] = Lh
    L = torch.as_tensor(Lp, device="cuda")
    x0 = W.gp_inputs(n, 1, seed=4)[:, 0]
    stream = torch.cuda.current_stream().cuda_stream
    for trans in (0, 1):
        x = torch.as_tensor(x0, device="cuda")
        assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), ldl, x.data_ptr(), trans, stream) == gp.GPC_OK
        assert rel(x.cpu().numpy(), O.trsv(Lh, x0, bool(trans))) <= TOL


def test_noalloc_matches_oracle_at_4096():
    n = 4096
    Lh = W.known_factor(n, seed=7)
    L = torch.as_tensor(Lh, device="cuda")
    x0 = W.gp_inputs(n, 1, seed=8)[:, 0]
    stream = torch.cuda.current_stream().cuda_stream
    for trans in (0, 1):
        x = torch.as_tensor(x0, device="cuda")
        assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x.data_ptr(), trans, stream) == gp.GPC_OK
        assert rel(x.cpu().numpy(), O.trsv(Lh, x0, bool(trans))) <= TOL


def test_noalloc_timeout_is_reported_in_the_error_word():
    # a withheld ready flag and a 1 ms wait budget (test hooks): the later
    # blocks give up, the call still returns GPC_OK (it is asynchronous) and
    # the error word says GPC_ERR_TIMEOUT; the next normal call is exact again
    n = 640
    Lh = W.known_factor(n, seed=9)
    L = torch.as_tensor(Lh, device="cuda")
    x0 = W.gp_inputs(n, 1, seed=10)[:, 0]
    stream = torch.cuda.current_stream().cuda_stream
    gp.get_error(clear=True)
    try:
        gp.set_test_fault(gp.GPC_TEST_WAIT_NS, 1_000_000)
        gp.set_test_fault(gp.GPC_TEST_TRSV_WITHHOLD, 4)
        x = torch.as_tensor(x0, device="cuda")
        assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x.data_ptr(), 0, stream) == gp.GPC_OK
        assert gp.get_error(clear=True) == gp.GPC_ERR_TIMEOUT
    finally:
        gp.set_test_fault(gp.GPC_TEST_TRSV_WITHHOLD, -1)
        gp.set_test_fault(gp.GPC_TEST_WAIT_NS, 0)
    x = torch.as_tensor(x0, device="cuda")
    assert gp.capi.gpc_trsv_noalloc(n, L.data_ptr(), n, x.data_ptr(), 0, stream) == gp.GPC_OK
    assert gp.get_error() == gp.GPC_OK
    assert rel(x.cpu().numpy(), O.trsv(Lh, x0, False)) <= TOL


def test_noalloc_rejects_sizes_above_its_limit():
    dummy = torch.zeros(4, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = gp.capi.gpc_trsv_noalloc(MAX_N + 1, dummy.data_ptr(), MAX_N + 1, dummy.data_ptr(), 0, stream)
    assert st == gp.GPC_ERR_INVALID_ARG
    assert gp.capi.gpc_trsv_noalloc(0, None, 0, None, 0, stream) == gp.GPC_OK
