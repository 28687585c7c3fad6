"""Bounded device waits that run out, made to run out on purpose.

Failure detection is tested without a GPU fault: the test hooks of
gpchol_testing.h shorten the budget of every bounded wait to a millisecond and
either withhold one block's ready flag in the triangular solve or stop the
split product's copy warp from issuing copies.  The waiting kernels must give
up, record GPC_ERR_TIMEOUT in the library error word (and in the per-call
status where the call has one), release what they hold (the product frees its
tensor memory) and return; the next normal call on the same context must be
exact again.  Every wait involved is bounded, so nothing here can hang.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu

SHORT_NS = 1_000_000  # 1 ms


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture
def faults():
    gp.get_error(clear=True)
    yield gp.set_test_fault
    gp.set_test_fault(gp.GPC_TEST_WAIT_NS, 0)
    gp.set_test_fault(gp.GPC_TEST_TRSV_WITHHOLD, -1)
    gp.set_test_fault(gp.GPC_TEST_OZAKI_NO_LOADS, 0)
    torch.cuda.synchronize()
    gp.get_error(clear=True)


def test_error_word_starts_clear_and_clears():
    assert gp.get_error(clear=True) in (gp.GPC_OK, gp.GPC_ERR_TIMEOUT)
    assert gp.get_error() == gp.GPC_OK


@pytest.mark.parametrize("n,withhold,trans", [(640, 3, False), (640, 0, True), (1000, 14, False)])
def test_trsv_withheld_flag_times_out_then_recovers(faults, n, withhold, trans):
    Lh = W.known_factor(n, seed=5)
    x0 = W.gp_inputs(n, 1, seed=6)[:, 0]
    L = torch.as_tensor(Lh, device="cuda")
    faults(gp.GPC_TEST_WAIT_NS, SHORT_NS)
    faults(gp.GPC_TEST_TRSV_WITHHOLD, withhold)
    x = torch.as_tensor(x0, device="cuda")
    gp.trsv(L, x, trans=trans)
    assert gp.get_error(clear=True) == gp.GPC_ERR_TIMEOUT
    # blocks before the withheld one finished normally: their rows are right
    ref = O.trsv(Lh, x0, trans)
    good = slice(0, 64 * withhold) if not trans else slice(n - 64 * withhold, n)
    if withhold > 0:
        assert rel(x.cpu().numpy()[good], ref[good]) <= 1e-12
    # normal budget, nothing withheld: exact again, no error recorded
    faults(gp.GPC_TEST_TRSV_WITHHOLD, -1)
    faults(gp.GPC_TEST_WAIT_NS, 0)
    x = torch.as_tensor(x0, device="cuda")
    gp.trsv(L, x, trans=trans)
    assert gp.get_error() == gp.GPC_OK
    assert rel(x.cpu().numpy(), ref) <= 1e-12


def test_split_product_abort_frees_tensor_memory_and_recovers(faults):
    g = np.random.default_rng(11)
    a = g.integers(-(2 ** 16 - 1), 2 ** 16, size=(300, 256)).astype(np.int64)
    b = g.integers(-(2 ** 16 - 1), 2 ** 16, size=(200, 256)).astype(np.int64)
    A = torch.as_tensor(a * 2.0 ** -16, device="cuda")
    B = torch.as_tensor(b * 2.0 ** -16, device="cuda")
    faults(gp.GPC_TEST_WAIT_NS, SHORT_NS)
    faults(gp.GPC_TEST_OZAKI_NO_LOADS, 1)
    with pytest.raises(gp.GpcholError) as e:
        gp.test_ozaki_gemm(A, B)  # the per-call status word reports the timeout
    assert e.value.status == gp.GPC_ERR_TIMEOUT
    assert gp.get_error(clear=True) == gp.GPC_ERR_TIMEOUT
    faults(gp.GPC_TEST_OZAKI_NO_LOADS, 0)
    faults(gp.GPC_TEST_WAIT_NS, 0)
    # every persistent CTA allocated and freed its tensor memory: a normal
    # product on all SMs runs and is exact (16-bit operands: every step exact)
    for _ in range(2):
        C = gp.test_ozaki_gemm(A, B).cpu().numpy()
        assert np.array_equal(C, (a @ b.T).astype(np.float64) * 2.0 ** -32)
    assert gp.get_error() == gp.GPC_OK


def test_gp_step_reports_no_error():
    n = 300
    X = W.gp_inputs(n, 2, seed=0)
    y = W.gp_targets(X, 1.0, 0.5, 0.1, seed=1)
    gp.get_error(clear=True)
    for precision in ("fp64", "mixed"):
        h = torch.tensor([1.0, 0.5, 0.1], dtype=torch.float64, requires_grad=True)
        v = gp.gp_lml_value(torch.as_tensor(X, device="cuda"), torch.as_tensor(y, device="cuda"), h, 1e-8,
                            precision=precision)
        v.backward()
    assert gp.get_error() == gp.GPC_OK
