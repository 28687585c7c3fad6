"""The mixed path's FP64 -> double-float conversion, pinned.

Every FP64 entry that enters a split product, the double-float covariance
gradient or the double-float solves is split into an FP32 pair hi + lo with
hi = x rounded to nearest FP32 and lo = the remainder x - hi rounded to
nearest FP32.  On GB300 the conversion instructions (FP64 to FP32 and integer
to FP32) issue on the slow FP64 pipe, so the library forms the pair from the
bit fields: the mantissa's top 23 bits rounded half-to-even on the 29 below,
and the signed 29-bit remainder rounded to FP32 through two exponent-field
conversions and one FMA.  Checked here bit for bit against the host's IEEE
conversions (numpy's float64 -> float32 is round-to-nearest-even) over the
whole range the field moves cover, its edges, every rounding tie and the
values outside it (which take the conversion instructions), and the exact
FP32 -> FP64 move back.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp

pytestmark = pytest.mark.gpu


def probe(x):
    xd = torch.as_tensor(x, device="cuda")
    hilo = torch.empty(2 * x.size, dtype=torch.float32, device="cuda")
    back = torch.empty(x.size, dtype=torch.float64, device="cuda")
    st = gp.capi.gpc_test_split_f64(x.size, xd.data_ptr(), hilo.data_ptr(), back.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)
    assert st == gp.GPC_OK
    hl = hilo.cpu().numpy().reshape(-1, 2)
    return hl[:, 0], hl[:, 1], back.cpu().numpy()


def host_split(x):
    hi = x.astype(np.float32)
    with np.errstate(over="ignore", invalid="ignore"):
        lo = (x - hi.astype(np.float64)).astype(np.float32)
    return hi, lo


def check(x):
    hi, lo, back = probe(x)
    rhi, rlo = host_split(x)
    assert np.array_equal(hi.view(np.uint32), rhi.view(np.uint32))
    assert np.array_equal(lo.view(np.uint32), rlo.view(np.uint32))
    with np.errstate(invalid="ignore"):
        ref_back = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.array_equal(back, ref_back, equal_nan=True)


def test_split_random_over_the_field_move_range():
    g = np.random.default_rng(0)
    n = 400000
    # |x| in [2^-74, 2^127): both parts normal FP32
    e = g.integers(-74, 127, size=n)
    x = np.ldexp(1.0 + g.random(n), e) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    check(x)


def test_split_rounding_ties_and_edges():
    g = np.random.default_rng(1)
    n = 100000
    e = g.integers(-74, 127, size=n)
    # mantissas whose 29 bits below the FP32 mantissa are exactly one half
    # (ties, both parities), just below and just above it, all ones and zero
    m23 = g.integers(0, 1 << 23, size=n, dtype=np.int64)
    low = np.array([1 << 28, (1 << 28) - 1, (1 << 28) + 1, (1 << 29) - 1, 0, 1], dtype=np.int64)
    rem = low[g.integers(0, low.size, size=n)]
    bits = ((e + 1023).astype(np.int64) << 52) | (m23 << 29) | rem
    x = bits.view(np.float64) * np.where(g.random(n) < 0.5, -1.0, 1.0)
    edges = np.array([np.ldexp(1.0, -74), -np.ldexp(1.0, -74), np.nextafter(np.ldexp(1.0, 127), 0.0),
                      np.ldexp(1.0 - 2.0 ** -30, 127), 1.0, -1.0, 3.0, 1.0 / 3.0, np.pi])
    check(np.concatenate([x, edges]))


def test_split_outside_the_range_takes_the_conversions():
    g = np.random.default_rng(2)
    n = 20000
    e = np.concatenate([g.integers(-140, -74, size=n), g.integers(127, 128, size=n)])
    x = np.ldexp(1.0 + g.random(2 * n), e)
    specials = np.array([0.0, -0.0, np.ldexp(1.0, -1074), 1e-300, -1e-300])
    check(np.concatenate([x, specials]))
