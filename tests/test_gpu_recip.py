"""The refined reciprocals of the diagonal-block factorisation, pinned.

The factorisation's serial path takes 1/x and 1/sqrt(x) of its pivots as the
hardware approximations refined by two Newton-Raphson steps (y <- y (2 - x y)
and y <- y (3 - x y^2) / 2).  Each step roughly doubles the correct bits, so
the result should sit within a couple of units in the last place of the
correctly rounded value.  Checked here over the whole normal exponent range
(x and 1/x both normal for the reciprocal; every positive normal x for the
reciprocal square root) against CUDA's own 1.0 / x and rsqrt(x) evaluated in
the same kernel, and against the host's IEEE division and square root.
"""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp

pytestmark = pytest.mark.gpu


def ulps(a, b):
    ia = np.asarray(a, dtype=np.float64).view(np.int64)
    ib = np.asarray(b, dtype=np.float64).view(np.int64)
    return np.abs(ia - ib)


def probe(x):
    xd = torch.as_tensor(x, device="cuda")
    out = torch.empty(4 * x.size, dtype=torch.float64, device="cuda")
    st = gp.capi.gpc_test_recip_rsqrt(x.size, xd.data_ptr(), out.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == gp.GPC_OK
    return out.cpu().numpy().reshape(-1, 4)


def inputs(lo_exp, hi_exp, count, seed):
    g = np.random.default_rng(seed)
    e = g.integers(lo_exp, hi_exp, size=count)
    m = 1.0 + g.random(count)
    x = np.ldexp(m, e)
    top = np.nextafter(np.ldexp(1.0, hi_exp - 1), 0.0) * 2.0  # the largest double below 2^hi_exp
    edges = np.array([1.0, 2.0, 3.0, 0.5, np.nextafter(1.0, 2.0), np.nextafter(2.0, 1.0),
                      np.ldexp(1.0, lo_exp), np.ldexp(1.0, hi_exp - 1), top])
    return np.concatenate([x, edges])


def test_refined_reciprocal_within_two_ulp():
    x = inputs(-1022, 1022, 200000, 0)  # x and 1/x normal
    r = probe(x)
    d_cuda = ulps(r[:, 0], r[:, 1])
    d_host = ulps(r[:, 0], 1.0 / x)
    print(f"recip: max ulp vs CUDA {d_cuda.max()}, vs host {d_host.max()}, "
          f"exact share {np.mean(d_cuda == 0):.4f}")
    assert np.array_equal(r[:, 1], 1.0 / x)  # CUDA's division is correctly rounded
    assert d_cuda.max() <= 2 and d_host.max() <= 2


def test_refined_rsqrt_within_two_ulp():
    x = inputs(-1022, 1024, 200000, 1)  # every positive normal x
    r = probe(x)
    d_cuda = ulps(r[:, 2], r[:, 3])
    d_host = ulps(r[:, 2], 1.0 / np.sqrt(x))
    print(f"rsqrt: max ulp vs CUDA {d_cuda.max()}, vs host {d_host.max()}, "
          f"exact share {np.mean(d_cuda == 0):.4f}")
    assert d_cuda.max() <= 2
    assert d_host.max() <= 3  # the host value itself is two roundings (sqrt, then divide)
