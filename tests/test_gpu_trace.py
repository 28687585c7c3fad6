"""Launch trace and timeline (measurement support) through the C ABI."""
import pytest
import torch

import paper_1907_01063_gb300 as gp
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_timeline_lists_every_launch_in_order():
    n = 300
    L0 = torch.as_tensor(W.known_factor(n, seed=1), device="cuda")
    K = L0 @ L0.T
    torch.cuda.synchronize()
    c0 = gp.launch_count()
    gp.trace_enable(True, timeline=True)
    gp.chol(K)
    torch.cuda.synchronize()
    gp.trace_enable(False)
    spans = gp.trace_timeline()
    assert len(spans) == gp.launch_count() - c0 > 0
    names = [s["kernel"] for s in spans]
    # FP64 block 128: blocks of 128, 128 and 44 rows; blocks of up to 64 rows
    # take the lookahead kernel
    assert names.count("potrf_diag_kernel") == 2 and names.count("potrf_la_kernel") == 1
    assert all("launch_k" not in nm and "<<<" not in nm for nm in names)
    assert all(s["dur_ms"] > 0 for s in spans)
    starts = [s["start_ms"] for s in spans]
    assert starts[0] == 0.0 and all(b >= a for a, b in zip(starts, starts[1:]))
    summary = gp.trace_summary()
    assert sum(v["launches"] for v in summary.values()) == len(spans)
    # plain tracing (no timeline) leaves the recorded spans alone
    gp.trace_enable(True)
    gp.chol(K)
    gp.trace_enable(False)
    assert len(gp.trace_timeline()) == len(spans)
