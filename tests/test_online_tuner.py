"""Online tuning across repeated calls (Section 5): the host-side logic of
``autotune.OnlineTuner`` with a fake timer and a fake knob (no GPU), and one
GPU run with the FP64 block size."""
import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from paper_1907_01063_gb300 import autotune


class FakeTimer:
    """Durations come from a table indexed by the knob value at start()."""

    def __init__(self, knob_state, ms_of_value):
        self.knob, self.ms = knob_state, ms_of_value
        self.reads = 0

    def start(self):
        return {"value": self.knob["v"], "stopped": False}

    def stop(self, tok):
        tok["stopped"] = True

    def elapsed_ms(self, tok):
        assert tok["stopped"]
        self.reads += 1
        return self.ms[tok["value"]]


def make(ms, candidates, reps=1):
    knob = {"v": 0}
    log = []

    def setter(k, v):
        knob["v"] = v
        log.append(v)

    timer = FakeTimer(knob, ms)
    t = autotune.OnlineTuner(7, candidates, reps=reps, timer=timer, setter=setter, getter=lambda k: knob["v"])
    return t, knob, log, timer


def test_explores_each_candidate_then_keeps_the_fastest():
    t, knob, log, timer = make({64: 3.0, 96: 2.0, 128: 2.5}, [64, 96, 128], reps=2)
    seen = []
    for _ in range(10):
        t("chol/4096", lambda: seen.append(knob["v"]))
    assert seen == [64, 64, 96, 96, 128, 128, 96, 96, 96, 96]
    assert t.best("chol/4096") == 96
    assert t.times("chol/4096") == {64: 3.0, 96: 2.0, 128: 2.5}
    assert timer.reads == 6  # each exploration call read once, at the decision
    assert knob["v"] == 0  # the knob is restored after every call
    assert log[-1] == 0


def test_keys_are_independent_and_ties_keep_the_earlier_candidate():
    t, knob, _, _ = make({32: 1.0, 64: 1.0}, [32, 64])
    for _ in range(3):
        t(("batch", 512), lambda: None)
    assert t.best(("batch", 512)) == 32
    assert t.best(("batch", 1024)) is None
    t(("batch", 1024), lambda: None)
    assert t.best(("batch", 1024)) is None  # one of two candidates seen
    t(("batch", 1024), lambda: None)
    assert t.best(("batch", 1024)) == 32


def test_result_and_exceptions_pass_through_and_restore_the_knob():
    t, knob, _, _ = make({1: 1.0, 2: 2.0}, [1, 2])
    assert t("k", lambda: 42) == 42
    with pytest.raises(RuntimeError):
        t("k", lambda: (_ for _ in ()).throw(RuntimeError("boom")))
    assert knob["v"] == 0


def test_rejects_empty_candidates():
    with pytest.raises(ValueError):
        autotune.OnlineTuner(0, [], timer=object(), setter=lambda k, v: None, getter=lambda k: 0)


@pytest.mark.gpu
def test_online_tuner_on_the_fp64_factorisation():
    from oracle import oracle as O
    from paper_1907_01063_gb300 import workloads as W
    n = 600
    L0 = W.known_factor(n, seed=0)
    K = torch.as_tensor(L0 @ L0.T, device="cuda")
    old = gp.get_tuning(gp.GPC_TUNE_BLOCK)
    t = autotune.OnlineTuner(gp.GPC_TUNE_BLOCK, [64, 128], reps=1)
    outs = [t(("chol", n), lambda: gp.chol(K)) for _ in range(4)]
    assert t.best(("chol", n)) in (64, 128)
    assert gp.get_tuning(gp.GPC_TUNE_BLOCK) == old
    ref = O.chol(L0 @ L0.T)
    for L in outs:
        assert np.linalg.norm(L.cpu().numpy() - ref) <= 1e-10 * np.linalg.norm(ref)
