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


def test_coordinate_search_walks_each_knob_with_the_others_at_their_best():
    from paper_1907_01063_gb300.autotune import coordinate_search
    # separable cost with a unique optimum at a=2, b=30; first candidates are the start
    cost = {("a", 1): 5.0, ("a", 2): 1.0, ("a", 3): 4.0, ("b", 10): 3.0, ("b", 20): 2.0, ("b", 30): 0.5}
    calls = []

    def measure(cfg):
        calls.append(dict(cfg))
        return cost[("a", cfg["a"])] + cost[("b", cfg["b"])]

    res = coordinate_search([("a", (1, 2, 3)), ("b", (10, 20, 30))], measure)
    assert res["best"] == {"a": 2, "b": 30}
    # a varied with b at its start value, then b varied with a at its best; no repeats
    assert calls == [{"a": 1, "b": 10}, {"a": 2, "b": 10}, {"a": 3, "b": 10}, {"a": 2, "b": 20}, {"a": 2, "b": 30}]
    assert len(res["ms"]) == 5
    # ties keep the earlier candidate; an explicit start is honoured
    res = coordinate_search([("a", (1, 2))], lambda cfg: 1.0, start={"a": 2})
    assert res["best"] == {"a": 1}


def test_n_bucket():
    from paper_1907_01063_gb300.autotune import n_bucket
    assert [n_bucket(n) for n in (1, 1024, 1025, 3000, 16384, 20000)] == [1024, 1024, 2048, 4096, 16384, 16384]


@pytest.mark.gpu
def test_tuned_mixed_schedule_runs_at_parity(tmp_path, monkeypatch):
    # tune the mixed schedule at a small order (cache in a scratch file), then
    # run the factorisation and adjoint with the chosen knobs against the oracle
    from oracle import oracle as O
    from paper_1907_01063_gb300 import workloads as W
    monkeypatch.setenv("GPCHOL_TUNE_CACHE", str(tmp_path / "tune.json"))
    ids = [gp.GPC_TUNE_MIXED_DEFER, gp.GPC_TUNE_MIXED_FREE_SMS, gp.GPC_TUNE_MIXED_ADJ_FREE_SMS]
    saved = [gp.get_tuning(k) for k in ids]
    try:
        rec = autotune.tune_mixed(1000)
        assert rec["n"] == 1024 and set(rec["best"]) == {"mixed_defer", "mixed_free_sms", "mixed_adj_free_sms"}
        assert gp.get_tuning(gp.GPC_TUNE_MIXED_DEFER) == rec["best"]["mixed_defer"]
        n = 1000
        X = W.gp_inputs(n, 3, seed=4)
        K = O.se_cov(X, 1.0, 1.0, 0.3, 1e-6)
        Lo = O.chol(K)
        Lbar = W.random_lower(n, seed=5)
        Go = O.chol_adjoint(Lo, Lbar)
        L = gp.chol(torch.as_tensor(K, device="cuda"), "mixed").cpu().numpy()
        G = gp.chol_adjoint(torch.as_tensor(Lo, device="cuda"), torch.as_tensor(Lbar, device="cuda"),
                            precision="mixed").cpu().numpy()
        assert np.linalg.norm(L - Lo) <= 1e-9 * np.linalg.norm(Lo)
        assert np.linalg.norm(G - Go) <= 1e-8 * np.linalg.norm(Go)
        # a second call reads the cache instead of timing again
        assert autotune.tune_mixed(1000)["when"] == rec["when"]
    finally:
        for k, v in zip(ids, saved):
            gp.set_tuning(k, v)
