"""Parity at the benchmark's full size (n = 16384, d = 16, condition ~1e5), in
the launch configuration bench.py times (se_cov -> gp_lml -> gp_lml_grad ->
se_hyper_grad, both precisions, one workspace).

Element by element against the oracle: the oracle's whole pass at this size
(covariance, factor, solves, log det, LML, L-bar, K-bar, hyperparameter
gradient) with its two O(n^3) steps taken by the multi-core routines whose
factor is bitwise the oracle's and whose adjoint is within 1e-13 of it
(tests/test_cpu_baseline.py), about two minutes on the host cores, computed
once per module.  The FP64 path must match it to relative Frobenius 1e-10 in
L, K-bar, alpha and the gradient and to 1e-10 in log det and the LML value;
the mixed path's errors against it are stated and held to the LML bar of
1e-8.  Besides that, (a) sampled covariance entries that the oracle computes
one by one and (b) properties that hold at any size: (L L^T)_ij = K_ij on
sampled pairs, K alpha = y, log det = 2 sum log L_ii, and the closed form of
the likelihood's adjoint, Kbar = (alpha alpha^T - K^{-1}) in the lower
convention, checked as K (K^{-1} e_j) = e_j for sampled columns j.  The mixed
path is also compared with the FP64 path.
"""
import json
import os

import numpy as np
import pytest
import torch

import paper_1907_01063_gb300 as gp
from oracle import oracle as O
from paper_1907_01063_gb300 import workloads as W

pytestmark = pytest.mark.gpu

N, D = 16384, 16
HERE = os.path.dirname(os.path.abspath(__file__))


def workload():
    rec = json.load(open(os.path.join(HERE, "golden", "cond_sigma.json")))
    assert rec["n"] == N and rec["d"] == D
    X = W.gp_inputs(N, D, seed=0)
    y = W.gp_targets(X, rec["alpha"], rec["rho"], rec["sigma"], seed=1)
    return X, y, (rec["alpha"], rec["rho"], rec["sigma"])


@pytest.fixture(scope="module")
def runs():
    X, y, (a, r, s) = workload()
    dev = torch.device("cuda")
    Xd = torch.as_tensor(X, device=dev)
    yd = torch.as_tensor(y, device=dev)
    ws = gp.workspace(N, "mixed", dev)
    hws = torch.empty(gp.se_hyper_grad_workspace_size(N), dtype=torch.uint8, device=dev)
    out = {}
    for prec in ("fp64", "mixed"):
        K = torch.empty(N, N, dtype=torch.float64, device=dev)
        L = torch.empty_like(K)
        Kbar = torch.empty_like(K)
        info = gp.new_info(dev)
        gp.se_cov(Xd, a, r, s, 0.0, out=K, precision=prec)
        res = gp.gp_lml(K, yd, prec, L=L, ws=ws, info=info, check=False)
        gp.gp_lml_grad(L, res["alpha"], 1.0, prec, out=Kbar, ws=ws)
        g = gp.se_hyper_grad(Xd, a, r, s, Kbar, ws=hws, precision=prec)
        torch.cuda.synchronize()
        out[prec] = {"K": K.cpu().numpy(), "L": L.cpu().numpy(), "Kbar": Kbar.cpu().numpy(),
                     "alpha": res["alpha"].cpu().numpy(), "value": res["value"].item(),
                     "logdet": res["logdet"].item(), "grad": g.cpu().numpy(), "info": info.tolist()}
        del K, L, Kbar
        torch.cuda.empty_cache()
    return X, y, (a, r, s), out


def pairs(count, seed):
    g = np.random.default_rng(seed)
    i = g.integers(0, N, size=count)
    j = (g.random(count) * (i + 1)).astype(np.int64)  # j <= i
    return list(zip(i.tolist(), j.tolist())) + [(N - 1, 0), (N - 1, N - 1), (0, 0), (8191, 8064)]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fullsize_status_and_covariance_samples(runs, prec):
    X, _, (a, r, s), out = runs
    assert out[prec]["info"][1] == gp.GPC_OK
    K = out[prec]["K"]
    tol = 1e-13 if prec == "fp64" else 1e-12
    for i, j in pairs(48, 1):
        if i == j:
            ko = O.se_cov(X[[i]], a, r, s, 0.0)[0, 0]
        else:
            ko = O.se_cov(X[[j, i]], a, r, s, 0.0)[1, 0]
        assert abs(K[i, j] - ko) <= tol * abs(ko), (i, j, K[i, j], ko)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-10)])
def test_fullsize_factor_reproduces_K(runs, prec, tol):
    _, _, _, out = runs
    K, L = out[prec]["K"], out[prec]["L"]
    assert np.all(np.diag(L) > 0)
    for i, j in pairs(64, 2):
        llt = float(np.dot(L[i, : j + 1], L[j, : j + 1]))
        assert abs(llt - K[i, j]) <= tol * np.sqrt(K[i, i] * K[j, j]), (i, j, llt, K[i, j])
    # upper triangle of L is zero (checked on sampled rows)
    for i in (0, 1, 4095, 8192, N - 2):
        assert not np.any(L[i, i + 1:])
    ld = 2.0 * np.sum(np.log(np.diag(L)))
    assert abs(ld - out[prec]["logdet"]) <= 1e-12 * abs(ld)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_fullsize_solve_residual(runs, prec):
    _, y, _, out = runs
    K, alpha = out[prec]["K"], out[prec]["alpha"]
    Ks = np.tril(K) + np.tril(K, -1).T
    r = y - Ks @ alpha
    # the mixed path refines in FP64 to the residual floor
    print(f"solve residual {prec}: {np.linalg.norm(r) / np.linalg.norm(y):.3e}")
    assert np.linalg.norm(r) <= 1e-11 * np.linalg.norm(y)


def test_fullsize_mixed_matches_fp64(runs):
    _, _, _, out = runs
    f, m = out["fp64"], out["mixed"]
    assert abs(m["value"] - f["value"]) <= 1e-8 * abs(f["value"])
    assert abs(m["logdet"] - f["logdet"]) <= 1e-10 * abs(f["logdet"])
    gf, gm = f["grad"], m["grad"]
    print(f"mixed vs fp64: value {abs(m['value'] - f['value']) / abs(f['value']):.3e} "
          f"grad {np.linalg.norm(gm - gf) / np.linalg.norm(gf):.3e}")
    assert np.linalg.norm(gm - gf) <= 1e-7 * np.linalg.norm(gf)


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("mixed", 1e-7)])
def test_fullsize_adjoint_closed_form(runs, prec, tol):
    # Kbar (lower) = alpha alpha^T - K^{-1} off the diagonal and
    # (alpha_i^2 - K^{-1}_ii) / 2 on it, so column j of K^{-1} can be read off
    # Kbar and alpha; K times it must give e_j.  The tolerance is relative to
    # |K| |K^{-1} e_j|, which carries the conditioning (about 1e5).
    _, _, _, out = runs
    K, Kbar, alpha = out[prec]["K"], out[prec]["Kbar"], out[prec]["alpha"]
    Ks = np.tril(K) + np.tril(K, -1).T
    for j in (0, 1234, 8191, N - 1):
        col = np.empty(N)
        col[j:] = alpha[j:] * alpha[j] - Kbar[j:, j]          # rows i >= j: lower column j
        col[:j] = alpha[:j] * alpha[j] - Kbar[j, :j]          # rows i < j: lower row j
        col[j] = alpha[j] ** 2 - 2.0 * Kbar[j, j]
        res = Ks @ col
        res[j] -= 1.0
        scale = np.abs(Ks) @ np.abs(col)
        print(f"adjoint closed form {prec} column {j}: {float(np.max(np.abs(res) / scale)):.3e}")
        assert np.max(np.abs(res) / scale) <= tol, (j, float(np.max(np.abs(res) / scale)))


@pytest.fixture(scope="module")
def oracle_ref(runs):
    X, y, (a, r, s), _ = runs
    return O.gp_lml_and_grad_multicore(X, y, a, r, s, 0.0)


def frob(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def errors_vs_oracle(out, ref):
    return {"L": frob(out["L"], ref["L"]), "Kbar": frob(out["Kbar"], ref["Kbar"]),
            "alpha": frob(out["alpha"], ref["alpha"]),
            "logdet": abs(out["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
            "value": abs(out["value"] - ref["value"]) / abs(ref["value"]),
            "grad": frob(out["grad"], ref["grad"])}


def report(name, rec):
    d = os.environ.get("GPCHOL_REPORT_DIR")
    if d:
        os.makedirs(d, exist_ok=True)
        with open(os.path.join(d, name), "w") as f:
            json.dump(rec, f, indent=1)


def test_fullsize_fp64_matches_oracle_elementwise(runs, oracle_ref):
    _, _, _, out = runs
    e = errors_vs_oracle(out["fp64"], oracle_ref)
    e_mixed = errors_vs_oracle(out["mixed"], oracle_ref)
    report("fullsize_oracle_parity.json", {"n": N, "d": D, "fp64": e, "mixed": e_mixed})
    print("fp64 vs oracle:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-10, e


def test_fullsize_mixed_errors_vs_oracle(runs, oracle_ref):
    _, _, _, out = runs
    e = errors_vs_oracle(out["mixed"], oracle_ref)
    print("mixed vs oracle:", {k: f"{v:.2e}" for k, v in e.items()})
    assert e["value"] <= 1e-8 and e["logdet"] <= 1e-8, e
    assert e["L"] <= 1e-8 and e["alpha"] <= 1e-8, e
    assert e["Kbar"] <= 1e-6 and e["grad"] <= 1e-7, e
