"""Parity at the two intermediate workload sizes.

* n = 4096, d = 8, rho = 1, sigma^2 = 1e-2: the SE covariance, its FP64
  Cholesky factor and the blocked adjoint of a random lower L-bar against the
  oracle's unblocked definitions (relative 1e-10); the mixed factor against
  the same oracle.
* n = 8192, d = 16, rho = 4, sigma = 0.1: the autograd gradient of the LML in
  (alpha, rho, sigma) against central finite differences of the LML with
  h = 1e-6 (FP64 path), and the mixed path's value and gradient against it.
* n = 4096, d = 16, rho = 4 with sigma^2 = lambda_max(K^f) / 1e6
  (tests/golden/cond_sigma_n4096_1e6.json: condition number 9.5e5), the edge
  of the conditioning range of the FP64 bar: the whole GP pass (covariance,
  factor, solves, LML, K-bar, hyperparameter gradient) against the oracle's
  pass at relative 1e-10 (FP64), and the mixed path's errors against it.
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


def rel(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def se4096():
    n, d = 4096, 8
    X = W.gp_inputs(n, d, seed=0)
    K = O.se_cov(X, 1.0, 1.0, 0.1, 0.0)
    Lo = O.chol(K)
    Lbar = W.random_lower(n, seed=1)
    Go = O.chol_adjoint(Lo, Lbar)
    return X, K, Lo, Lbar, Go


def test_se4096_covariance_factor_and_adjoint_fp64(se4096):
    X, K, Lo, Lbar, Go = se4096
    Kd = gp.se_cov(dev(X), 1.0, 1.0, 0.1, 0.0)
    assert rel(np.tril(Kd.cpu().numpy()), np.tril(K)) <= 1e-13
    L = gp.chol(Kd)
    print(f"n=4096 fp64: L {rel(L.cpu().numpy(), Lo):.3e}")
    assert rel(L.cpu().numpy(), Lo) <= 1e-10
    G = gp.chol_adjoint(dev(Lo), dev(Lbar)).cpu().numpy()
    print(f"n=4096 fp64: Kbar {rel(G, Go):.3e}")
    assert rel(G, Go) <= 1e-10


def test_se4096_mixed_factor_and_adjoint(se4096):
    X, K, Lo, Lbar, Go = se4096
    L = gp.chol(dev(K), precision="mixed").cpu().numpy()
    G = gp.chol_adjoint(dev(Lo), dev(Lbar), precision="mixed").cpu().numpy()
    print(f"n=4096 mixed: L {rel(L, Lo):.3e} Kbar {rel(G, Go):.3e}")
    # split-BF16 products (about 2^-39 relative per product) amplified by the
    # conditioning of the trailing updates
    assert rel(L, Lo) <= 1e-9
    assert rel(G, Go) <= 1e-8
    ld = 2.0 * np.sum(np.log(np.diag(Lo)))
    assert abs(2.0 * np.sum(np.log(np.diag(L))) - ld) <= 1e-10 * abs(ld)


@pytest.fixture(scope="module")
def gp8192():
    n, d = 8192, 16
    X = W.gp_inputs(n, d, seed=0)
    y = W.gp_targets(X, 1.0, 4.0, 0.1, seed=1)
    return dev(X), dev(y)


def lml(X, y, hyp, precision="fp64"):
    with torch.no_grad():
        return gp.gp_lml_value(X, y, torch.tensor(hyp, dtype=torch.float64), 0.0, precision).item()


def test_autograd_8192_matches_central_differences(gp8192):
    X, y = gp8192
    hyp = [1.0, 4.0, 0.1]
    h = torch.tensor(hyp, dtype=torch.float64, requires_grad=True)
    v = gp.gp_lml_value(X, y, h, 0.0)
    v.backward()
    g = h.grad.numpy()
    fd = np.empty(3)
    step = 1e-6
    for p in range(3):
        hp, hm = list(hyp), list(hyp)
        hp[p] += step
        hm[p] -= step
        fd[p] = (lml(X, y, hp) - lml(X, y, hm)) / (2 * step)
    err = np.abs(g - fd)
    print(f"n=8192 autograd vs central FD: {err / np.abs(fd)} (value {v.item():.6e})")
    # the difference quotient carries the rounding of the two LML values
    # (measured about 4e-14 |f| each at this size: log-determinant and
    # quadratic-form sums over 8192 terms) divided by 2h, plus O(h^2) truncation
    bound = 1e-13 * abs(v.item()) / step + 1e-7 * np.abs(fd)
    assert np.all(err <= bound), (g, fd, bound)


def test_autograd_8192_mixed_matches_fp64(gp8192):
    X, y = gp8192
    out = {}
    for prec in ("fp64", "mixed"):
        h = torch.tensor([1.0, 4.0, 0.1], dtype=torch.float64, requires_grad=True)
        v = gp.gp_lml_value(X, y, h, 0.0, prec)
        v.backward()
        out[prec] = (v.item(), h.grad.numpy().copy())
    (vf, gf), (vm, gm) = out["fp64"], out["mixed"]
    print(f"n=8192 mixed vs fp64: value {abs(vm - vf) / abs(vf):.3e} grad {rel(gm, gf):.3e}")
    assert abs(vm - vf) <= 1e-8 * abs(vf)
    assert rel(gm, gf) <= 1e-7


@pytest.fixture(scope="module")
def cond1e6():
    rec = json.load(open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                                      "cond_sigma_n4096_1e6.json")))
    n, d, a, r, s = rec["n"], rec["d"], rec["alpha"], rec["rho"], rec["sigma"]
    assert rec["cond"] > 5e5
    X = W.gp_inputs(n, d, seed=rec["seed"])
    y = W.gp_targets(X, a, r, s, seed=1)
    # the oracle's pass, its two O(n^3) steps by the multi-core routines whose
    # factor is bitwise the oracle's (tests/test_cpu_baseline.py)
    ref = O.gp_lml_and_grad_multicore(X, y, a, r, s, 0.0)
    return X, y, (a, r, s), ref


def gp_pass(X, y, hyp, prec):
    n = X.shape[0]
    a, r, s = hyp
    Xd, yd = dev(X), dev(y)
    K = gp.se_cov(Xd, a, r, s, 0.0, precision=prec)
    ws = gp.workspace(n, prec, Xd.device)
    info = gp.new_info(Xd.device)
    res = gp.gp_lml(K, yd, prec, ws=ws, info=info, check=False)
    L = res["L"]
    Kbar = torch.empty_like(K)
    gp.gp_lml_grad(L, res["alpha"], 1.0, prec, out=Kbar, ws=ws)
    g = gp.se_hyper_grad(Xd, a, r, s, Kbar, precision=prec)
    torch.cuda.synchronize()
    return {"L": L.cpu().numpy(), "Kbar": Kbar.cpu().numpy(), "alpha": res["alpha"].cpu().numpy(),
            "logdet": res["logdet"].item(), "value": res["value"].item(), "grad": g.cpu().numpy(),
            "info": info.tolist()}


def pass_errors(out, ref):
    return {"L": rel(out["L"], ref["L"]), "Kbar": rel(out["Kbar"], ref["Kbar"]),
            "alpha": rel(out["alpha"], ref["alpha"]),
            "logdet": abs(out["logdet"] - ref["logdet"]) / abs(ref["logdet"]),
            "value": abs(out["value"] - ref["value"]) / abs(ref["value"]), "grad": rel(out["grad"], ref["grad"])}


def test_cond1e6_fp64_pass_matches_oracle(cond1e6):
    X, y, hyp, ref = cond1e6
    out = gp_pass(X, y, hyp, "fp64")
    assert out["info"] == [-1, gp.GPC_OK]
    e = pass_errors(out, ref)
    print("cond 1e6, n=4096, fp64 vs oracle:", {k: f"{v:.2e}" for k, v in e.items()})
    assert max(e.values()) <= 1e-10, e


def test_cond1e6_mixed_pass_errors(cond1e6):
    X, y, hyp, ref = cond1e6
    out = gp_pass(X, y, hyp, "mixed")
    assert out["info"][1] in (gp.GPC_OK, gp.GPC_ERR_NO_CONVERGENCE)
    e = pass_errors(out, ref)
    print("cond 1e6, n=4096, mixed vs oracle:", {k: f"{v:.2e}" for k, v in e.items()},
          "refinement status", out["info"][1])
    assert e["value"] <= 1e-8 and e["logdet"] <= 1e-8, e
    assert e["grad"] <= 1e-6, e
