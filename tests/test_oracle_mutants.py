"""The oracle's pins must catch plausible mistakes.

Each mutant below is a one-line error planted in a temporary copy of the
oracle's C source (a dropped term, a wrong sign, index or factor, a transposed
operand).  The copy is compiled on the CPU and the pin suite is run against it
in a subprocess; every mutant must make at least one pin fail.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "gpchol_oracle.c")

MUTANTS = {
    "chol_wrong_index": ("s -= AT(L, ldl, i, k) * AT(L, ldl, j, k);",
                         "s -= AT(L, ldl, i, k) * AT(L, ldl, i, k);"),
    "chol_no_sqrt": ("AT(L, ldl, i, i) = sqrt(s);", "AT(L, ldl, i, i) = s;"),
    "adj_diag_factor": ("sbar = AT(W, n, i, i) / (2.0 * AT(L, ldl, i, i));",
                        "sbar = AT(W, n, i, i) / AT(L, ldl, i, i);"),
    "adj_drop_pivot_term": ("AT(W, n, j, j) -= AT(W, n, i, j) * AT(L, ldl, i, j) / ljj;", ""),
    "adj_sign": ("AT(W, n, j, k) -= sbar * AT(L, ldl, i, k);",
                 "AT(W, n, j, k) += sbar * AT(L, ldl, i, k);"),
    "trsv_transposed": ("for (int k = i + 1; k < n; ++k) s -= AT(L, ldl, k, i) * x[k];",
                        "for (int k = i + 1; k < n; ++k) s -= AT(L, ldl, i, k) * x[k];"),
    "sym_no_halving": ("if (i == j) s *= 0.5;", ""),
    "secov_scale": ("exp(-r2 / (2.0 * rho * rho));\n    }", "exp(-r2 / (rho * rho));\n    }"),
    "lml_logdet_weight": ("*value = -0.5 * q - 0.5 * ld", "*value = -0.5 * q - ld"),
    "lbar_sign": ("if (i == j) v -= 1.0 / AT(L, ldl, i, i);",
                  "if (i == j) v += 1.0 / AT(L, ldl, i, i);"),
    "hyper_rho_power": ("gr += kb * kf * r2 / (rho * rho * rho);",
                        "gr += kb * kf * r2 / (rho * rho);"),
    "hyper_alpha_factor": ("ga += kb * 2.0 * kf / alpha;", "ga += kb * kf / alpha;"),
    "trinv_diag_index": ("AT(X, ldx, i, j) = -s / AT(L, ldl, i, i);",
                         "AT(X, ldx, i, j) = -s / AT(L, ldl, j, j);"),
    "trinv_dropped_term": ("for (int k = j; k < i; ++k) s += AT(L, ldl, i, k) * AT(X, ldx, k, j);",
                           "for (int k = j + 1; k < i; ++k) s += AT(L, ldl, i, k) * AT(X, ldx, k, j);"),
    "trsolve_sign": ("s -= AT(L, ldl, i, k) * AT(C, ldc, k, j);", "s += AT(L, ldl, i, k) * AT(C, ldc, k, j);"),
    "trsolve_adj_untransposed": ("s -= AT(L, ldl, k, i) * AT(Bbar, ldbb, k, j);",
                                 "s -= AT(L, ldl, i, k) * AT(Bbar, ldbb, k, j);"),
    "trsolve_adj_lbar_transposed": ("s -= AT(Bbar, ldbb, i, t) * AT(C, ldc, j, t);",
                                    "s -= AT(Bbar, ldbb, j, t) * AT(C, ldc, i, t);"),
    "gemm_transposed_b": ("for (int t = 0; t < k; ++t) s += AT(A, lda, i, t) * AT(B, ldb, t, j);",
                          "for (int t = 0; t < k; ++t) s += AT(A, lda, i, t) * AT(B, ldb, j, t);"),
    "gemm_adj_untransposed": ("for (int j = 0; j < n; ++j) s += AT(Cbar, ldcb, i, j) * AT(B, ldb, t, j);",
                              "for (int j = 0; j < n; ++j) s += AT(Cbar, ldcb, i, j) * AT(B, ldb, j, t);"),
    "glm_logit_derivative_sign": ("di = y[i] - 1.0 / (1.0 + exp(-eta));", "di = y[i] - 1.0 / (1.0 + exp(eta));"),
    "glm_softplus_branch": ("double softplus = (eta > 0.0 ? eta : 0.0) + log1p(exp(-fabs(eta)));",
                            "double softplus = log1p(exp(-fabs(eta)));"),
    "glm_dropped_alpha": ("double eta = alpha;", "double eta = 0.0;"),
    "glm_poisson_lgamma": ("li = y[i] * eta - exp(eta) - lgamma(y[i] + 1.0);", "li = y[i] * eta - exp(eta);"),
    "glm_normal_dsigma": ("sds += (y[i] - eta) * (y[i] - eta) / (sigma * sigma * sigma) - 1.0 / sigma;",
                          "sds += (y[i] - eta) * (y[i] - eta) / (sigma * sigma) - 1.0 / sigma;"),
    "digamma_recurrence_sign": ("    acc -= 1.0 / x;\n", "    acc += 1.0 / x;\n"),
    "negbin_dropped_lgamma_phi": ("li = lgamma(y[i] + phi) - lgamma(y[i] + 1.0) - lgamma(phi) + phi",
                                  "li = lgamma(y[i] + phi) - lgamma(y[i] + 1.0) + phi"),
    "negbin_derivative_factor": ("di = y[i] - (y[i] + phi) * mu / (mu + phi);", "di = y[i] - y[i] * mu / (mu + phi);"),
    "categorical_wrong_class": ("slp += eta[yi] - lse;", "slp += eta[0] - lse;"),
    "categorical_dropped_alpha": ("    double e = alpha[c];\n", "    double e = 0.0;\n"),
    "ordinal_cut_sign": ("if (yi > 0) dcuts[yi - 1] -= du;", "if (yi > 0) dcuts[yi - 1] += du;"),
    "ordinal_wrong_cut_index": ("if (yi < C - 1) sv = 1.0 / (1.0 + exp(-(eta - cuts[yi])));",
                                "if (yi < C - 1) sv = 1.0 / (1.0 + exp(-(eta - cuts[yi > 0 ? yi - 1 : 0])));"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site for {name} not found exactly once"
    mut = tmp_path / "mutant.c"
    mut.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC",
                           "-o", str(lib), str(mut), "-lm"])
    env = dict(os.environ, GPCHOL_ORACLE_LIB=str(lib))
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle.py")],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
