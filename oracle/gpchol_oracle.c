/*
 * gpchol_oracle.c -- plain, slow, single-threaded FP64 CPU oracle for the
 * dense Cholesky / Cholesky-adjoint / Gaussian-process likelihood path of
 * "GPU-based Parallel Computation Support for Stan" (Cesnovar et al., 2019).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  The GPU library shares no code,
 * header, table or helper with this file, and nothing here is ever used on
 * the product path.
 *
 * Conventions: every matrix is FP64, row-major, element (i,j) at a[i*ld + j],
 * ld >= n.  Only the lower triangle (i >= j) of a symmetric input is read.
 * Lower-triangular outputs have their strict upper triangle set to zero.
 * Compile with -O2 -ffp-contract=off (no fused multiply-add contraction), so
 * every sum is an ordinary left-to-right FP64 sum in the order written.
 *
 * Every function is the plain unblocked definition of what the paper's
 * blocked GPU routines compute; none of them is blocked, fused or reordered.
 */
#include <math.h>

#define ORACLE_TWO_PI 6.283185307179586476925286766559
#include <stdlib.h>
#include <string.h>

#define AT(a, ld, i, j) ((a)[(size_t)(i) * (size_t)(ld) + (size_t)(j)])

/*
 * Cholesky factor L of an SPD matrix K (K = L L^T, L lower, L_ii > 0).
 * Section 3.3 (Cholesky decomposition, primitive function) partitions
 * K = [A11 .; A21 A22] into L11 = chol(A11), L21 = A21 L11^{-T},
 * L22 = chol(A22 - L21 L21^T).  Taking A11 to be 1x1 at every level gives
 * the row-by-row Cholesky-Banachiewicz recurrence written here:
 *   s = K_ij - sum_{k<j} L_ik L_jk  (k ascending),
 *   L_ii = sqrt(s) on the diagonal, L_ij = s / L_jj below it.
 * A pivot s that is not > 0 (this includes NaN) stops the factorisation.
 * Returns -1 on success, else the 0-based index of the first failing pivot
 * (rows from that index on are left as they were when it stopped).
 * K and L may be the same buffer.
 */
int oracle_chol(int n, const double *K, int ldk, double *L, int ldl) {
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double s = AT(K, ldk, i, j);
      for (int k = 0; k < j; ++k) s -= AT(L, ldl, i, k) * AT(L, ldl, j, k);
      if (i == j) {
        if (!(s > 0.0)) return i;
        AT(L, ldl, i, i) = sqrt(s);
      } else {
        AT(L, ldl, i, j) = s / AT(L, ldl, j, j);
      }
    }
    for (int j = i + 1; j < n; ++j) AT(L, ldl, i, j) = 0.0;
  }
  return -1;
}

/*
 * Reverse mode of oracle_chol: given L and an adjoint Lbar (lower), returns
 * Kbar (lower) = d f / d K_ij for i >= j, where f depends on K only through
 * the lower-triangle entries that chol reads (Section 3.3, reverse mode
 * function; Murray 2016 gives the unblocked form this follows).
 * Each statement of the forward recurrence is reversed, visiting (i,j) in the
 * exact reverse of the forward order (i descending, then j descending):
 *   diagonal  L_ii = sqrt(s):   sbar = Lbar_ii / (2 L_ii)
 *   off-diag  L_ij = s / L_jj:  sbar = Lbar_ij / L_jj,
 *                                Lbar_jj -= Lbar_ij L_ij / L_jj
 *   then Kbar_ij = sbar, and for k < j (from s -= L_ik L_jk):
 *                                Lbar_ik -= sbar L_jk,  Lbar_jk -= sbar L_ik.
 * Lbar is copied first and not modified.  Kbar may alias Lbar.
 * Returns 0, or -1 if the scratch copy cannot be allocated.
 */
int oracle_chol_adjoint(int n, const double *L, int ldl, const double *Lbar,
                        int ldlb, double *Kbar, int ldkb) {
  double *W = (double *)malloc((size_t)n * (size_t)n * sizeof(double) + 8);
  if (!W) return -1;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) AT(W, n, i, j) = (j <= i) ? AT(Lbar, ldlb, i, j) : 0.0;
  for (int i = n - 1; i >= 0; --i) {
    for (int j = i; j >= 0; --j) {
      double sbar;
      if (i == j) {
        sbar = AT(W, n, i, i) / (2.0 * AT(L, ldl, i, i));
      } else {
        double ljj = AT(L, ldl, j, j);
        sbar = AT(W, n, i, j) / ljj;
        AT(W, n, j, j) -= AT(W, n, i, j) * AT(L, ldl, i, j) / ljj;
      }
      AT(W, n, i, j) = sbar; /* this slot now holds Kbar_ij */
      for (int k = 0; k < j; ++k) {
        AT(W, n, i, k) -= sbar * AT(L, ldl, j, k);
        AT(W, n, j, k) -= sbar * AT(L, ldl, i, k);
      }
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) AT(Kbar, ldkb, i, j) = (j <= i) ? AT(W, n, i, j) : 0.0;
  free(W);
  return 0;
}

/* x <- L^{-1} x (trans = 0) or x <- L^{-T} x (trans = 1); plain forward /
 * back substitution with L lower (Section 3.2, solving triangular systems:
 * the result the inverse-based GPU solver reaches). */
void oracle_trsv(int n, const double *L, int ldl, double *x, int trans) {
  if (!trans) {
    for (int i = 0; i < n; ++i) {
      double s = x[i];
      for (int k = 0; k < i; ++k) s -= AT(L, ldl, i, k) * x[k];
      x[i] = s / AT(L, ldl, i, i);
    }
  } else {
    for (int i = n - 1; i >= 0; --i) {
      double s = x[i];
      for (int k = i + 1; k < n; ++k) s -= AT(L, ldl, k, i) * x[k];
      x[i] = s / AT(L, ldl, i, i);
    }
  }
}

/*
 * Symbolic Cholesky adjoint (Murray 2016, the identity the blocked gradient of
 * Section 3.3 applies block by block), as an independent cross-check of
 * oracle_chol_adjoint:
 *   P = Phi(L^T Lbar)   (Phi: lower triangle, diagonal halved)
 *   S = L^{-T} P L^{-1}
 *   Kbar_ij = S_ij + S_ji (i > j),  Kbar_ii = S_ii,  upper = 0.
 * L^{-1} is applied by substitution, column by column.
 * Returns 0, or -1 if scratch cannot be allocated.
 */
int oracle_chol_adjoint_symbolic(int n, const double *L, int ldl, const double *Lbar,
                                 int ldlb, double *Kbar, int ldkb) {
  double *P = (double *)malloc((size_t)n * (size_t)n * sizeof(double) + 8);
  double *col = (double *)malloc((size_t)n * sizeof(double) + 8);
  if (!P || !col) { free(P); free(col); return -1; }
  /* P = Phi(L^T Lbar): (L^T Lbar)_ij = sum_k L_ki Lbar_kj over k >= max(i,j). */
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      if (j <= i) {
        for (int k = i; k < n; ++k) s += AT(L, ldl, k, i) * AT(Lbar, ldlb, k, j);
        if (i == j) s *= 0.5;
      }
      AT(P, n, i, j) = s;
    }
  }
  /* T = P L^{-1}: row r of T solves t L = p_r, i.e. L^T t^T = p_r^T. */
  for (int r = 0; r < n; ++r) {
    for (int c = 0; c < n; ++c) col[c] = AT(P, n, r, c);
    oracle_trsv(n, L, ldl, col, 1);
    for (int c = 0; c < n; ++c) AT(P, n, r, c) = col[c];
  }
  /* S = L^{-T} T: column c of S solves L^T s = t_c. */
  for (int c = 0; c < n; ++c) {
    for (int r = 0; r < n; ++r) col[r] = AT(P, n, r, c);
    oracle_trsv(n, L, ldl, col, 1);
    for (int r = 0; r < n; ++r) AT(P, n, r, c) = col[r];
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      if (j < i) v = AT(P, n, i, j) + AT(P, n, j, i);
      else if (j == i) v = AT(P, n, i, i);
      AT(Kbar, ldkb, i, j) = v;
    }
  free(P);
  free(col);
  return 0;
}

/*
 * Squared-exponential covariance (the GP covariance of the Gaussian-process
 * regression example of Section 4.2; the kernel's form is not printed there):
 *   K_ij = alpha^2 exp(-sum_t (x_it - x_jt)^2 / (2 rho^2))  (i != j)
 *   K_ii = alpha^2 + sigma^2 + jitter
 * with direct coordinate differences.  Writes the lower triangle; when
 * full != 0 the upper triangle is mirrored, else it is set to zero.
 */
void oracle_se_cov(int n, int d, const double *X, int ldx, double alpha, double rho,
                   double sigma, double jitter, double *K, int ldk, int full) {
  double a2 = alpha * alpha;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < i; ++j) {
      double r2 = 0.0;
      for (int t = 0; t < d; ++t) {
        double df = AT(X, ldx, i, t) - AT(X, ldx, j, t);
        r2 += df * df;
      }
      AT(K, ldk, i, j) = a2 * exp(-r2 / (2.0 * rho * rho));
    }
    AT(K, ldk, i, i) = a2 + sigma * sigma + jitter;
    for (int j = i + 1; j < n; ++j) AT(K, ldk, i, j) = 0.0;
  }
  if (full)
    for (int i = 0; i < n; ++i)
      for (int j = i + 1; j < n; ++j) AT(K, ldk, i, j) = AT(K, ldk, j, i);
}

/*
 * Gaussian-process log marginal likelihood of y ~ N(0, K) through the
 * Cholesky factor (the quantity the GP regression model of Section 4.2
 * evaluates every gradient step):
 *   L = chol(K);  z = L^{-1} y;  alpha = L^{-T} z;
 *   logdet = 2 sum_i log L_ii;
 *   value = -1/2 z.z - 1/2 logdet - (n/2) log(2 pi).
 * oracle_gp_lml_factored takes the steps after L = chol(K) for a given factor
 * L; oracle_gp_lml is oracle_chol followed by it.
 * Writes L (may alias K), z and alpha (n each; may be NULL), logdet and value.
 * Returns -1 on success, the failing pivot of oracle_chol, or -2 if scratch
 * cannot be allocated.
 */
int oracle_gp_lml_factored(int n, const double *L, int ldl, const double *y, double *z, double *alpha,
                           double *logdet, double *value);

int oracle_gp_lml(int n, const double *K, int ldk, const double *y, double *L, int ldl,
                  double *z, double *alpha, double *logdet, double *value) {
  int info = oracle_chol(n, K, ldk, L, ldl);
  if (info >= 0) return info;
  return oracle_gp_lml_factored(n, L, ldl, y, z, alpha, logdet, value);
}

int oracle_gp_lml_factored(int n, const double *L, int ldl, const double *y, double *z, double *alpha,
                           double *logdet, double *value) {
  double *zz = (double *)malloc((size_t)n * sizeof(double) + 8);
  double *aa = (double *)malloc((size_t)n * sizeof(double) + 8);
  if (!zz || !aa) { free(zz); free(aa); return -2; }
  for (int i = 0; i < n; ++i) zz[i] = y[i];
  oracle_trsv(n, L, ldl, zz, 0);
  for (int i = 0; i < n; ++i) aa[i] = zz[i];
  oracle_trsv(n, L, ldl, aa, 1);
  double ld = 0.0, q = 0.0;
  for (int i = 0; i < n; ++i) ld += log(AT(L, ldl, i, i));
  ld *= 2.0;
  for (int i = 0; i < n; ++i) q += zz[i] * zz[i];
  if (logdet) *logdet = ld;
  if (value) *value = -0.5 * q - 0.5 * ld - 0.5 * (double)n * log(ORACLE_TWO_PI);
  if (z) memcpy(z, zz, (size_t)n * sizeof(double));
  if (alpha) memcpy(alpha, aa, (size_t)n * sizeof(double));
  free(zz);
  free(aa);
  return -1;
}

/*
 * Upstream adjoint of the log marginal likelihood with respect to L, scaled by
 * gbar (reverse mode of oracle_gp_lml's value for fixed y):
 *   Lbar = gbar * (tril(alpha z^T) - diag(1 / L_ii)).
 * d(-1/2 z.z) = alpha^T dL z gives the first term, d(-sum log L_ii) the second.
 */
void oracle_lml_lbar(int n, const double *L, int ldl, const double *alpha, const double *z,
                     double gbar, double *Lbar, int ldlb) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double v = 0.0;
      if (j <= i) {
        v = alpha[i] * z[j];
        if (i == j) v -= 1.0 / AT(L, ldl, i, i);
        v *= gbar;
      }
      AT(Lbar, ldlb, i, j) = v;
    }
}

/*
 * Hyperparameter gradient of a scalar f(K(alpha, rho, sigma)) from Kbar in the
 * lower-triangle convention of oracle_chol_adjoint (Kbar_ij = df/dK_ij over
 * the entries i >= j that chol reads), with K from oracle_se_cov:
 *   g_alpha = sum_{i>=j} Kbar_ij * 2 K^f_ij / alpha
 *   g_rho   = sum_{i>=j} Kbar_ij * K^f_ij * r2_ij / rho^3
 *   g_sigma = sum_i Kbar_ii * 2 sigma
 * where K^f_ij = alpha^2 exp(-r2_ij / (2 rho^2)) is the noise-free part and the
 * jitter is a constant.  grad3 = {g_alpha, g_rho, g_sigma}.
 */
void oracle_se_hyper_grad(int n, int d, const double *X, int ldx, double alpha, double rho,
                          double sigma, const double *Kbar, int ldkb, double *grad3) {
  double ga = 0.0, gr = 0.0, gs = 0.0;
  double a2 = alpha * alpha;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j <= i; ++j) {
      double r2 = 0.0;
      for (int t = 0; t < d; ++t) {
        double df = AT(X, ldx, i, t) - AT(X, ldx, j, t);
        r2 += df * df;
      }
      double kf = a2 * exp(-r2 / (2.0 * rho * rho));
      double kb = AT(Kbar, ldkb, i, j);
      ga += kb * 2.0 * kf / alpha;
      gr += kb * kf * r2 / (rho * rho * rho);
      if (i == j) gs += kb * 2.0 * sigma;
    }
  }
  grad3[0] = ga;
  grad3[1] = gr;
  grad3[2] = gs;
}

/*
 * Lower-triangular inverse X = L^{-1} (Section 3.2, solving triangular
 * systems, primitive function: the result the divide-and-conquer inverse
 * reaches).  Written as its definition L X = I, solved one column at a time
 * by forward substitution:
 *   X_ij = 0 (i < j),  X_jj = 1 / L_jj,
 *   X_ij = -(sum_{k=j}^{i-1} L_ik X_kj) / L_ii   (i > j, k ascending).
 * Only the lower triangle of L is read; the strict upper triangle of X is set
 * to zero.  X must not overlap L.
 */
void oracle_tri_inverse(int n, const double *L, int ldl, double *X, int ldx) {
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < j; ++i) AT(X, ldx, i, j) = 0.0;
    AT(X, ldx, j, j) = 1.0 / AT(L, ldl, j, j);
    for (int i = j + 1; i < n; ++i) {
      double s = 0.0;
      for (int k = j; k < i; ++k) s += AT(L, ldl, i, k) * AT(X, ldx, k, j);
      AT(X, ldx, i, j) = -s / AT(L, ldl, i, i);
    }
  }
}

/*
 * C = L^{-1} B for lower-triangular L (n x n) and B (n x m): Section 3.2's
 * general triangular solver (which the GPU reaches through the inverse and a
 * product), written as forward substitution per column of B:
 *   C_ij = (B_ij - sum_{k<i} L_ik C_kj) / L_ii   (k ascending).
 * C may alias B.
 */
void oracle_tri_solve(int n, int m, const double *L, int ldl, const double *B, int ldb,
                      double *C, int ldc) {
  for (int j = 0; j < m; ++j) {
    for (int i = 0; i < n; ++i) {
      double s = AT(B, ldb, i, j);
      for (int k = 0; k < i; ++k) s -= AT(L, ldl, i, k) * AT(C, ldc, k, j);
      AT(C, ldc, i, j) = s / AT(L, ldl, i, i);
    }
  }
}

/*
 * Reverse mode of C = L^{-1} B (Section 3.2, reverse mode function) for a
 * scalar f with Cbar = df/dC.  From dC = L^{-1} (dB - dL C):
 *   Bbar = L^{-T} Cbar                (back substitution per column)
 *   Lbar_ij = -sum_t Bbar_it C_jt     (i >= j; strict upper set to zero)
 * i.e. Lbar = -tril(Bbar C^T): the gradient with respect to the lower-triangle
 * entries of L, the only ones the solve reads.  The paper prints the adjoint
 * system with A rather than A^T; the transpose is what the differential
 * gives (the two agree only for symmetric A).
 */
void oracle_tri_solve_adjoint(int n, int m, const double *L, int ldl, const double *C, int ldc,
                              const double *Cbar, int ldcb, double *Bbar, int ldbb,
                              double *Lbar, int ldlb) {
  for (int j = 0; j < m; ++j) {
    for (int i = n - 1; i >= 0; --i) {
      double s = AT(Cbar, ldcb, i, j);
      for (int k = i + 1; k < n; ++k) s -= AT(L, ldl, k, i) * AT(Bbar, ldbb, k, j);
      AT(Bbar, ldbb, i, j) = s / AT(L, ldl, i, i);
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      if (j <= i)
        for (int t = 0; t < m; ++t) s -= AT(Bbar, ldbb, i, t) * AT(C, ldc, j, t);
      AT(Lbar, ldlb, i, j) = s;
    }
}

/*
 * General matrix product C = A B (A: m x k, B: k x n, row-major; Section 3.1,
 * primitive function), the plain triple loop with the sum over k ascending.
 */
void oracle_gemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                 double *C, int ldc) {
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int t = 0; t < k; ++t) s += AT(A, lda, i, t) * AT(B, ldb, t, j);
      AT(C, ldc, i, j) = s;
    }
}

/*
 * Reverse mode of C = A B (Section 3.1, reverse mode function) for a scalar f
 * with Cbar = df/dC:  Abar = Cbar B^T,  Bbar = A^T Cbar.
 */
void oracle_gemm_adjoint(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                         const double *Cbar, int ldcb, double *Abar, int ldab, double *Bbar, int ldbb) {
  for (int i = 0; i < m; ++i)
    for (int t = 0; t < k; ++t) {
      double s = 0.0;
      for (int j = 0; j < n; ++j) s += AT(Cbar, ldcb, i, j) * AT(B, ldb, t, j);
      AT(Abar, ldab, i, t) = s;
    }
  for (int t = 0; t < k; ++t)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int i = 0; i < m; ++i) s += AT(A, lda, i, t) * AT(Cbar, ldcb, i, j);
      AT(Bbar, ldbb, t, j) = s;
    }
}

/*
 * Digamma psi(x) for x > 0 (needed by the negative-binomial GLM's dphi):
 * the recurrence psi(x) = psi(x + 1) - 1/x (Abramowitz and Stegun 6.3.5)
 * moves x to 12 or above, then the asymptotic series (A&S 6.3.18)
 *   psi(x) ~ ln x - 1/(2x) - sum_k B_2k / (2k x^2k)
 * is summed through the x^-12 term (B_2 .. B_12 = 1/6, -1/30, 1/42, -1/30,
 * 5/66, -691/2730); the first omitted term is below 4e-16 at x = 12.
 */
static double oracle_digamma(double x) {
  double acc = 0.0;
  while (x < 12.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  double r = 1.0 / (x * x);
  double series = r * (1.0 / 12.0 - r * (1.0 / 120.0 - r * (1.0 / 252.0 - r * (1.0 / 240.0 - r * (1.0 / 132.0 - r * (691.0 / 32760.0))))));
  return acc + log(x) - 0.5 / x - series;
}

/*
 * GLM log likelihood and its gradient (Section 3.4): the linear predictor
 * eta_i = alpha + sum_j X_ij beta_j (j ascending), then per observation
 *   family 0, normal-identity:  lp_i = -((y_i - eta_i)/sigma)^2 / 2 - log sigma - log(2 pi) / 2,
 *                               d_i = (y_i - eta_i) / sigma^2
 *   family 1, Bernoulli-logit:  lp_i = y_i eta_i - log(1 + exp(eta_i)),
 *                               d_i = y_i - 1 / (1 + exp(-eta_i))
 *   family 2, Poisson-log:      lp_i = y_i eta_i - exp(eta_i) - lgamma(y_i + 1),
 *                               d_i = y_i - exp(eta_i)
 *   family 3, negative-binomial-log (mean mu_i = exp(eta_i), dispersion phi = sigma):
 *     lp_i = lgamma(y_i + phi) - lgamma(y_i + 1) - lgamma(phi)
 *            + phi (log phi - log(mu_i + phi)) + y_i (eta_i - log(mu_i + phi)),
 *     d_i = y_i - (y_i + phi) mu_i / (mu_i + phi),
 *     dphi_i = psi(y_i + phi) - psi(phi) + log phi - log(mu_i + phi) + 1 - (y_i + phi)/(mu_i + phi)
 * with d_i = d lp_i / d eta_i.  Outputs: lp = sum_i lp_i, dalpha = sum_i d_i,
 * dbeta_j = sum_i X_ij d_i (i ascending), and for family 0
 * dsigma = sum_i ((y_i - eta_i)^2 / sigma^3 - 1 / sigma), for family 3
 * dsigma = sum_i dphi_i (else 0).
 * log(1 + exp(eta)) is evaluated as max(eta, 0) + log1p(exp(-|eta|)), the
 * same quantity without overflow.  Returns -1 if scratch cannot be allocated.
 */
int oracle_glm(int family, int n, int k, const double *X, int ldx, const double *y, double alpha,
               const double *beta, double sigma, double *lp, double *dalpha, double *dbeta,
               double *dsigma) {
  double *d = (double *)malloc((size_t)n * sizeof(double) + 8);
  if (!d) return -1;
  double slp = 0.0, sda = 0.0, sds = 0.0;
  for (int i = 0; i < n; ++i) {
    double eta = alpha;
    for (int j = 0; j < k; ++j) eta += AT(X, ldx, i, j) * beta[j];
    double li, di;
    if (family == 0) {
      double r = (y[i] - eta) / sigma;
      li = -0.5 * r * r - log(sigma) - 0.5 * log(ORACLE_TWO_PI);
      di = (y[i] - eta) / (sigma * sigma);
      sds += (y[i] - eta) * (y[i] - eta) / (sigma * sigma * sigma) - 1.0 / sigma;
    } else if (family == 1) {
      double softplus = (eta > 0.0 ? eta : 0.0) + log1p(exp(-fabs(eta)));
      li = y[i] * eta - softplus;
      di = y[i] - 1.0 / (1.0 + exp(-eta));
    } else if (family == 2) {
      li = y[i] * eta - exp(eta) - lgamma(y[i] + 1.0);
      di = y[i] - exp(eta);
    } else {
      double phi = sigma, mu = exp(eta), lmp = log(mu + phi);
      li = lgamma(y[i] + phi) - lgamma(y[i] + 1.0) - lgamma(phi) + phi * (log(phi) - lmp) + y[i] * (eta - lmp);
      di = y[i] - (y[i] + phi) * mu / (mu + phi);
      sds += oracle_digamma(y[i] + phi) - oracle_digamma(phi) + log(phi) - lmp + 1.0 - (y[i] + phi) / (mu + phi);
    }
    d[i] = di;
    slp += li;
    sda += di;
  }
  for (int j = 0; j < k; ++j) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += AT(X, ldx, i, j) * d[i];
    dbeta[j] = s;
  }
  *lp = slp;
  *dalpha = sda;
  *dsigma = (family == 0 || family == 3) ? sds : 0.0;
  free(d);
  return 0;
}

/* exported for the pins: the digamma above */
double oracle_psi(double x) { return oracle_digamma(x); }

/*
 * Categorical-logit GLM (Section 3.4, multinomial logistic regression): C
 * classes, y_i in {0, .., C-1}; the class scores are
 *   eta_ic = alpha_c + sum_j X_ij beta_jc   (beta: k x C, row-major)
 * and lp_i = eta_{i,y_i} - log sum_c exp(eta_ic) (the maximum is subtracted
 * inside the log-sum-exp).  With p_ic = exp(eta_ic - logsumexp_i) and
 * d_ic = [c == y_i] - p_ic:  dalpha_c = sum_i d_ic,  dbeta_jc = sum_i X_ij d_ic.
 * Returns -1 if scratch cannot be allocated.
 */
int oracle_glm_categorical(int n, int k, int C, const double *X, int ldx, const double *y, const double *alpha,
                           const double *beta, double *lp, double *dalpha, double *dbeta) {
  double *eta = (double *)malloc((size_t)C * sizeof(double) + 8);
  if (!eta) return -1;
  double slp = 0.0;
  for (int c = 0; c < C; ++c) dalpha[c] = 0.0;
  for (int j = 0; j < k; ++j)
    for (int c = 0; c < C; ++c) dbeta[(size_t)j * C + c] = 0.0;
  for (int i = 0; i < n; ++i) {
    double mx = -HUGE_VAL;
    for (int c = 0; c < C; ++c) {
      double e = alpha[c];
      for (int j = 0; j < k; ++j) e += AT(X, ldx, i, j) * beta[(size_t)j * C + c];
      eta[c] = e;
      if (e > mx) mx = e;
    }
    double se = 0.0;
    for (int c = 0; c < C; ++c) se += exp(eta[c] - mx);
    double lse = mx + log(se);
    int yi = (int)y[i];
    slp += eta[yi] - lse;
    for (int c = 0; c < C; ++c) {
      double d = (c == yi ? 1.0 : 0.0) - exp(eta[c] - lse);
      dalpha[c] += d;
      for (int j = 0; j < k; ++j) dbeta[(size_t)j * C + c] += AT(X, ldx, i, j) * d;
    }
  }
  *lp = slp;
  free(eta);
  return 0;
}

/*
 * Ordinal-logit GLM (Section 3.4, ordinal logistic regression): C ordered
 * classes, y_i in {0, .., C-1}, increasing cut points c_0 < .. < c_{C-2},
 * eta_i = sum_j X_ij beta_j (the cut points take the intercept's place) and
 * with s(t) = 1/(1 + exp(-t)):
 *   P(y = 0) = 1 - s(eta - c_0),  P(y = m) = s(eta - c_{m-1}) - s(eta - c_m),
 *   P(y = C-1) = s(eta - c_{C-2}).
 * lp = sum_i log P(y_i).  With u = eta - c_{y-1} (absent for y = 0) and
 * v = eta - c_y (absent for y = C-1), log P = log(s(u) - s(v)) and, since
 * s' = s (1 - s),
 *   d log P / d u = s(u)(1 - s(u)) / P,   d log P / d v = -s(v)(1 - s(v)) / P,
 * so d/deta = (du + dv), d/dc_{y-1} = -du, d/dc_y = -dv, where the missing
 * ends read s = 1 (u side) and s = 0 (v side) with no derivative.
 * Outputs lp, dbeta (k) = sum_i X_ij d/deta_i, dcuts (C-1).
 */
void oracle_glm_ordinal(int n, int k, int C, const double *X, int ldx, const double *y, const double *beta,
                        const double *cuts, double *lp, double *dbeta, double *dcuts) {
  double slp = 0.0;
  for (int j = 0; j < k; ++j) dbeta[j] = 0.0;
  for (int m = 0; m + 1 < C; ++m) dcuts[m] = 0.0;
  for (int i = 0; i < n; ++i) {
    double eta = 0.0;
    for (int j = 0; j < k; ++j) eta += AT(X, ldx, i, j) * beta[j];
    int yi = (int)y[i];
    double su = 1.0, sv = 0.0;
    if (yi > 0) su = 1.0 / (1.0 + exp(-(eta - cuts[yi - 1])));
    if (yi < C - 1) sv = 1.0 / (1.0 + exp(-(eta - cuts[yi])));
    double P = su - sv;
    slp += log(P);
    double du = yi > 0 ? su * (1.0 - su) / P : 0.0;
    double dv = yi < C - 1 ? -sv * (1.0 - sv) / P : 0.0;
    double deta = du + dv;
    for (int j = 0; j < k; ++j) dbeta[j] += AT(X, ldx, i, j) * deta;
    if (yi > 0) dcuts[yi - 1] -= du;
    if (yi < C - 1) dcuts[yi] -= dv;
  }
  *lp = slp;
}

