/*
 * cpu_baseline.c -- the timed multi-core CPU baseline: the unblocked Cholesky
 * factorisation and its unblocked reverse mode, reordered by columns so the
 * rows of each column run in parallel on all host cores (OpenMP).  No
 * blocking and no BLAS.
 *
 * THIS IS MEASUREMENT AND TEST INFRASTRUCTURE, not the oracle: only the
 * benchmark's CPU legs and the tests load it.  The tests check that its factor
 * is bitwise equal to the oracle's (the same operations in the same order for
 * every entry; compiled, like the oracle, with -ffp-contract=off) and its
 * adjoint within 1e-13 of the oracle's; that lets the tests use it in place of
 * the single-threaded oracle for the two O(n^3) steps at n = 16384.
 * It shares no code with the GPU library or with the oracle.
 *
 * Storage: row-major, leading dimension n, lower triangle meaningful.
 *
 * Forward (column order, Section 3.3's recurrence with 1 x 1 diagonal
 * blocks): for j = 0 .. n-1
 *   L_jj = sqrt(K_jj - sum_{k<j} L_jk^2)
 *   L_ij = (K_ij - sum_{k<j} L_ik L_jk) / L_jj   for every i > j, in parallel.
 * Reverse: the same statements backwards, columns j = n-1 .. 0; first the
 * off-diagonal ones of column j (independent given the column's inputs, so
 * the rows run in parallel), then the diagonal one:
 *   tbar = Lbar_ij / L_jj;  Lbar_jj -= tbar L_ij;  Kbar_ij = tbar;
 *   Lbar_ik -= tbar L_jk (row i, private);  Lbar_jk -= tbar L_ik (row j,
 *   summed over i from per-thread accumulators);
 *   sbar = Lbar_jj / (2 L_jj);  Kbar_jj = sbar;  Lbar_jk -= 2 sbar L_jk.
 */
#include <math.h>
#include <omp.h>
#include <stdlib.h>
#include <string.h>

#define IDX(i, j, n) ((size_t)(i) * (size_t)(n) + (size_t)(j))

int cpu_baseline_threads(void) { return omp_get_max_threads(); }

/* L = chol(K); returns -1, or the first failing pivot.  K and L may alias. */
int cpu_baseline_chol(int n, const double *K, double *L) {
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) L[IDX(i, j, n)] = j <= i ? K[IDX(i, j, n)] : 0.0;
  for (int j = 0; j < n; ++j) {
    const double *lj = L + IDX(j, 0, n);
    double s = lj[j];
    for (int k = 0; k < j; ++k) s -= lj[k] * lj[k];
    if (!(s > 0.0)) return j;
    const double d = sqrt(s);
    L[IDX(j, j, n)] = d;
    /* Rows below the diagonal in groups of four: the four sums are independent
     * chains, so a core overlaps their latencies; each row's own sum is still
     * formed term by term with k ascending, so every L_ij is bitwise the value
     * of the row-by-row recurrence. */
    const int first = j + 1, groups = (n - first + 3) / 4;
#pragma omp parallel for schedule(static)
    for (int g = 0; g < groups; ++g) {
      const int i0 = first + 4 * g;
      if (i0 + 4 <= n) {
        double *l0 = L + IDX(i0, 0, n), *l1 = l0 + n, *l2 = l1 + n, *l3 = l2 + n;
        double t0 = l0[j], t1 = l1[j], t2 = l2[j], t3 = l3[j];
        for (int k = 0; k < j; ++k) {
          const double c = lj[k];
          t0 -= l0[k] * c;
          t1 -= l1[k] * c;
          t2 -= l2[k] * c;
          t3 -= l3[k] * c;
        }
        l0[j] = t0 / d;
        l1[j] = t1 / d;
        l2[j] = t2 / d;
        l3[j] = t3 / d;
      } else {
        for (int i = i0; i < n; ++i) {
          double *li = L + IDX(i, 0, n);
          double t = li[j];
          for (int k = 0; k < j; ++k) t -= li[k] * lj[k];
          li[j] = t / d;
        }
      }
    }
  }
  return -1;
}

/* Kbar (lower) from L and Lbar; returns 0, or -1 if scratch cannot be allocated. */
int cpu_baseline_chol_adjoint(int n, const double *L, const double *Lbar, double *Kbar) {
  const int T = omp_get_max_threads();
  double *W = (double *)malloc((size_t)n * (size_t)n * sizeof(double) + 8);
  double *acc = (double *)malloc((size_t)T * (size_t)n * sizeof(double) + 8);
  if (!W || !acc) {
    free(W);
    free(acc);
    return -1;
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) W[IDX(i, j, n)] = j <= i ? Lbar[IDX(i, j, n)] : 0.0;
  for (int j = n - 1; j >= 0; --j) {
    const double *lj = L + IDX(j, 0, n);
    const double d = lj[j];
    double dsum = 0.0;
    for (int t = 0; t < T; ++t) memset(acc + (size_t)t * (size_t)n, 0, (size_t)j * sizeof(double));
#pragma omp parallel reduction(+ : dsum)
    {
      double *a = acc + (size_t)omp_get_thread_num() * (size_t)n;
#pragma omp for schedule(static)
      for (int i = j + 1; i < n; ++i) {
        double *wi = W + IDX(i, 0, n);
        const double *li = L + IDX(i, 0, n);
        const double tb = wi[j] / d;
        dsum += tb * li[j];
        wi[j] = tb;
        for (int k = 0; k < j; ++k) {
          wi[k] -= tb * lj[k];
          a[k] += tb * li[k];
        }
      }
    }
    double *wj = W + IDX(j, 0, n);
    wj[j] -= dsum;
    for (int t = 0; t < T; ++t) {
      const double *a = acc + (size_t)t * (size_t)n;
      for (int k = 0; k < j; ++k) wj[k] -= a[k];
    }
    const double sb = wj[j] / (2.0 * d);
    wj[j] = sb;
    for (int k = 0; k < j; ++k) wj[k] -= 2.0 * sb * lj[k];
  }
#pragma omp parallel for schedule(static)
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Kbar[IDX(i, j, n)] = j <= i ? W[IDX(i, j, n)] : 0.0;
  free(W);
  free(acc);
  return 0;
}
