// C ABI of libgpchol: argument checks, workspace layout and the launch
// sequence of each entry point.  Every step of each call runs in this
// library's kernels on the caller's stream.
#include "common.cuh"

#include <algorithm>
#include <cstring>

namespace gpc {

Tuning &tuning() {
  static Tuning t;
  return t;
}

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cached[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 148;
    cached[dev] = v;
  }
  return cached[dev];
}

namespace {

struct ApiWs {
  void *core;
  double *vec;   // 4 n doubles
  void *refine;  // refinement residual, partial norms and state
  int *flags;    // triangular-solve tickets and ready flags
};

constexpr int kRefineMaxIters = 10;
constexpr double kRefineTol = 1e-14;

size_t core_bytes(int n, int precision) {
  size_t c = std::max(chol_workspace_bytes(n, precision), adjoint_workspace_bytes(n, precision));
  c = std::max(c, ltv_workspace_bytes(n));
  if (precision == GPC_MIXED) c = std::max(c, mixed_workspace_bytes(n));
  return align_up(c, 256);
}

bool valid_precision(int p) { return p == GPC_FP64 || p == GPC_MIXED; }

// Ticket and ready flags of either solve kernel (blocks of 64 rows, or of the
// factorisation's block size, which is at least 16).
size_t flags_bytes(int n) {
  return std::max(trsv_workspace_bytes(std::max(n, 1)), align_up(((size_t)(n + 15) / 16 + 1) * sizeof(int), 256));
}

size_t total_bytes(int n, int precision) {
  return core_bytes(n, precision) + align_up(4 * (size_t)std::max(n, 1) * sizeof(double), 256) +
         refine_workspace_bytes(std::max(n, 1)) + flags_bytes(n);
}

ApiWs carve(void *ws, int n, int precision) {
  ApiWs w;
  char *p = (char *)ws;
  w.core = p;
  p += core_bytes(n, precision);
  w.vec = (double *)p;
  p += align_up(4 * (size_t)std::max(n, 1) * sizeof(double), 256);
  w.refine = p;
  p += refine_workspace_bytes(std::max(n, 1));
  w.flags = (int *)p;
  return w;
}

int status_of(cudaError_t e) { return e == cudaSuccess ? GPC_OK : GPC_ERR_CUDA; }

bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
  const char *pa = (const char *)a, *pb = (const char *)b;
  return pa < pb + bbytes && pb < pa + abytes;
}

size_t mat_bytes(int n, int ld) { return n > 0 ? ((size_t)(n - 1) * ld + n) * sizeof(double) : 0; }

bool bad_square(int n, const void *p, int ld) { return n > 0 && (p == nullptr || ld < n); }

size_t rect_bytes(int rows, int cols, int ld) {
  return rows > 0 && cols > 0 ? ((size_t)(rows - 1) * ld + cols) * sizeof(double) : 0;
}

bool bad_rect(int rows, int cols, const void *p, int ld) {
  return rows > 0 && cols > 0 && (p == nullptr || ld < cols);
}

// L and its inverse: the same buffer with the same ld, or disjoint.
bool bad_inverse_pair(int n, const double *L, int ldl, const double *X, int ldx) {
  if ((const void *)L == (const void *)X) return ldl != ldx;
  return overlaps(L, mat_bytes(n, ldl), X, mat_bytes(n, ldx));
}

}  // namespace
}  // namespace gpc

using namespace gpc;

extern "C" {

const char *gpc_status_string(int status) {
  switch (status) {
    case GPC_OK: return "GPC_OK: success";
    case GPC_ERR_INVALID_ARG: return "GPC_ERR_INVALID_ARG: invalid argument";
    case GPC_ERR_NOT_PD: return "GPC_ERR_NOT_PD: matrix is not positive definite";
    case GPC_ERR_NAN: return "GPC_ERR_NAN: NaN or infinite pivot";
    case GPC_ERR_CUDA: return "GPC_ERR_CUDA: CUDA launch or runtime error";
    case GPC_ERR_TIMEOUT: return "GPC_ERR_TIMEOUT: bounded device wait gave up";
    case GPC_ERR_NO_CONVERGENCE: return "GPC_ERR_NO_CONVERGENCE: refinement above tolerance";
    default: return "unknown gpchol status";
  }
}

int gpc_version(void) { return 100; }

int gpc_set_tuning(int key, int value) {
  switch (key) {
    case GPC_TUNE_BLOCK:
      if (value < 16 || value > kMaxBlock || value % 16) return GPC_ERR_INVALID_ARG;
      tuning().block = value;
      return GPC_OK;
    case GPC_TUNE_SLICES:  // fixed by the product grouping of the split kernels
      return value == slices_count() ? GPC_OK : GPC_ERR_INVALID_ARG;
    case GPC_TUNE_SPLITK_MIN:
      if (value < 16 || value > (1 << 20)) return GPC_ERR_INVALID_ARG;
      tuning().splitk_min = value;
      return GPC_OK;
    case GPC_TUNE_BATCH_BLOCK:
      if (value != 32 && value != 64) return GPC_ERR_INVALID_ARG;
      tuning().batch_block = value;
      return GPC_OK;
    case GPC_TUNE_MIXED_DEFER:
      if (value < 1 || value > 8) return GPC_ERR_INVALID_ARG;
      tuning().mixed_defer = value;
      return GPC_OK;
    case GPC_TUNE_MIXED_FREE_SMS:
      if (value < 0 || value > 32) return GPC_ERR_INVALID_ARG;
      tuning().mixed_free_sms = value;
      return GPC_OK;
    case GPC_TUNE_MIXED_CTA_ITEMS:
      if (value < 0 || value > 1024) return GPC_ERR_INVALID_ARG;
      tuning().mixed_cta_items = value;
      return GPC_OK;
    case GPC_TUNE_MIXED_PRIORITY:
      if (value != 0 && value != 1) return GPC_ERR_INVALID_ARG;
      tuning().mixed_priority = value;
      return GPC_OK;
    case GPC_TUNE_MIXED_ADJ_FREE_SMS:
      if (value < 0 || value > 64) return GPC_ERR_INVALID_ARG;
      tuning().mixed_adj_free_sms = value;
      return GPC_OK;
    case GPC_TUNE_F64_SMALL_TILE:
      if (value < 0 || value > 4096) return GPC_ERR_INVALID_ARG;
      tuning().f64_small_tile = value;
      return GPC_OK;
    default:
      return GPC_ERR_INVALID_ARG;
  }
}

int gpc_get_tuning(int key, int *value) {
  if (!value) return GPC_ERR_INVALID_ARG;
  switch (key) {
    case GPC_TUNE_BLOCK: *value = tuning().block; return GPC_OK;
    case GPC_TUNE_SLICES: *value = slices_count(); return GPC_OK;
    case GPC_TUNE_SPLITK_MIN: *value = tuning().splitk_min; return GPC_OK;
    case GPC_TUNE_BATCH_BLOCK: *value = tuning().batch_block; return GPC_OK;
    case GPC_TUNE_MIXED_DEFER: *value = tuning().mixed_defer; return GPC_OK;
    case GPC_TUNE_MIXED_FREE_SMS: *value = tuning().mixed_free_sms; return GPC_OK;
    case GPC_TUNE_MIXED_CTA_ITEMS: *value = tuning().mixed_cta_items; return GPC_OK;
    case GPC_TUNE_MIXED_PRIORITY: *value = tuning().mixed_priority; return GPC_OK;
    case GPC_TUNE_MIXED_ADJ_FREE_SMS: *value = tuning().mixed_adj_free_sms; return GPC_OK;
    case GPC_TUNE_F64_SMALL_TILE: *value = tuning().f64_small_tile; return GPC_OK;
    default: return GPC_ERR_INVALID_ARG;
  }
}

int gpc_workspace_size(int n, int precision, size_t *bytes) {
  if (!bytes || n < 0 || (precision != GPC_FP64 && precision != GPC_MIXED)) return GPC_ERR_INVALID_ARG;
  *bytes = total_bytes(n, precision);
  return GPC_OK;
}

int gpc_se_cov(int n, int d, const double *X, int ldx, double alpha, double rho, double sigma,
               double jitter, double *K, int ldk, int full, int precision, gpc_stream_t stream) {
  if (n < 0 || d < 1 || d > kMaxDim || !valid_precision(precision)) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (!X || ldx < d || bad_square(n, K, ldk) || !(rho > 0.0)) return GPC_ERR_INVALID_ARG;
  return status_of(se_cov(n, d, X, ldx, alpha, rho, sigma, jitter, K, ldk, full, precision == GPC_MIXED, stream));
}

int gpc_chol(int n, const double *K, int ldk, double *L, int ldl, int precision, void *ws,
             size_t ws_bytes, int *info, gpc_stream_t stream) {
  if (n < 0 || !valid_precision(precision) || !info) return GPC_ERR_INVALID_ARG;
  if (n == 0) return status_of(reset_info(info, stream));
  if (bad_square(n, K, ldk) || bad_square(n, L, ldl) || !ws || ws_bytes < total_bytes(n, precision))
    return GPC_ERR_INVALID_ARG;
  if ((const void *)K == (const void *)L) {
    if (ldk != ldl) return GPC_ERR_INVALID_ARG;
  } else if (overlaps(K, mat_bytes(n, ldk), L, mat_bytes(n, ldl))) {
    return GPC_ERR_INVALID_ARG;
  }
  ApiWs w = carve(ws, n, precision);
  cudaError_t e = reset_info(info, stream);
  if (precision == GPC_MIXED) {
    if (e == cudaSuccess) e = to_df_lower(n, K, ldk, L, ldl, stream);
    if (e == cudaSuccess) e = chol_mixed(n, L, ldl, w.core, info, stream);
    return status_of(e);
  }
  if (e == cudaSuccess) e = copy_lower(n, K, ldk, L, ldl, stream);
  if (e == cudaSuccess) e = chol_fp64(n, L, ldl, w.core, info, stream);
  return status_of(e);
}

int gpc_chol_adjoint(int n, const double *L, int ldl, const double *Lbar, int ldlb, double *Kbar,
                     int ldkb, int precision, int symmetric_out, void *ws, size_t ws_bytes,
                     gpc_stream_t stream) {
  if (n < 0 || !valid_precision(precision)) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, L, ldl) || bad_square(n, Lbar, ldlb) || bad_square(n, Kbar, ldkb) || !ws ||
      ws_bytes < total_bytes(n, precision))
    return GPC_ERR_INVALID_ARG;
  if ((const void *)Lbar == (const void *)Kbar) {
    if (ldlb != ldkb) return GPC_ERR_INVALID_ARG;
  } else if (overlaps(Lbar, mat_bytes(n, ldlb), Kbar, mat_bytes(n, ldkb))) {
    return GPC_ERR_INVALID_ARG;
  }
  if (overlaps(L, mat_bytes(n, ldl), Kbar, mat_bytes(n, ldkb))) return GPC_ERR_INVALID_ARG;
  ApiWs w = carve(ws, n, precision);
  cudaError_t e;
  if (precision == GPC_MIXED) {
    e = to_df_lower(n, Lbar, ldlb, Kbar, ldkb, stream);
    if (e == cudaSuccess) e = chol_adjoint_mixed(n, L, ldl, Kbar, ldkb, w.core, w.flags, stream);
  } else {
    e = copy_lower(n, Lbar, ldlb, Kbar, ldkb, stream);
    if (e == cudaSuccess) e = chol_adjoint_fp64(n, L, ldl, Kbar, ldkb, w.core, stream);
  }
  if (e == cudaSuccess && symmetric_out) e = lower_to_symmetric_half(n, Kbar, ldkb, stream);
  return status_of(e);
}

int gpc_trsv(int n, const double *L, int ldl, double *x, int trans, void *ws, size_t ws_bytes,
             gpc_stream_t stream) {
  if (n < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, L, ldl) || !x || !ws || ws_bytes < trsv_workspace_bytes(n)) return GPC_ERR_INVALID_ARG;
  return status_of(trsv(n, L, ldl, x, trans, ws, nullptr, stream));
}

int gpc_gemm_workspace_size(size_t *bytes) {
  if (!bytes) return GPC_ERR_INVALID_ARG;
  *bytes = gemm_f64_scratch_bytes();
  return GPC_OK;
}

int gpc_gemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
             void *ws, size_t ws_bytes, gpc_stream_t stream) {
  if (m < 0 || n < 0 || k < 0) return GPC_ERR_INVALID_ARG;
  if (m == 0 || n == 0) return GPC_OK;
  if (bad_rect(m, k, A, lda) || bad_rect(k, n, B, ldb) || bad_rect(m, n, C, ldc) ||
      (ws && ws_bytes < gemm_f64_scratch_bytes()))
    return GPC_ERR_INVALID_ARG;
  const size_t cb = rect_bytes(m, n, ldc);
  if (overlaps(C, cb, A, rect_bytes(m, k, lda)) || overlaps(C, cb, B, rect_bytes(k, n, ldb)) ||
      (ws && overlaps(C, cb, ws, ws_bytes)))
    return GPC_ERR_INVALID_ARG;
  Gemm g;
  g.M = m; g.N = n; g.K = k;
  g.A = A; g.lda = lda;
  g.B = B; g.ldb = ldb;
  g.C = C; g.ldc = ldc;
  return status_of(gemm_f64(g, (double *)ws, stream));
}

int gpc_gemm_adjoint(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                     const double *Cbar, int ldcb, double *Abar, int ldab, double *Bbar, int ldbb, void *ws,
                     size_t ws_bytes, gpc_stream_t stream) {
  if (m < 0 || n < 0 || k < 0) return GPC_ERR_INVALID_ARG;
  if (bad_rect(m, k, A, lda) || bad_rect(k, n, B, ldb) || bad_rect(m, n, Cbar, ldcb) ||
      bad_rect(m, k, Abar, ldab) || bad_rect(k, n, Bbar, ldbb) || (ws && ws_bytes < gemm_f64_scratch_bytes()))
    return GPC_ERR_INVALID_ARG;
  const size_t ab = rect_bytes(m, k, lda), bb = rect_bytes(k, n, ldb), cbb = rect_bytes(m, n, ldcb);
  const size_t abb = rect_bytes(m, k, ldab), bbb = rect_bytes(k, n, ldbb);
  const size_t wb = ws ? ws_bytes : 0;
  if (overlaps(Abar, abb, A, ab) || overlaps(Abar, abb, B, bb) || overlaps(Abar, abb, Cbar, cbb) ||
      overlaps(Abar, abb, Bbar, bbb) || overlaps(Bbar, bbb, A, ab) || overlaps(Bbar, bbb, B, bb) ||
      overlaps(Bbar, bbb, Cbar, cbb) || overlaps(Abar, abb, ws, wb) || overlaps(Bbar, bbb, ws, wb))
    return GPC_ERR_INVALID_ARG;
  if (m > 0 && k > 0) {
    Gemm a;  // Abar (m x k) = Cbar (m x n) B^T; B (k x n) is stored N x K
    a.M = m; a.N = k; a.K = n;
    a.A = Cbar; a.lda = ldcb;
    a.transB = true; a.B = B; a.ldb = ldb;
    a.C = Abar; a.ldc = ldab;
    cudaError_t e = gemm_f64(a, (double *)ws, stream);
    if (e != cudaSuccess) return status_of(e);
  }
  if (k > 0 && n > 0) {
    Gemm b;  // Bbar (k x n) = A^T Cbar; A (m x k) is stored K x M
    b.M = k; b.N = n; b.K = m;
    b.transA = true; b.A = A; b.lda = lda;
    b.B = Cbar; b.ldb = ldcb;
    b.C = Bbar; b.ldc = ldbb;
    cudaError_t e = gemm_f64(b, (double *)ws, stream);
    if (e != cudaSuccess) return status_of(e);
  }
  return GPC_OK;
}

int gpc_glm_workspace_size(int k, size_t *bytes) {
  if (!bytes || k < 0 || k > GPC_GLM_MAX_K) return GPC_ERR_INVALID_ARG;
  *bytes = glm_workspace_bytes(k);
  return GPC_OK;
}

int gpc_glm(int family, long long n, int k, const double *X, long long ldx, const double *y, double alpha,
            const double *beta, double sigma, double *lp, double *dalpha, double *dbeta, double *dsigma,
            void *ws, size_t ws_bytes, gpc_stream_t stream) {
  if (family != GPC_GLM_NORMAL_ID && family != GPC_GLM_BERNOULLI_LOGIT && family != GPC_GLM_POISSON_LOG &&
      family != GPC_GLM_NEG_BINOMIAL_LOG)
    return GPC_ERR_INVALID_ARG;
  if (n < 0 || k < 0 || k > GPC_GLM_MAX_K || !lp || !dalpha || !dsigma || !ws ||
      ws_bytes < glm_workspace_bytes(k))
    return GPC_ERR_INVALID_ARG;
  if ((family == GPC_GLM_NORMAL_ID || family == GPC_GLM_NEG_BINOMIAL_LOG) &&
      !(sigma > 0.0 && sigma <= 1.79769313486231570e308))
    return GPC_ERR_INVALID_ARG;
  if (!(alpha == alpha) || (k > 0 && (!beta || !dbeta)) || (n > 0 && (!y || (k > 0 && (!X || ldx < k)))))
    return GPC_ERR_INVALID_ARG;
  return status_of(glm(family, n, k, X, ldx, y, alpha, beta, sigma, lp, dalpha, dbeta, dsigma, ws, stream));
}

int gpc_glm_ordinal(long long n, int k, int C, const double *X, long long ldx, const double *y,
                    const double *beta, const double *cuts, double *lp, double *dbeta, double *dcuts, void *ws,
                    size_t ws_bytes, gpc_stream_t stream) {
  if (n < 0 || k < 0 || k > GPC_GLM_MAX_K || C < 2 || C > GPC_GLM_MAX_CLASSES || !lp || !dcuts || !cuts || !ws ||
      ws_bytes < glm_workspace_bytes(k))
    return GPC_ERR_INVALID_ARG;
  if ((k > 0 && (!beta || !dbeta)) || (n > 0 && (!y || (k > 0 && (!X || ldx < k))))) return GPC_ERR_INVALID_ARG;
  return status_of(glm_ordinal(n, k, C, X, ldx, y, beta, cuts, lp, dbeta, dcuts, ws, stream));
}

int gpc_glm_categorical_workspace_size(int k, int C, size_t *bytes) {
  if (!bytes || k < 0 || C < 2 || C > GPC_GLM_MAX_CLASSES || (long long)k * C > GPC_GLM_MAX_KC)
    return GPC_ERR_INVALID_ARG;
  *bytes = glm_categorical_workspace_bytes(k, C);
  return GPC_OK;
}

int gpc_glm_categorical(long long n, int k, int C, const double *X, long long ldx, const double *y,
                        const double *alpha, const double *beta, double *lp, double *dalpha, double *dbeta,
                        void *ws, size_t ws_bytes, gpc_stream_t stream) {
  if (n < 0 || k < 0 || C < 2 || C > GPC_GLM_MAX_CLASSES || (long long)k * C > GPC_GLM_MAX_KC || !lp || !alpha ||
      !dalpha || !ws || ws_bytes < glm_categorical_workspace_bytes(k, C))
    return GPC_ERR_INVALID_ARG;
  if ((k > 0 && (!beta || !dbeta)) || (n > 0 && (!y || (k > 0 && (!X || ldx < k))))) return GPC_ERR_INVALID_ARG;
  return status_of(glm_categorical(n, k, C, X, ldx, y, alpha, beta, lp, dalpha, dbeta, ws, stream));
}

int gpc_tri_inverse(int n, const double *L, int ldl, double *Linv, int ldi, gpc_stream_t stream) {
  if (n < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, L, ldl) || bad_square(n, Linv, ldi) || bad_inverse_pair(n, L, ldl, Linv, ldi))
    return GPC_ERR_INVALID_ARG;
  return status_of(tri_inverse(n, L, ldl, Linv, ldi, stream));
}

int gpc_tri_solve(int n, int m, const double *L, int ldl, const double *B, int ldb, double *Linv, int ldi,
                  double *C, int ldc, gpc_stream_t stream) {
  if (n < 0 || m < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, L, ldl) || bad_square(n, Linv, ldi) || bad_inverse_pair(n, L, ldl, Linv, ldi) ||
      bad_rect(n, m, B, ldb) || bad_rect(n, m, C, ldc))
    return GPC_ERR_INVALID_ARG;
  if (m > 0) {
    const size_t bb = rect_bytes(n, m, ldb), cb = rect_bytes(n, m, ldc);
    if (overlaps(C, cb, B, bb) || overlaps(C, cb, L, mat_bytes(n, ldl)) || overlaps(C, cb, Linv, mat_bytes(n, ldi)) ||
        overlaps(B, bb, Linv, mat_bytes(n, ldi)))
      return GPC_ERR_INVALID_ARG;
  }
  return status_of(tri_solve(n, m, L, ldl, B, ldb, Linv, ldi, C, ldc, stream));
}

int gpc_tri_solve_adjoint(int n, int m, const double *Linv, int ldi, const double *C, int ldc,
                          const double *Cbar, int ldcb, double *Bbar, int ldbb, double *Lbar, int ldlb,
                          gpc_stream_t stream) {
  if (n < 0 || m < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, Linv, ldi) || bad_square(n, Lbar, ldlb) || bad_rect(n, m, C, ldc) ||
      bad_rect(n, m, Cbar, ldcb) || bad_rect(n, m, Bbar, ldbb))
    return GPC_ERR_INVALID_ARG;
  const size_t xb = mat_bytes(n, ldi), lb = mat_bytes(n, ldlb);
  const size_t cb = rect_bytes(n, m, ldc), cbb = rect_bytes(n, m, ldcb), bbb = rect_bytes(n, m, ldbb);
  if (overlaps(Lbar, lb, Linv, xb) || overlaps(Lbar, lb, C, cb) || overlaps(Lbar, lb, Cbar, cbb) ||
      overlaps(Lbar, lb, Bbar, bbb) || overlaps(Bbar, bbb, Linv, xb) || overlaps(Bbar, bbb, C, cb) ||
      overlaps(Bbar, bbb, Cbar, cbb))
    return GPC_ERR_INVALID_ARG;
  return status_of(tri_solve_adjoint(n, m, Linv, ldi, C, ldc, Cbar, ldcb, Bbar, ldbb, Lbar, ldlb, stream));
}

int gpc_gp_lml(int n, const double *K, int ldk, const double *y, double *L, int ldl,
               int precision, double *logdet, double *alpha, double *value, void *ws,
               size_t ws_bytes, int *info, gpc_stream_t stream) {
  if (n < 0 || !valid_precision(precision) || !info || !logdet || !value) return GPC_ERR_INVALID_ARG;
  if (n == 0) {
    cudaError_t e = reset_info(info, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(logdet, 0, sizeof(double), stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(value, 0, sizeof(double), stream);
    return status_of(e);
  }
  if (bad_square(n, K, ldk) || bad_square(n, L, ldl) || !y || !alpha || !ws ||
      ws_bytes < total_bytes(n, precision))
    return GPC_ERR_INVALID_ARG;
  if ((const void *)K == (const void *)L) {
    if (ldk != ldl || precision == GPC_MIXED) return GPC_ERR_INVALID_ARG;
  } else if (overlaps(K, mat_bytes(n, ldk), L, mat_bytes(n, ldl))) {
    return GPC_ERR_INVALID_ARG;
  }
  if (overlaps(alpha, n * sizeof(double), L, mat_bytes(n, ldl)) ||
      overlaps(alpha, n * sizeof(double), y, n * sizeof(double)))
    return GPC_ERR_INVALID_ARG;
  ApiWs w = carve(ws, n, precision);
  cudaError_t e = reset_info(info, stream);
  if (precision == GPC_MIXED) {
    if (e == cudaSuccess) e = to_df_lower(n, K, ldk, L, ldl, stream);
    if (e == cudaSuccess) e = chol_mixed(n, L, ldl, w.core, info, stream);
  } else {
    if (e == cudaSuccess) e = copy_lower(n, K, ldk, L, ldl, stream);
    if (e == cudaSuccess) e = chol_fp64(n, L, ldl, w.core, info, stream);
  }
  // the factorisation left every diagonal-block inverse at the start of the core workspace
  const double *inv = (const double *)w.core;
  const int b = chol_block_size(precision);
  if (e == cudaSuccess) e = cudaMemcpyAsync(alpha, y, n * sizeof(double), cudaMemcpyDeviceToDevice, stream);
  if (precision == GPC_MIXED) {
    // The mixed path solves in double-float: its factor's own error is far
    // larger, and the FP64 refinement against K removes both.  L's lower
    // triangle is converted once into the workspace core behind the block
    // inverses (free after the factorisation); the solved sub-blocks pass
    // through w.vec.
    const size_t inv_bytes = align_up((size_t)((n + b - 1) / b) * b * b * sizeof(double), 256);
    const bool room = core_bytes(n, precision) >= inv_bytes + (size_t)n * n * sizeof(float2);
    float2 *Ld = room ? (float2 *)((char *)w.core + inv_bytes) : nullptr;
    float2 *xdf = (float2 *)w.vec;
    if (Ld) {
      if (e == cudaSuccess) e = to_df_tri(n, L, ldl, Ld, n, stream);
      if (e == cudaSuccess) e = trsv_inv_df(n, Ld, n, inv, b, alpha, xdf, 0, w.flags, info, stream);
      if (e == cudaSuccess) e = trsv_inv_df(n, Ld, n, inv, b, alpha, xdf, 1, w.flags, info, stream);
    } else {
      if (e == cudaSuccess) e = trsv_inv(n, L, ldl, inv, b, alpha, 0, w.flags, info, stream);
      if (e == cudaSuccess) e = trsv_inv(n, L, ldl, inv, b, alpha, 1, w.flags, info, stream);
    }
    if (e == cudaSuccess)
      e = refine(n, K, ldk, L, ldl, inv, b, y, alpha, w.refine, w.flags, info, kRefineMaxIters, kRefineTol,
                 stream, Ld, n, xdf);
  } else {
    if (e == cudaSuccess) e = trsv_inv(n, L, ldl, inv, b, alpha, 0, w.flags, info, stream);
    if (e == cudaSuccess) e = trsv_inv(n, L, ldl, inv, b, alpha, 1, w.flags, info, stream);
  }
  if (e == cudaSuccess) e = lml_finalize(n, L, ldl, y, alpha, logdet, value, stream);
  return status_of(e);
}

int gpc_gp_lml_grad(int n, const double *L, int ldl, const double *alpha, double gbar,
                    double *Kbar, int ldkb, int precision, void *ws, size_t ws_bytes,
                    gpc_stream_t stream) {
  if (n < 0 || !valid_precision(precision)) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (bad_square(n, L, ldl) || bad_square(n, Kbar, ldkb) || !alpha || !ws ||
      ws_bytes < total_bytes(n, precision))
    return GPC_ERR_INVALID_ARG;
  if (overlaps(L, mat_bytes(n, ldl), Kbar, mat_bytes(n, ldkb))) return GPC_ERR_INVALID_ARG;
  ApiWs w = carve(ws, n, precision);
  double *z = w.vec;
  cudaError_t e = ltv(n, L, ldl, alpha, z, w.core, stream);
  if (e == cudaSuccess) e = lml_lbar(n, L, ldl, alpha, z, gbar, Kbar, ldkb, stream, precision == GPC_MIXED);
  if (precision == GPC_MIXED) {
    if (e == cudaSuccess) e = chol_adjoint_mixed(n, L, ldl, Kbar, ldkb, w.core, w.flags, stream);
  } else {
    if (e == cudaSuccess) e = chol_adjoint_fp64(n, L, ldl, Kbar, ldkb, w.core, stream);
  }
  return status_of(e);
}

int gpc_se_hyper_grad(int n, int d, const double *X, int ldx, double alpha, double rho,
                      double sigma, const double *Kbar, int ldkb, double *grad3, int precision, void *ws,
                      size_t ws_bytes, gpc_stream_t stream) {
  if (n < 0 || d < 1 || d > kMaxDim || !grad3 || !valid_precision(precision)) return GPC_ERR_INVALID_ARG;
  if (n > 0 && (!X || ldx < d || bad_square(n, Kbar, ldkb) || !(rho > 0.0) || !(alpha != 0.0) ||
                !ws || ws_bytes < se_hyper_grad_workspace_bytes(n)))
    return GPC_ERR_INVALID_ARG;
  return status_of(
      se_hyper_grad(n, d, X, ldx, alpha, rho, sigma, Kbar, ldkb, grad3, ws, precision == GPC_MIXED, stream));
}

constexpr int kBatchMaxN = 4096;

int gpc_batched_workspace_size(int batch, int nmax, int precision, size_t *bytes) {
  if (!bytes || batch < 0 || nmax < 1 || nmax > kBatchMaxN || !valid_precision(precision)) return GPC_ERR_INVALID_ARG;
  *bytes = batched_workspace_bytes(std::max(batch, 1), nmax, precision == GPC_MIXED);
  return GPC_OK;
}

int gpc_batched_gp_lml_grad(int batch, int nmax, const int *n, const long long *offK, const long long *rowX, int d,
                            const double *X, const double *y, const double *hyp, int precision, double *Kws,
                            double *value, double *grad3, int *info, void *ws, size_t ws_bytes,
                            gpc_stream_t stream) {
  if (batch < 0 || nmax < 1 || nmax > kBatchMaxN || d < 1 || d > kMaxDim || !valid_precision(precision))
    return GPC_ERR_INVALID_ARG;
  if (batch == 0) return GPC_OK;
  const bool mixed = precision == GPC_MIXED;
  if (!n || !offK || !rowX || !X || !y || !hyp || !Kws || !value || !grad3 || !info || !ws ||
      ws_bytes < batched_workspace_bytes(batch, nmax, mixed))
    return GPC_ERR_INVALID_ARG;
  return status_of(batched_gp_lml_grad(batch, n, offK, rowX, d, X, y, hyp, Kws, value, grad3, info, nmax, mixed,
                                       ws, stream));
}

int gpc_se_hyper_grad_workspace_size(int n, size_t *bytes) {
  if (n < 0 || !bytes) return GPC_ERR_INVALID_ARG;
  *bytes = se_hyper_grad_workspace_bytes(std::max(n, 1));
  return GPC_OK;
}

}  // extern "C"
