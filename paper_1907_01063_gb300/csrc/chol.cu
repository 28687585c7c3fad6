// Blocked Cholesky factorisation and blocked reverse-mode adjoint (FP64).
//
// Forward (Section 3.3, primitive function): right-looking over b-wide block
// columns.  Each step factors the diagonal block and forms its inverse in one
// thread block, computes the panel L21 = A21 L11^{-T} as a product with that
// inverse, and applies the trailing update A22 -= L21 L21^T to the lower tiles
// only.  The paper recurses on A22 with a partition parameter; a fixed block
// width gives the same factor up to rounding.
//
// Reverse (Section 3.3, reverse mode function; Murray 2016): a backward sweep
// over the same block columns, k = n, n-b, ..., with j = max(0, k-b) and
//   R = L[j:k, 0:j], D = L[j:k, j:k], B = L[k:n, 0:j], C = L[k:n, j:k]
// (and the same slices of the adjoint buffer, updated in place):
//   Cbar <- Cbar D^{-1}
//   Bbar -= Cbar R
//   Dbar -= Cbar^T C                        (lower part only; see below)
//   Dbar <- D^{-T} sym(tril(D^T Dbar)) D^{-1}   (symmetric)
//   Rbar -= Cbar^T B + Dbar R                (one product: [Dbar; Cbar]^T [R; B])
//   Dbar <- lower part of Dbar with its diagonal halved.
// tril(D^T Dbar) depends only on tril(Dbar) because D^T is upper triangular,
// so the Dbar update only needs its lower triangle.  The paper's last
// statement prints "diagonal * 0.5"; it is read as halving the diagonal of
// Dbar (not replacing Dbar by its diagonal), then zeroing the strict upper
// triangle -- the reading that reproduces the unblocked adjoint.
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

struct CholWs {
  double *inv, *panel, *scratch;
};
struct AdjWs {
  double *dinv, *m, *t, *panel, *scratch;
};

size_t block_sz() { return (size_t)tuning().block; }

size_t nblocks(int n) { return (size_t)std::max(1, (n + (int)block_sz() - 1) / (int)block_sz()); }

CholWs carve_chol(void *ws, int n) {
  const size_t b = block_sz();
  char *p = (char *)ws;
  CholWs w;
  w.inv = (double *)p;  // every diagonal-block inverse, block i at inv + i b^2
  p += align_up(nblocks(n) * b * b * sizeof(double), 256);
  w.panel = (double *)p;
  p += align_up((size_t)n * b * sizeof(double), 256);
  w.scratch = (double *)p;
  return w;
}

AdjWs carve_adj(void *ws, int n) {
  const size_t b = block_sz();
  char *p = (char *)ws;
  AdjWs w;
  w.dinv = (double *)p;  // every diagonal-block inverse (blocks counted from the bottom)
  p += align_up(nblocks(n) * b * b * sizeof(double), 256);
  w.m = (double *)p;
  p += align_up(b * b * sizeof(double), 256);
  w.t = (double *)p;
  p += align_up(b * b * sizeof(double), 256);
  w.panel = (double *)p;
  p += align_up((size_t)n * b * sizeof(double), 256);
  w.scratch = (double *)p;
  return w;
}

#define TRY(x)                                 \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return e_;          \
  } while (0)

}  // namespace

size_t chol_workspace_bytes(int n, int /*precision*/) {
  const size_t b = block_sz();
  return align_up(nblocks(n) * b * b * sizeof(double), 256) + align_up((size_t)n * b * sizeof(double), 256) +
         gemm_f64_scratch_bytes();
}

size_t adjoint_workspace_bytes(int n, int /*precision*/) {
  const size_t b = block_sz();
  return align_up(nblocks(n) * b * b * sizeof(double), 256) + 2 * align_up(b * b * sizeof(double), 256) +
         align_up((size_t)n * b * sizeof(double), 256) + gemm_f64_scratch_bytes();
}

int chol_block_size(int precision) { return precision == GPC_MIXED ? 128 : (int)block_sz(); }

cudaError_t chol_fp64(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s) {
  const int b = tuning().block;
  CholWs w = carve_chol(ws, n);
  for (int k0 = 0; k0 < n; k0 += b) {
    const int nb = std::min(b, n - k0), m = n - k0 - nb;
    double *A11 = L + (long long)k0 * ldl + k0;
    TRY(potrf_diag(nb, A11, ldl, info, k0, s));
    if (m <= 0) continue;
    double *A21 = L + (long long)(k0 + nb) * ldl + k0;
    TRY(trsm_rows(m, nb, A21, ldl, A11, ldl, 0, s));  // L21 = A21 L11^{-T}
    Gemm u;  // A22 -= L21 L21^T (lower tiles)
    u.M = m; u.N = m; u.K = nb;
    u.A = A21; u.lda = ldl;
    u.B = A21; u.ldb = ldl; u.transB = true;
    u.C = A21 + nb; u.ldc = ldl;
    u.alpha = -1.0; u.beta = 1.0; u.uplo = UPLO_LOWER;
    TRY(gemm_f64(u, w.scratch, s));
  }
  // every diagonal-block inverse, for the solves that follow the factorisation
  return trtri_batched(n, L, ldl, std::min(b, n), b, w.inv, s);
}

cudaError_t chol_adjoint_fp64(int n, const double *L, long long ldl, double *A, long long lda,
                              void *ws, cudaStream_t s) {
  const int b = tuning().block;
  AdjWs w = carve_adj(ws, n);
  const int nblk = (int)nblocks(n), first = n - (nblk - 1) * b;
  double *dinv_all = w.dinv;
  TRY(trtri_batched(n, L, ldl, first, b, dinv_all, s));  // independent of the sweep: one launch
  for (int k = n, ib = nblk - 1; k > 0; k -= b, --ib) {
    const int j = std::max(0, k - b), nb = k - j, m = n - k;
    const double *D = L + (long long)j * ldl + j;
    double *Dbar = A + (long long)j * lda + j;
    w.dinv = dinv_all + (size_t)ib * b * b;
    if (m > 0) {
      double *Cbar = A + (long long)k * lda + j;
      const double *C = L + (long long)k * ldl + j;
      TRY(trsm_rows(m, nb, Cbar, lda, D, ldl, 1, s));  // Cbar <- Cbar D^{-1}
      if (j > 0) {
        Gemm h;  // Bbar -= Cbar R
        h.M = m; h.N = j; h.K = nb;
        h.A = Cbar; h.lda = lda;
        h.B = L + (long long)j * ldl; h.ldb = ldl;
        h.C = A + (long long)k * lda; h.ldc = lda;
        h.alpha = -1.0; h.beta = 1.0;
        TRY(gemm_f64(h, w.scratch, s));
      }
      Gemm q;  // Dbar -= Cbar^T C (lower)
      q.M = nb; q.N = nb; q.K = m;
      q.A = Cbar; q.lda = lda; q.transA = true;
      q.B = C; q.ldb = ldl;
      q.C = Dbar; q.ldc = lda;
      q.alpha = -1.0; q.beta = 1.0; q.uplo = UPLO_LOWER;
      TRY(gemm_f64(q, w.scratch, s));
    }
    {
      Gemm p;  // M = sym(tril(D^T Dbar))
      p.M = nb; p.N = nb; p.K = nb;
      p.A = D; p.lda = ldl; p.transA = true;
      p.B = Dbar; p.ldb = lda;
      p.C = w.m; p.ldc = nb;
      p.uplo = UPLO_LOWER_MIRROR;
      p.kskip = KSKIP_ROWS;  // D^T upper triangular
      p.algo_flops = (double)nb * nb * nb / 3.0;  // triangular A and B, lower output
      TRY(gemm_f64(p, w.scratch, s));
      Gemm t;  // T = M D^{-1}
      t.M = nb; t.N = nb; t.K = nb;
      t.A = w.m; t.lda = nb;
      t.B = w.dinv; t.ldb = nb;
      t.C = w.t; t.ldc = nb;
      t.kskip = KSKIP_COLS;  // D^{-1} lower triangular
      t.algo_flops = (double)nb * nb * (nb + 1);  // triangular B
      TRY(gemm_f64(t, w.scratch, s));
      Gemm d;  // Dbar = D^{-T} T, symmetric
      d.M = nb; d.N = nb; d.K = nb;
      d.A = w.dinv; d.lda = nb; d.transA = true;
      d.B = w.t; d.ldb = nb;
      d.C = Dbar; d.ldc = lda;
      d.uplo = UPLO_LOWER_MIRROR;
      d.kskip = KSKIP_ROWS;  // D^{-T} upper triangular
      d.algo_flops = (double)nb * nb * nb / 3.0 * 2.0;  // triangular A, lower output
      TRY(gemm_f64(d, w.scratch, s));
    }
    if (j > 0) {
      Gemm r;  // Rbar -= [Dbar; Cbar]^T [R; B]
      r.M = nb; r.N = j; r.K = n - j;
      r.A = Dbar; r.lda = lda; r.transA = true;
      r.B = L + (long long)j * ldl; r.ldb = ldl;
      r.C = A + (long long)j * lda; r.ldc = lda;
      r.alpha = -1.0; r.beta = 1.0;
      TRY(gemm_f64(r, w.scratch, s));
    }
    TRY(phi_block(nb, Dbar, lda, s));
  }
  return cudaSuccess;
}

}  // namespace gpc
