// Mixed-precision blocked Cholesky and blocked adjoint (precision GPC_MIXED).
//
// Same block algorithms as the FP64 path (Section 3.3; see chol.cu), with the
// O(n^3) products moved to split-BF16 tensor-core products (ozaki.cu):
//   forward: the trailing update A22 -= L21 L21^T;
//   adjoint: Bbar -= Cbar R and Rbar -= [Dbar; Cbar]^T [R; B].
// The diagonal blocks, their inverses, the panel products with the inverses
// and the Dbar update stay FP64.  Matrices that the split products update
// (the trailing part of L, the not-yet-final part of Lbar) are held in
// double-float storage (FP32 hi + lo in each 8-byte element); each block
// column is converted back to FP64 in place when it becomes current, so every
// output is FP64 at the end.  The block size is fixed to the 128-wide chunk of
// the split products so chunk boundaries line up with the sweep's blocks.
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr int MB = 128;  // block size of the mixed path (== slice chunk)
constexpr size_t kPartialCap = size_t(40) << 20;

#define TRY(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

struct MixWs {
  double *inv, *m, *t, *panel, *scratch;  // FP64 pieces (scratch doubles as the split-K partials)
  void *sc, *sdc, *lt;                    // slices: panel rows, block-column columns, L^T
};

size_t b2() { return align_up((size_t)MB * MB * sizeof(double), 256); }
size_t scratch_bytes() { return std::max(gemm_f64_scratch_bytes(), kPartialCap); }
int nchunks(int n) { return std::max(1, (n + MB - 1) / MB); }

MixWs carve(void *ws, int n, bool adjoint) {
  char *p = (char *)ws;
  MixWs w{};
  w.inv = (double *)p; p += b2();
  w.m = (double *)p; p += b2();
  w.t = (double *)p; p += b2();
  w.panel = (double *)p; p += align_up((size_t)n * MB * sizeof(double), 256);
  w.scratch = (double *)p; p += scratch_bytes();
  w.sc = p; p += slice_bytes(n, 1);
  if (adjoint) {
    w.sdc = p; p += slice_bytes(MB, nchunks(n));
    w.lt = p; p += slice_bytes(n, nchunks(n));
  }
  return w;
}

}  // namespace

size_t mixed_workspace_bytes(int n) {
  n = std::max(n, 1);
  return 3 * b2() + align_up((size_t)n * MB * sizeof(double), 256) + scratch_bytes() + slice_bytes(n, 1) +
         slice_bytes(MB, nchunks(n)) + slice_bytes(n, nchunks(n)) + 1024;
}

cudaError_t chol_mixed(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s) {
  MixWs w = carve(ws, n, false);
  for (int k0 = 0; k0 < n; k0 += MB) {
    const int nb = std::min(MB, n - k0), m = n - k0 - nb;
    double *A11 = L + (long long)k0 * ldl + k0;
    TRY(from_df_rect(n - k0, nb, A11, ldl, s));
    TRY(potrf_trtri_diag(nb, A11, ldl, w.inv, info, k0, s));
    if (m <= 0) continue;
    double *A21 = L + (long long)(k0 + nb) * ldl + k0;
    TRY(copy_rect(m, nb, A21, ldl, w.panel, nb, s));
    Gemm g;  // L21 = A21 * L11^{-T} (FP64)
    g.M = m; g.N = nb; g.K = nb;
    g.A = w.panel; g.lda = nb;
    g.B = w.inv; g.ldb = nb; g.transB = true;
    g.C = A21; g.ldc = ldl;
    g.algo_flops = (double)m * nb * (nb + 1);
    TRY(gemm_f64(g, w.scratch, s));
    // A22 -= L21 L21^T on split-BF16 slices, lower tiles, double-float storage
    SliceBuf S = slice_view(w.sc, m, 1);
    TRY(split_operand(A21, ldl, 1, m, nb, nb, S, s));
    TRY(ozaki_gemm(S, 0, 0, S, 0, 0, m, m, 1, true, -1.0f, (float2 *)(A21 + nb), ldl, 1, nullptr,
                   info ? info + 1 : nullptr, s));
  }
  return cudaSuccess;
}

cudaError_t chol_adjoint_mixed(int n, const double *L, long long ldl, double *A, long long lda, void *ws,
                               int *err, cudaStream_t s) {
  MixWs w = carve(ws, n, true);
  const int nblk = nchunks(n);
  const int first = n - (nblk - 1) * MB;  // rows in the top-left block
  // L^T slices: operand row t = column t of L, K = rows of L, chunked like the sweep's blocks.
  SliceBuf LT = slice_view(w.lt, n, nblk);
  TRY(split_operand(L, 1, ldl, n, n, first, LT, s));
  for (int ib = nblk - 1; ib >= 0; --ib) {
    const int j = (ib == 0) ? 0 : first + (ib - 1) * MB;
    const int k = first + ib * MB;
    const int nb = k - j, m = n - k;
    const double *D = L + (long long)j * ldl + j;
    double *Dbar = A + (long long)j * lda + j;
    TRY(from_df_rect(n - j, nb, Dbar, lda, s));
    TRY(trtri_diag(nb, D, ldl, w.inv, s));
    if (m > 0) {
      double *Cbar = A + (long long)k * lda + j;
      const double *C = L + (long long)k * ldl + j;
      TRY(copy_rect(m, nb, Cbar, lda, w.panel, nb, s));
      Gemm g;  // Cbar <- Cbar D^{-1} (FP64)
      g.M = m; g.N = nb; g.K = nb;
      g.A = w.panel; g.lda = nb;
      g.B = w.inv; g.ldb = nb;
      g.C = Cbar; g.ldc = lda;
      g.algo_flops = (double)m * nb * (nb + 1);
      TRY(gemm_f64(g, w.scratch, s));
      if (j > 0) {  // Bbar -= Cbar R on slices (Bbar in double-float storage)
        SliceBuf SC = slice_view(w.sc, m, 1);
        TRY(split_operand(Cbar, lda, 1, m, nb, nb, SC, s));
        TRY(ozaki_gemm(SC, 0, 0, LT, 0, ib * MB, m, j, 1, false, -1.0f, (float2 *)(A + (long long)k * lda),
                       lda, 1, nullptr, err, s));
      }
      Gemm q;  // Dbar -= Cbar^T C (lower, FP64)
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
      p.algo_flops = (double)nb * nb * nb / 3.0;
      TRY(gemm_f64(p, w.scratch, s));
      Gemm t;  // T = M D^{-1}
      t.M = nb; t.N = nb; t.K = nb;
      t.A = w.m; t.lda = nb;
      t.B = w.inv; t.ldb = nb;
      t.C = w.t; t.ldc = nb;
      t.algo_flops = (double)nb * nb * (nb + 1);
      TRY(gemm_f64(t, w.scratch, s));
      Gemm d;  // Dbar = D^{-T} T, symmetric
      d.M = nb; d.N = nb; d.K = nb;
      d.A = w.inv; d.lda = nb; d.transA = true;
      d.B = w.t; d.ldb = nb;
      d.C = Dbar; d.ldc = lda;
      d.uplo = UPLO_LOWER_MIRROR;
      d.algo_flops = (double)nb * nb * nb / 3.0 * 2.0;
      TRY(gemm_f64(d, w.scratch, s));
    }
    if (j > 0) {  // Rbar -= [Dbar; Cbar]^T [R; B] on slices (Rbar in double-float storage)
      const int chunks = nblk - ib;
      SliceBuf SDC = slice_view(w.sdc, nb, chunks);
      TRY(split_operand(Dbar, 1, lda, nb, n - j, nb, SDC, s));
      const int tiles = (j + 63) / 64;
      int splits = std::max(1, std::min(chunks, (2 * sm_count() + tiles - 1) / tiles));
      while (splits > 1 && ozaki_partial_bytes(nb, j, splits) > kPartialCap) --splits;
      TRY(ozaki_gemm(SDC, 0, 0, LT, 0, ib * MB, nb, j, chunks, false, -1.0f, (float2 *)(A + (long long)j * lda),
                     lda, splits, (float2 *)w.scratch, err, s));
    }
    TRY(phi_block(nb, Dbar, lda, s));
  }
  return cudaSuccess;
}

}  // namespace gpc
