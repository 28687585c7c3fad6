// Lower-triangular inverse, triangular solve with a matrix right-hand side and
// the solve's reverse mode (Section 3.2).
//
// Inverse (Section 3.2, primitive function).  A lower-triangular matrix split
// as [[A1, 0], [A3, A2]] has the inverse [[C1, 0], [C3, C2]] with C1 = A1^{-1},
// C2 = A2^{-1} and C3 = -C2 A3 C1.  As in the paper's many-core version the
// recursion is run bottom-up: first every b x b diagonal block is inverted
// (one CTA each, in shared memory), then the block width doubles level by
// level, each level forming C3 for all pairs of neighbouring w-blocks at
// once.  Each level is two FP64 tensor-core products batched over the pairs
// (grid.y of the FP64 GEMM): T = C2 A3, then C3 = -T C1.  T is kept
// transposed in the strict upper triangle of the output, in the mirror image
// of the C3 block it feeds, which nothing reads until it is cleared at the
// end -- so the inverse needs no workspace and may overwrite its input.
// Triangular operands skip their zero K range tile by tile.
//
// Solve: C = L^{-1} B through the inverse and one product, as in the paper's
// general solver; the inverse is the caller's buffer and is kept for the
// reverse mode.
//
// Reverse mode (Section 3.2, reverse mode function): for C = L^{-1} B and an
// upstream Cbar, Bbar = L^{-T} Cbar (a product with the kept inverse) and
// Lbar = -tril(Bbar C^T) (lower output tiles only).  The paper prints the
// adjoint system with A where the transpose belongs; the transpose is what the
// differential of the solve gives.
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr int kInvBlock = 128;  // diagonal blocks inverted in shared memory (a multiple of the 64-wide tile)

#define TRY(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

__global__ void __launch_bounds__(256) zero_strict_upper_kernel(int n, double *X, long long ldx) {
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    double *row = X + (long long)i * ldx;
    for (int j = i + 1 + threadIdx.x; j < n; j += blockDim.x) row[j] = 0.0;
  }
}

cudaError_t zero_strict_upper(int n, double *X, long long ldx, cudaStream_t s) {
  if (n <= 1) return cudaSuccess;
  const int grid = std::min(n, 8 * sm_count());
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 4.0 * (double)n * (n - 1), s,
             zero_strict_upper_kernel<<<grid, 256, 0, s>>>(n, X, ldx));
  return cudaGetLastError();
}

// C3 = -C2 A3 C1 for `count` pairs of neighbouring diagonal blocks: the upper
// block of pair p has rows [r0 + 2wp, r0 + 2wp + w), the lower one the next h
// rows.  A3 is read from L, C1 and C2 from X, and C3 is written to X.
cudaError_t combine_pairs(int w, int h, int count, int r0, const double *L, long long ldl, double *X,
                          long long ldx, cudaStream_t s) {
  const long long stepL = 2LL * w * (ldl + 1), stepX = 2LL * w * (ldx + 1);
  // T^T (w x h) = A3^T C2^T, into the mirror image of C3 in X's upper triangle.
  // op(B) = C2^T is upper triangular: columns below n0 + 64 need k < n0 + 64.
  Gemm t;
  t.M = w; t.N = h; t.K = h;
  t.transA = true;  // A3 (h x w) stored K x M
  t.A = L + (long long)(r0 + w) * ldl + r0; t.lda = ldl;
  t.transB = true;  // C2 (h x h) stored N x K
  t.B = X + (long long)(r0 + w) * ldx + (r0 + w); t.ldb = ldx;
  t.C = X + (long long)r0 * ldx + (r0 + w); t.ldc = ldx;
  t.alpha = 1.0; t.beta = 0.0;
  t.kskip = KSKIP_COLS_END;
  t.batch = count; t.sA = stepL; t.sB = stepX; t.sC = stepX;
  t.algo_flops = (double)count * w * h * (h + 1.0);
  TRY(gemm_f64(t, nullptr, s));
  // C3 (h x w) = -T C1; op(B) = C1 is lower triangular: columns from n0 need k >= n0.
  Gemm c;
  c.M = h; c.N = w; c.K = w;
  c.transA = true;  // T^T (w x h) stored K x M
  c.A = X + (long long)r0 * ldx + (r0 + w); c.lda = ldx;
  c.B = X + (long long)r0 * ldx + r0; c.ldb = ldx;
  c.C = X + (long long)(r0 + w) * ldx + r0; c.ldc = ldx;
  c.alpha = -1.0; c.beta = 0.0;
  c.kskip = KSKIP_COLS;
  c.batch = count; c.sA = stepX; c.sB = stepX; c.sC = stepX;
  c.algo_flops = (double)count * h * w * (w + 1.0);
  return gemm_f64(c, nullptr, s);
}

}  // namespace

cudaError_t tri_inverse(int n, const double *L, long long ldl, double *X, long long ldx, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int b = kInvBlock;
  TRY(trtri_batched(n, L, ldl, std::min(b, n), b, X, s, ldx));
  for (long long w = b; w < n; w *= 2) {
    const long long full = n / (2 * w);  // pairs whose lower block has all w rows
    const long long rest = n - full * 2 * w;
    if (full > 0) TRY(combine_pairs((int)w, (int)w, (int)full, 0, L, ldl, X, ldx, s));
    if (rest > w) TRY(combine_pairs((int)w, (int)(rest - w), 1, (int)(full * 2 * w), L, ldl, X, ldx, s));
  }
  return zero_strict_upper(n, X, ldx, s);
}

cudaError_t tri_solve(int n, int m, const double *L, long long ldl, const double *B, long long ldb, double *X,
                      long long ldx, double *C, long long ldc, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  TRY(tri_inverse(n, L, ldl, X, ldx, s));
  if (m <= 0) return cudaSuccess;
  Gemm g;  // C = X B; op(A) = X is lower triangular: rows below m0 + 64 need k < m0 + 64
  g.M = n; g.N = m; g.K = n;
  g.A = X; g.lda = ldx;
  g.B = B; g.ldb = ldb;
  g.C = C; g.ldc = ldc;
  g.kskip = KSKIP_ROWS_END;
  g.algo_flops = (double)n * n * m;
  return gemm_f64(g, nullptr, s);
}

cudaError_t tri_solve_adjoint(int n, int m, const double *X, long long ldx, const double *C, long long ldc,
                              const double *Cbar, long long ldcb, double *Bbar, long long ldbb, double *Lbar,
                              long long ldlb, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  if (m <= 0)
    return cudaMemset2DAsync(Lbar, (size_t)ldlb * sizeof(double), 0, (size_t)n * sizeof(double), (size_t)n, s);
  Gemm g;  // Bbar = X^T Cbar; op(A) = X^T is upper triangular: rows from m0 need k >= m0
  g.M = n; g.N = m; g.K = n;
  g.transA = true; g.A = X; g.lda = ldx;
  g.B = Cbar; g.ldb = ldcb;
  g.C = Bbar; g.ldc = ldbb;
  g.kskip = KSKIP_ROWS;
  g.algo_flops = (double)n * n * m;
  TRY(gemm_f64(g, nullptr, s));
  Gemm l;  // Lbar = -tril(Bbar C^T), lower output tiles only
  l.M = n; l.N = n; l.K = m;
  l.A = Bbar; l.lda = ldbb;
  l.transB = true; l.B = C; l.ldb = ldc;
  l.C = Lbar; l.ldc = ldlb;
  l.alpha = -1.0;
  l.uplo = UPLO_LOWER;
  TRY(gemm_f64(l, nullptr, s));
  return zero_strict_upper(n, Lbar, ldlb, s);
}

}  // namespace gpc
