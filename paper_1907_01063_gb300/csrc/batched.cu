// Batched Gaussian-process likelihood and gradient: many independent GPs of
// uneven size in one persistent launch.
//
// Each CTA takes whole GPs from a device queue ordered by size, largest
// first (longest-processing-time-first), and runs the complete pass for that
// GP: SE covariance, blocked Cholesky (Section 3.3, primitive function),
// forward and backward solves, log det and log marginal likelihood, the
// upstream adjoint Lbar, the blocked reverse-mode sweep (Section 3.3, reverse
// mode function) and the hyperparameter gradient.  The batched diagonal
// inverses of Section 3.2 are the precedent for giving each small problem its
// own thread block, and they are used the same way here: the inverse of every
// diagonal block is formed once, right after the block is factored, and kept
// for the whole pass.
//
// FP64 is the scarce resource on this part (under two FP64 multiply-adds per
// cycle per SM, and a warp instruction occupies its sub-partition's FP64 unit
// for the full warp whatever its active lanes), so the pass is arranged to
// keep FP64 work in full-warp, independent form:
//   * panel solves are products with the stored inverses (L21 <- A21 L11^-T in
//     the factorisation, Cbar <- Cbar D^-1 in the adjoint) on the FP64 tensor
//     tiles, with the zero K steps of the triangular operand skipped;
//   * the forward and backward solves apply the stored block inverses as small
//     matrix-vector products and update the rest of the vector right-looking,
//     so no scalar substitution chain is left;
//   * the diagonal block is factored left-looking with the dot products split
//     over 1..32 threads per row and a refined 1/sqrt, and inverted
//     right-looking with the updates dealt evenly to all threads;
//   * the kernel values computed for the covariance are kept (packed lower
//     triangle) and reused by the gradient, which then needs no exponentials.
//
// Products inside a CTA are 64 x 64 output tiles on the FP64 tensor path
// (mma.sync m16n8k16 .f64), operands staged through shared memory with the
// next K step prefetched into registers.  Warps take interleaved 16-row and
// 8-column fragments, so skipped fragments (outside a ragged edge, above the
// diagonal of a triangular output, or in the zero part of a triangular
// operand) are spread over the four warps instead of idling one of them.
// In the mixed path the O(n^3) products instead run as split-BF16 slice
// products (slices.cuh) on the BF16 tensor path with FP32 group sums folded
// once per 32-wide K step into double-float accumulators; their FP64 operand
// tiles are double-buffered in shared memory with asynchronous copies.
// Each GP's factor overwrites its covariance in the caller's Kws; Kbar, the
// kernel values, the block inverses and the vectors live in a per-CTA slot of
// the workspace and are reused GP to GP.
#include "common.cuh"
#include "slices.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace gpc {
namespace {

constexpr int BT = 128;                  // threads per CTA (4 warps)
constexpr int TM = 64, TK = 16, TP = 4;  // FP64 product tile, K step, row padding
constexpr int MAXB = 64;                 // largest block size
constexpr int XLD = 40;                  // padded row of a BF16 slice tile (32 K + 8: conflict-free fragment loads)

// Structure of a tile product's operands and output.  A fragment's K step is
// skipped where the operand is known to be zero.
enum : int {
  TG_LOWER = 1,  // output: only col <= row is written; fragments above the diagonal are skipped
  TG_A_KGE = 2,  // op(A)(m, k) == 0 unless k >= m
  TG_B_KLE = 4,  // op(B)(k, n) == 0 unless k <= n
  TG_B_KGE = 8,  // op(B)(k, n) == 0 unless k >= n
};

struct BatchParams {
  int batch, d, nb, nmax;
  const int *n;
  const long long *offK, *rowX;
  const double *X, *y, *hyp;
  double *K;
  double *slots;
  long long slot_elems;
  const int *order;
  int *queue;
  double *value, *grad3;
  int *info;
};

// Shared memory: the FP64 working set, then a region used either for the
// diagonal block and its inverse or (mixed path, inside the products) for the
// two stages of slice tiles.
struct SmemF {
  double As[TM][TK + TP];
  double Bs[TM][TK + TP];
  double v[MAXB];
  double w[MAXB];
  double red[8];
  int flag;
};
struct SmemT {
  double D[MAXB][MAXB + 1];  // the diagonal block, factored in place
  double X[MAXB][MAXB + 1];  // its inverse
};
struct SmemS {
  __nv_bfloat16 A[2][kSlices][TM][XLD];
  __nv_bfloat16 B[2][kSlices][TM][XLD];
};
constexpr size_t kRegionOffset = (sizeof(SmemF) + 127) / 128 * 128;
constexpr size_t kSmemF64 = kRegionOffset + sizeof(SmemT);
constexpr size_t kSmemMixed = kRegionOffset + (sizeof(SmemS) > sizeof(SmemT) ? sizeof(SmemS) : sizeof(SmemT));

__device__ __forceinline__ void dmma(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
        "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// Fragment (mi, ni) of warp (wm, wn) in a 64 x 64 tile: rows 16 (wm + 2 mi) ..
// + 15 and columns 8 (wn + 2 ni) .. + 7 of the tile (interleaved, see above).
__device__ __forceinline__ int frag_row(int wm, int mi) { return 16 * (wm + 2 * mi); }
__device__ __forceinline__ int frag_col(int wn, int ni) { return 8 * (wn + 2 * ni); }

// Whether fragment rows [r0, r0+16) x cols [c0, c0+8) (tile-absolute) takes
// part in K step [k0, k0+16).
__device__ __forceinline__ bool frag_active(int r0, int c0, int k0, int M, int N, int flags) {
  if (r0 >= M || c0 >= N) return false;
  if ((flags & TG_LOWER) && c0 > r0 + 15) return false;
  if ((flags & TG_A_KGE) && k0 + 15 < r0) return false;
  if ((flags & TG_B_KLE) && k0 > c0 + 7) return false;
  if ((flags & TG_B_KGE) && k0 + 15 < c0) return false;
  return true;
}

// Global -> registers for one 16-wide K step of a 64 x 64 tile (8 + 8 values per thread).
template <bool TA, bool TB>
__device__ __forceinline__ void tile_fetch(const double *A, long long lda, const double *B, long long ldb, int M,
                                           int N, int K, int m0, int n0, int k0, double (&ra)[8],
                                           double (&rb)[8]) {
  const int t = threadIdx.x;
  if (!TA) {  // A[m][k]: 2 threads per row, 8 consecutive k each
    const int r = t >> 1, c0 = (t & 1) * 8, m = m0 + r;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + c0 + i;
      ra[i] = (m < M && k < K) ? A[(long long)m * lda + k] : 0.0;
    }
  } else {  // A[k][m]: 8 threads per k row, 8 consecutive m each
    const int kk = t >> 3, mm0 = (t & 7) * 8, k = k0 + kk;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int m = m0 + mm0 + i;
      ra[i] = (m < M && k < K) ? A[(long long)k * lda + m] : 0.0;
    }
  }
  if (!TB) {  // B[k][n]
    const int kk = t >> 3, nn0 = (t & 7) * 8, k = k0 + kk;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int nn = n0 + nn0 + i;
      rb[i] = (nn < N && k < K) ? B[(long long)k * ldb + nn] : 0.0;
    }
  } else {  // B[n][k]
    const int r = t >> 1, c0 = (t & 1) * 8, nn = n0 + r;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int k = k0 + c0 + i;
      rb[i] = (nn < N && k < K) ? B[(long long)nn * ldb + k] : 0.0;
    }
  }
}

template <bool TA, bool TB>
__device__ __forceinline__ void tile_stash(const double (&ra)[8], const double (&rb)[8], SmemF &sm) {
  const int t = threadIdx.x;
  if (!TA) {
    const int r = t >> 1, c0 = (t & 1) * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.As[r][c0 + i] = ra[i];
  } else {
    const int kk = t >> 3, mm0 = (t & 7) * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.As[mm0 + i][kk] = ra[i];
  }
  if (!TB) {
    const int kk = t >> 3, nn0 = (t & 7) * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.Bs[nn0 + i][kk] = rb[i];
  } else {
    const int r = t >> 1, c0 = (t & 1) * 8;
#pragma unroll
    for (int i = 0; i < 8; ++i) sm.Bs[r][c0 + i] = rb[i];
  }
}

// One 64 x 64 output tile of C = beta C + alpha op(A) op(B) over K, rows
// [m0, m0+64) and cols [n0, n0+64) clipped to M x N.
// op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k];  op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
// The tile reads all of its operands before it writes C, so C may alias
// op(A)'s rows when N <= 64 (a single tile column).
template <bool TA, bool TB>
__device__ __noinline__ void tile_gemm(const double *A, long long lda, const double *B, long long ldb, double *C,
                                       long long ldc, int M, int N, int K, double alpha, double beta, int flags,
                                       int m0, int n0, SmemF &sm) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
  double acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0;
  double ra[8], rb[8];
  tile_fetch<TA, TB>(A, lda, B, ldb, M, N, K, m0, n0, 0, ra, rb);
  for (int k0 = 0; k0 < K; k0 += TK) {
    __syncthreads();
    tile_stash<TA, TB>(ra, rb, sm);
    __syncthreads();
    if (k0 + TK < K) tile_fetch<TA, TB>(A, lda, B, ldb, M, N, K, m0, n0, k0 + TK, ra, rb);
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = frag_row(wm, mi);
      double a[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = sm.As[r + g + 8 * (i & 1)][tg + 4 * (i >> 1)];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = frag_col(wn, ni);
        if (!frag_active(m0 + r, n0 + c, k0, M, N, flags)) continue;
        double b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) b[i] = sm.Bs[c + g][tg + 4 * i];
        dmma(acc[mi][ni], a, b);
      }
    }
  }
  // epilogue: the outputs of a thread are loaded together (when beta != 0)
  double cv[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + frag_row(wm, mi) + g + ((r >> 1) << 3);
        const int col = n0 + frag_col(wn, ni) + 2 * tg + (r & 1);
        const bool in = row < M && col < N && !((flags & TG_LOWER) && col > row);
        cv[mi][ni][r] = (in && beta != 0.0) ? C[(long long)row * ldc + col] : 0.0;
      }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + frag_row(wm, mi) + g + ((r >> 1) << 3);
        const int col = n0 + frag_col(wn, ni) + 2 * tg + (r & 1);
        if (row >= M || col >= N || ((flags & TG_LOWER) && col > row)) continue;
        double v;
        if (beta == 0.0) v = alpha * acc[mi][ni][r];
        else if (beta == 1.0) v = fma(alpha, acc[mi][ni][r], cv[mi][ni][r]);  // alpha = +-1 in every call
        else v = fma(beta, cv[mi][ni][r], alpha * acc[mi][ni][r]);
        C[(long long)row * ldc + col] = v;
      }
  __syncthreads();
}

template <bool TA, bool TB>
__device__ void cta_gemm(const double *A, long long lda, const double *B, long long ldb, double *C, long long ldc,
                         int M, int N, int K, double alpha, double beta, int flags, SmemF &sm) {
  for (int m0 = 0; m0 < M; m0 += TM)
    for (int n0 = 0; n0 < N; n0 += TM) {
      if ((flags & TG_LOWER) && n0 > m0 + TM - 1) break;
      tile_gemm<TA, TB>(A, lda, B, ldb, C, ldc, M, N, K, alpha, beta, flags, m0, n0, sm);
    }
}

// ------------------------------------------------------------------ mixed products
// Operands of the mixed products are split into BF16 slices once per use (the
// factorisation's panel once per block step, L^T once per pass, the adjoint's
// block column once per step) into slice buffers of the workspace:
// slice p of operand row r, K index k at S[p * plane + r * kpad + k], K
// contiguous, one scale per (row, 32-wide K chunk) folded into the values,
// chunks padded with zeros.  The tiles then only copy slices.
using bf16 = __nv_bfloat16;
constexpr int SL_CH = 32;  // K chunk of one scale (= one K step of a tile)

struct SliceOp {
  const bf16 *S;
  long long plane;  // elements between slices
  int kpad;         // elements between operand rows
  int k0;           // first K index used
};

// Slices of the rows of A (rows x K, row-major, ld lda): operand row r is row
// r of A.  A warp takes (row, chunk) units, a lane one K index, so reads and
// slice writes are contiguous; the chunk's exponent is a warp max.  A warp
// loads eight units before it splits them, so one memory latency covers eight.
__device__ __noinline__ void split_rows_cta(const double *A, long long lda, int rows, int K, bf16 *S, long long plane, int kpad) {
  constexpr int U = 8;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int chunks = (K + SL_CH - 1) / SL_CH, units = rows * chunks;
  for (int u0 = warp * U; u0 < units; u0 += U * (BT / 32)) {
    unsigned long long bits[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int u = u0 + q, r = u / chunks, k = (u - r * chunks) * SL_CH + lane;
      bits[q] = (u < units && k < K) ? (unsigned long long)__double_as_longlong(A[(long long)r * lda + k]) : 0ull;
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int u = u0 + q, r = u / chunks, k = (u - r * chunks) * SL_CH + lane;
      if (u >= units) break;
      const int ex = __reduce_max_sync(0xffffffffu, slice_exponent(bits[q]));
      float v[kSlices];
      split_value(bits[q], ex, v);
      bf16 *dst = S + (long long)r * kpad + k;
#pragma unroll
      for (int pp = 0; pp < kSlices; ++pp) dst[pp * plane] = __float2bfloat16_rn(v[pp]);
    }
  }
  __syncthreads();
}

// Slices of the columns of A (Krows x cols, row-major, ld lda): operand row c is
// column c of A, its K index k is row k of A, stored at K offset koff (a
// multiple of the chunk).  32 x 32 blocks of A pass through shared memory
// (T, 32 x 33 doubles) so that both the reads of A and the slice writes are
// contiguous; the next block is loaded into registers while one is split.
__device__ __noinline__ void split_cols_cta(const double *A, long long lda, int Krows, int cols, bf16 *S, long long plane,
                               int kpad, int koff, double (*T)[33]) {
  constexpr int RW = SL_CH / (BT / 32);  // rows of a block per warp
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int rch = (Krows + SL_CH - 1) / SL_CH, cch = (cols + 31) / 32, nblk = rch * cch;
  double nxt[RW];
  auto load = [&](int blk) {
    const int r0 = (blk / cch) * SL_CH, c0 = (blk - (blk / cch) * cch) * 32, col = c0 + lane;
#pragma unroll
    for (int q = 0; q < RW; ++q) {
      const int row = r0 + warp + q * (BT / 32);
      nxt[q] = (row < Krows && col < cols) ? A[(long long)row * lda + col] : 0.0;
    }
  };
  if (nblk > 0) load(0);
  for (int blk = 0; blk < nblk; ++blk) {
    const int r0 = (blk / cch) * SL_CH, c0 = (blk - (blk / cch) * cch) * 32;
    __syncthreads();
#pragma unroll
    for (int q = 0; q < RW; ++q) T[warp + q * (BT / 32)][lane] = nxt[q];
    __syncthreads();
    if (blk + 1 < nblk) load(blk + 1);
    for (int cc = warp; cc < 32; cc += BT / 32) {
      const int col = c0 + cc;
      if (col >= cols) break;
      const unsigned long long bits = (unsigned long long)__double_as_longlong(T[lane][cc]);
      const int ex = __reduce_max_sync(0xffffffffu, slice_exponent(bits));
      float v[kSlices];
      split_value(bits, ex, v);
      bf16 *dst = S + (long long)col * kpad + koff + r0 + lane;
#pragma unroll
      for (int pp = 0; pp < kSlices; ++pp) dst[pp * plane] = __float2bfloat16_rn(v[pp]);
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void hmma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void two_sum_f(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float v = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, v)), __fsub_rn(b, v));
}
// (hi, lo) += g2 + g3 + g4 + g5 (slice groups in decreasing scale): exact
// two-sums for the three exact groups, the rounded last group into the low part
__device__ __forceinline__ void df_acc4(float &hi, float &lo, float g2, float g3, float g4, float g5) {
  float s, e1, e2, e3;
  two_sum_f(hi, g2, s, e1);
  two_sum_f(s, g3, s, e2);
  two_sum_f(s, g4, s, e3);
  const float e = __fadd_rn(__fadd_rn(__fadd_rn(lo, g5), __fadd_rn(e1, e2)), e3);
  hi = __fadd_rn(s, e);
  lo = __fsub_rn(e, __fsub_rn(hi, s));
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Copy the slices of one K step of a 64-row operand tile into a stage
// (5 slices x 64 rows x 32 K = 1280 copies of 16 bytes); rows >= rows_valid
// are zero-filled.
__device__ __forceinline__ void slice_fetch(const SliceOp &op, int row0, int rows_valid, int kstep,
                                            bf16 (*dst)[TM][XLD]) {
  const long long kbase = (long long)op.k0 + (long long)kstep * SL_CH;
#pragma unroll 2
  for (int idx = threadIdx.x; idx < kSlices * TM * 4; idx += BT) {
    const int pp = idx >> 8, rem = idx & 255, r = rem >> 2, q = rem & 3;
    const bool in = row0 + r < rows_valid;
    const bf16 *src = in ? op.S + pp * op.plane + (long long)(row0 + r) * op.kpad + kbase + 8 * q : op.S;
    cp_async16(&dst[pp][r][8 * q], src, in ? 16 : 0);
  }
}

// One 64 x 64 tile of C -= A B^T from slices: op(A) rows [m0, m0+64) of A,
// op(B)(k, n) = row n of B, K steps of one chunk.  Per 16 x 8 fragment and
// step the 15 slice products with p + q <= 4 (0-based) go to ten independent
// FP32 accumulators (so no long chain of dependent tensor instructions), which
// are combined into the four groups p + q = 0, 1, 2 (exact: integer sums
// below 2^22 in units of their scale) and 3-4 (rounded) and added once into
// a double-float accumulator.  The epilogue loads its 32 outputs per thread
// together, then writes C - (hi + lo) in FP64.  TG_LOWER is the only flag used.
__device__ __noinline__ void tile_gemm_sl(const SliceOp &A, const SliceOp &B, double *C, long long ldc, int M, int N,
                                          int K, int flags, int m0, int n0, SmemS &ss) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
  const bool lower = (flags & TG_LOWER) != 0;
  float hi[2][4][4], lo[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) hi[i][j][r] = lo[i][j][r] = 0.0f;
  const int steps = (K + SL_CH - 1) / SL_CH;
  __syncthreads();  // the previous user of the stages is done
  slice_fetch(A, m0, M, 0, ss.A[0]);
  slice_fetch(B, n0, N, 0, ss.B[0]);
  cp_async_commit();
  for (int s = 0; s < steps; ++s) {
    const int b = s & 1;
    if (s + 1 < steps) {
      slice_fetch(A, m0, M, s + 1, ss.A[b ^ 1]);
      slice_fetch(B, n0, N, s + 1, ss.B[b ^ 1]);
      cp_async_commit();
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int rbase = frag_row(wm, mi);
      if (m0 + rbase >= M) continue;
      const int ra = rbase + g;
      uint32_t a[2][kSlices][4];
#pragma unroll
      for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int pp = 0; pp < kSlices; ++pp) {
          a[kk][pp][0] = *(const uint32_t *)&ss.A[b][pp][ra][16 * kk + 2 * tg];
          a[kk][pp][1] = *(const uint32_t *)&ss.A[b][pp][ra + 8][16 * kk + 2 * tg];
          a[kk][pp][2] = *(const uint32_t *)&ss.A[b][pp][ra][16 * kk + 2 * tg + 8];
          a[kk][pp][3] = *(const uint32_t *)&ss.A[b][pp][ra + 8][16 * kk + 2 * tg + 8];
        }
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const int c = frag_col(wn, ni);
        if (n0 + c >= N || (lower && n0 + c > m0 + rbase + 15)) continue;
        const int cb = c + g;
        // accumulators: 0 (0,0) | 1 (0,1) 2 (1,0) | 3 (0,2) 4 (1,1) 5 (2,0) |
        // 6 (0,3)(3,0) 7 (1,2)(2,1) 8 (0,4)(4,0) 9 (1,3)(3,1)(2,2)
        float ac[10][4];
#pragma unroll
        for (int q = 0; q < 10; ++q)
#pragma unroll
          for (int r = 0; r < 4; ++r) ac[q][r] = 0.0f;
#pragma unroll
        for (int kk = 0; kk < 2; ++kk) {
          uint32_t bf[kSlices][2];
#pragma unroll
          for (int pp = 0; pp < kSlices; ++pp) {
            bf[pp][0] = *(const uint32_t *)&ss.B[b][pp][cb][16 * kk + 2 * tg];
            bf[pp][1] = *(const uint32_t *)&ss.B[b][pp][cb][16 * kk + 2 * tg + 8];
          }
          hmma_bf16(ac[0], a[kk][0], bf[0]);
          hmma_bf16(ac[1], a[kk][0], bf[1]);
          hmma_bf16(ac[2], a[kk][1], bf[0]);
          hmma_bf16(ac[3], a[kk][0], bf[2]);
          hmma_bf16(ac[4], a[kk][1], bf[1]);
          hmma_bf16(ac[5], a[kk][2], bf[0]);
          hmma_bf16(ac[6], a[kk][0], bf[3]);
          hmma_bf16(ac[7], a[kk][1], bf[2]);
          hmma_bf16(ac[8], a[kk][0], bf[4]);
          hmma_bf16(ac[9], a[kk][1], bf[3]);
          hmma_bf16(ac[6], a[kk][3], bf[0]);
          hmma_bf16(ac[7], a[kk][2], bf[1]);
          hmma_bf16(ac[8], a[kk][4], bf[0]);
          hmma_bf16(ac[9], a[kk][3], bf[1]);
          hmma_bf16(ac[9], a[kk][2], bf[2]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          const float g1 = __fadd_rn(ac[1][r], ac[2][r]);                   // exact
          const float g2 = __fadd_rn(__fadd_rn(ac[3][r], ac[4][r]), ac[5][r]);  // exact
          const float g3 = __fadd_rn(__fadd_rn(ac[6][r], ac[7][r]), __fadd_rn(ac[8][r], ac[9][r]));
          df_acc4(hi[mi][ni][r], lo[mi][ni][r], ac[0][r], g1, g2, g3);
        }
      }
    }
    __syncthreads();  // stage b is free for the step after next
  }
  // epilogue: C -= hi + lo, the 32 outputs of a thread loaded together
  double cv[2][4][4];
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + frag_row(wm, mi) + g + ((r >> 1) << 3);
        const int col = n0 + frag_col(wn, ni) + 2 * tg + (r & 1);
        const bool in = row < M && col < N && !(lower && col > row);
        cv[mi][ni][r] = in ? C[(long long)row * ldc + col] : 0.0;
      }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + frag_row(wm, mi) + g + ((r >> 1) << 3);
        const int col = n0 + frag_col(wn, ni) + 2 * tg + (r & 1);
        if (row >= M || col >= N || (lower && col > row)) continue;
        const double v = exact_f64(hi[mi][ni][r]) + exact_f64(lo[mi][ni][r]);  // exact
        C[(long long)row * ldc + col] = cv[mi][ni][r] - v;
      }
}

// C -= op(A) op(B) over all tiles (lower tiles only with TG_LOWER).
__device__ void cta_gemm_sl(const SliceOp &A, const SliceOp &B, double *C, long long ldc, int M, int N, int K,
                            int flags, SmemS &ss) {
  for (int m0 = 0; m0 < M; m0 += TM)
    for (int n0 = 0; n0 < N; n0 += TM) {
      if ((flags & TG_LOWER) && n0 > m0 + TM - 1) break;
      tile_gemm_sl(A, B, C, ldc, M, N, K, flags, m0, n0, ss);
    }
  __syncthreads();
}

// ------------------------------------------------------------------ FP64 pieces
__device__ double cta_sum(double v, SmemF &sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
  __syncthreads();
  const double s = (sm.red[0] + sm.red[1]) + (sm.red[2] + sm.red[3]);
  __syncthreads();
  return s;
}

// Factor the nb x nb diagonal block at A (ld) into st.D, left-looking by
// columns: for column j every row i >= j forms a_ij - sum_k l_ik l_jk with the
// dot product split over tpr threads (the largest power of two <= 32 with
// (nb - j) tpr <= 128) and a fixed-order shuffle reduction, then every thread
// takes r = 1/sqrt(pivot) itself and the column is scaled by r.  L11 (upper
// part zeroed) is written back to A.  Returns false on a failing pivot, after
// recording it in info.
__device__ bool cta_potrf(int nb, double *A, long long lda, int *info, int offset, SmemF &sm, SmemT &st) {
  const int t = threadIdx.x;
  for (int idx = t; idx < nb * nb; idx += BT) {
    const int i = idx / nb, j = idx - i * nb;
    st.D[i][j] = (j <= i) ? A[(long long)i * lda + j] : 0.0;
  }
  __syncthreads();
  bool ok = true;
  for (int j = 0; j < nb; ++j) {
    const int R = nb - j;
    int tpr = 1;
    while (tpr < 32 && 2 * tpr * R <= BT) tpr *= 2;
    const int row = j + t / tpr, part = t & (tpr - 1);
    double s = 0.0;
    if (row < nb)
      for (int k = part; k < j; k += tpr) s = fma(st.D[row][k], st.D[j][k], s);
    for (int o = tpr >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (part == 0 && row < nb) sm.v[row] = st.D[row][j] - s;
    __syncthreads();
    const double p = sm.v[j];
    if (!(p > 0.0 && p <= 1.79769313486231570e308)) {
      if (t == 0 && info[1] == 0) {
        info[0] = offset + j;
        info[1] = (p != p || p > 1.79769313486231570e308) ? GPC_ERR_NAN : GPC_ERR_NOT_PD;
      }
      ok = false;
      break;
    }
    const double r = rsqrt_nr(p);
    if (t < R) st.D[j + t][j] = sm.v[j + t] * r;
    __syncthreads();
  }
  __syncthreads();
  for (int idx = t; idx < nb * nb; idx += BT) {
    const int r = idx / nb, c = idx - r * nb;
    A[(long long)r * lda + c] = (c <= r) ? st.D[r][c] : 0.0;
  }
  __syncthreads();
  return ok;
}

// Inverse of the lower nb x nb factor in st.D into st.X (lower), by forward
// substitution on the identity with right-looking updates: for j = 0, 1, ..
// row j of the inverse is finished (scaled by 1/l_jj) and then every later row
// i takes x_ic -= l_ij x_jc for c <= j; the (nb - 1 - j)(j + 1) updates of a
// step are dealt evenly to all threads.  The inverse is written, compact
// (ld nb), to Xg.
__device__ void cta_trtri(int nb, double *Xg, SmemF &sm, SmemT &st) {
  const int t = threadIdx.x;
  for (int idx = t; idx < nb * MAXB; idx += BT) st.X[idx / MAXB][idx % MAXB] = 0.0;
  if (t < nb) sm.w[t] = recip_nr(st.D[t][t]);
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const double rj = sm.w[j];
    for (int c = t; c <= j; c += BT) st.X[j][c] = (c == j) ? rj : st.X[j][c] * rj;
    __syncthreads();
    const int w = j + 1, E = (nb - 1 - j) * w;
    for (int e = t; e < E; e += BT) {
      const int i = j + 1 + e / w, c = e - (e / w) * w;
      st.X[i][c] = fma(-st.D[i][j], st.X[j][c], st.X[i][c]);
    }
    __syncthreads();
  }
  for (int idx = t; idx < nb * nb; idx += BT) {
    const int r = idx / nb, c = idx - r * nb;
    Xg[idx] = (c <= r) ? st.X[r][c] : 0.0;
  }
  __syncthreads();
}

// x <- L^{-1} x (trans 0) or L^{-T} x (trans 1) with the stored inverses of the
// nb x nb diagonal blocks (Dinv: block s at s nb^2, compact ld = its order):
// per block, x_blk = inv(L_ss) x_blk (or its transpose) as a small
// matrix-vector product (two threads per row), then the rest of x is updated
// right-looking: rows below the block (trans 0: x_i -= L_i,blk x_blk, one
// thread per row) or columns left of it (trans 1: x_c -= L_blk,c^T x_blk, one
// thread per column, coalesced).
__device__ void cta_trsv_inv(int n, const double *L, long long ldl, const double *Dinv, int nb, double *x, int trans,
                             SmemF &sm) {
  const int t = threadIdx.x, nblk = (n + nb - 1) / nb;
  for (int s2 = 0; s2 < nblk; ++s2) {
    const int s = trans ? nblk - 1 - s2 : s2;
    const int i0 = s * nb, bn = min(nb, n - i0);
    const double *Di = Dinv + (size_t)s * nb * nb;
    __syncthreads();
    if (t < bn) sm.v[t] = x[i0 + t];
    __syncthreads();
    {
      const int r = t >> 1, h = t & 1;
      double acc = 0.0;
      if (r < bn) {
        if (!trans)
          for (int c = h; c <= r; c += 2) acc = fma(Di[r * bn + c], sm.v[c], acc);
        else
          for (int c = r + h; c < bn; c += 2) acc = fma(Di[c * bn + r], sm.v[c], acc);
      }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (h == 0 && r < bn) {
        sm.w[r] = acc;
        x[i0 + r] = acc;
      }
    }
    __syncthreads();
    if (!trans) {
      for (int i = i0 + bn + t; i < n; i += BT) {
        const double *row = L + (long long)i * ldl + i0;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int c = 0;
        for (; c + 3 < bn; c += 4) {
          a0 = fma(row[c], sm.w[c], a0);
          a1 = fma(row[c + 1], sm.w[c + 1], a1);
          a2 = fma(row[c + 2], sm.w[c + 2], a2);
          a3 = fma(row[c + 3], sm.w[c + 3], a3);
        }
        for (; c < bn; ++c) a0 = fma(row[c], sm.w[c], a0);
        x[i] -= (a0 + a1) + (a2 + a3);
      }
    } else {
      for (int c = t; c < i0; c += BT) {
        const double *col = L + (long long)i0 * ldl + c;
        double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
        int r = 0;
        for (; r + 3 < bn; r += 4) {
          a0 = fma(col[(long long)r * ldl], sm.w[r], a0);
          a1 = fma(col[(long long)(r + 1) * ldl], sm.w[r + 1], a1);
          a2 = fma(col[(long long)(r + 2) * ldl], sm.w[r + 2], a2);
          a3 = fma(col[(long long)(r + 3) * ldl], sm.w[r + 3], a3);
        }
        for (; r < bn; ++r) a0 = fma(col[(long long)r * ldl], sm.w[r], a0);
        x[c] -= (a0 + a1) + (a2 + a3);
      }
    }
  }
  __syncthreads();
}

// Index of (i, j), j <= i, in packed lower storage.
__device__ __forceinline__ long long packed(int i, int j) { return (long long)i * (i + 1) / 2 + j; }

// r = y - K x for the symmetric K held packed (lower); returns |r|^2 (all
// threads).  Four partial sums per thread keep FP64 latency hidden.
__device__ double cta_residual(int n, const double *Kp, const double *y, const double *x, double *r, SmemF &sm) {
  double rr = 0.0;
  for (int i = threadIdx.x; i < n; i += BT) {
    const double *row = Kp + packed(i, 0);
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = 0;
    for (; j + 3 <= i; j += 4) {
      a0 = fma(row[j], x[j], a0);
      a1 = fma(row[j + 1], x[j + 1], a1);
      a2 = fma(row[j + 2], x[j + 2], a2);
      a3 = fma(row[j + 3], x[j + 3], a3);
    }
    for (; j <= i; ++j) a0 = fma(row[j], x[j], a0);
    for (j = i + 1; j + 3 < n; j += 4) {
      a0 = fma(Kp[packed(j, i)], x[j], a0);
      a1 = fma(Kp[packed(j + 1, i)], x[j + 1], a1);
      a2 = fma(Kp[packed(j + 2, i)], x[j + 2], a2);
      a3 = fma(Kp[packed(j + 3, i)], x[j + 3], a3);
    }
    for (; j < n; ++j) a0 = fma(Kp[packed(j, i)], x[j], a0);
    const double ri = y[i] - ((a0 + a1) + (a2 + a3));
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  return cta_sum(rr, sm);
}

// Workspace slot of one CTA (doubles): Kbar (nmax^2) | kernel values k_ij,
// packed lower (nmax (nmax + 1) / 2) | k_ij r_ij^2, packed the same way | z,
// alpha, r (3 nmax) | block inverses
// ((nmax + MAXB) MAXB) | M and T of the diagonal adjoint step (2 MAXB^2);
// the mixed path adds slice buffers (BF16): L^T (5 nmax kp), a row-split
// panel (5 nmax 64) and the adjoint's block column (5 64 kp), kp = nmax
// rounded up to the chunk.
__host__ __device__ inline long long slot_kp_offset(long long nmax) { return nmax * nmax; }
__host__ __device__ inline long long packed_elems(long long nmax) { return (nmax * (nmax + 1) / 2 + 1) / 2 * 2; }
__host__ __device__ inline long long slot_kr_offset(long long nmax) { return slot_kp_offset(nmax) + packed_elems(nmax); }
__host__ __device__ inline long long slot_vec_offset(long long nmax) { return slot_kr_offset(nmax) + packed_elems(nmax); }
__host__ __device__ inline long long slot_inv_offset(long long nmax) { return slot_vec_offset(nmax) + 3 * nmax; }
__host__ __device__ inline long long slot_mt_offset(long long nmax) {
  return slot_inv_offset(nmax) + (nmax + MAXB) * MAXB;
}
__host__ __device__ inline long long round32(long long v) { return (v + 31) / 32 * 32; }
__host__ __device__ inline long long slot_f64_elems(long long nmax) {
  return round32(slot_mt_offset(nmax) + 2 * MAXB * MAXB);
}
// slice buffers, in BF16 elements from the end of the FP64 part
__host__ __device__ inline long long sl_lt_plane(long long nmax) { return nmax * round32(nmax); }
__host__ __device__ inline long long sl_pan_offset(long long nmax) { return kSlices * sl_lt_plane(nmax); }
__host__ __device__ inline long long sl_pan_plane(long long nmax) { return nmax * 64; }
__host__ __device__ inline long long sl_bc_offset(long long nmax) {
  return sl_pan_offset(nmax) + kSlices * sl_pan_plane(nmax);
}
__host__ __device__ inline long long sl_bc_plane(long long nmax) { return 64 * round32(nmax); }
__host__ __device__ inline long long slot_elems(long long nmax, bool mixed) {
  const long long bf = sl_bc_offset(nmax) + kSlices * sl_bc_plane(nmax);
  return slot_f64_elems(nmax) + (mixed ? round32((bf + 3) / 4) : 0);
}

template <bool MIXED>
__global__ void __launch_bounds__(BT)
batched_gp_kernel(BatchParams p) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  SmemF &sm = *reinterpret_cast<SmemF *>(smem_raw);
  SmemT &st = *reinterpret_cast<SmemT *>(smem_raw + kRegionOffset);
  SmemS *ss = MIXED ? reinterpret_cast<SmemS *>(smem_raw + kRegionOffset) : nullptr;
  __shared__ int s_item;
  const int t = threadIdx.x;
  double *slot = p.slots + (size_t)blockIdx.x * p.slot_elems;
  const int nb = p.nb, nmax = p.nmax;
  double *Kb = slot;
  double *Kp = slot + slot_kp_offset(nmax);
  double *Kr = slot + slot_kr_offset(nmax);
  double *z = slot + slot_vec_offset(nmax);
  double *alpha = z + nmax;
  double *rv = alpha + nmax;
  double *Dinv = slot + slot_inv_offset(nmax);
  double *Mw = slot + slot_mt_offset(nmax);
  double *Tw = Mw + MAXB * MAXB;
  bf16 *sl = reinterpret_cast<bf16 *>(slot + slot_f64_elems(nmax));
  const int kpl = (int)round32(nmax);
  const SliceOp pan{sl + sl_pan_offset(nmax), sl_pan_plane(nmax), 64, 0};
  double(*tbuf)[33] = reinterpret_cast<double(*)[33]>(&sm.As[0][0]);  // split transpose buffer (FP64 tiles idle)
  static_assert(sizeof(SmemF::As) >= 32 * 33 * sizeof(double), "transpose buffer");
  for (;;) {
    if (t == 0) s_item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= p.batch) break;
    const int gi = p.order[item];
    const int n = p.n[gi];
    if (n < 1 || n > nmax) {  // rejected on the device: sizes travel in device memory
      if (t == 0) {
        p.info[2 * gi] = -1;
        p.info[2 * gi + 1] = GPC_ERR_INVALID_ARG;
      }
      __syncthreads();
      continue;
    }
    const int d = p.d;
    const double *Xg = p.X + p.rowX[gi] * d;
    const double *yg = p.y + p.rowX[gi];
    const double al = p.hyp[3 * gi], rho = p.hyp[3 * gi + 1], sig = p.hyp[3 * gi + 2];
    double *L = p.K + p.offK[gi];
    const long long ld = n;
    int *info = p.info + 2 * gi;
    const int nblk = (n + nb - 1) / nb;
    if (t == 0) {
      info[0] = -1;
      info[1] = GPC_OK;
    }
    // ---- covariance: L gets the lower triangle (zero upper), Kp the kernel
    // values and Kr the products k_ij r_ij^2 (both packed, for the gradient);
    // a warp per row, lanes along the row
    {
      const double a2 = al * al, inv2r2 = 1.0 / (2.0 * rho * rho), dg = a2 + sig * sig;
      const int warp = t >> 5, lane = t & 31;
      for (int i = warp; i < n; i += BT / 32) {
        const double *xi = Xg + (long long)i * d;
        double *Li = L + (long long)i * ld;
        double *Kpi = Kp + packed(i, 0);
        double *Kri = Kr + packed(i, 0);
        for (int j = lane; j <= i; j += 32) {
          double v = dg, kr = 0.0;
          if (j < i) {
            double r2 = 0.0;
            for (int q = 0; q < d; ++q) {
              const double df = xi[q] - Xg[(long long)j * d + q];
              r2 = fma(df, df, r2);
            }
            v = a2 * exp(-r2 * inv2r2);
            kr = v * r2;
          }
          Li[j] = v;
          Kpi[j] = v;
          Kri[j] = kr;
        }
        for (int j = i + 1 + lane; j < n; j += 32) Li[j] = 0.0;
      }
    }
    __syncthreads();
    // ---- blocked Cholesky; the inverse of each diagonal block is kept in Dinv
    bool ok = true;
    for (int s = 0; s < nblk && ok; ++s) {
      const int k0 = s * nb, bn = min(nb, n - k0), m = n - k0 - bn;
      double *A11 = L + (long long)k0 * ld + k0;
      double *Di = Dinv + (size_t)s * nb * nb;
      ok = cta_potrf(bn, A11, ld, info, k0, sm, st);
      if (!ok) break;
      cta_trtri(bn, Di, sm, st);
      if (m <= 0) continue;
      double *A21 = L + (long long)(k0 + bn) * ld + k0;
      // L21 = A21 L11^{-T} (FP64), then the trailing update A22 -= L21 L21^T
      cta_gemm<false, true>(A21, ld, Di, bn, A21, ld, m, bn, bn, 1.0, 0.0, TG_B_KLE, sm);
      if constexpr (MIXED) {
        split_rows_cta(A21, ld, m, bn, const_cast<bf16 *>(pan.S), pan.plane, pan.kpad);
        cta_gemm_sl(pan, pan, A21 + bn, ld, m, m, bn, TG_LOWER, *ss);
      } else {
        cta_gemm<false, true>(A21, ld, A21, ld, A21 + bn, ld, m, m, bn, -1.0, 1.0, TG_LOWER, sm);
      }
    }
    if (!ok) {
      if (t == 0) {
        p.value[gi] = __longlong_as_double(0x7ff8000000000000LL);
        p.grad3[3 * gi] = p.grad3[3 * gi + 1] = p.grad3[3 * gi + 2] = __longlong_as_double(0x7ff8000000000000LL);
      }
      __syncthreads();
      continue;
    }
    // ---- solves, log det, value
    for (int i = t; i < n; i += BT) z[i] = yg[i];
    __syncthreads();
    cta_trsv_inv(n, L, ld, Dinv, nb, z, 0, sm);
    for (int i = t; i < n; i += BT) alpha[i] = z[i];
    __syncthreads();
    cta_trsv_inv(n, L, ld, Dinv, nb, alpha, 1, sm);
    if constexpr (MIXED) {
      // FP64 refinement against the kept covariance until |r| <= 1e-14 |y| or
      // the residual stops halving (the FP64 floor); then z = L^T alpha
      double yy = 0.0;
      for (int i = t; i < n; i += BT) yy = fma(yg[i], yg[i], yy);
      yy = cta_sum(yy, sm);
      double prev = -1.0;
      for (int it = 0; it < 8; ++it) {
        const double rr = cta_residual(n, Kp, yg, alpha, rv, sm);
        if (rr <= 1e-28 * yy || (prev >= 0.0 && rr > 0.25 * prev)) break;
        prev = rr;
        cta_trsv_inv(n, L, ld, Dinv, nb, rv, 0, sm);
        cta_trsv_inv(n, L, ld, Dinv, nb, rv, 1, sm);
        for (int i = t; i < n; i += BT) alpha[i] += rv[i];
        __syncthreads();
      }
      for (int jc = t; jc < n; jc += BT) {
        double acc = 0.0;
        for (int i = jc; i < n; ++i) acc = fma(L[(long long)i * ld + jc], alpha[i], acc);
        z[jc] = acc;
      }
      __syncthreads();
    }
    double lsum = 0.0, q = 0.0;
    for (int i = t; i < n; i += BT) {
      lsum += log(L[(long long)i * ld + i]);
      q = fma(yg[i], alpha[i], q);
    }
    lsum = cta_sum(lsum, sm);
    q = cta_sum(q, sm);
    if (t == 0) p.value[gi] = -0.5 * q - lsum - 0.5 * (double)n * 1.8378770664093454835606594728112;
    // ---- upstream adjoint Lbar = tril(alpha z^T) - diag(1/L_ii)  (z = L^{-1} y)
    {
      const int warp = t >> 5, lane = t & 31;
      for (int i = warp; i < n; i += BT / 32) {
        const double ai = alpha[i];
        double *Kbi = Kb + (long long)i * ld;
        for (int j = lane; j < n; j += 32) {
          double v = 0.0;
          if (j <= i) {
            v = ai * z[j];
            if (i == j) v -= 1.0 / L[(long long)i * ld + i];
          }
          Kbi[j] = v;
        }
      }
    }
    __syncthreads();
    // ---- blocked adjoint sweep over the factorisation's blocks, last first
    const SliceOp lt{sl, sl_lt_plane(nmax), kpl, 0};  // operand row c = column c of L, K = rows of L
    const SliceOp bc{sl + sl_bc_offset(nmax), sl_bc_plane(nmax), kpl, 0};  // the block column [Dbar; Cbar]^T
    if constexpr (MIXED) {
      split_cols_cta(L, ld, n, n, const_cast<bf16 *>(lt.S), lt.plane, lt.kpad, 0, tbuf);
      __syncthreads();
    }
    for (int s = nblk - 1; s >= 0; --s) {
      const int j = s * nb, k = min(j + nb, n);
      const int bn = k - j, m = n - k;
      const double *D = L + (long long)j * ld + j;
      double *Dbar = Kb + (long long)j * ld + j;
      const double *Di = Dinv + (size_t)s * nb * nb;
      if (m > 0) {
        double *Cbar = Kb + (long long)k * ld + j;
        const double *C = L + (long long)k * ld + j;
        cta_gemm<false, false>(Cbar, ld, Di, bn, Cbar, ld, m, bn, bn, 1.0, 0.0, TG_B_KGE, sm);  // Cbar D^{-1}
        if constexpr (MIXED) {
          split_rows_cta(Cbar, ld, m, bn, const_cast<bf16 *>(pan.S), pan.plane, pan.kpad);
          split_cols_cta(Cbar, ld, m, bn, const_cast<bf16 *>(bc.S), bc.plane, bc.kpad, bn, tbuf);
          __syncthreads();
          if (j > 0)  // Bbar -= Cbar R
            cta_gemm_sl(pan, SliceOp{lt.S, lt.plane, lt.kpad, j}, Kb + (long long)k * ld, ld, m, j, bn, 0, *ss);
          // Dbar -= Cbar^T C (lower)
          cta_gemm_sl(SliceOp{bc.S, bc.plane, bc.kpad, bn}, SliceOp{lt.S + (long long)j * lt.kpad, lt.plane, lt.kpad, k},
                      Dbar, ld, bn, bn, m, TG_LOWER, *ss);
        } else {
          if (j > 0)  // Bbar -= Cbar R
            cta_gemm<false, false>(Cbar, ld, L + (long long)j * ld, ld, Kb + (long long)k * ld, ld, m, j, bn, -1.0,
                                   1.0, 0, sm);
          // Dbar -= Cbar^T C (lower)
          cta_gemm<true, false>(Cbar, ld, C, ld, Dbar, ld, bn, bn, m, -1.0, 1.0, TG_LOWER, sm);
        }
      }
      // Dbar <- D^{-T} sym(tril(D^T Dbar)) D^{-1}
      cta_gemm<true, false>(D, ld, Dbar, ld, Mw, bn, bn, bn, bn, 1.0, 0.0, TG_LOWER | TG_A_KGE | TG_B_KGE, sm);
      for (int idx = t; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        if (c > r) Mw[idx] = Mw[c * bn + r];
      }
      __syncthreads();
      cta_gemm<false, false>(Mw, bn, Di, bn, Tw, bn, bn, bn, bn, 1.0, 0.0, TG_B_KGE, sm);
      cta_gemm<true, false>(Di, bn, Tw, bn, Dbar, ld, bn, bn, bn, 1.0, 0.0, TG_LOWER | TG_A_KGE, sm);
      for (int idx = t; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        if (c > r) Dbar[(long long)r * ld + c] = Dbar[(long long)c * ld + r];
      }
      __syncthreads();
      if (j > 0) {  // Rbar -= [Dbar; Cbar]^T [R; B]
        if constexpr (MIXED) {
          split_cols_cta(Dbar, ld, bn, bn, const_cast<bf16 *>(bc.S), bc.plane, bc.kpad, 0, tbuf);
          __syncthreads();
          cta_gemm_sl(bc, SliceOp{lt.S, lt.plane, lt.kpad, j}, Kb + (long long)j * ld, ld, bn, j, n - j, 0, *ss);
        } else {
          cta_gemm<true, false>(Dbar, ld, L + (long long)j * ld, ld, Kb + (long long)j * ld, ld, bn, j, n - j,
                                -1.0, 1.0, 0, sm);
        }
      }
      for (int idx = t; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        double *q2 = Dbar + (long long)r * ld + c;
        if (c > r) *q2 = 0.0;
        else if (c == r) *q2 *= 0.5;
      }
      __syncthreads();
    }
    // ---- hyperparameter gradient from Kbar and the kept kernel values:
    // dk_ij/dalpha = 2 k_ij / alpha (k_ii without the noise), dk_ij/drho =
    // k_ij r_ij^2 / rho^3, dk_ii/dsigma = 2 sigma; the constant factors are
    // applied to the sums
    {
      const double a2 = al * al;
      double sk = 0.0, skr = 0.0, sd = 0.0;  // sum kb k (off-diagonal), sum kb k r^2, sum of the diagonal kb
      const int warp = t >> 5, lane = t & 31;
      for (int i = warp; i < n; i += BT / 32) {
        const double *Kbi = Kb + (long long)i * ld;
        const double *Kpi = Kp + packed(i, 0);
        const double *Kri = Kr + packed(i, 0);
        for (int j = lane; j <= i; j += 32) {
          const double kb = Kbi[j];
          if (j == i) {
            sd += kb;
          } else {
            sk = fma(kb, Kpi[j], sk);
            skr = fma(kb, Kri[j], skr);
          }
        }
      }
      sk = cta_sum(sk, sm);
      skr = cta_sum(skr, sm);
      sd = cta_sum(sd, sm);
      const double ga = 2.0 * (sk + sd * a2) / al;
      const double gr = skr / (rho * rho * rho);
      const double gs = 2.0 * sig * sd;
      if (t == 0) {
        p.grad3[3 * gi] = ga;
        p.grad3[3 * gi + 1] = gr;
        p.grad3[3 * gi + 2] = gs;
      }
    }
    __syncthreads();
  }
}

// Order of the GPs by size, largest first (ties by index): one CTA, rank by counting.
__global__ void order_kernel(int batch, const int *n, int *order) {
  for (int i = threadIdx.x; i < batch; i += blockDim.x) {
    const int ni = n[i];
    int rank = 0;
    for (int j = 0; j < batch; ++j) {
      const int nj = n[j];
      rank += (nj > ni) || (nj == ni && j < i);
    }
    order[rank] = i;
  }
}

}  // namespace

size_t batched_workspace_bytes(int batch, int nmax, bool mixed) {
  const size_t slot = (size_t)slot_elems(nmax, mixed);
  return align_up((size_t)sm_count() * slot * sizeof(double), 256) + align_up((size_t)batch * sizeof(int), 256) + 256;
}

cudaError_t batched_gp_lml_grad(int batch, const int *n, const long long *offK, const long long *rowX, int d,
                                const double *X, const double *y, const double *hyp, double *K, double *value,
                                double *grad3, int *info, int nmax, bool mixed, void *ws, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const int nb = std::min(std::max(tuning().batch_block, 16), MAXB);
  const size_t slot = (size_t)slot_elems(nmax, mixed);
  char *p = (char *)ws;
  double *slots = (double *)p;
  p += align_up((size_t)sm_count() * slot * sizeof(double), 256);
  int *order = (int *)p;
  p += align_up((size_t)batch * sizeof(int), 256);
  int *queue = (int *)p;
  cudaError_t e = cudaMemsetAsync(queue, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * batch, s, order_kernel<<<1, 256, 0, s>>>(batch, n, order));
  BatchParams bp;
  bp.batch = batch;
  bp.d = d;
  bp.nb = nb;
  bp.nmax = nmax;
  bp.n = n;
  bp.offK = offK;
  bp.rowX = rowX;
  bp.X = X;
  bp.y = y;
  bp.hyp = hyp;
  bp.K = K;
  bp.slots = slots;
  bp.slot_elems = (long long)slot;
  bp.order = order;
  bp.queue = queue;
  bp.value = value;
  bp.grad3 = grad3;
  bp.info = info;
  // one CTA per SM: the slots cover that many
  const int grid = sm_count();
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    e = cudaFuncSetAttribute(batched_gp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemF64);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batched_gp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)kSmemMixed);
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (mixed)
    GPC_LAUNCH(GPC_TRACE_GEMM_MIXED, 0.0, 0.0, s, batched_gp_kernel<true><<<grid, BT, kSmemMixed, s>>>(bp));
  else
    GPC_LAUNCH(GPC_TRACE_GEMM_F64, 0.0, 0.0, s, batched_gp_kernel<false><<<grid, BT, kSmemF64, s>>>(bp));
  return cudaGetLastError();
}

}  // namespace gpc
