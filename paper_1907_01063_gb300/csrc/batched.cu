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
// own thread block.  On this part one SM's FP64 rate bounds a GP's time, so a
// GP is not spread over SMs: with the queue in LPT order the makespan is close
// to total work / SMs unless a single GP dominates.
//
// Products inside a CTA are 64 x 64 output tiles on the FP64 tensor path
// (mma.sync m16n8k16 .f64), operands staged through shared memory; the
// diagonal block is factored and inverted in shared memory; panels are solved
// by row-parallel substitution.  Block size b (32 or 64) is a tuning knob.
// Each GP's factor overwrites its covariance in the caller's Kws; Kbar and the
// vectors live in a per-CTA slot of the workspace and are reused GP to GP.
#include "common.cuh"
#include "slices.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace gpc {
namespace {

constexpr int BT = 128;                    // threads per CTA (4 warps)
constexpr int TM = 64, TK = 16, TP = 4;    // product tile and K step
constexpr int MAXB = 64;                   // largest block size

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

constexpr int XK = 32;          // K step of the mixed product (one scale per row and step)
constexpr int XLD = XK + 8;     // padded row of a BF16 slice tile (conflict-free fragment loads)

struct Smem {
  double As[TM][TK + TP];
  double Bs[TM][TK + TP];
  double D[MAXB][MAXB + 1];  // diagonal block / inverse / solve block
  double v[MAXB];
  double red[8];
  int flag;
};

// Extra shared memory of the mixed products: the FP64 operand tiles of one
// 32-wide K step and their BF16 slices.
constexpr size_t kSmemXOffset = (sizeof(Smem) + 127) / 128 * 128;
struct SmemX {
  double Ax[TM][XK + 1];
  double Bx[TM][XK + 1];
  __nv_bfloat16 As[kSlices][TM][XLD];
  __nv_bfloat16 Bs[kSlices][TM][XLD];
};

__device__ __forceinline__ void dmma(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
        "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// One 64 x 64 output tile of C = beta C + alpha op(A) op(B) over K, rows
// [m0, m0+64) and cols [n0, n0+64) clipped to M x N; lower: only col <= row.
// op(A)(m, k) = TA ? A[k lda + m] : A[m lda + k];  op(B)(k, n) = TB ? B[n ldb + k] : B[k ldb + n].
template <bool TA, bool TB>
__device__ void tile_gemm(const double *A, long long lda, const double *B, long long ldb, double *C,
                          long long ldc, int M, int N, int K, double alpha, double beta, bool lower, int m0,
                          int n0, Smem &sm) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
  double acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0;
  for (int k0 = 0; k0 < K; k0 += TK) {
    __syncthreads();
    if (!TA) {
      const int r = t >> 1, c0 = (t & 1) * 8, m = m0 + r;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + c0 + i;
        sm.As[r][c0 + i] = (m < M && k < K) ? A[(long long)m * lda + k] : 0.0;
      }
    } else {
      const int kk = t >> 3, mm0 = (t & 7) * 8, k = k0 + kk;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int m = m0 + mm0 + i;
        sm.As[mm0 + i][kk] = (m < M && k < K) ? A[(long long)k * lda + m] : 0.0;
      }
    }
    if (!TB) {
      const int kk = t >> 3, nn0 = (t & 7) * 8, k = k0 + kk;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int n = n0 + nn0 + i;
        sm.Bs[nn0 + i][kk] = (n < N && k < K) ? B[(long long)k * ldb + n] : 0.0;
      }
    } else {
      const int r = t >> 1, c0 = (t & 1) * 8, n = n0 + r;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + c0 + i;
        sm.Bs[r][c0 + i] = (n < N && k < K) ? B[(long long)n * ldb + k] : 0.0;
      }
    }
    __syncthreads();
    double a[2][8], b[4][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
      const int r = wm * 32 + mi * 16 + g;
#pragma unroll
      for (int i = 0; i < 8; ++i) a[mi][i] = sm.As[r + 8 * (i & 1)][tg + 4 * (i >> 1)];
    }
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int c = wn * 32 + ni * 8 + g;
#pragma unroll
      for (int i = 0; i < 4; ++i) b[ni][i] = sm.Bs[c][tg + 4 * i];
    }
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) dmma(acc[mi][ni], a[mi], b[ni]);
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * 32 + mi * 16 + g + ((r >> 1) << 3);
        const int col = n0 + wn * 32 + ni * 8 + 2 * tg + (r & 1);
        if (row >= M || col >= N || (lower && col > row)) continue;
        double *dst = C + (long long)row * ldc + col;
        const double v = alpha * acc[mi][ni][r];
        *dst = (beta == 0.0) ? v : fma(beta, *dst, v);
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

// The mixed tile product: the same contract as tile_gemm, with the products
// of each 32-wide K step taken as split-BF16 slices (slices.cuh; one scale per
// operand row and step) on the warp-level BF16 tensor instruction with FP32
// accumulation.  Per 16-wide K sub-step and 16 x 8 fragment the 15 slice
// products with p + q <= 6 go to four FP32 groups (p + q = 2, 3, 4 exact:
// integer sums below 2^21 in units of their scale; 5-6 rounded), which are
// added into a double-float accumulator; the tile is converted to FP64 once,
// when it is written.  No FP64 arithmetic is in the K loop.
template <bool TA, bool TB>
__device__ __noinline__ void tile_gemm_mixed(const double *A, long long lda, const double *B, long long ldb, double *C,
                                long long ldc, int M, int N, int K, double alpha, double beta, bool lower, int m0,
                                int n0, SmemX &sx) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int wm = warp >> 1, wn = warp & 1, g = lane >> 2, tg = lane & 3;
  float hi[2][4][4], lo[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) hi[i][j][r] = lo[i][j][r] = 0.0f;
  for (int k0 = 0; k0 < K; k0 += XK) {
    __syncthreads();
    // FP64 operand tiles, row-major [m][k] and [n][k]
    for (int idx = t; idx < TM * XK; idx += BT) {
      int r, k;
      if (!TA) { r = idx / XK; k = idx - r * XK; } else { k = idx / TM; r = idx - k * TM; }
      const int m = m0 + r, kk = k0 + k;
      sx.Ax[r][k] = (m < M && kk < K) ? (TA ? A[(long long)kk * lda + m] : A[(long long)m * lda + kk]) : 0.0;
    }
    for (int idx = t; idx < TM * XK; idx += BT) {
      int r, k;
      if (TB) { r = idx / XK; k = idx - r * XK; } else { k = idx / TM; r = idx - k * TM; }
      const int nn = n0 + r, kk = k0 + k;
      sx.Bx[r][k] = (nn < N && kk < K) ? (TB ? B[(long long)nn * ldb + kk] : B[(long long)kk * ldb + nn]) : 0.0;
    }
    __syncthreads();
    // slices: thread (row, half) splits 16 values of a row; the pair shares the row's exponent
    {
      const int r = t >> 1, h = t & 1;
#pragma unroll
      for (int op = 0; op < 2; ++op) {
        const double *src = op == 0 ? &sx.Ax[r][16 * h] : &sx.Bx[r][16 * h];
        int ex = 0;
#pragma unroll
        for (int i = 0; i < 16; ++i)
          ex = max(ex, slice_exponent((unsigned long long)__double_as_longlong(src[i])));
        ex = max(ex, __shfl_xor_sync(0xffffffffu, ex, 1));
        __nv_bfloat16(*dst)[TM][XLD] = op == 0 ? sx.As : sx.Bs;
#pragma unroll 4
        for (int i = 0; i < 16; ++i) {
          float v[kSlices];
          split_value((unsigned long long)__double_as_longlong(src[i]), ex, v);
#pragma unroll
          for (int pp = 0; pp < kSlices; ++pp) dst[pp][r][16 * h + i] = __float2bfloat16_rn(v[pp]);
        }
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < XK; kk += 16) {
#pragma unroll
      for (int mi = 0; mi < 2; ++mi) {
        const int ra = wm * 32 + mi * 16 + g;
        uint32_t a[kSlices][4];
#pragma unroll
        for (int pp = 0; pp < kSlices; ++pp) {
          a[pp][0] = *(const uint32_t *)&sx.As[pp][ra][kk + 2 * tg];
          a[pp][1] = *(const uint32_t *)&sx.As[pp][ra + 8][kk + 2 * tg];
          a[pp][2] = *(const uint32_t *)&sx.As[pp][ra][kk + 2 * tg + 8];
          a[pp][3] = *(const uint32_t *)&sx.As[pp][ra + 8][kk + 2 * tg + 8];
        }
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) {
          const int cb = wn * 32 + ni * 8 + g;
          uint32_t b[kSlices][2];
#pragma unroll
          for (int pp = 0; pp < kSlices; ++pp) {
            b[pp][0] = *(const uint32_t *)&sx.Bs[pp][cb][kk + 2 * tg];
            b[pp][1] = *(const uint32_t *)&sx.Bs[pp][cb][kk + 2 * tg + 8];
          }
          float gr[4][4];
#pragma unroll
          for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int r = 0; r < 4; ++r) gr[q][r] = 0.0f;
          // slice pairs (p, q), 0-based, p + q <= 4: group min(p + q, 3)
#pragma unroll
          for (int pp = 0; pp < kSlices; ++pp)
#pragma unroll
            for (int qq = 0; qq < kSlices; ++qq)
              if (pp + qq <= 4) hmma_bf16(gr[pp + qq < 3 ? pp + qq : 3], a[pp], b[qq]);
#pragma unroll
          for (int r = 0; r < 4; ++r) df_acc4(hi[mi][ni][r], lo[mi][ni][r], gr[0][r], gr[1][r], gr[2][r], gr[3][r]);
        }
      }
    }
  }
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * 32 + mi * 16 + g + ((r >> 1) << 3);
        const int col = n0 + wn * 32 + ni * 8 + 2 * tg + (r & 1);
        if (row >= M || col >= N || (lower && col > row)) continue;
        double *dst = C + (long long)row * ldc + col;
        const double v = alpha * ((double)hi[mi][ni][r] + (double)lo[mi][ni][r]);
        *dst = (beta == 0.0) ? v : fma(beta, *dst, v);
      }
  __syncthreads();
}

template <bool TA, bool TB>
__device__ void cta_gemm(const double *A, long long lda, const double *B, long long ldb, double *C, long long ldc,
                         int M, int N, int K, double alpha, double beta, bool lower, Smem &sm) {
  for (int m0 = 0; m0 < M; m0 += TM)
    for (int n0 = 0; n0 < N; n0 += TM) {
      if (lower && n0 > m0 + TM - 1) break;
      tile_gemm<TA, TB>(A, lda, B, ldb, C, ldc, M, N, K, alpha, beta, lower, m0, n0, sm);
    }
}

// The O(n^3) products of a GP: split-BF16 tensor products when MIXED.
template <bool MIXED, bool TA, bool TB>
__device__ void cta_gemm_big(const double *A, long long lda, const double *B, long long ldb, double *C,
                             long long ldc, int M, int N, int K, double alpha, double beta, bool lower, Smem &sm,
                             SmemX *sx) {
  if constexpr (!MIXED) {
    cta_gemm<TA, TB>(A, lda, B, ldb, C, ldc, M, N, K, alpha, beta, lower, sm);
  } else {
    for (int m0 = 0; m0 < M; m0 += TM)
      for (int n0 = 0; n0 < N; n0 += TM) {
        if (lower && n0 > m0 + TM - 1) break;
        tile_gemm_mixed<TA, TB>(A, lda, B, ldb, C, ldc, M, N, K, alpha, beta, lower, m0, n0, *sx);
      }
  }
}

__device__ double cta_sum(double v, Smem &sm) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sm.red[threadIdx.x >> 5] = v;
  __syncthreads();
  const double s = (sm.red[0] + sm.red[1]) + (sm.red[2] + sm.red[3]);
  __syncthreads();
  return s;
}

// Factor the nb x nb diagonal block at A (ld) in shared memory, left-looking by
// columns; write L11 back (upper part zeroed).  Returns false on a failing pivot.
__device__ bool cta_potrf(int nb, double *A, long long lda, int *info, int offset, Smem &sm) {
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int i = idx / nb, j = idx - i * nb;
    sm.D[i][j] = (j <= i) ? A[(long long)i * lda + j] : 0.0;
  }
  if (threadIdx.x == 0) sm.flag = 0;
  __syncthreads();
  const int i = threadIdx.x >> 1, h = threadIdx.x & 1;
  for (int j = 0; j < nb; ++j) {
    double s = 0.0;
    if (i >= j && i < nb)
      for (int k = h; k < j; k += 2) s = fma(sm.D[i][k], sm.D[j][k], s);
    s += __shfl_xor_sync(0xffffffffu, s, 1);
    if (h == 0 && i >= j && i < nb) sm.v[i] = sm.D[i][j] - s;
    __syncthreads();
    if (threadIdx.x == 0) {
      const double p = sm.v[j];
      if (p > 0.0 && p <= 1.79769313486231570e308) {
        sm.D[j][j] = sqrt(p);
      } else {
        sm.flag = 1;
        if (info[1] == 0) {
          info[0] = offset + j;
          info[1] = (p != p || p > 1.79769313486231570e308) ? GPC_ERR_NAN : GPC_ERR_NOT_PD;
        }
      }
    }
    __syncthreads();
    if (sm.flag) break;
    if (h == 0 && i > j && i < nb) sm.D[i][j] = sm.v[i] / sm.D[j][j];
    __syncthreads();
  }
  const bool ok = !sm.flag;
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int r = idx / nb, c = idx - r * nb;
    A[(long long)r * lda + c] = (c <= r) ? sm.D[r][c] : 0.0;
  }
  __syncthreads();
  return ok;
}

// Inverse of the lower nb x nb block T (global) into sm.D (lower), by the
// backward column sweep L^{-1} = [[1/l, 0], [-L2^{-1} x / l, L2^{-1}]].
__device__ void cta_trtri(int nb, const double *T, long long ldt, Smem &sm) {
  for (int idx = threadIdx.x; idx < nb * nb; idx += BT) {
    const int i = idx / nb, j = idx - i * nb;
    sm.D[i][j] = (j <= i) ? T[(long long)i * ldt + j] : 0.0;
  }
  __syncthreads();
  for (int j = nb - 1; j >= 0; --j) {
    const double ljj = sm.D[j][j];
    for (int i = j + 1 + threadIdx.x; i < nb; i += BT) {
      double s = 0.0;
      for (int k = j + 1; k <= i; ++k) s = fma(sm.D[i][k], sm.D[k][j], s);
      sm.v[i] = -s / ljj;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += BT) sm.D[i][j] = sm.v[i];
    if (threadIdx.x == 0) sm.D[j][j] = 1.0 / ljj;
    __syncthreads();
  }
}

// Row-parallel panel solve against the lower nb x nb block T (global):
// mode 0: X <- X T^{-T};  mode 1: X <- X T^{-1}.  32 rows at a time through sm.D.
__device__ void cta_trsm(int m, int nb, double *X, long long ldx, const double *T, long long ldt, int mode,
                         Smem &sm) {
  for (int j = threadIdx.x; j < nb; j += BT) sm.v[j] = 1.0 / T[(long long)j * ldt + j];
  for (int r0 = 0; r0 < m; r0 += 32) {
    const int rows = min(32, m - r0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < 32 * nb; idx += BT) {
      const int r = idx / nb, c = idx - r * nb;
      sm.D[r][c] = (r < rows) ? X[(long long)(r0 + r) * ldx + c] : 0.0;
    }
    __syncthreads();
    const int r = threadIdx.x & 31, cg = threadIdx.x >> 5;
    for (int step = 0; step < nb; ++step) {
      const int j = mode == 0 ? step : nb - 1 - step;
      if (threadIdx.x < 32) sm.D[r][j] *= sm.v[j];
      __syncthreads();
      const double xj = sm.D[r][j];
      if (mode == 0) {
        for (int k = j + 1 + cg; k < nb; k += 4) sm.D[r][k] = fma(-xj, T[(long long)k * ldt + j], sm.D[r][k]);
      } else {
        for (int k = cg; k < j; k += 4) sm.D[r][k] = fma(-xj, T[(long long)j * ldt + k], sm.D[r][k]);
      }
      __syncthreads();
    }
    for (int idx = threadIdx.x; idx < 32 * nb; idx += BT) {
      const int rr = idx / nb, c = idx - rr * nb;
      if (rr < rows) X[(long long)(r0 + rr) * ldx + c] = sm.D[rr][c];
    }
  }
  __syncthreads();
}

// x <- L^{-1} x (trans 0) or L^{-T} x (trans 1), blocked by nb with
// substitution inside each diagonal block.
__device__ void cta_trsv(int n, const double *L, long long ldl, double *x, int trans, int nb, Smem &sm) {
  const int nblk = (n + nb - 1) / nb;
  for (int s = 0; s < nblk; ++s) {
    const int blk = trans ? nblk - 1 - s : s;
    const int i0 = blk * nb, bn = min(nb, n - i0);
    __syncthreads();
    // rhs of the block: x_I - (off-diagonal part) with the finished entries
    for (int r = threadIdx.x; r < bn; r += BT) {
      double acc = 0.0;
      if (!trans) {
        const double *row = L + (long long)(i0 + r) * ldl;
        for (int k = 0; k < i0; ++k) acc = fma(row[k], x[k], acc);
      } else {
        for (int k = i0 + bn; k < n; ++k) acc = fma(L[(long long)k * ldl + i0 + r], x[k], acc);
      }
      sm.v[r] = x[i0 + r] - acc;
    }
    __syncthreads();
    if (!trans) {
      for (int j = 0; j < bn; ++j) {
        if (threadIdx.x == 0) sm.v[j] /= L[(long long)(i0 + j) * ldl + i0 + j];
        __syncthreads();
        for (int r = j + 1 + threadIdx.x; r < bn; r += BT)
          sm.v[r] = fma(-L[(long long)(i0 + r) * ldl + i0 + j], sm.v[j], sm.v[r]);
        __syncthreads();
      }
    } else {
      for (int j = bn - 1; j >= 0; --j) {
        if (threadIdx.x == 0) sm.v[j] /= L[(long long)(i0 + j) * ldl + i0 + j];
        __syncthreads();
        for (int r = threadIdx.x; r < j; r += BT) sm.v[r] = fma(-L[(long long)(i0 + j) * ldl + i0 + r], sm.v[j], sm.v[r]);
        __syncthreads();
      }
    }
    for (int r = threadIdx.x; r < bn; r += BT) x[i0 + r] = sm.v[r];
  }
  __syncthreads();
}

// r = y - K x for the symmetric K held in its lower triangle (ld n); returns
// |r|^2 (all threads).  Four partial sums per thread keep FP64 latency hidden.
__device__ double cta_residual(int n, const double *Kc, const double *y, const double *x, double *r, Smem &sm) {
  double rr = 0.0;
  for (int i = threadIdx.x; i < n; i += BT) {
    const double *row = Kc + (long long)i * n;
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
      a0 = fma(Kc[(long long)j * n + i], x[j], a0);
      a1 = fma(Kc[(long long)(j + 1) * n + i], x[j + 1], a1);
      a2 = fma(Kc[(long long)(j + 2) * n + i], x[j + 2], a2);
      a3 = fma(Kc[(long long)(j + 3) * n + i], x[j + 3], a3);
    }
    for (; j < n; ++j) a0 = fma(Kc[(long long)j * n + i], x[j], a0);
    const double ri = y[i] - ((a0 + a1) + (a2 + a3));
    r[i] = ri;
    rr = fma(ri, ri, rr);
  }
  return cta_sum(rr, sm);
}

template <bool MIXED>
__global__ void __launch_bounds__(BT)
batched_gp_kernel(BatchParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  Smem &sm = *reinterpret_cast<Smem *>(smem_raw);
  SmemX *sx = MIXED ? reinterpret_cast<SmemX *>(smem_raw + kSmemXOffset) : nullptr;
  __shared__ int s_item;
  double *slot = p.slots + (size_t)blockIdx.x * p.slot_elems;
  const int nb = p.nb;
  for (;;) {
    if (threadIdx.x == 0) s_item = atomicAdd(p.queue, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= p.batch) break;
    const int gi = p.order[item];
    const int n = p.n[gi];
    if (n < 1 || n > p.nmax) {  // rejected on the device: sizes travel in device memory
      if (threadIdx.x == 0) {
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
    double *Kb = slot;
    double *z = slot + (size_t)p.nmax * p.nmax;
    double *alpha = z + p.nmax;
    double *Mw = alpha + p.nmax;         // MAXB^2: sym(tril(D^T Dbar))
    double *Tw = Mw + MAXB * MAXB;       // MAXB^2: M D^{-1}
    double *Dinv = Tw + MAXB * MAXB;     // MAXB^2
    double *Kc = Dinv + MAXB * MAXB;     // mixed: the covariance kept for refinement (nmax^2)
    double *rv = Kc + (size_t)p.nmax * p.nmax;  // mixed: residual / correction (nmax)
    if (threadIdx.x == 0) {
      info[0] = -1;
      info[1] = GPC_OK;
    }
    // ---- covariance (lower triangle, ld = n)
    {
      const double a2 = al * al, inv2r2 = 1.0 / (2.0 * rho * rho), dg = a2 + sig * sig;
      const long long tot = (long long)n * n;
      for (long long idx = threadIdx.x; idx < tot; idx += BT) {
        const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
        double v = 0.0;
        if (j < i) {
          double r2 = 0.0;
          for (int t = 0; t < d; ++t) {
            const double df = Xg[(long long)i * d + t] - Xg[(long long)j * d + t];
            r2 = fma(df, df, r2);
          }
          v = a2 * exp(-r2 * inv2r2);
        } else if (j == i) {
          v = dg;
        }
        L[idx] = v;
        if (MIXED) Kc[idx] = v;
      }
    }
    __syncthreads();
    // ---- blocked Cholesky
    bool ok = true;
    for (int k0 = 0; k0 < n && ok; k0 += nb) {
      const int bn = min(nb, n - k0), m = n - k0 - bn;
      double *A11 = L + (long long)k0 * ld + k0;
      ok = cta_potrf(bn, A11, ld, info, k0, sm);
      if (!ok || m <= 0) continue;
      double *A21 = L + (long long)(k0 + bn) * ld + k0;
      cta_trsm(m, bn, A21, ld, A11, ld, 0, sm);
      cta_gemm_big<MIXED, false, true>(A21, ld, A21, ld, A21 + bn, ld, m, m, bn, -1.0, 1.0, true, sm, sx);
    }
    if (!ok) {
      if (threadIdx.x == 0) {
        p.value[gi] = __longlong_as_double(0x7ff8000000000000LL);
        p.grad3[3 * gi] = p.grad3[3 * gi + 1] = p.grad3[3 * gi + 2] = __longlong_as_double(0x7ff8000000000000LL);
      }
      __syncthreads();
      continue;
    }
    // ---- solves, log det, value
    for (int i = threadIdx.x; i < n; i += BT) z[i] = yg[i];
    __syncthreads();
    cta_trsv(n, L, ld, z, 0, nb, sm);
    for (int i = threadIdx.x; i < n; i += BT) alpha[i] = z[i];
    __syncthreads();
    cta_trsv(n, L, ld, alpha, 1, nb, sm);
    if constexpr (MIXED) {
      // FP64 refinement against the kept covariance until |r| <= 1e-14 |y| or
      // the residual stops halving (the FP64 floor); then z = L^T alpha
      double yy = 0.0;
      for (int i = threadIdx.x; i < n; i += BT) yy = fma(yg[i], yg[i], yy);
      yy = cta_sum(yy, sm);
      double prev = -1.0;
      for (int it = 0; it < 8; ++it) {
        const double rr = cta_residual(n, Kc, yg, alpha, rv, sm);
        if (rr <= 1e-28 * yy || (prev >= 0.0 && rr > 0.25 * prev)) break;
        prev = rr;
        cta_trsv(n, L, ld, rv, 0, nb, sm);
        cta_trsv(n, L, ld, rv, 1, nb, sm);
        for (int i = threadIdx.x; i < n; i += BT) alpha[i] += rv[i];
        __syncthreads();
      }
      for (int jc = threadIdx.x; jc < n; jc += BT) {
        double acc = 0.0;
        for (int i = jc; i < n; ++i) acc = fma(L[(long long)i * ld + jc], alpha[i], acc);
        z[jc] = acc;
      }
      __syncthreads();
    }
    double lsum = 0.0, q = 0.0;
    for (int i = threadIdx.x; i < n; i += BT) {
      lsum += log(L[(long long)i * ld + i]);
      q = fma(yg[i], alpha[i], q);
    }
    lsum = cta_sum(lsum, sm);
    q = cta_sum(q, sm);
    if (threadIdx.x == 0) p.value[gi] = -0.5 * q - lsum - 0.5 * (double)n * 1.8378770664093454835606594728112;
    // ---- upstream adjoint Lbar = tril(alpha z^T) - diag(1/L_ii)  (z = L^{-1} y)
    for (long long idx = threadIdx.x; idx < (long long)n * n; idx += BT) {
      const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
      double v = 0.0;
      if (j <= i) {
        v = alpha[i] * z[j];
        if (i == j) v -= 1.0 / L[(long long)i * ld + i];
      }
      Kb[idx] = v;
    }
    __syncthreads();
    // ---- blocked adjoint sweep (blocks counted from the bottom)
    const int nblk = (n + nb - 1) / nb, first = n - (nblk - 1) * nb;
    for (int ib = nblk - 1; ib >= 0; --ib) {
      const int j = (ib == 0) ? 0 : first + (ib - 1) * nb;
      const int k = first + ib * nb;
      const int bn = k - j, m = n - k;
      const double *D = L + (long long)j * ld + j;
      double *Dbar = Kb + (long long)j * ld + j;
      cta_trtri(bn, D, ld, sm);
      for (int idx = threadIdx.x; idx < bn * bn; idx += BT) Dinv[idx] = sm.D[idx / bn][idx % bn];
      __syncthreads();
      if (m > 0) {
        double *Cbar = Kb + (long long)k * ld + j;
        const double *C = L + (long long)k * ld + j;
        cta_trsm(m, bn, Cbar, ld, D, ld, 1, sm);
        if (j > 0)
          cta_gemm_big<MIXED, false, false>(Cbar, ld, L + (long long)j * ld, ld, Kb + (long long)k * ld, ld, m, j,
                                            bn, -1.0, 1.0, false, sm, sx);
        cta_gemm_big<MIXED, true, false>(Cbar, ld, C, ld, Dbar, ld, bn, bn, m, -1.0, 1.0, true, sm, sx);
      }
      // Dbar <- D^{-T} sym(tril(D^T Dbar)) D^{-1}
      cta_gemm<true, false>(D, ld, Dbar, ld, Mw, bn, bn, bn, bn, 1.0, 0.0, true, sm);
      for (int idx = threadIdx.x; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        if (c > r) Mw[idx] = Mw[c * bn + r];
      }
      __syncthreads();
      cta_gemm<false, false>(Mw, bn, Dinv, bn, Tw, bn, bn, bn, bn, 1.0, 0.0, false, sm);
      cta_gemm<true, false>(Dinv, bn, Tw, bn, Dbar, ld, bn, bn, bn, 1.0, 0.0, true, sm);
      for (int idx = threadIdx.x; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        if (c > r) Dbar[(long long)r * ld + c] = Dbar[(long long)c * ld + r];
      }
      __syncthreads();
      if (j > 0)
        cta_gemm_big<MIXED, true, false>(Dbar, ld, L + (long long)j * ld, ld, Kb + (long long)j * ld, ld, bn, j,
                                         n - j, -1.0, 1.0, false, sm, sx);
      for (int idx = threadIdx.x; idx < bn * bn; idx += BT) {
        const int r = idx / bn, c = idx - r * bn;
        double *q2 = Dbar + (long long)r * ld + c;
        if (c > r) *q2 = 0.0;
        else if (c == r) *q2 *= 0.5;
      }
      __syncthreads();
    }
    // ---- hyperparameter gradient from Kbar
    {
      const double a2 = al * al, inv2r2 = 1.0 / (2.0 * rho * rho), ir3 = 1.0 / (rho * rho * rho);
      double ga = 0.0, gr = 0.0, gs = 0.0;
      const long long tot = (long long)n * n;
      for (long long idx = threadIdx.x; idx < tot; idx += BT) {
        const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
        if (j > i) continue;
        double r2 = 0.0;
        for (int t = 0; t < d; ++t) {
          const double df = Xg[(long long)i * d + t] - Xg[(long long)j * d + t];
          r2 = fma(df, df, r2);
        }
        const double kf = a2 * exp(-r2 * inv2r2);
        const double kb = Kb[idx];
        ga = fma(kb, 2.0 * kf / al, ga);
        gr = fma(kb, kf * r2 * ir3, gr);
        if (i == j) gs = fma(kb, 2.0 * sig, gs);
      }
      ga = cta_sum(ga, sm);
      gr = cta_sum(gr, sm);
      gs = cta_sum(gs, sm);
      if (threadIdx.x == 0) {
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

size_t batch_slot_elems(int nmax, bool mixed) {
  const size_t base = (size_t)nmax * nmax + 2 * (size_t)nmax + 3 * MAXB * MAXB;
  return mixed ? base + (size_t)nmax * nmax + nmax : base;
}
size_t batched_smem_bytes(bool mixed) {
  return mixed ? kSmemXOffset + sizeof(SmemX) : sizeof(Smem);
}

}  // namespace

size_t batched_workspace_bytes(int batch, int nmax, bool mixed) {
  const size_t slot = batch_slot_elems(nmax, mixed);
  return align_up((size_t)sm_count() * slot * sizeof(double), 256) + align_up((size_t)batch * sizeof(int), 256) + 256;
}

cudaError_t batched_gp_lml_grad(int batch, const int *n, const long long *offK, const long long *rowX, int d,
                                const double *X, const double *y, const double *hyp, double *K, double *value,
                                double *grad3, int *info, int nmax, bool mixed, void *ws, cudaStream_t s) {
  if (batch <= 0) return cudaSuccess;
  const int nb = std::min(std::max(tuning().batch_block, 16), MAXB);
  const int ctas = sm_count() * std::max(1, tuning().batch_ctas_per_sm);
  const size_t slot = batch_slot_elems(nmax, mixed);
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
  // the slots cover one CTA per SM; more CTAs than that would share slots
  const int grid = std::min(ctas, sm_count());
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    e = cudaFuncSetAttribute(batched_gp_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)batched_smem_bytes(false));
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(batched_gp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)batched_smem_bytes(true));
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (mixed)
    GPC_LAUNCH(GPC_TRACE_GEMM_MIXED, 0.0, 0.0, s,
               batched_gp_kernel<true><<<grid, BT, batched_smem_bytes(true), s>>>(bp));
  else
    GPC_LAUNCH(GPC_TRACE_GEMM_F64, 0.0, 0.0, s,
               batched_gp_kernel<false><<<grid, BT, batched_smem_bytes(false), s>>>(bp));
  return cudaGetLastError();
}

}  // namespace gpc
