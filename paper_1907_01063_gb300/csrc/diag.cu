// Diagonal-block kernels and elementwise helpers of the blocked factorisation.
//
// potrf_trtri_diag: the small-block factorisation of Section 3.3 (one thread
// block factors a b x b diagonal block with the classic sequential algorithm,
// its inner loops spread over the threads), followed by the block's inverse
// (the per-block inverses of Section 3.2's divide-and-conquer triangular
// inverse), which turns the panel solve L21 = A21 L11^{-T} into a product.
// The block lives in shared memory for the whole kernel.
#include "common.cuh"

namespace gpc {
namespace {

constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ double &S(double *s, int ld, int i, int j) { return s[i * ld + j]; }

// In-place inverse of the lower nb x nb factor held in shared memory
// (backward column sweep: with L = [[l, 0], [x, L2]],
//  L^{-1} = [[1/l, 0], [-L2^{-1} x / l, L2^{-1}]]).
__device__ void invert_lower_smem(double *s, int ld, int nb) {
  __shared__ double col[kMaxBlock];
  for (int j = nb - 1; j >= 0; --j) {
    const double ljj = S(s, ld, j, j);
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) {
      double t = 0.0;
      for (int k = j + 1; k <= i; ++k) t = fma(S(s, ld, i, k), S(s, ld, k, j), t);
      col[i] = -t / ljj;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) S(s, ld, i, j) = col[i];
    if (threadIdx.x == 0) S(s, ld, j, j) = 1.0 / ljj;
    __syncthreads();
  }
}

__device__ void potrf_trtri_body(int nb, double *A, long long lda, double *Winv, long long ldw, int *info,
                                 int pivot_offset, int factor) {
  extern __shared__ double smem[];
  const int ld = nb + 1;
  __shared__ int fail;
  if (threadIdx.x == 0) fail = 0;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx - i * nb;
    S(smem, ld, i, j) = (j <= i) ? A[(long long)i * lda + j] : 0.0;
  }
  __syncthreads();

  if (factor) {
    for (int j = 0; j < nb; ++j) {
      if (threadIdx.x == 0) {
        const double p = S(smem, ld, j, j);
        if (p > 0.0 && p <= 1.79769313486231570e308) {
          S(smem, ld, j, j) = sqrt(p);
        } else {
          fail = 1;
          if (info && info[1] == 0) {
            info[0] = pivot_offset + j;
            info[1] = (p != p || p > 1.79769313486231570e308) ? GPC_ERR_NAN : GPC_ERR_NOT_PD;
          }
        }
      }
      __syncthreads();
      if (fail) break;
      const double d = S(smem, ld, j, j);
      for (int i = j + 1 + threadIdx.x; i < nb; i += blockDim.x) S(smem, ld, i, j) /= d;
      __syncthreads();
      const int m = nb - j - 1;
      for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
        const int r = idx / m, c = idx - r * m;
        if (c <= r)
          S(smem, ld, j + 1 + r, j + 1 + c) -= S(smem, ld, j + 1 + r, j) * S(smem, ld, j + 1 + c, j);
      }
      __syncthreads();
    }
    // L11 back in place, upper part of the block zeroed.
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int i = idx / nb, j = idx - i * nb;
      A[(long long)i * lda + j] = (j <= i) ? S(smem, ld, i, j) : 0.0;
    }
    if (fail) return;
  }
  invert_lower_smem(smem, ld, nb);
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx - i * nb;
    Winv[(long long)i * ldw + j] = (j <= i) ? S(smem, ld, i, j) : 0.0;
  }
}

__global__ void __launch_bounds__(DIAG_THREADS)
potrf_trtri_kernel(int nb, double *A, long long lda, double *Winv, int *info, int pivot_offset,
                   int factor) {
  potrf_trtri_body(nb, A, lda, Winv, nb, info, pivot_offset, factor);
}

// All diagonal-block inverses of L at once, one CTA per block.  Block 0 is
// rows [0, first), block ib >= 1 is [first + (ib - 1) b, first + ib b).  With
// ldo == 0 the inverse of block ib goes to out + ib * b * b with leading
// dimension equal to its size; otherwise to its diagonal position in an
// n x n matrix out with leading dimension ldo (out may be L itself: each block
// is read into shared memory before its inverse is written).  (The per-block
// inverses of Section 3.2, computed as a batch.)
__global__ void __launch_bounds__(DIAG_THREADS)
trtri_batched_kernel(int n, const double *L, long long ldl, int first, int b, double *out, long long ldo) {
  const int ib = blockIdx.x;
  const int j0 = (ib == 0) ? 0 : first + (ib - 1) * b;
  const int nb = (ib == 0) ? first : min(b, n - j0);
  double *dst = ldo ? out + (long long)j0 * ldo + j0 : out + (size_t)ib * b * b;
  potrf_trtri_body(nb, const_cast<double *>(L) + (long long)j0 * ldl + j0, ldl, dst, ldo ? ldo : nb, nullptr,
                   0, 0);
}

// Cholesky factor of one nb x nb diagonal block in shared memory (the small-
// block step of Section 3.3), blocked right-looking with panels of PF_PW
// columns.  Per panel:
//  1. the PF_PW x PF_PW diagonal sub-block by Schur-complement updates
//     without square roots (a_ik -= a_ij a_kj / a_jj), one thread per
//     element, one barrier per column; the thread that owns the next pivot
//     forms its reciprocal right after its own update.  Column k is then
//     scaled by 1/sqrt(a_kk) (L = L' D^{1/2}).
//  2. one thread per row below solves that row against the sub-block,
//     column by column with the later columns' updates independent, and
//     writes it, transposed, into a panel buffer;
//  3. every thread updates 4 x 4 tiles of the trailing lower triangle from
//     the panel buffer (row and column quadruples read as contiguous pairs).
// The FP64 pipe of one SM bounds step 3 (about nb^3/6 fused multiply-adds);
// steps 1 and 2 are short dependent chains.  Writes L11 in place with the
// upper part of the block zeroed; the first failing pivot is recorded in info
// (GPC_ERR_NOT_PD, or GPC_ERR_NAN for NaN/Inf) and the rest of the block is
// written back unfinished.  No inverse is formed: the panel below is solved
// by substitution (trsm_rows_kernel).
// An FP64 entry, or a double-float one (FP32 hi + lo in the same 8 bytes) when df.
__device__ __forceinline__ double load_entry(const double *p, int df) {
  if (df) {
    const float2 v = *reinterpret_cast<const float2 *>(p);
    return exact_f64(v.x) + exact_f64(v.y);
  }
  return *p;
}

constexpr int PF_PW = 16;
static_assert(PF_PW * PF_PW == DIAG_THREADS, "one thread per sub-block element");
__global__ void __launch_bounds__(DIAG_THREADS)
potrf_diag_kernel(int nb, double *A, long long lda, int *info, int pivot_offset, int df) {
  extern __shared__ double smem[];                            // nb x (nb + 1)
  __shared__ __align__(16) double pt[PF_PW][kMaxBlock + 4];  // panel rows below, transposed
  __shared__ double rdiag[PF_PW], pinv[PF_PW];
  __shared__ int fail;
  const int ld = nb + 1;
  if (threadIdx.x == 0) fail = 0;
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int i = idx / nb, j = idx - i * nb;
    S(smem, ld, i, j) = (j <= i) ? load_entry(A + (long long)i * lda + j, df) : 0.0;
  }
  __syncthreads();
  const int si = threadIdx.x / PF_PW, sk = threadIdx.x % PF_PW;  // sub-block element of this thread
  for (int p0 = 0; p0 < nb; p0 += PF_PW) {
    const int pw = min(PF_PW, nb - p0), m0 = p0 + pw;
    const bool mine = si < pw && sk <= si;
    // 1. diagonal sub-block
    auto pivot = [&](int j) {  // by the owner of (j, j), after its last update
      const double pv = S(smem, ld, p0 + j, p0 + j);
      if (!(pv > 0.0 && pv <= 1.79769313486231570e308)) {
        fail = 1;
        if (info && info[1] == 0) {
          info[0] = pivot_offset + p0 + j;
          info[1] = (pv != pv || pv > 1.79769313486231570e308) ? GPC_ERR_NAN : GPC_ERR_NOT_PD;
        }
      } else {
        pinv[j] = recip_nr(pv);
      }
    };
    if (threadIdx.x == 0) pivot(0);
    __syncthreads();
    for (int j = 0; j < pw && !fail; ++j) {
      if (mine && sk > j) {
        const double t = S(smem, ld, p0 + si, p0 + j) * pinv[j];
        S(smem, ld, p0 + si, p0 + sk) = fma(-t, S(smem, ld, p0 + sk, p0 + j), S(smem, ld, p0 + si, p0 + sk));
        if (si == j + 1 && sk == j + 1) pivot(j + 1);
      }
      __syncthreads();
    }
    if (fail) break;
    if (mine && si == sk) rdiag[sk] = rsqrt_nr(S(smem, ld, p0 + sk, p0 + sk));
    __syncthreads();
    if (mine) {
      double &e = S(smem, ld, p0 + si, p0 + sk);
      e *= rdiag[sk];  // on the diagonal: a_kk / sqrt(a_kk) = sqrt(a_kk)
    }
    __syncthreads();
    // 2. rows below the sub-block: x = a L_pp^{-T} by forward substitution
    for (int i = m0 + threadIdx.x; i < nb; i += blockDim.x) {
      double x[PF_PW];
#pragma unroll
      for (int j = 0; j < PF_PW; ++j) x[j] = (j < pw) ? S(smem, ld, i, p0 + j) : 0.0;
#pragma unroll
      for (int j = 0; j < PF_PW; ++j) {
        if (j < pw) {
          x[j] *= rdiag[j];
#pragma unroll
          for (int t = j + 1; t < PF_PW; ++t)
            if (t < pw) x[t] = fma(-x[j], S(smem, ld, p0 + t, p0 + j), x[t]);
        }
      }
#pragma unroll
      for (int j = 0; j < PF_PW; ++j) {
        if (j < pw) {
          S(smem, ld, i, p0 + j) = x[j];
          pt[j][i - m0] = x[j];
        }
      }
    }
    __syncthreads();
    // 3. trailing update of the lower triangle, rows and columns in [m0, nb)
    const int m = nb - m0;
    if (m > 0) {
      const int tb = (m + 3) >> 2, ntiles = tb * (tb + 1) / 2;
      for (int t = threadIdx.x; t < ntiles; t += blockDim.x) {
        int ti = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
        while ((ti + 1) * (ti + 2) / 2 <= t) ++ti;
        while (ti * (ti + 1) / 2 > t) --ti;
        const int tk = t - ti * (ti + 1) / 2;
        const int r0 = 4 * ti, c0 = 4 * tk;  // offsets from m0
        double acc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = 0.0;
#pragma unroll
        for (int q = 0; q < PF_PW; ++q) {
          if (q < pw) {
            const double2 a01 = *(const double2 *)&pt[q][r0], a23 = *(const double2 *)&pt[q][r0 + 2];
            const double2 b01 = *(const double2 *)&pt[q][c0], b23 = *(const double2 *)&pt[q][c0 + 2];
            const double a[4] = {a01.x, a01.y, a23.x, a23.y}, bc[4] = {b01.x, b01.y, b23.x, b23.y};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bc[v], acc[u][v]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int i = m0 + r0 + u, k = m0 + c0 + v;
            if (i < nb && k <= i) S(smem, ld, i, k) -= acc[u][v];
          }
      }
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    A[(long long)r * lda + c] = (c <= r) ? S(smem, ld, r, c) : 0.0;
  }
}

// Row-parallel triangular solve of an m x nb panel X (in place) against the
// nb x nb lower block T (Section 3.3's panel step, by substitution instead of
// a product with the inverse):
//   mode 0: X <- X T^{-T}  (forward panel L21 = A21 L11^{-T}; columns ascending)
//   mode 1: X <- X T^{-1}  (adjoint panel Cbar D^{-1}; columns descending)
// One CTA per ROWS rows, the rows in shared memory; T is read through L1.
// Thread (r, g) owns the columns k = g (mod 256 / ROWS) of row r; the owner of
// the next column scales it right after its last update, so one barrier per
// column suffices.  Fewer rows per CTA for short panels keep every SM busy.
template <int ROWS>
__global__ void __launch_bounds__(256)
trsm_rows_kernel(int m, int nb, double *X, long long ldx, const double *T, long long ldt, int mode, int df) {
  constexpr int CG = 256 / ROWS;
  __shared__ double xs[ROWS][kMaxBlock + 1];
  __shared__ double rdiag[kMaxBlock];
  const int r0 = blockIdx.x * ROWS, rows = min(ROWS, m - r0);
  for (int idx = threadIdx.x; idx < ROWS * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    xs[r][c] = (r < rows) ? load_entry(X + (long long)(r0 + r) * ldx + c, df) : 0.0;
  }
  for (int j = threadIdx.x; j < nb; j += blockDim.x) rdiag[j] = 1.0 / __ldg(&T[(long long)j * ldt + j]);
  __syncthreads();
  const int r = threadIdx.x % ROWS, cg = threadIdx.x / ROWS;
  const int jfirst = mode == 0 ? 0 : nb - 1;
  if (cg == jfirst % CG) xs[r][jfirst] *= rdiag[jfirst];
  __syncthreads();
  for (int step = 0; step < nb; ++step) {
    const int j = mode == 0 ? step : nb - 1 - step;
    const double xj = xs[r][j];
    if (mode == 0) {
      int k = j + 1 + ((cg - (j + 1)) % CG + CG) % CG;
      if (k == j + 1 && k < nb) {  // the next column: last update, then scale
        xs[r][k] = fma(-xj, __ldg(&T[(long long)k * ldt + j]), xs[r][k]) * rdiag[k];
        k += CG;
      }
      for (; k < nb; k += CG) xs[r][k] = fma(-xj, __ldg(&T[(long long)k * ldt + j]), xs[r][k]);
    } else {
      const int kl = j - 1;
      for (int k = cg; k < kl; k += CG) xs[r][k] = fma(-xj, __ldg(&T[(long long)j * ldt + k]), xs[r][k]);
      if (kl >= 0 && kl % CG == cg)
        xs[r][kl] = fma(-xj, __ldg(&T[(long long)j * ldt + kl]), xs[r][kl]) * rdiag[kl];
    }
    __syncthreads();
  }
  for (int idx = threadIdx.x; idx < ROWS * nb; idx += blockDim.x) {
    const int rr = idx / nb, c = idx - rr * nb;
    if (rr < rows) X[(long long)(r0 + rr) * ldx + c] = xs[rr][c];
  }
}

// The same panel solve with TPR threads per row (4, or 16 for short panels)
// and no block barriers, for the block sizes the factorisations use (NB = 64
// or 128).  Thread t of a row holds columns k = TPR c + t (c < NB / TPR) in
// registers; at step j the owner of column j (final by then) passes it to the
// row's other threads with a warp shuffle, every thread updates its columns
// still to be solved, and the owner of the next column scales it.  Columns
// are dealt round-robin so the shrinking work stays balanced; the loops are
// unrolled at compile time so the row stays in registers.  The FP64 pipe, not
// synchronisation, bounds it: one FP64 warp instruction holds a sub-partition's
// FP64 unit for about 64 cycles, so a short panel (the 64 x 64 solve of a
// diagonal block's halves) is spread over 16 threads per row and more warps.
// Every element sees the same operations in the same order for any TPR.
constexpr int TQ_THREADS = 64;  // 16 rows per CTA at TPR = 4: enough CTAs that every SM gets an even share
template <int NB, int MODE, int TPR>
__global__ void __launch_bounds__(TQ_THREADS)
trsm_quad_kernel(int m, double *X, long long ldx, const double *T, long long ldt, int df) {
  constexpr int C = NB / TPR;
  __shared__ double rdiag[NB];
  for (int k = threadIdx.x; k < NB; k += blockDim.x) rdiag[k] = 1.0 / __ldg(&T[(long long)k * ldt + k]);
  __syncthreads();
  const int lane = threadIdx.x & 31, t = lane & (TPR - 1), src0 = lane & ~(TPR - 1);
  const int row = blockIdx.x * (TQ_THREADS / TPR) + (threadIdx.x / TPR);
  const bool live = row < m;
  double *xr = X + (long long)(live ? row : 0) * ldx;
  double x[C];
#pragma unroll
  for (int c = 0; c < C; ++c) x[c] = live ? load_entry(xr + TPR * c + t, df) : 0.0;
  if (MODE == 0) {  // X <- X T^{-T}: columns ascending, x_k -= x_j T[k][j] for k > j
    if (t == 0) x[0] *= rdiag[0];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const double xj = __shfl_sync(0xffffffffu, x[j / TPR], src0 | (j % TPR));
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (TPR * c + TPR - 1 <= j) continue;  // every column of this group is already final
        const int k = TPR * c + t;
        const double tv = __ldg(&T[(long long)k * ldt + j]);
        if (TPR * c > j || k > j) x[c] = fma(-xj, tv, x[c]);
      }
      if (j + 1 < NB && t == ((j + 1) % TPR)) x[(j + 1) / TPR] *= rdiag[j + 1];
    }
  } else {  // X <- X T^{-1}: columns descending, x_k -= x_j T[j][k] for k < j
    if (t == ((NB - 1) % TPR)) x[C - 1] *= rdiag[NB - 1];
#pragma unroll
    for (int j = NB - 1; j >= 0; --j) {
      const double xj = __shfl_sync(0xffffffffu, x[j / TPR], src0 | (j % TPR));
#pragma unroll
      for (int c = 0; c < C; ++c) {
        if (TPR * c >= j) continue;  // every column of this group is at or past j
        const int k = TPR * c + t;
        const double tv = __ldg(&T[(long long)j * ldt + k]);
        if (TPR * c + TPR - 1 < j || k < j) x[c] = fma(-xj, tv, x[c]);
      }
      if (j > 0 && t == ((j - 1) % TPR)) x[(j - 1) / TPR] *= rdiag[j - 1];
    }
  }
  if (live) {
#pragma unroll
    for (int c = 0; c < C; ++c) xr[TPR * c + t] = x[c];
  }
}

__global__ void copy_lower_kernel(int n, const double *src, long long lds, double *dst,
                                  long long ldd) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
  dst[(long long)i * ldd + j] = (j <= i) ? src[(long long)i * lds + j] : 0.0;
}

__global__ void copy_rect_kernel(int m, int c, const double *src, long long lds, double *dst,
                                 long long ldd) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * c) return;
  const int i = (int)(idx / c), j = (int)(idx - (long long)i * c);
  dst[(long long)i * ldd + j] = src[(long long)i * lds + j];
}

__global__ void phi_block_kernel(int nb, double *A, long long lda) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nb * nb) return;
  const int i = idx / nb, j = idx - i * nb;
  double *p = A + (long long)i * lda + j;
  if (j > i) *p = 0.0;
  else if (j == i) *p *= 0.5;
}

__global__ void lower_to_symmetric_half_kernel(int n, double *A, long long lda) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
  if (j >= i) return;
  const double v = 0.5 * A[(long long)i * lda + j];
  A[(long long)i * lda + j] = v;
  A[(long long)j * lda + i] = v;
}

__global__ void reset_info_kernel(int *info) {
  info[0] = -1;
  info[1] = GPC_OK;
}

unsigned blocks_for(long long total, int threads) { return (unsigned)((total + threads - 1) / threads); }

// Test hook: the refined reciprocals next to CUDA's own 1.0 / x and rsqrt(x).
__global__ void recip_rsqrt_probe_kernel(int n, const double *x, double *out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double v = x[i];
  out[4 * i + 0] = recip_nr(v);
  out[4 * i + 1] = 1.0 / v;
  out[4 * i + 2] = rsqrt_nr(v);
  out[4 * i + 3] = rsqrt(v);
}

// Cholesky factor of one nb x nb diagonal block, nb <= 64, with a one-column
// lookahead (the small-block step of Section 3.3).  Column k+1 is finished
// (pivot, 1/sqrt, scaling) by one warp while six other warps apply column k
// to the rest of the block.  On this part a dependent FP64 operation costs
// about 60 cycles and one SM sustains under two FP64 multiply-adds per cycle,
// so the pivot chain and the trailing updates must overlap, and no FP64
// instruction may issue with lanes that have nothing to do (a warp
// instruction costs the FP64 pipe the same time whatever its active mask):
//   * warp 0 (the pivot warp) finishes columns: for column k+1 it applies the
//     column-k update itself, takes r = 1/sqrt(pivot) and writes the final
//     column to shared memory, then publishes col_ready = k+1;
//   * warps 1-3 and 5-7 (the updaters, u = 0..5) own whole columns j = u mod 6,
//     lane l holding rows j + l and j + l + 32 in registers, so whether a
//     column takes part in a step is the same for the whole warp; at step k,
//     once column k is final, the owner of column k+2 (the one the pivot warp
//     finishes next) updates and stores it first and marks rounds[k+1], then
//     every warp updates its later columns (rounds[0]: columns 0 and 1 stored
//     as loaded, one mark per warp);
//   * warp 4 idles, so the pivot warp has its SM sub-partition to itself.
// Every wait is a bounded spin on a shared-memory word; a wait that runs out
// records GPC_ERR_TIMEOUT and stops the block.  The first failing pivot is
// recorded like potrf_diag_kernel does, and the rest of the block is written
// back unfinished.
constexpr int PL_NB = 64, PL_LD = PL_NB + 1, PL_W = 6, PL_COLS = (PL_NB + PL_W - 1) / PL_W;
constexpr long long PL_SPIN = 1LL << 24;

__global__ void __launch_bounds__(256)
potrf_la_kernel(int nb, double *A, long long lda, int *info, int pivot_offset, int df, int *gerr) {
  __shared__ double M[PL_NB * PL_LD];
  __shared__ int col_ready, stop;
  __shared__ int rounds[PL_NB];  // rounds[r]: marks of round r
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    col_ready = -1;
    stop = 0;
  }
  if (threadIdx.x < PL_NB) rounds[threadIdx.x] = 0;
  const bool updater = warp != 0 && warp != 4;
  const int uw = updater ? warp - 1 - (warp > 4) : 0;
  double a0[PL_COLS], a1[PL_COLS];  // column uw + 6 c: rows j + lane, j + lane + 32
  if (updater) {
#pragma unroll
    for (int c = 0; c < PL_COLS; ++c) {
      const int j = uw + PL_W * c, r0 = j + lane, r1 = r0 + 32;
      a0[c] = (j < nb && r0 < nb) ? load_entry(A + (long long)r0 * lda + j, df) : 0.0;
      a1[c] = (j < nb && r1 < nb) ? load_entry(A + (long long)r1 * lda + j, df) : 0.0;
    }
  }
  __syncthreads();
  volatile int *vready = &col_ready, *vstop = &stop;
  // Polls: the updaters back off between polls, so that their loads do not
  // queue in front of the pivot warp's shared-memory accesses.
  auto spin_ge = [&](volatile int *w, int target) -> bool {
    for (long long it = 0; it < PL_SPIN; ++it) {
      if (*w >= target) return true;
      if (*vstop) return false;
      if (updater) __nanosleep(64);
    }
    return false;
  };
  auto give_up = [&]() {  // a wait ran out: report and stop the block
    if (info && info[1] == 0) info[1] = GPC_ERR_TIMEOUT;
    record_error(gerr, GPC_ERR_TIMEOUT);
    *vstop = 1;
  };
  if (updater) {
    // round 0: columns 0 and 1 as loaded (owned by updaters 0 and 1)
    if (uw <= 1 && uw < nb) {
      const int j = uw, r0 = j + lane, r1 = r0 + 32;
      if (r0 < nb) M[r0 * PL_LD + j] = a0[0];
      if (r1 < nb) M[r1 * PL_LD + j] = a1[0];
    }
    __threadfence_block();
    __syncwarp();
    if (lane == 0) atomicAdd(&rounds[0], 1);
  }
  if (warp == 0) {
    // ---- pivot warp: lanes own rows lane and lane + 32
    for (int c = 0; c < nb; ++c) {
      // column c comes from round max(c - 1, 0)
      if (!spin_ge((volatile int *)&rounds[max(c - 1, 0)], c <= 1 ? PL_W : 1)) {
        if (!*vstop && lane == 0) give_up();
        break;
      }
      __threadfence_block();
      const int i0 = lane, i1 = lane + 32;
      double v0 = (i0 >= c && i0 < nb) ? M[i0 * PL_LD + c] : 0.0;
      double v1 = (i1 >= c && i1 < nb) ? M[i1 * PL_LD + c] : 0.0;
      if (c > 0) {  // the update by column c - 1, finished by this warp just before
        const double lc = M[c * PL_LD + c - 1];
        if (i0 >= c && i0 < nb) v0 = fma(-M[i0 * PL_LD + c - 1], lc, v0);
        if (i1 >= c && i1 < nb) v1 = fma(-M[i1 * PL_LD + c - 1], lc, v1);
      }
      const double pv = (c < 32) ? __shfl_sync(0xffffffffu, v0, c) : __shfl_sync(0xffffffffu, v1, c - 32);
      if (!(pv > 0.0 && pv <= 1.79769313486231570e308)) {
        if (lane == 0) {
          if (info && info[1] == 0) {
            info[0] = pivot_offset + c;
            info[1] = (pv != pv || pv > 1.79769313486231570e308) ? GPC_ERR_NAN : GPC_ERR_NOT_PD;
          }
          *vstop = 1;
        }
        break;
      }
      const double r = rsqrt_nr(pv);  // every lane: no broadcast on the chain
      if (i0 >= c && i0 < nb) M[i0 * PL_LD + c] = (i0 == c) ? pv * r : v0 * r;
      if (i1 >= c && i1 < nb) M[i1 * PL_LD + c] = (i1 == c) ? pv * r : v1 * r;
      __threadfence_block();
      __syncwarp();
      if (lane == 0) *vready = c;
    }
  } else if (updater) {
    // ---- updaters: step k applies column k to columns k + 2 .. nb - 1
    for (int k = 0; k + 2 < nb; ++k) {
      if (!spin_ge(vready, k)) {
        if (!*vstop && lane == 0) give_up();
        break;
      }
      __threadfence_block();
#pragma unroll
      for (int c = 0; c < PL_COLS; ++c) {
        const int j = uw + PL_W * c;
        if (j == k + 2) {  // warp-uniform: the column the pivot warp needs next
          const double ljk = M[j * PL_LD + k];
          const int r0 = j + lane, r1 = r0 + 32;
          if (r0 < nb) {
            a0[c] = fma(-M[r0 * PL_LD + k], ljk, a0[c]);
            M[r0 * PL_LD + j] = a0[c];
          }
          if (r1 < nb) {
            a1[c] = fma(-M[r1 * PL_LD + k], ljk, a1[c]);
            M[r1 * PL_LD + j] = a1[c];
          }
          __threadfence_block();
          __syncwarp();
          if (lane == 0) atomicAdd(&rounds[k + 1], 1);
        }
      }
#pragma unroll
      for (int c = 0; c < PL_COLS; ++c) {
        const int j = uw + PL_W * c;
        if (j > k + 2 && j < nb) {  // warp-uniform
          const double ljk = M[j * PL_LD + k];
          const int r0 = j + lane, r1 = r0 + 32;
          if (r0 < nb) a0[c] = fma(-M[r0 * PL_LD + k], ljk, a0[c]);
          if (j + 32 < nb && r1 < nb) a1[c] = fma(-M[r1 * PL_LD + k], ljk, a1[c]);
        }
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
    const int r = idx / nb, c = idx - r * nb;
    A[(long long)r * lda + c] = (c <= r) ? M[r * PL_LD + c] : 0.0;
  }
}

}  // namespace

static cudaError_t launch_diag(int nb, double *A, long long lda, double *Winv, int *info,
                               int pivot_offset, int factor, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  if (nb > kMaxBlock) return cudaErrorInvalidValue;
  const size_t smem = (size_t)nb * (nb + 1) * sizeof(double);
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(potrf_trtri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)kMaxBlock * (kMaxBlock + 1) * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const double nb3 = (double)nb * nb * nb;
  GPC_LAUNCH(GPC_TRACE_DIAG, (factor ? nb3 / 3.0 : 0.0) + nb3 / 3.0, 8.0 * 1.5 * nb * nb, s,
             potrf_trtri_kernel<<<1, DIAG_THREADS, smem, s>>>(nb, A, lda, Winv, info, pivot_offset,
                                                               factor));
  return cudaGetLastError();
}

cudaError_t potrf_trtri_diag(int nb, double *A, long long lda, double *Winv, int *info,
                             int pivot_offset, cudaStream_t s) {
  return launch_diag(nb, A, lda, Winv, info, pivot_offset, 1, s);
}

cudaError_t trtri_diag(int nb, const double *D, long long ldd, double *Dinv, cudaStream_t s) {
  return launch_diag(nb, const_cast<double *>(D), ldd, Dinv, nullptr, 0, 0, s);
}

cudaError_t trtri_batched(int n, const double *L, long long ldl, int first, int b, double *out,
                          cudaStream_t s, long long ldo) {
  if (n <= 0) return cudaSuccess;
  if (b > kMaxBlock || first < 1 || first > b) return cudaErrorInvalidValue;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(trtri_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)kMaxBlock * (kMaxBlock + 1) * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  const int nblk = 1 + (n - first + b - 1) / b;
  const size_t smem = (size_t)b * (b + 1) * sizeof(double);
  GPC_LAUNCH(GPC_TRACE_DIAG, (double)n * b * b / 3.0, 16.0 * (double)n * b, s,
             trtri_batched_kernel<<<nblk, DIAG_THREADS, smem, s>>>(n, L, ldl, first, b, out, ldo));
  return cudaGetLastError();
}

cudaError_t potrf_diag(int nb, double *A, long long lda, int *info, int pivot_offset, cudaStream_t s, bool df) {
  if (nb <= 0) return cudaSuccess;
  if (nb > kMaxBlock) return cudaErrorInvalidValue;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_set[dev]) {
    cudaError_t e = cudaFuncSetAttribute(potrf_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((size_t)kMaxBlock * (kMaxBlock + 1) * sizeof(double)));
    if (e != cudaSuccess) return e;
    attr_set[dev] = true;
  }
  if (nb <= PL_NB) {  // blocks of up to 64: the lookahead kernel
    GPC_LAUNCH(GPC_TRACE_DIAG, (double)nb * nb * nb / 3.0, 16.0 * nb * nb, s,
               launch_k(potrf_la_kernel, 1, 256, 0, s, nb, A, lda, info, pivot_offset, df ? 1 : 0, error_word()));
    return cudaGetLastError();
  }
  const size_t smem = (size_t)nb * (nb + 1) * sizeof(double);
  GPC_LAUNCH(GPC_TRACE_DIAG, (double)nb * nb * nb / 3.0, 16.0 * nb * nb, s,
             launch_k(potrf_diag_kernel, 1, DIAG_THREADS, smem, s, nb, A, lda, info, pivot_offset, df ? 1 : 0));
  return cudaGetLastError();
}

// The panel solves run beside the split products' CTAs (one product CTA per
// SM holds ~219 KB of shared memory, leaving room for a small solve CTA).  An
// SM runs CTAs of one shared-memory configuration at a time, so the solve
// kernels ask for the same maximal shared-memory carveout as the products.
bool g_trsm_carveout[64];
cudaError_t trsm_carveout() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaSuccess;
  if (g_trsm_carveout[dev]) return cudaSuccess;
  const void *fns[] = {(const void *)trsm_quad_kernel<64, 0, 4>, (const void *)trsm_quad_kernel<64, 1, 4>,
                       (const void *)trsm_quad_kernel<128, 0, 4>, (const void *)trsm_quad_kernel<128, 1, 4>,
                       (const void *)trsm_quad_kernel<64, 0, 16>, (const void *)trsm_quad_kernel<64, 1, 16>,
                       (const void *)trsm_quad_kernel<128, 0, 16>, (const void *)trsm_quad_kernel<128, 1, 16>,
                       (const void *)trsm_rows_kernel<8>, (const void *)trsm_rows_kernel<16>,
                       (const void *)trsm_rows_kernel<32>};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  g_trsm_carveout[dev] = true;
  return cudaSuccess;
}

cudaError_t trsm_rows(int m, int nb, double *X, long long ldx, const double *T, long long ldt, int mode,
                      cudaStream_t s, bool df) {
  if (m <= 0 || nb <= 0) return cudaSuccess;
  if (nb > kMaxBlock) return cudaErrorInvalidValue;
  if (cudaError_t ce = trsm_carveout(); ce != cudaSuccess) return ce;
  const double fl = (double)m * nb * nb, by = 16.0 * (double)m * nb + 4.0 * nb * nb;
  if (nb == 64 || nb == 128) {
    // short panels (at most 256 rows): 16 threads per row, so the row's FP64
    // work is spread over four times as many warps
    const bool short_panel = m <= 256;
    const int tpr = short_panel ? 16 : 4;
    const unsigned qgrid = (unsigned)((m + TQ_THREADS / tpr - 1) / (TQ_THREADS / tpr));
#define GPC_TRSM_QUAD(NB_, MODE_, TPR_)                                                                      \
  GPC_LAUNCH(GPC_TRACE_TRSM, fl, by, s,                                                                     \
             launch_k(trsm_quad_kernel<NB_, MODE_, TPR_>, qgrid, TQ_THREADS, 0, s, m, X, ldx, T, ldt, df))
    if (short_panel) {
      if (nb == 64 && mode == 0) GPC_TRSM_QUAD(64, 0, 16);
      else if (nb == 64) GPC_TRSM_QUAD(64, 1, 16);
      else if (mode == 0) GPC_TRSM_QUAD(128, 0, 16);
      else GPC_TRSM_QUAD(128, 1, 16);
    } else {
      if (nb == 64 && mode == 0) GPC_TRSM_QUAD(64, 0, 4);
      else if (nb == 64) GPC_TRSM_QUAD(64, 1, 4);
      else if (mode == 0) GPC_TRSM_QUAD(128, 0, 4);
      else GPC_TRSM_QUAD(128, 1, 4);
    }
#undef GPC_TRSM_QUAD
    return cudaGetLastError();
  }
  // other block sizes: 32 rows per CTA when that still gives two CTAs per SM, else 16 or 8
  const int sms = sm_count();
  if ((m + 31) / 32 >= 2 * sms) {
    GPC_LAUNCH(GPC_TRACE_TRSM, (double)m * nb * nb, 16.0 * (double)m * nb + 4.0 * nb * nb, s,
               launch_k(trsm_rows_kernel<32>, (m + 31) / 32, 256, 0, s, m, nb, X, ldx, T, ldt, mode,
                        df ? 1 : 0));
  } else if ((m + 15) / 16 >= sms) {
    GPC_LAUNCH(GPC_TRACE_TRSM, (double)m * nb * nb, 16.0 * (double)m * nb + 4.0 * nb * nb, s,
               launch_k(trsm_rows_kernel<16>, (m + 15) / 16, 256, 0, s, m, nb, X, ldx, T, ldt, mode,
                        df ? 1 : 0));
  } else {
    GPC_LAUNCH(GPC_TRACE_TRSM, (double)m * nb * nb, 16.0 * (double)m * nb + 4.0 * nb * nb, s,
               launch_k(trsm_rows_kernel<8>, (m + 7) / 8, 256, 0, s, m, nb, X, ldx, T, ldt, mode,
                        df ? 1 : 0));
  }
  return cudaGetLastError();
}

cudaError_t copy_lower(int n, const double *src, long long lds, double *dst, long long ldd,
                       cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (double)n * n * 1.5, s,
             copy_lower_kernel<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(n, src, lds, dst, ldd));
  return cudaGetLastError();
}

cudaError_t copy_rect(int m, int c, const double *src, long long lds, double *dst, long long ldd,
                      cudaStream_t s) {
  if (m <= 0 || c <= 0) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 16.0 * (double)m * c, s,
             copy_rect_kernel<<<blocks_for((long long)m * c, 256), 256, 0, s>>>(m, c, src, lds, dst, ldd));
  return cudaGetLastError();
}

cudaError_t phi_block(int nb, double *A, long long lda, cudaStream_t s) {
  if (nb <= 0) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 16.0 * (double)nb * nb, s,
             phi_block_kernel<<<blocks_for((long long)nb * nb, 256), 256, 0, s>>>(nb, A, lda));
  return cudaGetLastError();
}

cudaError_t lower_to_symmetric_half(int n, double *A, long long lda, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 16.0 * (double)n * n, s,
             lower_to_symmetric_half_kernel<<<blocks_for((long long)n * n, 256), 256, 0, s>>>(n, A, lda));
  return cudaGetLastError();
}

cudaError_t recip_rsqrt_probe(int n, const double *x, double *out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 40.0 * n, s, recip_rsqrt_probe_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, out));
  return cudaGetLastError();
}

cudaError_t reset_info(int *info, cudaStream_t s) {
  if (!info) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0, s, reset_info_kernel<<<1, 1, 0, s>>>(info));
  return cudaGetLastError();
}

}  // namespace gpc
