// Fused categorical-logit GLM likelihood with its gradient (Section 3.4,
// multinomial logistic regression).
//
// C classes, y_i in {0, .., C - 1}; class scores eta_ic = alpha_c + x_i . beta_c
// (beta: k x C, row-major, column c = class c); lp_i = eta_{i,y_i} - lse_i with
// lse_i = log sum_c exp(eta_ic) (the row maximum subtracted inside); with
// p_ic = exp(eta_ic - lse_i) and d_ic = [c == y_i] - p_ic the outputs are
// lp = sum_i lp_i, dalpha_c = sum_i d_ic and dbeta_jc = sum_i X_ij d_ic.
//
// Same one-pass layout as the single-predictor kernel (glm.cu): a CTA walks
// blocks of R rows; its warps form the C scores of a row at a time (lanes
// strided over the columns, C independent FMA chains per lane, a fixed-order
// butterfly per class), one thread per row evaluates the log-sum-exp and
// d_i., and every thread adds X_ij d_ic for the columns it owns over the
// block's rows, re-reading the block from L1/L2.  The k x C column sums stay
// in shared memory for the CTA's whole share of rows; one partial row per CTA
// goes to the workspace and a second kernel adds them in CTA order, so
// results are bitwise reproducible.  A y_i outside {0, .., C - 1} makes lp
// NaN without indexing anything.
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr int CT_T = 256;    // threads per CTA
constexpr int CT_R = 32;     // rows per block
constexpr int CMAX = GPC_GLM_MAX_CLASSES;

struct CatParams {
  int k, C;
  long long n, ldx;
  const double *X, *y, *alpha, *beta;
  double *part, *part_s;  // per CTA: k C column sums; 1 + C scalars (lp, dalpha)
};

__global__ void __launch_bounds__(CT_T) glm_cat_kernel(CatParams p) {
  extern __shared__ double sm[];
  const int kc = p.k * p.C;
  double *bs = sm;                  // beta, k x C
  double *acc = bs + kc;            // dbeta sums, k x C
  double *al = acc + kc;            // alpha, C
  double *eta_s = al + CMAX;        // CT_R x CMAX scores of the block's rows
  double *dblk = eta_s + CT_R * CMAX;  // CT_R x CMAX d values
  __shared__ double red[CT_T / 32][CMAX + 1];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, C = p.C;
  for (int q = t; q < kc; q += CT_T) {
    bs[q] = p.beta[q];
    acc[q] = 0.0;
  }
  if (t < C) al[t] = p.alpha[t];
  __syncthreads();
  double slp = 0.0, sda[CMAX];
#pragma unroll
  for (int c = 0; c < CMAX; ++c) sda[c] = 0.0;
  const long long nblk = (p.n + CT_R - 1) / CT_R;
  for (long long b = blockIdx.x; b < nblk; b += gridDim.x) {
    const long long i0 = b * CT_R;
    const int rows = (int)min((long long)CT_R, p.n - i0);
    // scores: one row per warp pass, C chains per lane
    for (int r = warp; r < rows; r += CT_T / 32) {
      const double *x = p.X + (i0 + r) * p.ldx;
      double sc[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c) sc[c] = 0.0;
      for (int j = lane; j < p.k; j += 32) {
        const double xj = x[j];
        const double *bj = bs + (long long)j * C;
#pragma unroll
        for (int c = 0; c < CMAX; ++c)
          if (c < C) sc[c] = fma(xj, bj[c], sc[c]);
      }
#pragma unroll
      for (int c = 0; c < CMAX; ++c) {
        if (c < C) {
          double v = sc[c];
          for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
          if (lane == 0) eta_s[r * CMAX + c] = v + al[c];
        }
      }
    }
    __syncthreads();
    // log-sum-exp and d per row, one row per thread
    if (t < rows) {
      const double yv = p.y[i0 + t];
      const int yi = (int)yv;
      const double *e = eta_s + t * CMAX;
      double mx = e[0];
      for (int c = 1; c < C; ++c) mx = fmax(mx, e[c]);
      double se = 0.0;
      for (int c = 0; c < C; ++c) se += exp(e[c] - mx);
      const double lse = mx + log(se);
      const bool ok = yv >= 0.0 && yi < C && (double)yi == yv;
      slp += ok ? e[yi] - lse : __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
      for (int c = 0; c < CMAX; ++c) {
        if (c < C) {
          const double dc = (ok && c == yi ? 1.0 : 0.0) - (ok ? exp(e[c] - lse) : 0.0);
          dblk[t * CMAX + c] = dc;
          sda[c] += dc;
        }
      }
    }
    __syncthreads();
    // dbeta: column-owned sums over the block's rows
    for (int j = t; j < p.k; j += CT_T) {
      const double *xc = p.X + i0 * p.ldx + j;
      double a[CMAX];
#pragma unroll
      for (int c = 0; c < CMAX; ++c) a[c] = 0.0;
      for (int r = 0; r < rows; ++r) {
        const double xv = xc[(long long)r * p.ldx];
        const double *dr = dblk + r * CMAX;
#pragma unroll
        for (int c = 0; c < CMAX; ++c)
          if (c < C) a[c] = fma(xv, dr[c], a[c]);
      }
#pragma unroll
      for (int c = 0; c < CMAX; ++c)
        if (c < C) acc[(long long)j * C + c] += a[c];
    }
    __syncthreads();
  }
  for (int q = t; q < kc; q += CT_T) p.part[(long long)blockIdx.x * kc + q] = acc[q];
  // lp and dalpha: warp sums, then the warps in order
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) slp += __shfl_down_sync(0xffffffffu, slp, o);
#pragma unroll
  for (int c = 0; c < CMAX; ++c) {
    if (c < C) {
      double v = sda[c];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      sda[c] = v;
    }
  }
  if (lane == 0) {
    red[warp][0] = slp;
#pragma unroll
    for (int c = 0; c < CMAX; ++c)
      if (c < C) red[warp][1 + c] = sda[c];
  }
  __syncthreads();
  if (t < 1 + C) {
    double v = 0.0;
    for (int w = 0; w < CT_T / 32; ++w) v += red[w][t];
    p.part_s[(long long)blockIdx.x * (CMAX + 1) + t] = v;
  }
}

__global__ void glm_cat_reduce_kernel(int kc, int C, int ctas, const double *part, const double *part_s,
                                      double *dbeta, double *lp, double *dalpha) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < kc) {
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s += part[(long long)c * kc + q];
    dbeta[q] = s;
  } else if (q < kc + 1 + C) {
    const int m = q - kc;
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s += part_s[(long long)c * (CMAX + 1) + m];
    if (m == 0) *lp = s;
    else dalpha[m - 1] = s;
  }
}

size_t cat_smem_bytes(int k, int C) {
  return (2 * (size_t)k * C + CMAX + 2 * (size_t)CT_R * CMAX) * sizeof(double);
}

int cat_max_ctas(int k, int C) {
  const size_t per = cat_smem_bytes(k, C) + 1024 + sizeof(double) * (CT_T / 32) * (CMAX + 1);
  const int by_smem = (int)std::max<size_t>(1, (size_t)(228 * 1024) / per);
  return sm_count() * std::max(1, std::min(4, by_smem));
}

}  // namespace

size_t glm_categorical_workspace_bytes(int k, int C) {
  const size_t ctas = (size_t)cat_max_ctas(k, C);
  return align_up(ctas * (size_t)std::max(k * C, 1) * sizeof(double), 256) +
         align_up(ctas * (CMAX + 1) * sizeof(double), 256);
}

cudaError_t glm_categorical(long long n, int k, int C, const double *X, long long ldx, const double *y,
                            const double *alpha, const double *beta, double *lp, double *dalpha, double *dbeta,
                            void *ws, cudaStream_t s) {
  CatParams p;
  p.n = n;
  p.k = k;
  p.C = C;
  p.ldx = ldx;
  p.X = X;
  p.y = y;
  p.alpha = alpha;
  p.beta = beta;
  const int kc = k * C;
  const long long nblk = std::max<long long>(1, (n + CT_R - 1) / CT_R);
  const int ctas = (int)std::min<long long>(nblk, cat_max_ctas(k, C));
  char *w = (char *)ws;
  p.part = (double *)w;
  p.part_s = (double *)(w + align_up((size_t)cat_max_ctas(k, C) * (size_t)std::max(kc, 1) * sizeof(double), 256));
  const size_t smem = cat_smem_bytes(k, C);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(glm_cat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  GPC_LAUNCH(GPC_TRACE_GLM, 4.0 * (double)n * kc, 8.0 * ((double)n * k + 2.0 * n + 2.0 * kc), s,
             glm_cat_kernel<<<ctas, CT_T, smem, s>>>(p));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int outs = kc + 1 + C;
  GPC_LAUNCH(GPC_TRACE_ELEM, (double)ctas * outs, 8.0 * (double)ctas * outs, s,
             glm_cat_reduce_kernel<<<(outs + 255) / 256, 256, 0, s>>>(kc, C, ctas, p.part, p.part_s, dbeta, lp,
                                                                      dalpha));
  return cudaGetLastError();
}

}  // namespace gpc
