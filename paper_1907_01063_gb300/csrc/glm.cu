// Fused GLM log likelihoods with their gradients (Section 3.4).
//
// For observations (x_i, y_i), i < n, the linear predictor is
// eta_i = alpha + x_i . beta; each family gives lp_i and d_i = d lp_i / d eta_i:
//   normal-identity  lp_i = -((y_i - eta_i)/sigma)^2/2 - log sigma - log(2 pi)/2,  d_i = (y_i - eta_i)/sigma^2
//   Bernoulli-logit  lp_i = y_i eta_i - log(1 + e^eta_i),                          d_i = y_i - 1/(1 + e^-eta_i)
//   Poisson-log      lp_i = y_i eta_i - e^eta_i - lgamma(y_i + 1),                  d_i = y_i - e^eta_i
//   negative-binomial-log (mu_i = e^eta_i, dispersion phi = sigma)
//                    lp_i = lgamma(y_i + phi) - lgamma(y_i + 1) - lgamma(phi)
//                           + phi (log phi - log(mu_i + phi)) + y_i (eta_i - log(mu_i + phi)),
//                    d_i = y_i - (y_i + phi) mu_i / (mu_i + phi)
//   ordinal-logit    (C ordered classes, cut points c_0 < .. < c_{C-2}, no intercept)
//                    lp_i = log(s(eta_i - c_{y_i - 1}) - s(eta_i - c_{y_i})), s(t) = 1/(1 + e^-t),
//                    the missing ends reading s = 1 (y_i = 0) and s = 0 (y_i = C - 1)
// and the outputs are lp = sum lp_i, dalpha = sum d_i, dbeta = X^T d and, for
// the normal family, dsigma = sum ((y_i - eta_i)^2/sigma^3 - 1/sigma); for the
// negative binomial dsigma = d lp / d phi = sum (psi(y_i + phi) - psi(phi) +
// log phi - log(mu_i + phi) + 1 - (y_i + phi)/(mu_i + phi)); for the ordinal
// family dcuts_m = d lp / d c_m.
//
// As in the paper each likelihood is one kernel that produces the value and
// the analytic gradient together; here the GEMV for dbeta is fused in as well,
// so X (the only large operand) crosses HBM once.  A CTA walks blocks of R
// rows: its warps first form eta_i for the block (four rows per warp, lanes
// strided over the columns, a fixed-order shuffle reduction), then one thread
// per row evaluates the family's terms, then every thread adds d_i x_ij for
// the columns it owns (j = thread, thread + 256, ...) over the block's rows,
// re-reading the block from L1/L2.  FP64 work (two multiply-adds per element
// of X) rather than HBM bounds this on GB300, so every FP64 instruction
// carries 32 active lanes: the per-row exp/log1p run one row per thread, not
// on one lane of a warp.  The column sums stay in
// shared memory for the CTA's whole share of rows and go out once as one
// partial row; a second kernel adds the partial rows in CTA order.  Every sum
// has a fixed order, so results are bitwise reproducible.
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr int GT = 256;  // threads per CTA
constexpr int kMaxRowsPerBlock = 64;
constexpr int kFamilyOrdinal = 100;  // internal family id of the ordinal-logit GLM
constexpr int kMaxCuts = GPC_GLM_MAX_CLASSES - 1;
constexpr int kScalars = 3 + kMaxCuts;  // per-CTA partial scalars: lp, dalpha, dsigma, dcuts

struct GlmParams {
  int family, k, R, ncut;
  long long n, ldx;
  const double *X, *y, *beta, *cuts;
  double alpha, inv_sigma, log_norm;  // log_norm = log(sigma) + log(2 pi)/2
  double phi, log_phi, lgamma_phi;    // negative binomial
  double *part, *part_s;
};

// Digamma psi(x), x > 0: the recurrence psi(x) = psi(x + 1) - 1/x (Abramowitz
// and Stegun 6.3.5) until x >= 10, then the asymptotic expansion (A&S 6.3.18)
//   psi(x) = ln x - 1/(2x) - sum_{k=1..7} B_2k / (2k x^2k) + O(x^-16),
// with B_2 .. B_14 = 1/6, -1/30, 1/42, -1/30, 5/66, -691/2730, 7/6; the first
// omitted term is below 5e-17 at x = 10.
__device__ double digamma_dev(double x) {
  double acc = 0.0;
  while (x < 10.0) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  const double r = 1.0 / (x * x);
  double t = 1.0 / 12.0;  // B_14 / 14
  t = fma(t, r, -691.0 / 32760.0);
  t = fma(t, r, 1.0 / 132.0);
  t = fma(t, r, -1.0 / 240.0);
  t = fma(t, r, 1.0 / 252.0);
  t = fma(t, r, -1.0 / 120.0);
  t = fma(t, r, 1.0 / 12.0);
  return acc + log(x) - 0.5 / x - t * r;
}

// cut: the ordinal family's contributions to its cut-point derivatives
// (index lo gets -du, lo + 1 gets -dv; lo = -2 when there are none).
__device__ __forceinline__ void glm_row(const GlmParams &p, double eta, double y, double &lp, double &d,
                                        double &ds, int &lo, double &du, double &dv, double psi_phi) {
  lo = -2;
  du = dv = 0.0;
  if (p.family == GPC_GLM_NORMAL_ID) {
    const double r = y - eta, z = r * p.inv_sigma;
    lp = -0.5 * z * z - p.log_norm;
    d = z * p.inv_sigma;
    ds = (z * z - 1.0) * p.inv_sigma;
  } else if (p.family == GPC_GLM_BERNOULLI_LOGIT) {
    const double e = exp(-fabs(eta));  // log(1 + e^eta) = max(eta, 0) + log1p(e^-|eta|)
    lp = y * eta - (fmax(eta, 0.0) + log1p(e));
    d = y - (eta >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e));
    ds = 0.0;
  } else if (p.family == GPC_GLM_POISSON_LOG) {
    const double mu = exp(eta);
    lp = y * eta - mu - lgamma(y + 1.0);
    d = y - mu;
    ds = 0.0;
  } else if (p.family == GPC_GLM_NEG_BINOMIAL_LOG) {
    const double phi = p.phi, mu = exp(eta), ypp = y + phi, mpp = mu + phi, lmp = log(mpp);
    lp = lgamma(ypp) - lgamma(y + 1.0) - p.lgamma_phi + phi * (p.log_phi - lmp) + y * (eta - lmp);
    d = y - ypp * mu / mpp;
    ds = digamma_dev(ypp) - psi_phi + p.log_phi - lmp + 1.0 - ypp / mpp;
  } else {  // ordinal logit: y in {0 .. ncut}
    const int C = p.ncut + 1, yi = (int)y;
    ds = 0.0;
    if (!(y >= 0.0) || yi >= C || (double)yi != y) {  // outside the support: NaN, nothing indexed
      lp = __longlong_as_double(0x7ff8000000000000ll);
      d = 0.0;
      return;
    }
    const double su = yi > 0 ? 1.0 / (1.0 + exp(-(eta - p.cuts[yi - 1]))) : 1.0;
    const double sv = yi < C - 1 ? 1.0 / (1.0 + exp(-(eta - p.cuts[yi]))) : 0.0;
    const double P = su - sv;
    lp = log(P);
    du = yi > 0 ? su * (1.0 - su) / P : 0.0;
    dv = yi < C - 1 ? -sv * (1.0 - sv) / P : 0.0;
    d = du + dv;
    lo = yi - 1;
  }
}

__global__ void __launch_bounds__(GT) glm_kernel(GlmParams p) {
  extern __shared__ double sm[];
  double *acc = sm;                      // k column sums; thread t owns j = t, t + GT, ...
  double *bs = sm + p.k;                 // beta
  double *eta_s = bs + p.k;              // eta of the current block's rows
  double *dblk = eta_s + kMaxRowsPerBlock;  // d_i of the current block's rows
  double *cut_s = dblk + kMaxRowsPerBlock;  // ordinal: per-thread cut sums, kMaxRowsPerBlock x kMaxCuts
  __shared__ double red[3][GT / 32];
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  for (int j = t; j < p.k; j += GT) {
    acc[j] = 0.0;
    bs[j] = p.beta[j];
  }
  if (p.family == kFamilyOrdinal)
    for (int q = t; q < kMaxRowsPerBlock * kMaxCuts; q += GT) cut_s[q] = 0.0;
  const double psi_phi = p.family == GPC_GLM_NEG_BINOMIAL_LOG ? digamma_dev(p.phi) : 0.0;
  __syncthreads();
  double slp = 0.0, sda = 0.0, sds = 0.0;  // per thread (threads below R)
  const long long nblk = (p.n + p.R - 1) / p.R;
  for (long long b = blockIdx.x; b < nblk; b += gridDim.x) {
    const long long i0 = b * p.R;
    const int rows = (int)min((long long)p.R, p.n - i0);
    // eta for four rows per warp: four independent FMA chains per lane, then a
    // transposed butterfly that leaves row 2 bit4 + bit3 of the lane index in
    // every lane (6 adds for the four rows).  Missing rows of a short last
    // group re-read the group's first row and are not stored.
    for (int g = warp; 4 * g < rows; g += GT / 32) {
      const int r0 = 4 * g, nr = min(4, rows - r0);
      const double *x0 = p.X + (i0 + r0) * p.ldx;
      const double *x1 = nr > 1 ? x0 + p.ldx : x0;
      const double *x2 = nr > 2 ? x0 + 2 * p.ldx : x0;
      const double *x3 = nr > 3 ? x0 + 3 * p.ldx : x0;
      double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
#pragma unroll 2
      for (int j = lane; j < p.k; j += 32) {
        const double bj = bs[j];
        s0 = fma(x0[j], bj, s0);
        s1 = fma(x1[j], bj, s1);
        s2 = fma(x2[j], bj, s2);
        s3 = fma(x3[j], bj, s3);
      }
      const bool h16 = (lane & 16) != 0, h8 = (lane & 8) != 0;
      double k0 = h16 ? s2 : s0, k1 = h16 ? s3 : s1;
      k0 += __shfl_xor_sync(0xffffffffu, h16 ? s0 : s2, 16);
      k1 += __shfl_xor_sync(0xffffffffu, h16 ? s1 : s3, 16);
      double v = h8 ? k1 : k0;
      v += __shfl_xor_sync(0xffffffffu, h8 ? k0 : k1, 8);
      v += __shfl_xor_sync(0xffffffffu, v, 4);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      const int row = ((lane >> 4) << 1) | ((lane >> 3) & 1);
      if ((lane & 7) == 0 && row < nr) eta_s[r0 + row] = v + p.alpha;
    }
    __syncthreads();
    // the family's terms, one row per thread
    if (t < rows) {
      double lp, d, ds, du, dv;
      int lo;
      glm_row(p, eta_s[t], p.y[i0 + t], lp, d, ds, lo, du, dv, psi_phi);
      dblk[t] = d;
      slp += lp;
      sda += d;
      sds += ds;
      if (lo >= 0) cut_s[t * kMaxCuts + lo] -= du;
      if (lo >= -1 && lo + 1 < p.ncut) cut_s[t * kMaxCuts + lo + 1] -= dv;
    }
    __syncthreads();
    // dbeta: column-owned sums over the block's rows (two chains), X from L1/L2
    for (int j = t; j < p.k; j += GT) {
      const double *xc = p.X + i0 * p.ldx + j;
      double a0 = 0.0, a1 = 0.0;
      int r = 0;
      for (; r + 1 < rows; r += 2) {
        a0 = fma(xc[(long long)r * p.ldx], dblk[r], a0);
        a1 = fma(xc[(long long)(r + 1) * p.ldx], dblk[r + 1], a1);
      }
      if (r < rows) a0 = fma(xc[(long long)r * p.ldx], dblk[r], a0);
      acc[j] += a0 + a1;
    }
    __syncthreads();
  }
  for (int j = t; j < p.k; j += GT) p.part[(long long)blockIdx.x * p.k + j] = acc[j];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    slp += __shfl_down_sync(0xffffffffu, slp, o);
    sda += __shfl_down_sync(0xffffffffu, sda, o);
    sds += __shfl_down_sync(0xffffffffu, sds, o);
  }
  if (lane == 0) {
    red[0][warp] = slp;
    red[1][warp] = sda;
    red[2][warp] = sds;
  }
  __syncthreads();
  if (t < 3) {
    double v = 0.0;
    for (int w = 0; w < GT / 32; ++w) v += red[t][w];
    p.part_s[(long long)kScalars * blockIdx.x + t] = v;
  } else if (t < 3 + p.ncut) {  // ordinal: this CTA's cut sums, rows' threads in order
    const int m = t - 3;
    double v = 0.0;
    for (int r = 0; r < kMaxRowsPerBlock; ++r) v += cut_s[r * kMaxCuts + m];
    p.part_s[(long long)kScalars * blockIdx.x + t] = v;
  }
}

// dbeta_j = sum over CTAs of the partial rows, and the scalars (lp, dalpha,
// dsigma, then the ordinal family's ncut cut derivatives), in CTA order.
__global__ void glm_reduce_kernel(int k, int ctas, int ncut, const double *part, const double *part_s,
                                  double *dbeta, double *lp, double *dalpha, double *dsigma, double *dcuts) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < k) {
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s += part[(long long)c * k + j];
    dbeta[j] = s;
  } else if (j < k + 3 + ncut) {
    const int q = j - k;
    double s = 0.0;
    for (int c = 0; c < ctas; ++c) s += part_s[(long long)kScalars * c + q];
    double *dst = q == 0 ? lp : (q == 1 ? dalpha : (q == 2 ? dsigma : dcuts + (q - 3)));
    if (dst) *dst = s;
  }
}

int rows_per_block(int k) {
  const int r = 16384 / std::max(k, 1);  // about 128 KiB of X per block, re-read from L1/L2
  return std::max(8, std::min(kMaxRowsPerBlock, r / 8 * 8));
}

size_t smem_bytes(int k) {
  return (2 * (size_t)k + 2 * kMaxRowsPerBlock + (size_t)kMaxRowsPerBlock * kMaxCuts) * sizeof(double);
}

int max_ctas(int k) {
  const size_t per = smem_bytes(k) + 1024;
  const int by_smem = (int)std::max<size_t>(1, (size_t)(228 * 1024) / per);
  return sm_count() * std::max(1, std::min(4, by_smem));
}

}  // namespace

size_t glm_workspace_bytes(int k) {
  const size_t ctas = (size_t)max_ctas(k);
  return align_up(ctas * (size_t)std::max(k, 1) * sizeof(double), 256) +
         align_up(ctas * kScalars * sizeof(double), 256);
}

namespace {

cudaError_t glm_launch(GlmParams &p, long long n, int k, double *lp, double *dalpha, double *dbeta, double *dsigma,
                       double *dcuts, void *ws, cudaStream_t s) {
  p.n = n;
  p.k = k;
  p.R = rows_per_block(k);
  const long long nblk = std::max<long long>(1, (n + p.R - 1) / p.R);
  const int ctas = (int)std::min<long long>(nblk, max_ctas(k));
  char *w = (char *)ws;
  p.part = (double *)w;
  p.part_s = (double *)(w + align_up((size_t)max_ctas(k) * (size_t)std::max(k, 1) * sizeof(double), 256));
  const size_t smem = smem_bytes(k);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(glm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const double bytes = 8.0 * ((double)n * k + 2.0 * n + k);
  GPC_LAUNCH(GPC_TRACE_GLM, 4.0 * (double)n * k, bytes, s, glm_kernel<<<ctas, GT, smem, s>>>(p));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int outs = k + 3 + p.ncut;
  GPC_LAUNCH(GPC_TRACE_ELEM, (double)ctas * outs, 8.0 * (double)ctas * outs, s,
             glm_reduce_kernel<<<(outs + 255) / 256, 256, 0, s>>>(k, ctas, p.ncut, p.part, p.part_s, dbeta, lp,
                                                                   dalpha, dsigma, dcuts));
  return cudaGetLastError();
}

GlmParams base_params(int family, long long ldx, const double *X, const double *y, const double *beta) {
  GlmParams p{};
  p.family = family;
  p.ldx = ldx;
  p.X = X;
  p.y = y;
  p.beta = beta;
  p.cuts = nullptr;
  p.ncut = 0;
  p.inv_sigma = 1.0;
  p.log_norm = 0.0;
  return p;
}

}  // namespace

cudaError_t glm(int family, long long n, int k, const double *X, long long ldx, const double *y, double alpha,
                const double *beta, double sigma, double *lp, double *dalpha, double *dbeta, double *dsigma,
                void *ws, cudaStream_t s) {
  GlmParams p = base_params(family, ldx, X, y, beta);
  p.alpha = alpha;
  if (family == GPC_GLM_NORMAL_ID) {
    p.inv_sigma = 1.0 / sigma;
    p.log_norm = log(sigma) + 0.91893853320467274178;
  } else if (family == GPC_GLM_NEG_BINOMIAL_LOG) {
    p.phi = sigma;
    p.log_phi = log(sigma);
    p.lgamma_phi = lgamma(sigma);
  }
  return glm_launch(p, n, k, lp, dalpha, dbeta, dsigma, nullptr, ws, s);
}

cudaError_t glm_ordinal(long long n, int k, int C, const double *X, long long ldx, const double *y,
                        const double *beta, const double *cuts, double *lp, double *dbeta, double *dcuts, void *ws,
                        cudaStream_t s) {
  GlmParams p = base_params(kFamilyOrdinal, ldx, X, y, beta);
  p.alpha = 0.0;  // the cut points take the intercept's place
  p.cuts = cuts;
  p.ncut = C - 1;
  return glm_launch(p, n, k, lp, nullptr, dbeta, nullptr, dcuts, ws, s);
}

}  // namespace gpc
