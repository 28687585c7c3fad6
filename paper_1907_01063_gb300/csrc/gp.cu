// Gaussian-process pieces around the factorisation: squared-exponential
// covariance build, triangular solves, log-likelihood reduction, the upstream
// adjoint Lbar and the hyperparameter gradient (GP regression of Section 4.2;
// triangular solves of Section 3.2).
#include "common.cuh"
#include "df.cuh"

namespace gpc {
namespace {

constexpr int CT = 32;  // covariance / gradient tile (CT x CT entries per CTA)

__device__ __forceinline__ void tri_tile(long long x, int &ti, int &tj) {
  long long t = (long long)((sqrt(8.0 * (double)x + 1.0) - 1.0) * 0.5);
  while ((t + 1) * (t + 2) / 2 <= x) ++t;
  while (t * (t + 1) / 2 > x) --t;
  ti = (int)t;
  tj = (int)(x - t * (t + 1) / 2);
}

// ---------------------------------------------------------------- covariance
__global__ void __launch_bounds__(256)
se_cov_kernel(int n, int d, const double *X, long long ldx, double a2, double inv2r2,
              double diagv, double *K, long long ldk, int full) {
  extern __shared__ double xs[];  // [2][CT][d]
  double *xi = xs, *xj = xs + CT * d;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = ti * CT, j0 = tj * CT;
  for (int idx = threadIdx.x; idx < CT * d; idx += blockDim.x) {
    const int r = idx / d, t = idx - r * d;
    xi[idx] = (i0 + r < n) ? X[(long long)(i0 + r) * ldx + t] : 0.0;
    xj[t * CT + r] = (j0 + r < n) ? X[(long long)(j0 + r) * ldx + t] : 0.0;  // dimension-major: no bank conflicts
  }
  __syncthreads();
  const int c = threadIdx.x & (CT - 1);
  const int j = j0 + c;
  for (int r = threadIdx.x >> 5; r < CT; r += blockDim.x >> 5) {
    const int i = i0 + r;
    if (i >= n || j >= n || j > i) continue;
    double v;
    if (i == j) {
      v = a2 + diagv;
    } else {
      double r2 = 0.0;
      for (int t = 0; t < d; ++t) {
        const double df = xi[r * d + t] - xj[t * CT + c];
        r2 = fma(df, df, r2);
      }
      v = a2 * exp(-r2 * inv2r2);
    }
    K[(long long)i * ldk + j] = v;
    if (full && i != j) K[(long long)j * ldk + i] = v;
  }
}

// Mixed-precision covariance: the same matrix with r^2 and the exponential in
// double-float arithmetic (FP32 pairs, about 2^-46 relative per entry; see
// df.cuh) and one conversion to FP64 per entry.  Entries with
// r^2 / (2 rho^2) > 80 (below 2^-115 alpha^2) take FP64's exp instead.
// xi: the row's d coordinates (contiguous); xj: the column's, d apart by CT
// (the tile's column coordinates are stored dimension-major so that the 32
// lanes of a warp read 32 consecutive entries)
__device__ __forceinline__ dfa::df se_r2_df(const dfa::df *xi, const dfa::df *xj, int d) {
  dfa::df r2 = {0.0f, 0.0f};
  for (int t = 0; t < d; ++t) {
    const dfa::df df_ = dfa::add(xi[t], dfa::neg(xj[t * CT]));
    r2 = dfa::add_same_sign(r2, dfa::mul(df_, df_));
  }
  return r2;
}

// FP64 -> double-float pair by field moves (the same pair as dfa::from_double)
__device__ __forceinline__ dfa::df df_of(double x) {
  const float2 v = split_f64(x);
  return dfa::df{v.x, v.y};
}

__global__ void __launch_bounds__(256)
se_cov_df_kernel(int n, int d, const double *X, long long ldx, double a2, dfa::df inv2r2, double diagv,
                 double *K, long long ldk, int full) {
  extern __shared__ double xs_raw[];  // [2][CT][d] double-floats
  dfa::df *xi = (dfa::df *)xs_raw, *xj = xi + CT * d;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = ti * CT, j0 = tj * CT;
  for (int idx = threadIdx.x; idx < CT * d; idx += blockDim.x) {
    const int r = idx / d, t = idx - r * d;
    xi[idx] = df_of((i0 + r < n) ? X[(long long)(i0 + r) * ldx + t] : 0.0);
    xj[t * CT + r] = df_of((j0 + r < n) ? X[(long long)(j0 + r) * ldx + t] : 0.0);
  }
  __syncthreads();
  const int c = threadIdx.x & (CT - 1);
  const int j = j0 + c;
  for (int r = threadIdx.x >> 5; r < CT; r += blockDim.x >> 5) {
    const int i = i0 + r;
    if (i >= n || j >= n || j > i) continue;
    double v;
    if (i == j) {
      v = a2 + diagv;
    } else {
      const dfa::df t = dfa::mul(se_r2_df(xi + r * d, xj + c, d), inv2r2);
      if (t.hi <= 80.0f) {
        int k;
        const dfa::df m = dfa::exp_neg(t, k);
        // (hi + lo) a2 2^k: the conversions and the power of two by field
        // moves (exact), one FP64 add and one multiply
        const int ea = (int)((unsigned long long)__double_as_longlong(a2) >> 52) & 0x7FF;
        const double a2k = (ea > 116 && ea < 2047)  // a2 and a2 2^k normal (k >= -116)
                               ? __longlong_as_double(__double_as_longlong(a2) + ((long long)k << 52))
                               : a2 * dfa::pow2(k);
        v = (exact_f64(m.hi) + exact_f64(m.lo)) * a2k;
      } else {
        v = a2 * exp(-dfa::to_double(t));
      }
    }
    K[(long long)i * ldk + j] = v;
    if (full && i != j) K[(long long)j * ldk + i] = v;
  }
}

__device__ __forceinline__ double block_sum_256(double v, double *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) s += red[k];
  return s;  // valid in thread 0
}

__global__ void __launch_bounds__(256)
se_hyper_grad_kernel(int n, int d, const double *X, long long ldx, double alpha, double rho,
                     double sigma, const double *Kbar, long long ldkb, double *partial) {
  extern __shared__ double xs[];
  __shared__ double red[8];
  double *xi = xs, *xj = xs + CT * d;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = ti * CT, j0 = tj * CT;
  for (int idx = threadIdx.x; idx < CT * d; idx += blockDim.x) {
    const int r = idx / d, t = idx - r * d;
    xi[idx] = (i0 + r < n) ? X[(long long)(i0 + r) * ldx + t] : 0.0;
    xj[t * CT + r] = (j0 + r < n) ? X[(long long)(j0 + r) * ldx + t] : 0.0;  // dimension-major: no bank conflicts
  }
  __syncthreads();
  const double a2 = alpha * alpha, inv2r2 = 1.0 / (2.0 * rho * rho), inv_r3 = 1.0 / (rho * rho * rho);
  const int c = threadIdx.x & (CT - 1);
  const int j = j0 + c;
  double ga = 0.0, gr = 0.0, gs = 0.0;
  for (int r = threadIdx.x >> 5; r < CT; r += blockDim.x >> 5) {
    const int i = i0 + r;
    if (i >= n || j >= n || j > i) continue;
    double r2 = 0.0;
    for (int t = 0; t < d; ++t) {
      const double df = xi[r * d + t] - xj[t * CT + c];
      r2 = fma(df, df, r2);
    }
    const double kf = a2 * exp(-r2 * inv2r2);
    const double kb = Kbar[(long long)i * ldkb + j];
    ga = fma(kb, 2.0 * kf / alpha, ga);
    gr = fma(kb, kf * r2 * inv_r3, gr);
    if (i == j) gs = fma(kb, 2.0 * sigma, gs);
  }
  const double sa = block_sum_256(ga, red);
  const double sr = block_sum_256(gr, red);
  const double ss = block_sum_256(gs, red);
  if (threadIdx.x == 0) {
    partial[3 * (size_t)blockIdx.x + 0] = sa;
    partial[3 * (size_t)blockIdx.x + 1] = sr;
    partial[3 * (size_t)blockIdx.x + 2] = ss;
  }
}

// Mixed-precision hyperparameter gradient: the sums sum Kbar_ij e_ij and
// sum Kbar_ij e_ij r2_ij (e_ij = exp(-r2_ij / (2 rho^2))) are accumulated per
// thread in double-float (a running FP32 sum of the terms' high parts with
// the two-sum errors and the low parts collected beside it), then reduced in
// FP64; partial = (2 alpha S_e,
// alpha^2 / rho^3 S_er, 2 sigma sum Kbar_ii) per tile as in the FP64 kernel.
__global__ void __launch_bounds__(256)
se_hyper_grad_df_kernel(int n, int d, const double *X, long long ldx, double alpha, double rho,
                        double sigma, dfa::df inv2r2, const double *Kbar, long long ldkb, double *partial) {
  extern __shared__ double xs_raw[];
  __shared__ double red[8];
  dfa::df *xi = (dfa::df *)xs_raw, *xj = xi + CT * d;
  int ti, tj;
  tri_tile(blockIdx.x, ti, tj);
  const int i0 = ti * CT, j0 = tj * CT;
  for (int idx = threadIdx.x; idx < CT * d; idx += blockDim.x) {
    const int r = idx / d, t = idx - r * d;
    xi[idx] = df_of((i0 + r < n) ? X[(long long)(i0 + r) * ldx + t] : 0.0);
    xj[t * CT + r] = df_of((j0 + r < n) ? X[(long long)(j0 + r) * ldx + t] : 0.0);
  }
  __syncthreads();
  const int c = threadIdx.x & (CT - 1);
  const int j = j0 + c;
  // the two sums as running FP32 sums with their two-sum errors beside them
  float seS = 0.0f, seE = 0.0f, serS = 0.0f, serE = 0.0f;
  auto acc = [](float &S, float &E, dfa::df w) {
    const dfa::df u = dfa::two_sum(S, w.hi);
    S = u.hi;
    E = __fadd_rn(E, __fadd_rn(u.lo, w.lo));
  };
  double big_e = 0.0, big_er = 0.0, gs = 0.0;  // entries past the double-float range, in FP64
  for (int r = threadIdx.x >> 5; r < CT; r += blockDim.x >> 5) {
    const int i = i0 + r;
    if (i >= n || j >= n || j > i) continue;
    const double kb = Kbar[(long long)i * ldkb + j];
    if (i == j) {
      const float2 kd = split_f64(kb);
      acc(seS, seE, dfa::df{kd.x, kd.y});  // e_ii = 1, r2_ii = 0
      gs = fma(kb, 2.0 * sigma, gs);
      continue;
    }
    const dfa::df r2 = se_r2_df(xi + r * d, xj + c, d);
    const dfa::df t = dfa::mul(r2, inv2r2);
    if (t.hi <= 80.0f) {
      int k;
      const dfa::df m = dfa::exp_neg(t, k);
      const float sc = __int_as_float((k + 127) << 23);  // 2^k, k >= -116
      const dfa::df e = {m.hi * sc, m.lo * sc};
      const float2 kd = split_f64(kb);
      const dfa::df w = dfa::mul(dfa::df{kd.x, kd.y}, e);
      acc(seS, seE, w);
      acc(serS, serE, dfa::mul(w, r2));
    } else {
      const double r2d = dfa::to_double(r2);
      const double w = kb * exp(-dfa::to_double(t));
      big_e += w;
      big_er = fma(w, r2d, big_er);
    }
  }
  const double a2 = alpha * alpha, inv_r3 = 1.0 / (rho * rho * rho);
  const double ga = 2.0 * alpha * (((double)seS + (double)seE) + big_e);
  const double gr = a2 * inv_r3 * (((double)serS + (double)serE) + big_er);
  const double sa = block_sum_256(ga, red);
  const double sr = block_sum_256(gr, red);
  const double ss = block_sum_256(gs, red);
  if (threadIdx.x == 0) {
    partial[3 * (size_t)blockIdx.x + 0] = sa;
    partial[3 * (size_t)blockIdx.x + 1] = sr;
    partial[3 * (size_t)blockIdx.x + 2] = ss;
  }
}

__global__ void __launch_bounds__(256)
sum3_kernel(const double *partial, long long count, double *out) {
  __shared__ double red[8];
  double a = 0.0, b = 0.0, c = 0.0;
  for (long long k = threadIdx.x; k < count; k += blockDim.x) {
    a += partial[3 * k + 0];
    b += partial[3 * k + 1];
    c += partial[3 * k + 2];
  }
  const double sa = block_sum_256(a, red);
  const double sb = block_sum_256(b, red);
  const double sc = block_sum_256(c, red);
  if (threadIdx.x == 0) {
    out[0] = sa;
    out[1] = sb;
    out[2] = sc;
  }
}

// ---------------------------------------------------------------- triangular solve
// One CTA per 64-row block of the solve.  CTAs take their block from a ticket
// counter in launch order, so a CTA only ever waits on blocks owned by CTAs
// that started before it.  Each finished block publishes a ready flag (1 =
// solved, 2 = gave up); every wait is bounded and a timeout is reported as
// GPC_ERR_TIMEOUT and propagated to later blocks as flag 2.
constexpr int TB = 64;

__device__ __forceinline__ int ld_volatile(const int *p) { return *(const volatile int *)p; }
__device__ __forceinline__ unsigned long long clock_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait until *flag is non-zero (value receives it) or wait_ns of %globaltimer
// have passed (returns false).
__device__ __forceinline__ bool wait_flag(const int *flag, int &value, unsigned long long wait_ns) {
  const unsigned long long t0 = clock_ns();
  for (unsigned it = 0;; ++it) {
    value = ld_volatile(flag);
    if (value != 0) return true;
    if ((it & 255) == 255 && clock_ns() - t0 > wait_ns) return false;
    if (it > 1024) __nanosleep(32);
  }
}

// The same wait with an acquire load: the block's other threads, released by
// the barrier that follows, see everything the flag's writer published.
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ bool wait_flag_acquire(const int *flag, int &value, unsigned long long wait_ns) {
  const unsigned long long t0 = clock_ns();
  for (unsigned it = 0;; ++it) {
    value = ld_acquire(flag);
    if (value != 0) return true;
    if ((it & 255) == 255 && clock_ns() - t0 > wait_ns) return false;
    if (it > 1024) __nanosleep(32);
  }
}
// Publish a flag after a barrier: the acquire-release fence makes the writes
// of every thread of the block that reached the barrier visible before it.
__device__ __forceinline__ void publish_flag(int *p, int v) {
  asm volatile("fence.acq_rel.gpu;\n\tst.relaxed.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// withhold >= 0 (test hook): the block with that index in solve order computes
// its rows but never publishes its ready flag.
__global__ void __launch_bounds__(256)
trsv_kernel(int n, const double *L, long long ldl, double *x, int trans, int *sync, int *info,
            const int *skip, int *gerr, unsigned long long wait_ns, int withhold) {
  if (skip && *skip) return;  // the same value for every CTA: nothing waits on anything
  __shared__ int s_order, s_abort;
  __shared__ double diag[TB][TB + 1];
  __shared__ double red[4][TB];
  __shared__ double rhs[TB];
  const int nblk = (n + TB - 1) / TB;
  if (threadIdx.x == 0) {
    s_order = atomicAdd(&sync[0], 1);
    s_abort = 0;
  }
  __syncthreads();
  const int order = s_order;
  const int blk = trans ? (nblk - 1 - order) : order;
  const int b0 = blk * TB, nb = min(TB, n - b0);
  const int q = threadIdx.x & 63, rg = threadIdx.x >> 6;
  double acc[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) acc[r] = 0.0;

  for (int step = 0; step < order; ++step) {
    const int c = trans ? (nblk - 1 - step) : step;
    if (threadIdx.x == 0) {
      int f;
      if (!wait_flag(&sync[1 + c], f, wait_ns) || f != 1) s_abort = 1;
      __threadfence();
    }
    __syncthreads();
    if (s_abort) break;
    const int c0 = c * TB, cn = min(TB, n - c0);
    if (!trans) {
      if (q < cn) {
        const double xq = __ldcg(&x[c0 + q]);
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const int row = rg * 16 + rr;
          if (row < nb) acc[rr] = fma(L[(long long)(b0 + row) * ldl + c0 + q], xq, acc[rr]);
        }
      }
    } else {
      if (q < nb) {
#pragma unroll
        for (int rr = 0; rr < 16; ++rr) {
          const int r = rg * 16 + rr;
          if (r < cn) acc[0] = fma(L[(long long)(c0 + r) * ldl + b0 + q], __ldcg(&x[c0 + r]), acc[0]);
        }
      }
    }
  }
  if (s_abort) {
    if (threadIdx.x == 0) {
      if (info && info[1] == 0) info[1] = GPC_ERR_TIMEOUT;
      record_error(gerr, GPC_ERR_TIMEOUT);
      __threadfence();
      if (order != withhold) atomicExch(&sync[1 + blk], 2);
    }
    return;
  }

  // Reduce the partial products of this block.
  if (!trans) {
    // rows rg*16 + rr, summed over q (two warps per row group)
    const int w = (threadIdx.x >> 5) & 1, l = threadIdx.x & 31;
#pragma unroll
    for (int rr = 0; rr < 16; ++rr) {
      double v = acc[rr];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (l == 0) red[w][rg * 16 + rr] = v;
    }
    __syncthreads();
    if (threadIdx.x < TB) {
      const int r = threadIdx.x;
      rhs[r] = (r < nb) ? x[b0 + r] - (red[0][r] + red[1][r]) : 0.0;
    }
  } else {
    red[rg][q] = acc[0];
    __syncthreads();
    if (threadIdx.x < TB) {
      const int r = threadIdx.x;
      rhs[r] = (r < nb) ? x[b0 + r] - ((red[0][r] + red[1][r]) + (red[2][r] + red[3][r])) : 0.0;
    }
  }
  for (int idx = threadIdx.x; idx < TB * TB; idx += blockDim.x) {
    const int i = idx >> 6, j = idx & 63;
    diag[i][j] = (i < nb && j < nb) ? L[(long long)(b0 + i) * ldl + b0 + j] : 0.0;
  }
  __syncthreads();

  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    double v0 = rhs[lane], v1 = rhs[lane + 32];
    if (!trans) {
      for (int k = 0; k < nb; ++k) {
        const double vk = (k < 32) ? __shfl_sync(0xffffffffu, v0, k) : __shfl_sync(0xffffffffu, v1, k - 32);
        const double zk = vk / diag[k][k];
        if (lane > k) v0 = fma(-diag[lane][k], zk, v0);
        if (lane + 32 > k) v1 = fma(-diag[lane + 32][k], zk, v1);
        if (lane == k) v0 = zk;
        if (lane + 32 == k) v1 = zk;
      }
    } else {
      for (int k = nb - 1; k >= 0; --k) {
        const double vk = (k < 32) ? __shfl_sync(0xffffffffu, v0, k) : __shfl_sync(0xffffffffu, v1, k - 32);
        const double zk = vk / diag[k][k];
        if (lane < k) v0 = fma(-diag[k][lane], zk, v0);
        if (lane + 32 < k) v1 = fma(-diag[k][lane + 32], zk, v1);
        if (lane == k) v0 = zk;
        if (lane + 32 == k) v1 = zk;
      }
    }
    if (lane < nb) x[b0 + lane] = v0;
    if (lane + 32 < nb) x[b0 + lane + 32] = v1;
    __threadfence();
    __syncwarp();
    if (lane == 0 && order != withhold) atomicExch(&sync[1 + blk], 1);
  }
}

// Blocked solve with the diagonal-block inverses the factorisation kept (the
// paper's solve through the inverse, Section 3.2, applied block by block):
//   forward   x_I = Dinv_I (y_I - L[I, <I] x_<I)
//   transpose x_I = Dinv_I^T (z_I - L[>I, I]^T x_>I)
// Blocks are b rows from the top (the last may be shorter); Dinv_I is at
// inv + I b^2 with leading dimension equal to the block size.  Same ticket
// order, ready flags and bounded waits as trsv_kernel.

// Latency matters more than bandwidth here: every block waits for the one
// before it, and on GB300 each dependent FP64 instruction costs about 64
// cycles.  So the solve runs on sub-blocks of at most 64 rows (half a
// factorisation block; the inverse of a diagonal sub-block is the matching
// diagonal sub-block of the stored block inverse), with 256 threads as 64 rows
// x 4 column quarters and no cross-lane FP64 reductions: each CTA loads its
// sub-block inverse into shared memory at start, keeps the next L slice in
// registers while it waits for the previous sub-block's flag, and after the
// last flag only a 16-term product per thread, two four-way sums through
// shared memory and the 16-term product with the inverse remain.  The abort
// word is double-buffered by step parity so that a CTA's thread 0 can record a
// failed wait while slower warps still read the previous step's.
constexpr int TS = 64, TQ = 4, TW = TS / TQ;

__global__ void __launch_bounds__(256)
trsv_inv_kernel(int n, const double *L, long long ldl, const double *inv, int b, int sb, double *x, int trans,
                int *sync, int *info, const int *skip, int *gerr, unsigned long long wait_ns) {
  if (skip && *skip) return;
  __shared__ double dinv_s[TS][TS + 1];
  __shared__ int s_order, s_ab[2];
  __shared__ double vbuf[TS], xs[TS];
  __shared__ double red[TQ][TS];
  const int nsb = (n + sb - 1) / sb;
  if (threadIdx.x == 0) {
    s_order = atomicAdd(&sync[0], 1);
    s_ab[0] = s_ab[1] = 0;
  }
  __syncthreads();
  const int order = s_order;
  const int sbk = trans ? (nsb - 1 - order) : order;
  const int i0 = sbk * sb, nb = min(sb, n - i0);
  {
    const int B = i0 / b, off = i0 - B * b, nbB = min(b, n - B * b);
    const double *Dinv = inv + (size_t)B * b * b + (size_t)off * nbB + off;  // leading dimension nbB
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int rr = idx / nb, kk = idx - rr * nb;
      dinv_s[rr][kk] = __ldg(Dinv + (size_t)rr * nbB + kk);
    }
  }
  const int r = threadIdx.x % TS, q = threadIdx.x / TS;
  bool aborted = false;
  double acc = 0.0, lv[TW];
  // this sub-block's right-hand side, read now so that no global load is left
  // on the chain after the last wait
  const double rhs = (q == 0 && r < nb) ? x[i0 + r] : 0.0;

  if (!trans) {
    // lv[u] = L[i0 + r][c0 + q TW + u] for the next sub-block c
#pragma unroll
    for (int u = 0; u < TW; ++u) {
      const int k = q * TW + u;
      lv[u] = (sbk > 0 && r < nb && k < sb) ? __ldg(L + (long long)(i0 + r) * ldl + k) : 0.0;
    }
    for (int c = 0; c < sbk; ++c) {
      if (threadIdx.x == 0) {
        int f;
        if (!wait_flag(&sync[1 + c], f, wait_ns) || f != 1) s_ab[c & 1] = 1;
        __threadfence();
      }
      __syncthreads();
      if (s_ab[c & 1]) {
        aborted = true;
        break;
      }
      const int c0 = c * sb;  // c < sbk: a full sub-block
      double p[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int u = 0; u < TW; ++u) {
        const int k = q * TW + u;
        const double xv = (k < sb) ? __ldcg(&x[c0 + k]) : 0.0;
        p[u & 3] = fma(lv[u], xv, p[u & 3]);
      }
      acc += (p[0] + p[1]) + (p[2] + p[3]);
      if (c + 1 < sbk) {
        const int c1 = c0 + sb;
#pragma unroll
        for (int u = 0; u < TW; ++u) {
          const int k = q * TW + u;
          lv[u] = (r < nb && k < sb) ? __ldg(L + (long long)(i0 + r) * ldl + c1 + k) : 0.0;
        }
      }
    }
    red[q][r] = acc;
    __syncthreads();  // red and dinv_s complete
    if (!aborted && q == 0 && r < nb) vbuf[r] = rhs - ((red[0][r] + red[1][r]) + (red[2][r] + red[3][r]));
    __syncthreads();
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    if (!aborted && r < nb) {
#pragma unroll
      for (int u = 0; u < TW; ++u) {
        const int k = q * TW + u;
        if (k <= r) p[u & 3] = fma(dinv_s[r][k], vbuf[k], p[u & 3]);
      }
    }
    red[q][r] = (p[0] + p[1]) + (p[2] + p[3]);
    __syncthreads();
    if (!aborted && q == 0 && r < nb) {
      x[i0 + r] = (red[0][r] + red[1][r]) + (red[2][r] + red[3][r]);
      __threadfence();
    }
  } else {
    // thread (i = r, row quarter q): lv[u] = L[c0 + q TW + u][i0 + i] for the next sub-block c below
    {
      const int c0 = (nsb - 1) * sb, cn = n - c0;
#pragma unroll
      for (int u = 0; u < TW; ++u) {
        const int k = q * TW + u;
        lv[u] = (order > 0 && r < nb && k < cn) ? __ldg(L + (long long)(c0 + k) * ldl + i0 + r) : 0.0;
      }
    }
    for (int step = 0; step < order; ++step) {
      const int c = nsb - 1 - step;
      if (threadIdx.x == 0) {
        int f;
        if (!wait_flag(&sync[1 + c], f, wait_ns) || f != 1) s_ab[step & 1] = 1;
        __threadfence();
      }
      __syncthreads();
      if (s_ab[step & 1]) {
        aborted = true;
        break;
      }
      const int c0 = c * sb, cn = min(sb, n - c0);
      if (threadIdx.x < TS) xs[threadIdx.x] = threadIdx.x < cn ? __ldcg(&x[c0 + threadIdx.x]) : 0.0;
      __syncthreads();
      double p[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int u = 0; u < TW; ++u) p[u & 3] = fma(lv[u], xs[q * TW + u], p[u & 3]);
      acc += (p[0] + p[1]) + (p[2] + p[3]);
      if (step + 1 < order) {
        const int p0 = c0 - sb;  // the next sub-block up is a full one
#pragma unroll
        for (int u = 0; u < TW; ++u) {
          const int k = q * TW + u;
          lv[u] = (r < nb && k < sb) ? __ldg(L + (long long)(p0 + k) * ldl + i0 + r) : 0.0;
        }
      }
    }
    red[q][r] = acc;
    __syncthreads();  // red and dinv_s complete
    if (!aborted && q == 0 && r < nb) vbuf[r] = rhs - ((red[0][r] + red[1][r]) + (red[2][r] + red[3][r]));
    __syncthreads();
    double p[4] = {0.0, 0.0, 0.0, 0.0};
    if (!aborted && r < nb) {
#pragma unroll
      for (int u = 0; u < TW; ++u) {
        const int k = q * TW + u;
        if (k >= r && k < nb) p[u & 3] = fma(dinv_s[k][r], vbuf[k], p[u & 3]);
      }
    }
    red[q][r] = (p[0] + p[1]) + (p[2] + p[3]);
    __syncthreads();
    if (!aborted && q == 0 && r < nb) {
      x[i0 + r] = (red[0][r] + red[1][r]) + (red[2][r] + red[3][r]);
      __threadfence();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (aborted && info && info[1] == 0) info[1] = GPC_ERR_TIMEOUT;
    if (aborted) record_error(gerr, GPC_ERR_TIMEOUT);
    __threadfence();
    atomicExch(&sync[1 + sbk], aborted ? 2 : 1);
  }
}

// The same blocked solve in double-float arithmetic, for the mixed path: its
// initial solve and its refinement corrections.  There the factor's own error
// (split-BF16 trailing updates) is far above the 2^-44 or so that a
// double-float solve adds, and the FP64 residual of the refinement removes
// both, so the correction solves need not run on the FP64 pipe, which on this
// part issues about one warp instruction per 64 cycles per sub-partition.  L
// is read from a copy already split into FP32 pairs (Ld: hi = nearest FP32,
// lo = nearest FP32 to the remainder; one conversion pass per factor, reused
// by every solve), the sub-block inverses are split as they are loaded.
// Every product l x = (lh + ll)(xh + xl) keeps lh xh exactly (FMA
// two-product) plus the cross terms lh xl + ll xh, and the sums are kept as a
// running FP32 sum with its two-sum errors collected beside it (renormalised
// every few sub-blocks).  Solved sub-blocks are published to the later ones
// as FP32 pairs in xdf (n pairs, 8-byte aligned) behind an acquire/release
// flag; x receives hi + lo in FP64.  Measured at n = 16384 (mixed factor):
// forward 0.82 ms and transposed 0.74 ms against about 1.4-1.8 ms each for
// the FP64 kernel; reading L as FP64 and splitting it in the loop left each
// CTA's walk over the earlier sub-blocks instruction-bound (about 1000
// instructions per warp and sub-block, 10-13 us per step).
__device__ __forceinline__ void df_dot_term(float2 l, float2 v, float &S, float &E) {
  const float ph = __fmul_rn(l.x, v.x);
  float pl = __fmaf_rn(l.x, v.x, -ph);
  pl = __fmaf_rn(l.x, v.y, pl);
  pl = __fmaf_rn(l.y, v.x, pl);
  const dfa::df t = dfa::two_sum(S, ph);
  S = t.hi;
  E = __fadd_rn(E, __fadd_rn(t.lo, pl));
}

__global__ void __launch_bounds__(256)
trsv_inv_df_kernel(int n, const float2 *Ld, long long ldd, const double *inv, int b, int sb, double *x,
                   float2 *xdf, int trans, int *sync, int *info, const int *skip, int *gerr,
                   unsigned long long wait_ns) {
  if (skip && *skip) return;
  __shared__ float2 dinv_s[TS][TS + 1];
  __shared__ int s_order, s_ab[2];
  __shared__ float2 vbuf[TS], xs[TS];
  __shared__ float2 red[TQ][TS];
  const int nsb = (n + sb - 1) / sb;
  if (threadIdx.x == 0) {
    s_order = atomicAdd(&sync[0], 1);
    s_ab[0] = s_ab[1] = 0;
  }
  __syncthreads();
  const int order = s_order;
  const int sbk = trans ? (nsb - 1 - order) : order;
  const int i0 = sbk * sb, nb = min(sb, n - i0);
  {
    const int B = i0 / b, off = i0 - B * b, nbB = min(b, n - B * b);
    const double *Dinv = inv + (size_t)B * b * b + (size_t)off * nbB + off;  // leading dimension nbB
    for (int idx = threadIdx.x; idx < nb * nb; idx += blockDim.x) {
      const int rr = idx / nb, kk = idx - rr * nb;
      dinv_s[rr][kk] = split_f64(__ldg(Dinv + (size_t)rr * nbB + kk));
    }
  }
  const int r = threadIdx.x % TS, q = threadIdx.x / TS;
  bool aborted = false;
  float S = 0.f, E = 0.f;
  float2 lv[TW];
  const float2 rhs = (q == 0 && r < nb) ? split_f64(x[i0 + r]) : make_float2(0.f, 0.f);
  const float2 zero2 = make_float2(0.f, 0.f);

  if (!trans) {
    // Thread (column kk of the sub-block, row quarter rq) keeps one partial
    // sum per row rq TW + rr over its column, so that a warp reads 32
    // consecutive entries of a row of L; the 64 column partials of every row
    // meet in shared memory after the last flag.
    extern __shared__ float2 part[];  // [TS][TS + 1]
    const int kk = threadIdx.x % TS, rq = threadIdx.x / TS;
    float aS[TW], aE[TW];
#pragma unroll
    for (int rr = 0; rr < TW; ++rr) {
      aS[rr] = aE[rr] = 0.f;
      const int row = rq * TW + rr;
      lv[rr] = (sbk > 0 && row < nb && kk < sb) ? __ldg(Ld + (long long)(i0 + row) * ldd + kk) : zero2;
    }
    for (int c = 0; c < sbk; ++c) {
      if (threadIdx.x == 0) {
        int f;
        if (!wait_flag_acquire(&sync[1 + c], f, wait_ns) || f != 1) s_ab[c & 1] = 1;
      }
      __syncthreads();
      if (s_ab[c & 1]) {
        aborted = true;
        break;
      }
      const int c0 = c * sb;  // c < sbk: a full sub-block
      const float2 xk = kk < sb ? __ldcg(&xdf[c0 + kk]) : zero2;
#pragma unroll
      for (int rr = 0; rr < TW; ++rr) df_dot_term(lv[rr], xk, aS[rr], aE[rr]);
      if ((c & 15) == 15) {
#pragma unroll
        for (int rr = 0; rr < TW; ++rr) {
          const dfa::df t = dfa::two_sum(aS[rr], aE[rr]);
          aS[rr] = t.hi;
          aE[rr] = t.lo;
        }
      }
      if (c + 1 < sbk) {
        const int c1 = c0 + sb;
#pragma unroll
        for (int rr = 0; rr < TW; ++rr) {
          const int row = rq * TW + rr;
          lv[rr] = (row < nb && kk < sb) ? __ldg(Ld + (long long)(i0 + row) * ldd + c1 + kk) : zero2;
        }
      }
    }
#pragma unroll
    for (int rr = 0; rr < TW; ++rr) {
      const dfa::df t = dfa::two_sum(aS[rr], aE[rr]);
      part[(rq * TW + rr) * (TS + 1) + kk] = make_float2(t.hi, t.lo);
    }
    __syncthreads();
    // thread (r, q): row r's partials of columns q TW .. q TW + TW - 1
    float S1 = 0.f, E1 = 0.f;
#pragma unroll
    for (int u = 0; u < TW; u += 2) {
      const float2 p0 = part[r * (TS + 1) + q * TW + u], p1 = part[r * (TS + 1) + q * TW + u + 1];
      dfa::df t = dfa::two_sum(S, p0.x);
      S = t.hi;
      E = __fadd_rn(E, __fadd_rn(t.lo, p0.y));
      t = dfa::two_sum(S1, p1.x);
      S1 = t.hi;
      E1 = __fadd_rn(E1, __fadd_rn(t.lo, p1.y));
    }
    const dfa::df t = dfa::two_sum(S, S1);
    const dfa::df u2 = dfa::two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(E, E1)));
    S = u2.hi;
    E = u2.lo;
  } else {
    // thread (i = r, row quarter q): lv[u] = Ld[c0 + q TW + u][i0 + i] for the next sub-block c below
    {
      const int c0 = (nsb - 1) * sb, cn = n - c0;
#pragma unroll
      for (int u = 0; u < TW; ++u) {
        const int k = q * TW + u;
        lv[u] = (order > 0 && r < nb && k < cn) ? __ldg(Ld + (long long)(c0 + k) * ldd + i0 + r) : zero2;
      }
    }
    for (int step = 0; step < order; ++step) {
      const int c = nsb - 1 - step;
      if (threadIdx.x == 0) {
        int f;
        if (!wait_flag_acquire(&sync[1 + c], f, wait_ns) || f != 1) s_ab[step & 1] = 1;
      }
      __syncthreads();
      if (s_ab[step & 1]) {
        aborted = true;
        break;
      }
      const int c0 = c * sb, cn = min(sb, n - c0);
      if (threadIdx.x < TS) xs[threadIdx.x] = threadIdx.x < cn ? __ldcg(&xdf[c0 + threadIdx.x]) : zero2;
      __syncthreads();
      float S1 = 0.f, E1 = 0.f;
#pragma unroll
      for (int u = 0; u < TW; u += 2) {
        df_dot_term(lv[u], xs[q * TW + u], S, E);
        df_dot_term(lv[u + 1], xs[q * TW + u + 1], S1, E1);
      }
      {
        const dfa::df t = dfa::two_sum(S, S1);
        const dfa::df u2 = dfa::two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(E, E1)));
        S = u2.hi;
        E = u2.lo;
      }
      if (step + 1 < order) {
        const int p0 = c0 - sb;  // the next sub-block up is a full one
#pragma unroll
        for (int u = 0; u < TW; ++u) {
          const int k = q * TW + u;
          lv[u] = (r < nb && k < sb) ? __ldg(Ld + (long long)(p0 + k) * ldd + i0 + r) : zero2;
        }
      }
    }
  }
  red[q][r] = make_float2(S, E);
  __syncthreads();  // red and dinv_s complete
  if (!aborted && q == 0 && r < nb) {
    const dfa::df a = dfa::add(dfa::df{red[0][r].x, red[0][r].y}, dfa::df{red[1][r].x, red[1][r].y});
    const dfa::df c = dfa::add(dfa::df{red[2][r].x, red[2][r].y}, dfa::df{red[3][r].x, red[3][r].y});
    const dfa::df v = dfa::add(dfa::df{rhs.x, rhs.y}, dfa::neg(dfa::add(a, c)));
    vbuf[r] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  S = 0.f;
  E = 0.f;
  if (!aborted && r < nb) {
    float S1 = 0.f, E1 = 0.f;
    if (!trans) {
#pragma unroll
      for (int u = 0; u < TW; u += 2) {
        const int k = q * TW + u;
        if (k <= r) df_dot_term(dinv_s[r][k], vbuf[k], S, E);
        if (k + 1 <= r) df_dot_term(dinv_s[r][k + 1], vbuf[k + 1], S1, E1);
      }
    } else {
#pragma unroll
      for (int u = 0; u < TW; u += 2) {
        const int k = q * TW + u;
        if (k >= r && k < nb) df_dot_term(dinv_s[k][r], vbuf[k], S, E);
        if (k + 1 >= r && k + 1 < nb) df_dot_term(dinv_s[k + 1][r], vbuf[k + 1], S1, E1);
      }
    }
    const dfa::df t = dfa::two_sum(S, S1);
    S = t.hi;
    E = __fadd_rn(t.lo, __fadd_rn(E, E1));
  }
  red[q][r] = make_float2(S, E);
  __syncthreads();
  if (!aborted && q == 0 && r < nb) {
    const dfa::df a = dfa::add(dfa::df{red[0][r].x, red[0][r].y}, dfa::df{red[1][r].x, red[1][r].y});
    const dfa::df c = dfa::add(dfa::df{red[2][r].x, red[2][r].y}, dfa::df{red[3][r].x, red[3][r].y});
    const dfa::df v = dfa::add(a, c);
    xdf[i0 + r] = make_float2(v.hi, v.lo);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (aborted && info && info[1] == 0) info[1] = GPC_ERR_TIMEOUT;
    if (aborted) record_error(gerr, GPC_ERR_TIMEOUT);
    publish_flag(&sync[1 + sbk], aborted ? 2 : 1);
  }
  // the FP64 result after the flag: nothing in this launch reads x of another sub-block
  if (!aborted && q == 0 && r < nb) {
    const float2 v = xdf[i0 + r];
    x[i0 + r] = exact_f64(v.x) + exact_f64(v.y);
  }
}

// ---------------------------------------------------------------- likelihood pieces
__global__ void __launch_bounds__(256)
lml_finalize_kernel(int n, const double *L, long long ldl, const double *y, const double *alpha,
                    double *logdet, double *value) {
  __shared__ double red[8];
  double ld = 0.0, q = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    ld += log(L[(long long)i * ldl + i]);
    q = fma(y[i], alpha[i], q);
  }
  const double sld = block_sum_256(ld, red);
  const double sq = block_sum_256(q, red);
  if (threadIdx.x == 0) {
    const double lg = 2.0 * sld;
    if (logdet) *logdet = lg;
    if (value) *value = -0.5 * sq - 0.5 * lg - 0.5 * (double)n * 1.8378770664093454835606594728112;
  }
}

constexpr int LTV_ROWS = 256, LTV_COLS = 256;

__global__ void __launch_bounds__(LTV_COLS)
ltv_partial_kernel(int n, const double *L, long long ldl, const double *v, double *partial) {
  const int rc = blockIdx.y, col = blockIdx.x * LTV_COLS + threadIdx.x;
  const int r0 = rc * LTV_ROWS, r1 = min(n, r0 + LTV_ROWS);
  if (col >= n) return;
  double acc = 0.0;
  for (int i = max(r0, col); i < r1; ++i) acc = fma(L[(long long)i * ldl + col], v[i], acc);
  partial[(size_t)rc * n + col] = acc;
}

__global__ void ltv_reduce_kernel(int n, int chunks, const double *partial, double *z) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n) return;
  double s = 0.0;
  for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * n + col];
  z[col] = s;
}

// Lbar = gbar (tril(alpha z^T) - diag(1 / L_ii)), zero strict upper triangle.
// 2-D tiles of 32 rows x 128 columns, 16 entries per thread (4 rows x 4
// columns 32 apart, so every store of a warp covers one contiguous row piece).
// FP64 path: v = alpha_i z_j (one FP64 multiply per lower entry, then gbar).
// Double-float path (the mixed adjoint's input): alpha_i gbar and z_j are
// split into FP32 pairs once per row / column and their product is formed
// with the FMA-based two-product in FP32 arithmetic (about 2^-46 relative),
// so no FP64 instruction runs per entry; the diagonal is formed in FP64.
constexpr int LB_ROWS = 32, LB_COLS = 128;
__global__ void __launch_bounds__(256)
lml_lbar_kernel(int n, const double *L, long long ldl, const double *alpha, const double *z, double gbar,
                double *Lbar, long long ldlb, int df) {
  const int r0 = blockIdx.y * LB_ROWS, c0 = blockIdx.x * LB_COLS;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  if (c0 > r0 + LB_ROWS - 1) {  // tile wholly above the diagonal: zeros
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = r0 + ty + 8 * v;
      if (i >= n) continue;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = c0 + tx + 32 * u;
        if (j < n) Lbar[(long long)i * ldlb + j] = 0.0;
      }
    }
    return;
  }
  if (!df) {
    double zj[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = c0 + tx + 32 * u;
      zj[u] = j < n ? z[j] : 0.0;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = r0 + ty + 8 * v;
      if (i >= n) continue;
      const double ai = alpha[i];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int j = c0 + tx + 32 * u;
        if (j >= n) continue;
        double val = 0.0;
        if (j <= i) {
          val = ai * zj[u];
          if (i == j) val -= 1.0 / L[(long long)i * ldl + i];
          val *= gbar;
        }
        Lbar[(long long)i * ldlb + j] = val;
      }
    }
    return;
  }
  dfa::df zj[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int j = c0 + tx + 32 * u;
    zj[u] = dfa::from_double(j < n ? z[j] : 0.0);
  }
  float2 *out = reinterpret_cast<float2 *>(Lbar);
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const int i = r0 + ty + 8 * v;
    if (i >= n) continue;
    const dfa::df ai = dfa::from_double(alpha[i] * gbar);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int j = c0 + tx + 32 * u;
      if (j >= n) continue;
      float2 val = make_float2(0.f, 0.f);
      if (j < i) {
        const dfa::df p = dfa::mul(ai, zj[u]);
        val = make_float2(p.hi, p.lo);
      } else if (j == i) {
        const double d = (alpha[i] * z[i] - 1.0 / L[(long long)i * ldl + i]) * gbar;
        const dfa::df p = dfa::from_double(d);
        val = make_float2(p.hi, p.lo);
      }
      out[(long long)i * ldlb + j] = val;
    }
  }
}

bool g_attr[64][5];

cudaError_t set_dyn_smem(const void *fn, int which) {
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) return cudaSuccess;
  if (g_attr[dev][which]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       2 * CT * kMaxDim * (int)sizeof(double));
  if (e == cudaSuccess) g_attr[dev][which] = true;
  return e;
}

dfa::df host_df(double v) {
  const float h = (float)v;
  return dfa::df{h, (float)(v - (double)h)};
}

}  // namespace

cudaError_t se_cov(int n, int d, const double *X, long long ldx, double alpha, double rho,
                   double sigma, double jitter, double *K, long long ldk, int full, bool mixed,
                   cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  cudaError_t e = mixed ? set_dyn_smem((const void *)se_cov_df_kernel, 2)
                        : set_dyn_smem((const void *)se_cov_kernel, 0);
  if (e != cudaSuccess) return e;
  const long long T = (n + CT - 1) / CT;
  const size_t smem = 2 * CT * (size_t)d * sizeof(double);
  const double tri = 0.5 * (double)n * (n + 1);
  const double inv2r2 = 1.0 / (2.0 * rho * rho);
  if (mixed) {
    GPC_LAUNCH(GPC_TRACE_SECOV, tri * 3.0 * d, 8.0 * (full ? 2.0 * tri - n : tri) + 8.0 * n * d, s,
               se_cov_df_kernel<<<(unsigned)(T * (T + 1) / 2), 256, smem, s>>>(
                   n, d, X, ldx, alpha * alpha, host_df(inv2r2), sigma * sigma + jitter, K, ldk, full));
  } else {
    GPC_LAUNCH(GPC_TRACE_SECOV, tri * 3.0 * d, 8.0 * (full ? 2.0 * tri - n : tri) + 8.0 * n * d, s,
               se_cov_kernel<<<(unsigned)(T * (T + 1) / 2), 256, smem, s>>>(
                   n, d, X, ldx, alpha * alpha, inv2r2, sigma * sigma + jitter, K, ldk, full));
  }
  return cudaGetLastError();
}

size_t se_hyper_grad_workspace_bytes(int n) {
  const long long T = (n + CT - 1) / CT;
  return align_up((size_t)(T * (T + 1) / 2) * 3 * sizeof(double), 256);
}

cudaError_t se_hyper_grad(int n, int d, const double *X, long long ldx, double alpha, double rho,
                          double sigma, const double *Kbar, long long ldkb, double *grad3,
                          void *ws, bool mixed, cudaStream_t s) {
  if (n <= 0) return cudaMemsetAsync(grad3, 0, 3 * sizeof(double), s);
  cudaError_t e = mixed ? set_dyn_smem((const void *)se_hyper_grad_df_kernel, 3)
                        : set_dyn_smem((const void *)se_hyper_grad_kernel, 1);
  if (e != cudaSuccess) return e;
  const long long T = (n + CT - 1) / CT;
  const long long tiles = T * (T + 1) / 2;
  const size_t smem = 2 * CT * (size_t)d * sizeof(double);
  double *partial = (double *)ws;
  const double tri = 0.5 * (double)n * (n + 1);
  if (mixed) {
    GPC_LAUNCH(GPC_TRACE_HYPER, tri * (3.0 * d + 6.0), 8.0 * tri + 8.0 * n * d, s,
               se_hyper_grad_df_kernel<<<(unsigned)tiles, 256, smem, s>>>(
                   n, d, X, ldx, alpha, rho, sigma, host_df(1.0 / (2.0 * rho * rho)), Kbar, ldkb, partial));
  } else {
    GPC_LAUNCH(GPC_TRACE_HYPER, tri * (3.0 * d + 6.0), 8.0 * tri + 8.0 * n * d, s,
               se_hyper_grad_kernel<<<(unsigned)tiles, 256, smem, s>>>(n, d, X, ldx, alpha, rho,
                                                                       sigma, Kbar, ldkb, partial));
  }
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 24.0 * tiles, s, sum3_kernel<<<1, 256, 0, s>>>(partial, tiles, grad3));
  return cudaGetLastError();
}

size_t trsv_workspace_bytes(int n) {
  const int nblk = (n + TB - 1) / TB;
  return align_up((size_t)(nblk + 1) * sizeof(int), 256);
}

cudaError_t trsv(int n, const double *L, long long ldl, double *x, int trans, void *ws,
                 int *info, cudaStream_t s, const int *skip) {
  if (n <= 0) return cudaSuccess;
  const int nblk = (n + TB - 1) / TB;
  int *sync = (int *)ws;
  cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)(nblk + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  GPC_LAUNCH(GPC_TRACE_TRSV, (double)n * n, 4.0 * (double)n * (n + 1) + 16.0 * n, s,
             trsv_kernel<<<nblk, 256, 0, s>>>(n, L, ldl, x, trans ? 1 : 0, sync, info, skip, error_word(),
                                              faults().wait_ns, faults().trsv_withhold));
  return cudaGetLastError();
}

cudaError_t trsv_inv(int n, const double *L, long long ldl, const double *inv, int b, double *x, int trans,
                     void *ws, int *info, cudaStream_t s, const int *skip) {
  if (n <= 0) return cudaSuccess;
  if (b < 1 || b > 2 * TS) return cudaErrorInvalidValue;
  const int sb = b > TS ? (b + 1) / 2 : b;  // sub-blocks of at most 64 rows (b is even when > 64)
  if (sb > TS || (b > TS && 2 * sb != b)) return cudaErrorInvalidValue;
  const int nsb = (n + sb - 1) / sb;
  int *sync = (int *)ws;
  cudaError_t e = cudaMemsetAsync(sync, 0, (size_t)(nsb + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  GPC_LAUNCH(GPC_TRACE_TRSV, (double)n * n + 2.0 * n * b, 4.0 * (double)n * (n + 1) + 8.0 * n * b, s,
             trsv_inv_kernel<<<nsb, 256, 0, s>>>(n, L, ldl, inv, b, sb, x, trans ? 1 : 0, sync, info, skip,
                                                 error_word(), faults().wait_ns));
  return cudaGetLastError();
}

cudaError_t trsv_inv_df(int n, const float2 *Ld, long long ldd, const double *inv, int b, double *x,
                        float2 *xdf, int trans, void *ws, int *info, cudaStream_t s, const int *skip) {
  if (n <= 0) return cudaSuccess;
  if (b < 1 || b > 2 * TS || !Ld || !xdf || ((uintptr_t)xdf & 7u) || ((uintptr_t)Ld & 7u))
    return cudaErrorInvalidValue;
  const int sb = b > TS ? (b + 1) / 2 : b;
  if (sb > TS || (b > TS && 2 * sb != b)) return cudaErrorInvalidValue;
  const int nsb = (n + sb - 1) / sb;
  int *sync = (int *)ws;
  cudaError_t e = set_dyn_smem((const void *)trsv_inv_df_kernel, 4);  // the forward solve's row partials
  if (e == cudaSuccess) e = cudaMemsetAsync(sync, 0, (size_t)(nsb + 1) * sizeof(int), s);
  if (e != cudaSuccess) return e;
  const size_t dyn = trans ? 0 : (size_t)TS * (TS + 1) * sizeof(float2);
  GPC_LAUNCH(GPC_TRACE_TRSV, (double)n * n + 2.0 * n * b, 4.0 * (double)n * (n + 1) + 8.0 * n * b, s,
             trsv_inv_df_kernel<<<nsb, 256, dyn, s>>>(n, Ld, ldd, inv, b, sb, x, xdf, trans ? 1 : 0, sync, info,
                                                      skip, error_word(), faults().wait_ns));
  return cudaGetLastError();
}

// ---------------------------------------------------------------- iterative refinement
namespace {

// r = y - K x with K symmetric, read from its lower triangle.  One CTA per
// 64-row block I: row segments K[i, 0..i] (i in I) and column segments
// K[j, I] (j > first row of I) cover every stored entry that row block needs,
// so each lower entry is read twice over the grid and nothing is atomic.
// FP64 is throughput- and latency-bound here (n^2 fused multiply-adds, 64
// cycles per dependent one), so every thread carries four independent partial
// sums.  partial[block] = sum of r_i^2 over the block.
constexpr int RB = 64;
__global__ void __launch_bounds__(256)
symv_residual_kernel(int n, const double *K, long long ldk, const double *y, const double *x, double *r,
                     double *partial, const int *skip) {
  if (skip && *skip) return;
  __shared__ double part1[RB];
  __shared__ double part2[4][RB];
  __shared__ double red[8];
  const int i0 = blockIdx.x * RB, rows = min(RB, n - i0);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int rr = warp; rr < rows; rr += 8) {
    const int i = i0 + rr;
    const double *row = K + (long long)i * ldk;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = lane;
    for (; j + 96 <= i; j += 128) {
      a0 = fma(row[j], x[j], a0);
      a1 = fma(row[j + 32], x[j + 32], a1);
      a2 = fma(row[j + 64], x[j + 64], a2);
      a3 = fma(row[j + 96], x[j + 96], a3);
    }
    for (; j <= i; j += 32) a0 = fma(row[j], x[j], a0);
    double acc = (a0 + a1) + (a2 + a3);
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) part1[rr] = acc;
  }
  // column segments: thread (c, g) takes rows j = g (mod 4) below the block's diagonal
  const int c = threadIdx.x & (RB - 1), jg = threadIdx.x >> 6;
  double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
  if (c < rows) {
    const double *col = K + i0 + c;
    const int jd = min(n, i0 + RB);  // rows inside the diagonal block need j > i0 + c
    for (int j = i0 + 1 + jg; j < jd; j += 4)
      if (j > i0 + c) b0 = fma(col[(long long)j * ldk], x[j], b0);
    int j = jd + jg;
    for (; j + 12 < n; j += 16) {
      b0 = fma(col[(long long)j * ldk], x[j], b0);
      b1 = fma(col[(long long)(j + 4) * ldk], x[j + 4], b1);
      b2 = fma(col[(long long)(j + 8) * ldk], x[j + 8], b2);
      b3 = fma(col[(long long)(j + 12) * ldk], x[j + 12], b3);
    }
    for (; j < n; j += 4) b0 = fma(col[(long long)j * ldk], x[j], b0);
  }
  part2[jg][c] = (b0 + b1) + (b2 + b3);
  __syncthreads();
  double rr2 = 0.0;
  if (threadIdx.x < RB && threadIdx.x < rows) {
    const int i = i0 + threadIdx.x;
    const double kx = part1[threadIdx.x] + ((part2[0][threadIdx.x] + part2[1][threadIdx.x]) +
                                            (part2[2][threadIdx.x] + part2[3][threadIdx.x]));
    const double ri = y[i] - kx;
    r[i] = ri;
    rr2 = ri * ri;
  }
  const double tot = block_sum_256(rr2, red);
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// state[0] = done flag, state[1] = corrections applied; norms[0] = |y|^2,
// norms[1] = previous |r|^2.  Ends the refinement when |r| <= tol |y| or when
// |r| stopped halving (the FP64 residual floor has been reached).
__global__ void __launch_bounds__(256)
refine_check_kernel(int nblk, const double *partial, double *norms, double tol2, int *state) {
  __shared__ double red[8];
  if (state[0]) return;
  double a = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) a += partial[b];
  const double rr = block_sum_256(a, red);
  if (threadIdx.x == 0) {
    const bool small = rr <= tol2 * norms[0];
    const bool stalled = state[1] > 0 && rr > 0.25 * norms[1];
    if (small || stalled) state[0] = 1;
    norms[1] = rr;
  }
}

__global__ void refine_axpy_kernel(int n, double *x, const double *d, int *state) {
  if (state[0]) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[i] += d[i];
  if (i == 0) atomicAdd(&state[1], 1);
}

__global__ void __launch_bounds__(256)
refine_init_kernel(int n, const double *y, double *norms, int *state) {
  __shared__ double red[8];
  double a = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) a = fma(y[i], y[i], a);
  const double yy = block_sum_256(a, red);
  if (threadIdx.x == 0) {
    norms[0] = yy;
    norms[1] = 0.0;
    state[0] = 0;
    state[1] = 0;
  }
}

__global__ void refine_finish_kernel(int *state, int *info) {
  if (!state[0] && info && info[1] == 0) info[1] = GPC_ERR_NO_CONVERGENCE;
}

}  // namespace

size_t refine_workspace_bytes(int n) {
  const int nblk = (n + RB - 1) / RB;
  return align_up((size_t)n * sizeof(double), 256) + align_up((size_t)nblk * sizeof(double), 256) + 256;
}

cudaError_t refine(int n, const double *K, long long ldk, const double *L, long long ldl, const double *inv,
                   int b, const double *y, double *x, void *ws, void *trsv_ws, int *info, int max_iters,
                   double tol, cudaStream_t s, const float2 *Ld, long long ldd, float2 *xdf) {
  if (n <= 0) return cudaSuccess;
  const int nblk = (n + RB - 1) / RB;
  char *p = (char *)ws;
  double *r = (double *)p;
  p += align_up((size_t)n * sizeof(double), 256);
  double *partial = (double *)p;
  p += align_up((size_t)nblk * sizeof(double), 256);
  double *norms = (double *)p;
  int *state = (int *)(p + 2 * sizeof(double));
  GPC_LAUNCH(GPC_TRACE_ELEM, 2.0 * n, 8.0 * n, s, refine_init_kernel<<<1, 256, 0, s>>>(n, y, norms, state));
  for (int it = 0; it <= max_iters; ++it) {
    GPC_LAUNCH(GPC_TRACE_TRSV, 2.0 * (double)n * n, 8.0 * (double)n * (n + 1), s,
               symv_residual_kernel<<<nblk, 256, 0, s>>>(n, K, ldk, y, x, r, partial, state));
    GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * nblk, s,
               refine_check_kernel<<<1, 256, 0, s>>>(nblk, partial, norms, tol * tol, state));
    if (it == max_iters) break;
    cudaError_t e = Ld ? trsv_inv_df(n, Ld, ldd, inv, b, r, xdf, 0, trsv_ws, info, s, state)
                       : trsv_inv(n, L, ldl, inv, b, r, 0, trsv_ws, info, s, state);
    if (e == cudaSuccess)
      e = Ld ? trsv_inv_df(n, Ld, ldd, inv, b, r, xdf, 1, trsv_ws, info, s, state)
             : trsv_inv(n, L, ldl, inv, b, r, 1, trsv_ws, info, s, state);
    if (e != cudaSuccess) return e;
    GPC_LAUNCH(GPC_TRACE_ELEM, (double)n, 24.0 * n, s,
               refine_axpy_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, r, state));
  }
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0, s, refine_finish_kernel<<<1, 1, 0, s>>>(state, info));
  return cudaGetLastError();
}

cudaError_t lml_finalize(int n, const double *L, long long ldl, const double *y,
                         const double *alpha, double *logdet, double *value, cudaStream_t s) {
  GPC_LAUNCH(GPC_TRACE_ELEM, 3.0 * n, 24.0 * n, s,
             lml_finalize_kernel<<<1, 256, 0, s>>>(n, L, ldl, y, alpha, logdet, value));
  return cudaGetLastError();
}

size_t ltv_workspace_bytes(int n) {
  const int chunks = (n + LTV_ROWS - 1) / LTV_ROWS;
  return align_up((size_t)chunks * n * sizeof(double), 256);
}

cudaError_t ltv(int n, const double *L, long long ldl, const double *v, double *z, void *ws,
                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const int chunks = (n + LTV_ROWS - 1) / LTV_ROWS;
  double *partial = (double *)ws;
  dim3 grid((n + LTV_COLS - 1) / LTV_COLS, chunks);
  GPC_LAUNCH(GPC_TRACE_ELEM, (double)n * n, 4.0 * (double)n * (n + 1), s,
             ltv_partial_kernel<<<grid, LTV_COLS, 0, s>>>(n, L, ldl, v, partial));
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (double)chunks * n, s,
             ltv_reduce_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, chunks, partial, z));
  return cudaGetLastError();
}

cudaError_t lml_lbar(int n, const double *L, long long ldl, const double *alpha, const double *z,
                     double gbar, double *Lbar, long long ldlb, cudaStream_t s, bool df) {
  if (n <= 0) return cudaSuccess;
  const long long total = (long long)n * n;
  dim3 grid((unsigned)((n + LB_COLS - 1) / LB_COLS), (unsigned)((n + LB_ROWS - 1) / LB_ROWS));
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (double)total, s,
             lml_lbar_kernel<<<grid, 256, 0, s>>>(n, L, ldl, alpha, z, gbar, Lbar, ldlb, df ? 1 : 0));
  return cudaGetLastError();
}

}  // namespace gpc
