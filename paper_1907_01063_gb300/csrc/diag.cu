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

__global__ void __launch_bounds__(DIAG_THREADS)
potrf_trtri_kernel(int nb, double *A, long long lda, double *Winv, int *info, int pivot_offset,
                   int factor) {
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
    Winv[idx] = (j <= i) ? S(smem, ld, i, j) : 0.0;
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

cudaError_t reset_info(int *info, cudaStream_t s) {
  if (!info) return cudaSuccess;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0, s, reset_info_kernel<<<1, 1, 0, s>>>(info));
  return cudaGetLastError();
}

}  // namespace gpc
