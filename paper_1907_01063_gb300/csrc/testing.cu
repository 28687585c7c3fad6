// Test hooks declared in include/gpchol_testing.h.
#include "../../include/gpchol_testing.h"
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr size_t kTestPartialCap = size_t(64) << 20;

int chunks_of(int K) { return std::max(1, (K + 127) / 128); }

__global__ void split_probe_kernel(int n, const double *x, float2 *hilo, double *back) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float2 v = split_f64(x[i]);
  hilo[i] = v;
  back[i] = exact_f64(v.x) + exact_f64(v.y);
}

size_t test_bytes(int M, int N, int K) {
  const int c = chunks_of(K);
  return slice_bytes(M, c) + slice_bytes(N, c) + kTestPartialCap;
}

}  // namespace
}  // namespace gpc

using namespace gpc;

extern "C" int gpc_test_ozaki_workspace_size(int M, int N, int K, size_t *bytes) {
  if (M < 0 || N < 0 || K < 0 || !bytes) return GPC_ERR_INVALID_ARG;
  *bytes = test_bytes(std::max(M, 1), std::max(N, 1), std::max(K, 1));
  return GPC_OK;
}

extern "C" int gpc_test_ozaki_gemm(int M, int N, int K, const double *A, const double *B, double *C, void *ws,
                                   size_t ws_bytes, int *err, gpc_stream_t stream) {
  if (M < 0 || N < 0 || K < 0) return GPC_ERR_INVALID_ARG;
  if (M == 0 || N == 0) return GPC_OK;
  if (!A || !B || !C || !ws || ws_bytes < test_bytes(M, N, std::max(K, 1))) return GPC_ERR_INVALID_ARG;
  cudaStream_t s = stream;
  cudaError_t e = cudaMemsetAsync(C, 0, (size_t)M * N * sizeof(double), s);  // double-float zero
  if (e != cudaSuccess) return GPC_ERR_CUDA;
  if (K == 0) return GPC_OK;
  const int chunks = chunks_of(K), first = std::min(K, 128);
  char *p = (char *)ws;
  SliceBuf SA = slice_view(p, M, chunks);
  p += slice_bytes(M, chunks);
  SliceBuf SB = slice_view(p, N, chunks);
  p += slice_bytes(N, chunks);
  float2 *partial = (float2 *)p;
  e = split_operand(A, K, 1, M, K, first, SA, s);
  if (e == cudaSuccess) e = split_operand(B, K, 1, N, K, first, SB, s);
  const long long tiles = (long long)((M + 127) / 128) * ((N + 63) / 64);
  int splits = (int)std::max<long long>(1, std::min<long long>(chunks, (2LL * sm_count() + tiles - 1) / tiles));
  while (splits > 1 && ozaki_partial_bytes(M, N, splits) > kTestPartialCap) --splits;
  if (e == cudaSuccess)
    e = ozaki_gemm(SA, 0, 0, SB, 0, 0, M, N, chunks, false, 1.0f, (float2 *)C, N, splits, partial, err, s, 0,
                   chunks == 1 ? (K + 31) / 32 * 32 : 0);  // a single short chunk multiplies only its K range
  if (e == cudaSuccess) e = from_df_rect(M, N, C, N, s);
  return e == cudaSuccess ? GPC_OK : GPC_ERR_CUDA;
}

extern "C" int gpc_test_recip_rsqrt(int n, const double *x, double *out, gpc_stream_t stream) {
  if (n < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (!x || !out) return GPC_ERR_INVALID_ARG;
  return recip_rsqrt_probe(n, x, out, stream) == cudaSuccess ? GPC_OK : GPC_ERR_CUDA;
}

extern "C" int gpc_test_split_f64(int n, const double *x, float *hilo, double *back, gpc_stream_t stream) {
  if (n < 0) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (!x || !hilo || !back || ((uintptr_t)hilo & 7u)) return GPC_ERR_INVALID_ARG;
  cudaStream_t s = stream;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 24.0 * n, s,
             split_probe_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, x, (float2 *)hilo, back));
  return cudaGetLastError() == cudaSuccess ? GPC_OK : GPC_ERR_CUDA;
}
