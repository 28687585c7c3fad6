// FP64 register-tiled GEMM on the FP64 tensor path (mma.sync m16n8k16 .f64).
//
// This is the workhorse of the FP64 blocked Cholesky (panel product with the
// diagonal-block inverse, trailing update A22 -= L21 L21^T of Section 3.3) and
// of the blocked adjoint sweep (the products of the reverse-mode procedure of
// Section 3.3).  tcgen05 has no FP64 kind, so the FP64 tensor instruction on
// sm_103a is the warp-level DMMA; the m16n8k16 shape sustains the part's FP64
// peak (about 1.05 TFLOP/s measured, the rate of plain DFMA at full occupancy)
// with far fewer instructions and shared-memory operand reads than DFMA.
//
// Tile: 64 x 64 per CTA, K step 16, 4 warps in a 2 x 2 grid, 32 x 32 per warp
// (2 x 4 m16n8 fragments); single products of at most 256 x 256 take 32 x 32
// tiles instead (16 x 16 per warp), so that they spread over the part.  Operands are staged through shared memory with a
// register prefetch of the next K step; FP64 throughput on this part is low
// enough that one stage of prefetch hides global latency completely.
// Triangular outputs launch only the lower tiles; thin-output / long-K
// products split K over grid.z into partial tiles summed in fixed order by a
// second kernel (deterministic).
#include "common.cuh"

#include <algorithm>

namespace gpc {
namespace {

constexpr int BK = 16, PAD = 4, THREADS = 128;
constexpr size_t kScratchCap = size_t(40) << 20;  // split-K partial tiles, bytes

struct Params {
  int M, N, K;
  double alpha, beta;
  const double *A;
  long long lda;
  const double *B;
  long long ldb;
  double *C;
  long long ldc;
  int uplo, tiles_n, kchunk, kskip;
  long long sA, sB, sC;  // per-product offsets of a batch (grid.y)
  double *partial;  // non-null when grid.z > 1
};

__device__ __forceinline__ void tri_index(int x, int &ti, int &tj) {
  int t = (int)((sqrtf(8.0f * (float)x + 1.0f) - 1.0f) * 0.5f);
  while ((t + 1) * (t + 2) / 2 <= x) ++t;
  while (t * (t + 1) / 2 > x) --t;
  ti = t;
  tj = x - t * (t + 1) / 2;
}

__device__ __forceinline__ void dmma16816(double (&c)[4], const double (&a)[8], const double (&b)[4]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
      "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
      : "+d"(c[0]), "+d"(c[1]), "+d"(c[2]), "+d"(c[3])
      : "d"(a[0]), "d"(a[1]), "d"(a[2]), "d"(a[3]), "d"(a[4]), "d"(a[5]), "d"(a[6]), "d"(a[7]),
        "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
}

// Global -> registers for one K step of a T x T tile.  Each thread holds V A
// and V B values (V = 8 for T = 64, 4 for T = 32).
template <int T, bool TA, bool TB>
__device__ __forceinline__ void load_tiles(const Params &p, int m0, int n0, int k0, int kend,
                                           double (&ra)[T * BK / THREADS], double (&rb)[T * BK / THREADS]) {
  constexpr int V = T * BK / THREADS, RK = BK / V, RM = T / V;  // threads per K row / per operand row
  const int t = threadIdx.x;
  const double *A = p.A + (long long)blockIdx.y * p.sA, *B = p.B + (long long)blockIdx.y * p.sB;
  if (!TA) {  // A[m][k]: RK threads per row, V consecutive k each
    const int r = t / RK, c0 = (t % RK) * V, m = m0 + r;
    const double *src = A + (long long)m * p.lda;
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int k = k0 + c0 + i;
      ra[i] = (m < p.M && k < kend) ? src[k] : 0.0;
    }
  } else {  // A[k][m]: RM threads per k-row, V consecutive m each
    const int kk = t / RM, mm0 = (t % RM) * V, k = k0 + kk;
    const double *src = A + (long long)k * p.lda;
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int m = m0 + mm0 + i;
      ra[i] = (m < p.M && k < kend) ? src[m] : 0.0;
    }
  }
  if (!TB) {  // B[k][n]
    const int kk = t / RM, nn0 = (t % RM) * V, k = k0 + kk;
    const double *src = B + (long long)k * p.ldb;
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int n = n0 + nn0 + i;
      rb[i] = (n < p.N && k < kend) ? src[n] : 0.0;
    }
  } else {  // B[n][k]
    const int r = t / RK, c0 = (t % RK) * V, n = n0 + r;
    const double *src = B + (long long)n * p.ldb;
#pragma unroll
    for (int i = 0; i < V; ++i) {
      const int k = k0 + c0 + i;
      rb[i] = (n < p.N && k < kend) ? src[k] : 0.0;
    }
  }
}

// Row padding of the operand stages: 4 doubles for 64-wide tiles, 2 for
// 32-wide ones (9 KB per stage pair, room to spare beside a product CTA).
template <int T>
constexpr int tile_pad() { return T == 64 ? PAD : 2; }

template <int T, bool TA, bool TB>
__device__ __forceinline__ void store_tiles(double (*As)[BK + tile_pad<T>()], double (*Bs)[BK + tile_pad<T>()],
                                            const double (&ra)[T * BK / THREADS], const double (&rb)[T * BK / THREADS]) {
  constexpr int V = T * BK / THREADS, RK = BK / V, RM = T / V;
  const int t = threadIdx.x;
  if (!TA) {
    const int r = t / RK, c0 = (t % RK) * V;
#pragma unroll
    for (int i = 0; i < V; ++i) As[r][c0 + i] = ra[i];
  } else {
    const int kk = t / RM, mm0 = (t % RM) * V;
#pragma unroll
    for (int i = 0; i < V; ++i) As[mm0 + i][kk] = ra[i];
  }
  if (!TB) {
    const int kk = t / RM, nn0 = (t % RM) * V;
#pragma unroll
    for (int i = 0; i < V; ++i) Bs[nn0 + i][kk] = rb[i];
  } else {
    const int r = t / RK, c0 = (t % RK) * V;
#pragma unroll
    for (int i = 0; i < V; ++i) Bs[r][c0 + i] = rb[i];
  }
}

// T x T output tile per CTA (T = 64, or 32 for products too small to fill the
// part with 64-wide tiles); 4 warps in a 2 x 2 grid, (T/2) x (T/2) per warp.
// T = 64 double-buffers its operand stage; T = 32 keeps one stage (9 KB of
// shared memory), so that a CTA fits beside a split-product CTA on the same
// SM (which leaves about 11 KB free): the small products of the adjoint's
// chain then use every SM while a product runs in the background.
template <int T, bool TA, bool TB>
__global__ void __launch_bounds__(THREADS) gemm_f64_kernel(Params p) {
  constexpr int V = T * BK / THREADS, MI = T / 32, NI = T / 16, NS = (T == 64) ? 2 : 1;
  __shared__ double As[NS][T][BK + tile_pad<T>()];
  __shared__ double Bs[NS][T][BK + tile_pad<T>()];

  int tm, tn;
  if (p.uplo != UPLO_FULL) {
    tri_index(blockIdx.x, tm, tn);
  } else {
    tm = blockIdx.x / p.tiles_n;
    tn = blockIdx.x - tm * p.tiles_n;
  }
  const int m0 = tm * T, n0 = tn * T;
  // a skipped leading K range is a multiple of T, so kbeg stays on a K step
  const int kfirst = p.kskip == KSKIP_ROWS ? m0 : (p.kskip == KSKIP_COLS ? n0 : 0);
  const int klast = p.kskip == KSKIP_ROWS_END ? m0 + T : (p.kskip == KSKIP_COLS_END ? n0 + T : p.K);
  const int kbeg = max((int)blockIdx.z * p.kchunk, kfirst);
  const int kend = min(min(p.K, klast), (int)blockIdx.z * p.kchunk + p.kchunk);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wm = warp >> 1, wn = warp & 1;
  const int g = lane >> 2, tg = lane & 3;

  double acc[MI][NI][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < NI; ++j)
#pragma unroll
      for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.0;

  double ra[V], rb[V];
  auto compute = [&](int buf) {
    double a[MI][8], b[NI][4];
#pragma unroll
    for (int mi = 0; mi < MI; ++mi) {
      const int r = wm * (T / 2) + mi * 16 + g;
#pragma unroll
      for (int i = 0; i < 8; ++i) a[mi][i] = As[buf][r + 8 * (i & 1)][tg + 4 * (i >> 1)];
    }
#pragma unroll
    for (int ni = 0; ni < NI; ++ni) {
      const int c = wn * (T / 2) + ni * 8 + g;
#pragma unroll
      for (int i = 0; i < 4; ++i) b[ni][i] = Bs[buf][c][tg + 4 * i];
    }
#pragma unroll
    for (int mi = 0; mi < MI; ++mi)
#pragma unroll
      for (int ni = 0; ni < NI; ++ni) dmma16816(acc[mi][ni], a[mi], b[ni]);
  };
  if constexpr (NS == 2) {
    int buf = 0;
    if (kbeg < kend) {
      load_tiles<T, TA, TB>(p, m0, n0, kbeg, kend, ra, rb);
      store_tiles<T, TA, TB>(As[0], Bs[0], ra, rb);
    }
    __syncthreads();
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      const bool more = k0 + BK < kend;
      if (more) load_tiles<T, TA, TB>(p, m0, n0, k0 + BK, kend, ra, rb);
      compute(buf);
      if (more) {
        store_tiles<T, TA, TB>(As[buf ^ 1], Bs[buf ^ 1], ra, rb);
        __syncthreads();
        buf ^= 1;
      }
    }
  } else {  // one stage: the next K step waits in registers while this one is computed
    if (kbeg < kend) load_tiles<T, TA, TB>(p, m0, n0, kbeg, kend, ra, rb);
    for (int k0 = kbeg; k0 < kend; k0 += BK) {
      __syncthreads();  // the previous step's reads of the stage are done
      store_tiles<T, TA, TB>(As[0], Bs[0], ra, rb);
      __syncthreads();
      if (k0 + BK < kend) load_tiles<T, TA, TB>(p, m0, n0, k0 + BK, kend, ra, rb);
      compute(0);
    }
  }

  // Epilogue: fragment (mi, ni) element r sits at row g (+8 for r >= 2),
  // column 2*tg + (r & 1) of the 16 x 8 tile.
  const bool split = p.partial != nullptr;
  double *part = split ? p.partial + (size_t)blockIdx.z * p.M * p.N : nullptr;
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int ni = 0; ni < NI; ++ni)
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        const int row = m0 + wm * (T / 2) + mi * 16 + g + ((r >> 1) << 3);
        const int col = n0 + wn * (T / 2) + ni * 8 + 2 * tg + (r & 1);
        if (row >= p.M || col >= p.N) continue;
        const double v = p.alpha * acc[mi][ni][r];
        if (split) {
          part[(size_t)row * p.N + col] = v;
          continue;
        }
        if (p.uplo != UPLO_FULL && col > row) continue;
        double *C = p.C + (long long)blockIdx.y * p.sC;
        double *dst = C + (long long)row * p.ldc + col;
        const double out = (p.beta == 0.0) ? v : fma(p.beta, *dst, v);
        *dst = out;
        if (p.uplo == UPLO_LOWER_MIRROR && col < row) C[(long long)col * p.ldc + row] = out;
      }
}

__global__ void splitk_reduce_kernel(Params p, int splits) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long total = (long long)p.M * p.N;
  if (idx >= total) return;
  const int row = (int)(idx / p.N), col = (int)(idx - (long long)row * p.N);
  if (p.uplo != UPLO_FULL && col > row) return;
  double s = 0.0;
  for (int z = 0; z < splits; ++z) s += p.partial[(size_t)z * total + idx];
  double *dst = p.C + (long long)row * p.ldc + col;
  const double out = (p.beta == 0.0) ? s : fma(p.beta, *dst, s);
  *dst = out;
  if (p.uplo == UPLO_LOWER_MIRROR && col < row) p.C[(long long)col * p.ldc + row] = out;
}

}  // namespace

size_t gemm_f64_scratch_bytes() { return kScratchCap; }

namespace {
// The 32-wide instantiations share SMs with split-product CTAs only when they
// run in the same (maximal) shared-memory configuration.
bool g_small_carveout[64];
cudaError_t small_tile_carveout() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return cudaSuccess;
  if (g_small_carveout[dev]) return cudaSuccess;
  const void *fns[] = {(const void *)gemm_f64_kernel<32, false, false>, (const void *)gemm_f64_kernel<32, false, true>,
                       (const void *)gemm_f64_kernel<32, true, false>, (const void *)gemm_f64_kernel<32, true, true>};
  for (const void *f : fns) {
    cudaError_t e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
  }
  g_small_carveout[dev] = true;
  return cudaSuccess;
}
}  // namespace

cudaError_t gemm_f64(const Gemm &g, double *scratch, cudaStream_t s) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.uplo != UPLO_FULL && g.M != g.N) return cudaErrorInvalidValue;
  if (g.batch > 65535) return cudaErrorInvalidValue;
  Params p;
  p.M = g.M;
  p.N = g.N;
  p.K = std::max(g.K, 0);
  p.alpha = g.alpha;
  p.beta = g.beta;
  p.A = g.A;
  p.lda = g.lda;
  p.B = g.B;
  p.ldb = g.ldb;
  p.C = g.C;
  p.ldc = g.ldc;
  p.uplo = g.uplo;
  p.kskip = g.kskip;
  p.sA = g.sA;
  p.sB = g.sB;
  p.sC = g.sC;
  // 64-wide tiles; a single product that 64-wide tiles and split K cannot
  // spread over every SM takes 32-wide tiles and K steps down to 16 (the
  // symbolic steps of the adjoint, 128 x 128 x 128: 16 CTAs with 64-wide
  // tiles, 128 with 32-wide).  A long-K product of the same output (split
  // K reaches every SM) keeps 64-wide tiles, which read fewer operands per
  // DMMA.  The size limit is a tuning knob (0: never 32-wide).
  const long long target = 3LL * sm_count();  // three CTAs fit per SM
  const long long cap_splits = (long long)(kScratchCap / (sizeof(double) * (size_t)g.M * g.N));
  auto tile_count = [&](int T) {
    const long long tm_ = (g.M + T - 1) / T, tn_ = (g.N + T - 1) / T;
    return (g.uplo != UPLO_FULL) ? tm_ * (tm_ + 1) / 2 : tm_ * tn_;
  };
  auto max_splits = [&](int kmin) {
    return std::max<long long>(1, std::min<long long>(std::min<long long>(64, p.K / kmin), cap_splits));
  };
  const int kmin64 = std::max(tuning().splitk_min, BK);
  const int small_max = tuning().f64_small_tile;
  const bool small = g.batch == 1 && scratch != nullptr && g.M <= small_max && g.N <= small_max &&
                     tile_count(64) * max_splits(kmin64) < sm_count();
  const int T = small ? 32 : 64;
  p.tiles_n = (g.N + T - 1) / T;
  const long long tiles = tile_count(T);

  // Split K when the output alone cannot fill the machine.
  int splits = 1;
  const int kmin = small ? BK : kmin64;
  if (scratch && g.batch == 1 && tiles < target && p.K >= 2 * kmin) {
    long long want = (target + tiles - 1) / tiles;
    want = std::min(want, max_splits(kmin));
    splits = (int)std::max<long long>(want, 1);
  }
  int kchunk = (p.K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  if (kchunk == 0) kchunk = BK;
  splits = std::max(1, (p.K + kchunk - 1) / kchunk);
  p.kchunk = kchunk;
  p.partial = splits > 1 ? scratch : nullptr;

  dim3 grid((unsigned)tiles, (unsigned)g.batch, (unsigned)splits);
  const double mn = (g.uplo != UPLO_FULL) ? 0.5 * (double)g.M * (g.M + 1) : (double)g.M * g.N;
  const double flops = g.algo_flops > 0.0 ? g.algo_flops : 2.0 * mn * (double)p.K * g.batch;
  const double bytes =
      8.0 * g.batch * ((double)g.M * p.K + (double)p.K * g.N + (g.beta != 0.0 ? 2.0 : 1.0) * mn);
  if (small) {
    if (cudaError_t ce = small_tile_carveout(); ce != cudaSuccess) return ce;
    GPC_LAUNCH(GPC_TRACE_GEMM_F64, flops, bytes, s, {
      if (!g.transA && !g.transB) gemm_f64_kernel<32, false, false><<<grid, THREADS, 0, s>>>(p);
      else if (!g.transA && g.transB) gemm_f64_kernel<32, false, true><<<grid, THREADS, 0, s>>>(p);
      else if (g.transA && !g.transB) gemm_f64_kernel<32, true, false><<<grid, THREADS, 0, s>>>(p);
      else gemm_f64_kernel<32, true, true><<<grid, THREADS, 0, s>>>(p);
    });
  } else {
    GPC_LAUNCH(GPC_TRACE_GEMM_F64, flops, bytes, s, {
      if (!g.transA && !g.transB) gemm_f64_kernel<64, false, false><<<grid, THREADS, 0, s>>>(p);
      else if (!g.transA && g.transB) gemm_f64_kernel<64, false, true><<<grid, THREADS, 0, s>>>(p);
      else if (g.transA && !g.transB) gemm_f64_kernel<64, true, false><<<grid, THREADS, 0, s>>>(p);
      else gemm_f64_kernel<64, true, true><<<grid, THREADS, 0, s>>>(p);
    });
  }
  if (splits > 1) {
    const long long total = (long long)g.M * g.N;
    GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (splits + 2) * mn, s,
               splitk_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(p, splits));
  }
  return cudaGetLastError();
}

}  // namespace gpc
