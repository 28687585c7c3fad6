// Internal declarations shared by the CUDA translation units of libgpchol.
// Nothing here is part of the public C ABI (include/gpchol.h).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "../../include/gpchol.h"

namespace gpc {

// ---------------------------------------------------------------- tuning
struct Tuning {
  int block = 128;        // b: block size of the blocked factorisation / adjoint
  int splitk_min = 32;    // minimum K per split of a split-K product
  int batch_block = 64;   // block size inside the batched per-GP pass (32 or 64)
  int batch_ctas_per_sm = 1;
  int mixed_defer = 6;    // mixed path: block columns whose trailing updates are merged (K = 128 x this)
  int mixed_free_sms = 2; // mixed factorisation: SMs the background products leave to the FP64 chain
  int mixed_adj_free_sms = 16;  // mixed adjoint: the same
  int f64_small_tile = 256;  // FP64 products with M, N <= this take 32 x 32 tiles (0: never)
  int mixed_cta_items = 0;  // mixed path: work items per CTA of a background product (0: persistent)
  int mixed_priority = 1;   // mixed path: launch the critical chain at the device's greatest priority
};
Tuning &tuning();

// ---------------------------------------------------------------- launch priority
// Priority given to the launches this thread makes through launch_k (0: the
// stream's own).  The mixed factorisation raises it for its critical chain so
// that pending CTAs of the chain's kernels are scheduled before pending CTAs
// of the products running in the background.
int launch_priority();
int greatest_priority();  // of the current device (numerically lowest value)
struct PriorityScope {
  int saved;
  explicit PriorityScope(int p);
  ~PriorityScope();
};
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  const int prio = launch_priority();
  if (prio != 0) {
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = prio;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Number of SMs of the current device (cached per device).
int sm_count();

// ---------------------------------------------------------------- double-float conversions
// On this part the FP64 pipe (which also runs the FP32 <-> FP64 conversion
// instructions) is a small fraction of the integer and FP32 rates, so the
// conversions between FP64 and double-float storage (an FP32 pair hi + lo)
// move the fields with integer instructions where the result is exact.

// FP32 -> FP64, exact for every normal value and zero; subnormals, Inf and
// NaN take the conversion instruction.
__device__ __forceinline__ double exact_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xFFu;
  if (e == 0u || e == 0xFFu) {
    if ((u & 0x7FFFFFFFu) == 0u) return __longlong_as_double((long long)(u & 0x80000000u) << 32);
    return (double)f;
  }
  const unsigned long long d = ((unsigned long long)(u & 0x80000000u) << 32) |
                               ((unsigned long long)(e + 896u) << 52) | ((unsigned long long)(u & 0x7FFFFFu) << 29);
  return __longlong_as_double((long long)d);
}

// Signed integer |v| <= 2^28 -> nearest FP32 without the integer-to-float
// instruction (which issues on the FP64 pipe on this part): v = a 2^14 + b with
// a = v >> 14 and b = v & (2^14 - 1) each exact in FP32 by the exponent-field
// trick (2^23 + b and 1.5 * 2^23 + a are FP32 numbers whose low mantissa bits
// hold b and a), then one FMA rounds a 2^14 + b once.
__device__ __forceinline__ float int29_to_float_rn(int v) {
  const float a = __fsub_rn(__int_as_float(0x4B400000 + (v >> 14)), 12582912.0f);
  const float b = __fsub_rn(__int_as_float(0x4B000000 | (v & 0x3FFF)), 8388608.0f);
  return __fmaf_rn(a, 16384.0f, b);
}

// FP64 x -> (hi, lo): hi = x rounded to nearest FP32 (ties to even), lo = the
// exact remainder x - hi rounded to nearest FP32 -- the same pair as
// hi = (float)x, lo = (float)(x - (double)hi).  For 2^-74 <= |x| < 2^127 both
// are normal FP32 numbers and the pair is formed from the fields: the 52-bit
// mantissa splits into its top 23 bits (rounded on the 29 below) and the
// signed remainder r (|r| <= 2^28, exact in an int), so lo = r 2^(E - 1075)
// rounds r to FP32 (int29_to_float_rn) and scales by a power of two.  Other
// values take the FP64 conversions.
__device__ __forceinline__ float2 split_f64(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned E = (unsigned)(b >> 52) & 0x7FFu;
  if (E >= 949u && E <= 1149u) {
    const unsigned s = (unsigned)(b >> 63);
    const unsigned m23 = (unsigned)((b >> 29) & 0x7FFFFFull);
    const int rem = (int)(b & 0x1FFFFFFFull);  // the 29 bits below m23
    const bool up = rem > 0x10000000 || (rem == 0x10000000 && (m23 & 1u));
    const unsigned hb = (s << 31) | (((E - 896u) << 23) + m23 + (up ? 1u : 0u));
    const int r = up ? rem - 0x20000000 : rem;   // x - hi in units of 2^(E - 1075)
    const float lo = __fmul_rn(int29_to_float_rn(s ? -r : r), __uint_as_float((E - 948u) << 23));  // 2^(E - 1075)
    return make_float2(__uint_as_float(hb), lo);
  }
  const float hi = __double2float_rn(x);
  return make_float2(hi, __double2float_rn(x - (double)hi));
}


// ---------------------------------------------------------------- error word, symbols, test faults
// Device address of a file-scope __device__ variable on the current device,
// cached per device together with the context it was looked up in (a new
// context triggers a new lookup).  The first lookup on a device is a runtime
// query: make it before any stream capture.
struct SymbolCache {
  static constexpr int kMaxDevices = 64;
  std::mutex mu;
  void *ctx[kMaxDevices] = {};
  void *addr[kMaxDevices] = {};
};
cudaError_t symbol_address(const void *symbol, SymbolCache &cache, void **out);
// The library error word of the current device (gpc_get_error), or null if
// the lookup failed.  Kernels record device-side conditions with record_error.
int *error_word();
__device__ __forceinline__ void record_error(int *word, int status) {
  if (word) atomicCAS(word, 0, status);
}
// 1/x and 1/sqrt(x) for normal positive x: the hardware's approximations
// refined, 1/x by two Newton-Raphson steps y <- y (2 - x y) (each doubles the
// correct bits), 1/sqrt(x) as below; the results are
// within 2 ulp of the correctly rounded value, checked against CUDA's 1.0 / x
// and rsqrt over the normal range by gpc_test_recip_rsqrt's test; recip_nr
// needs 1/x normal too, x < 2^1022, which holds for any pivot of a matrix whose
// entries are below 2^511).  FP64 instructions are scarce on this part, so this
// short dependent chain is what the diagonal factorisation's serial part waits on.
__device__ __forceinline__ double recip_nr(double x) {
  if (!(x >= 2.2250738585072014e-308)) return 1.0 / x;
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
// 1/sqrt(x) refines the hardware seed y with one third-order step of the
// series (1 - e)^(-1/2) = 1 + e/2 + 3e^2/8 + ..., e = 1 - x y^2 (the error of
// a seed with relative error d is cubed, about 2.5 d^3): four dependent FP64
// operations instead of the six of two Newton-Raphson steps.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x >= 2.2250738585072014e-308)) return 1.0 / sqrt(x);
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y * y, 1.0);
  const double p = fma(0.375, e, 0.5);
  return fma(y * e, p, y);
}

// Fault-injection knobs of the test hooks (gpc_test_set_fault).  wait_ns is
// the budget of every bounded device wait in the solve and product kernels.
struct Faults {
  static constexpr unsigned long long kDefaultWaitNs = 2000000000ull;  // 2 s
  unsigned long long wait_ns = kDefaultWaitNs;
  int trsv_withhold = -1;  // 64-row block of trsv_kernel that never publishes its ready flag
  int ozaki_no_loads = 0;  // the split product's producer issues no copies
};
Faults &faults();

// ---------------------------------------------------------------- FP64 GEMM
// C = beta * C + alpha * op(A) * op(B), row-major, op(A) M x K, op(B) K x N.
// transA: A is stored K x M (element (m,k) at A[k*lda + m]); else M x K.
// transB: B is stored N x K (element (k,n) at B[n*ldb + k]); else K x N.
// uplo: 0 full; 1 lower triangle only (M == N, entries with col > row are
// neither computed nor touched); 2 lower, mirrored into the upper triangle.
// beta == 0 never reads C.
enum { UPLO_FULL = 0, UPLO_LOWER = 1, UPLO_LOWER_MIRROR = 2 };
enum { KSKIP_NONE = 0, KSKIP_ROWS = 1, KSKIP_COLS = 2, KSKIP_ROWS_END = 3, KSKIP_COLS_END = 4 };
struct Gemm {
  int M = 0, N = 0, K = 0;
  double algo_flops = 0.0;  // algorithmic flops for the trace (0: 2MNK, or M(M+1)K lower)
  bool transA = false, transB = false;
  double alpha = 1.0, beta = 0.0;
  const double *A = nullptr;
  long long lda = 0;
  const double *B = nullptr;
  long long ldb = 0;
  double *C = nullptr;
  long long ldc = 0;
  int uplo = UPLO_FULL;
  // Known-zero K ranges of a triangular operand, skipped per output tile:
  // KSKIP_ROWS when op(A)[i][k] = 0 for k < i (op(A) upper triangular), so
  // the tile's rows from m0 need k >= m0; KSKIP_COLS when op(B)[k][j] = 0
  // for k < j (op(B) lower triangular), so columns from n0 need k >= n0.
  // KSKIP_ROWS_END when op(A)[i][k] = 0 for k > i (op(A) lower triangular):
  // rows below m0 + 64 need k < m0 + 64; KSKIP_COLS_END when op(B)[k][j] = 0
  // for k > j (op(B) upper triangular): columns below n0 + 64 need k < n0 + 64.
  // Entries of the diagonal 64 x 64 tile on the zero side are still read and
  // must hold zeros.
  int kskip = KSKIP_NONE;
  // batch > 1: grid.y runs over independent products of the same shape whose
  // A, B and C start sA, sB and sC elements after the previous product's
  // (never split over K).
  int batch = 1;
  long long sA = 0, sB = 0, sC = 0;
};
// Bytes of split-K scratch any gemm_f64 call may use (a fixed cap).
size_t gemm_f64_scratch_bytes();
cudaError_t gemm_f64(const Gemm &g, double *scratch, cudaStream_t s);

// ---------------------------------------------------------------- diagonal blocks
constexpr int kMaxBlock = 128;
// Factor the nb x nb lower block at A (in place, upper part of the block set
// to zero) and write its inverse (lower, ld = nb) to Winv.  On a failing
// pivot p records {pivot_offset + p, status} in info if info[1] is still 0.
cudaError_t potrf_trtri_diag(int nb, double *A, long long lda, double *Winv, int *info,
                             int pivot_offset, cudaStream_t s);
// Factor only (no inverse) of the nb x nb block at A, in place.
// df: the block is read in double-float storage (written back as FP64).
cudaError_t potrf_diag(int nb, double *A, long long lda, int *info, int pivot_offset, cudaStream_t s,
                       bool df = false);
// In-place panel solve against the lower nb x nb block T: mode 0 X <- X T^{-T},
// mode 1 X <- X T^{-1}.  df: X is read in double-float storage (written back as FP64).
cudaError_t trsm_rows(int m, int nb, double *X, long long ldx, const double *T, long long ldt, int mode,
                      cudaStream_t s, bool df = false);
// Inverse (lower, ld = nb) of the nb x nb lower block D.
cudaError_t trtri_diag(int nb, const double *D, long long ldd, double *Dinv, cudaStream_t s);
// Inverses of all diagonal blocks of L in one launch: block 0 = rows [0, first),
// block ib >= 1 = [first + (ib-1) b, first + ib b); inverse ib at out + ib b^2
// (leading dimension = block size), or, when ldo != 0, at its diagonal
// position of the n x n matrix out (leading dimension ldo; out may be L).
cudaError_t trtri_batched(int n, const double *L, long long ldl, int first, int b, double *out,
                          cudaStream_t s, long long ldo = 0);

// ---------------------------------------------------------------- elementwise helpers
// dst(i,j) = src(i,j) for j <= i; strict upper of dst set to 0 (src may == dst).
cudaError_t copy_lower(int n, const double *src, long long lds, double *dst, long long ldd,
                       cudaStream_t s);
// dst (m x c) = src (m x c).
cudaError_t copy_rect(int m, int c, const double *src, long long lds, double *dst,
                      long long ldd, cudaStream_t s);
// Block nb x nb at A: halve the diagonal, zero the strict upper triangle.
cudaError_t phi_block(int nb, double *A, long long lda, cudaStream_t s);
// Lower Kbar -> full symmetric G: G_ii = Kbar_ii, G_ij = G_ji = Kbar_ij / 2.
cudaError_t lower_to_symmetric_half(int n, double *A, long long lda, cudaStream_t s);
cudaError_t reset_info(int *info, cudaStream_t s);
// Test hook: out[4 i ..] = {recip_nr(x_i), 1.0 / x_i, rsqrt_nr(x_i), rsqrt(x_i)}.
cudaError_t recip_rsqrt_probe(int n, const double *x, double *out, cudaStream_t s);

// ---------------------------------------------------------------- drivers
// Fused GLM likelihood and gradient (glm.cu).
size_t glm_workspace_bytes(int k);
cudaError_t glm(int family, long long n, int k, const double *X, long long ldx, const double *y, double alpha,
                const double *beta, double sigma, double *lp, double *dalpha, double *dbeta, double *dsigma,
                void *ws, cudaStream_t s);
// Ordinal-logit GLM (C ordered classes, C - 1 cut points); workspace as glm.
cudaError_t glm_ordinal(long long n, int k, int C, const double *X, long long ldx, const double *y,
                        const double *beta, const double *cuts, double *lp, double *dbeta, double *dcuts, void *ws,
                        cudaStream_t s);
// Categorical-logit GLM (C classes, beta k x C row-major).
size_t glm_categorical_workspace_bytes(int k, int C);
cudaError_t glm_categorical(long long n, int k, int C, const double *X, long long ldx, const double *y,
                            const double *alpha, const double *beta, double *lp, double *dalpha, double *dbeta,
                            void *ws, cudaStream_t s);
// Triangular inverse, solve and solve adjoint (trinv.cu); X is the inverse.
cudaError_t tri_inverse(int n, const double *L, long long ldl, double *X, long long ldx, cudaStream_t s);
cudaError_t tri_solve(int n, int m, const double *L, long long ldl, const double *B, long long ldb, double *X,
                      long long ldx, double *C, long long ldc, cudaStream_t s);
cudaError_t tri_solve_adjoint(int n, int m, const double *X, long long ldx, const double *C, long long ldc,
                              const double *Cbar, long long ldcb, double *Bbar, long long ldbb, double *Lbar,
                              long long ldlb, cudaStream_t s);
size_t chol_workspace_bytes(int n, int precision);
size_t adjoint_workspace_bytes(int n, int precision);
size_t trsv_workspace_bytes(int n);
cudaError_t chol_fp64(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s);
cudaError_t chol_adjoint_fp64(int n, const double *L, long long ldl, double *A, long long lda,
                              void *ws, cudaStream_t s);
// skip (device int, may be null): when *skip != 0 the solve does nothing.
cudaError_t trsv(int n, const double *L, long long ldl, double *x, int trans, void *ws,
                 int *info, cudaStream_t s, const int *skip = nullptr);
// FP64 iterative refinement of K x = y with the factor L (Section 3.2 solves):
// r = y - K x, x += L^{-T} L^{-1} r, until |r| <= tol |y|, the residual stops
// halving, or max_iters corrections; info[1] = GPC_ERR_NO_CONVERGENCE otherwise.
size_t refine_workspace_bytes(int n);
// With Ld (the lower triangle of L as FP32 pairs, leading dimension ldd) the
// correction solves run in double-float (trsv_inv_df) through xdf.
cudaError_t refine(int n, const double *K, long long ldk, const double *L, long long ldl, const double *inv,
                   int b, const double *y, double *x, void *ws, void *trsv_ws, int *info, int max_iters,
                   double tol, cudaStream_t s, const float2 *Ld = nullptr, long long ldd = 0,
                   float2 *xdf = nullptr);
// Blocked solve with stored diagonal-block inverses (blocks of b rows from the
// top, inverse I at inv + I b^2); ws as for trsv.
cudaError_t trsv_inv(int n, const double *L, long long ldl, const double *inv, int b, double *x, int trans,
                     void *ws, int *info, cudaStream_t s, const int *skip = nullptr);
// The same solve in double-float arithmetic on Ld, the lower triangle of L as
// FP32 pairs (hi, lo) with leading dimension ldd (to_df_tri); x is FP64 in and
// out, xdf (n pairs, 8-byte aligned) is scratch through which the solved
// sub-blocks pass.
cudaError_t trsv_inv_df(int n, const float2 *Ld, long long ldd, const double *inv, int b, double *x,
                        float2 *xdf, int trans, void *ws, int *info, cudaStream_t s, const int *skip = nullptr);
// Lower triangle of the FP64 matrix src as FP32 pairs (hi, lo) into dst; the
// strict upper triangle of dst is not written.
cudaError_t to_df_tri(int n, const double *src, long long lds, float2 *dst, long long ldd, cudaStream_t s);
// Block size the factorisation uses at a precision, and where it leaves its
// diagonal-block inverses (start of the workspace core).
int chol_block_size(int precision);

// ---------------------------------------------------------------- GP pieces
constexpr int kMaxDim = 256;
// mixed: r^2 and the exponential in double-float arithmetic (about 2^-46 per entry)
cudaError_t se_cov(int n, int d, const double *X, long long ldx, double alpha, double rho,
                   double sigma, double jitter, double *K, long long ldk, int full, bool mixed,
                   cudaStream_t s);
size_t se_hyper_grad_workspace_bytes(int n);
cudaError_t se_hyper_grad(int n, int d, const double *X, long long ldx, double alpha,
                          double rho, double sigma, const double *Kbar, long long ldkb,
                          double *grad3, void *ws, bool mixed, cudaStream_t s);
// scal[0] = logdet = 2 sum log L_ii, scal[1] = y . alpha, value = -1/2 scal[1] - 1/2 logdet
// - n/2 log(2 pi).  logdet/value may be null.
cudaError_t lml_finalize(int n, const double *L, long long ldl, const double *y,
                         const double *alpha, double *logdet, double *value, cudaStream_t s);
size_t ltv_workspace_bytes(int n);
// z = L^T v (L lower n x n).
cudaError_t ltv(int n, const double *L, long long ldl, const double *v, double *z, void *ws,
                cudaStream_t s);
// Lbar = gbar (tril(alpha z^T) - diag(1/L_ii)), strict upper zero.
// df: write L-bar in double-float storage (the mixed adjoint's input format).
cudaError_t lml_lbar(int n, const double *L, long long ldl, const double *alpha,
                     const double *z, double gbar, double *Lbar, long long ldlb, cudaStream_t s, bool df = false);

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// ---------------------------------------------------------------- mixed precision (ozaki.cu)
// BF16 slice planes of an operand, K-major: plane p, row r, K index k at
// base[p * rows_pad * kpad + r * kpad + k]; K is cut into 128-wide chunks.
struct SliceBuf {
  void *base = nullptr;
  int rows_pad = 0;
  int kpad = 0;
};
int slices_count();
int slice_chunk();
size_t slice_bytes(int rows, int kchunks);
SliceBuf slice_view(void *base, int rows, int kchunks);
// Operand element (r, k) = src[r * rs + k * ks]; chunk 0 is k in [0, first).
// chunk_offset: operand chunk c is written to slice chunk c + chunk_offset.
// row_offset: operand row r is written to slice row r + row_offset, and only
// rows row_offset .. row_offset + M - 1 are written (row_offset == 0 also
// zeroes the padding rows up to the buffer's rows_pad).
cudaError_t split_operand(const double *src, long long rs, long long ks, int M, int K, int first,
                          const SliceBuf &out, cudaStream_t s, int chunk_offset = 0, int row_offset = 0);
size_t ozaki_partial_bytes(int M, int N, int splits);
// C (double-float storage, ld in 8-byte elements) += alpha * A[a_row0 + i, a_k0 + k] B[b_row0 + j, b_k0 + k], alpha = +1 or -1
// over `chunks` K chunks; lower: only col <= row (M == N).  splits > 1 sums
// K ranges through `partial` (ozaki_partial_bytes) in fixed order.
// lower with M != N keeps the entries with (local) col <= row.  max_ctas > 0
// caps the persistent grid (leaves SMs free for work on another stream).
// kdepth (multiple of 32, at most 128; 0 = 128): K entries of each chunk that
// are multiplied -- the rest of the chunk must be zero slices.
// max_items > 0: at most that many work items per CTA (the grid grows past
// the SM count, so CTAs retire regularly and pending CTAs of other kernels,
// higher-priority ones first, get SMs).
cudaError_t ozaki_gemm(const SliceBuf &A, int a_row0, int a_k0, const SliceBuf &B, int b_row0, int b_k0,
                       int M, int N, int chunks, bool lower, float alpha, float2 *C, long long ldc,
                       int splits, float2 *partial, int *err, cudaStream_t s, int max_ctas = 0,
                       int kdepth = 0, int max_items = 0);
// Lower triangle of src (FP64) -> dst in double-float storage (upper set to 0); src may == dst.
cudaError_t to_df_lower(int n, const double *src, long long lds, double *dst, long long ldd, cudaStream_t s);
// m x c block in double-float storage -> FP64, in place.
cudaError_t from_df_rect(int m, int c, double *p, long long ld, cudaStream_t s);
size_t mixed_workspace_bytes(int n);
cudaError_t chol_mixed(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s);
// Batched per-GP pass (batched.cu); rowX[i] = first row of GP i in X (d per row) and y.
// mixed: split-BF16 products for the O(n^3) work and FP64 refinement of alpha.
size_t batched_workspace_bytes(int batch, int nmax, bool mixed);
cudaError_t batched_gp_lml_grad(int batch, const int *n, const long long *offK, const long long *rowX, int d,
                                const double *X, const double *y, const double *hyp, double *K, double *value,
                                double *grad3, int *info, int nmax, bool mixed, void *ws, cudaStream_t s);
cudaError_t chol_adjoint_mixed(int n, const double *L, long long ldl, double *A, long long lda, void *ws,
                               int *err, cudaStream_t s);

// ---------------------------------------------------------------- launch trace
// Every kernel launch site brackets its launch with trace_begin/trace_end.
// A process-wide counter always counts launches; when tracing is enabled
// (gpc_trace_enable) CUDA events are also recorded on the launching stream
// so per-class device time can be read back with gpc_trace_summary.
// Classes match the GPC_TRACE_* values of the public header.
// The launch expression's text names the kernel in the timeline.
void trace_begin(int cls, const char *what, cudaStream_t s);
void trace_end(int cls, double flops, double bytes, cudaStream_t s);
#define GPC_LAUNCH(cls, flops, bytes, stream, ...)     \
  do {                                                  \
    ::gpc::trace_begin((cls), #__VA_ARGS__, (stream));  \
    __VA_ARGS__;                                        \
    ::gpc::trace_end((cls), (flops), (bytes), (stream)); \
  } while (0)

}  // namespace gpc
