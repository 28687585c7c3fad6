/*
 * gpchol_testing.h -- test hooks of libgpchol (not part of the paper's
 * operations; they expose internal building blocks so tests can check them
 * in isolation).  Conventions as in gpchol.h: device pointers, caller-owned,
 * asynchronous on `stream`, GPC_ERR_INVALID_ARG before any launch on bad
 * arguments.
 */
#ifndef GPCHOL_TESTING_H
#define GPCHOL_TESTING_H

#include "gpchol.h"

#ifdef __cplusplus
extern "C" {
#endif

/*
 * C = A B^T through the mixed path's product: both FP64 operands are split
 * into BF16 slices (K cut into 128-wide chunks), multiplied on tcgen05 into
 * exact and rounded FP32 accumulators, and accumulated in double-float
 * storage; C is then converted to FP64.  A: M x K, B: N x K, C: M x N, all
 * row-major with leading dimension = column count.  ws: at least
 * gpc_test_ozaki_workspace_size bytes.  *err (device int) receives
 * GPC_ERR_TIMEOUT if a bounded device wait gave up; it is not reset here.
 */
int gpc_test_ozaki_workspace_size(int M, int N, int K, size_t *bytes);
int gpc_test_ozaki_gemm(int M, int N, int K, const double *A, const double *B, double *C, void *ws,
                        size_t ws_bytes, int *err, gpc_stream_t stream);

/*
 * The reciprocal and reciprocal square root that the diagonal-block
 * factorisation uses on its serial path (the hardware approximations refined
 * by two Newton-Raphson steps), evaluated on the n device doubles x next to
 * CUDA's own correctly rounded 1.0 / x and its rsqrt(x):
 *   out[4 i + 0] = refined 1/x_i      out[4 i + 1] = CUDA 1.0 / x_i
 *   out[4 i + 2] = refined 1/sqrt(x_i) out[4 i + 3] = CUDA rsqrt(x_i)
 * out: 4 n device doubles.  Meant for positive normal x; other x fall back to
 * the plain division and square root.
 */
int gpc_test_recip_rsqrt(int n, const double *x, double *out, gpc_stream_t stream);

/*
 * The FP64 -> double-float conversion of the mixed path (the split of every
 * FP64 matrix entry into an FP32 pair, formed from the bit fields without
 * the conversion instructions) and its inverse, on the n device doubles x:
 *   hilo[2 i] = hi_i, hilo[2 i + 1] = lo_i, meant to equal hi = (float)x_i
 *   and lo = (float)(x_i - (double)hi) with round-to-nearest-even;
 *   back[i] = (double)hi_i + (double)lo_i formed by the exact FP32 -> FP64
 *   field move.
 * hilo: 2 n device floats; back: n device doubles.
 */
int gpc_test_split_f64(int n, const double *x, float *hilo, double *back, gpc_stream_t stream);

/*
 * Fault injection for the tests of the bounded device waits.  These knobs
 * change what later launches do (process-wide, host-side; not thread-safe):
 *   GPC_TEST_WAIT_NS         budget of every bounded wait of the solve and
 *                            split-product kernels, in ns (1 .. 1e10);
 *                            0 restores the default of 2 s.
 *   GPC_TEST_TRSV_WITHHOLD   gpc_trsv / gpc_trsv_noalloc: the 64-row block
 *                            (0-based, in solve order) that computes its
 *                            rows but never publishes its ready flag, so the
 *                            blocks after it run out their waits and record
 *                            GPC_ERR_TIMEOUT; -1 (default) withholds none.
 *   GPC_TEST_OZAKI_NO_LOADS  1: the split product's copy warp issues no
 *                            copies, so the MMA warp's waits run out; the
 *                            kernel records GPC_ERR_TIMEOUT, releases its
 *                            tensor memory and returns.  0 (default): normal.
 * Every wait stays bounded, so no setting can hang a kernel.  Returns
 * GPC_ERR_INVALID_ARG for an unknown key or an out-of-range value.
 */
#define GPC_TEST_WAIT_NS 0
#define GPC_TEST_TRSV_WITHHOLD 1
#define GPC_TEST_OZAKI_NO_LOADS 2
int gpc_test_set_fault(int key, long long value);

#ifdef __cplusplus
}
#endif

#endif /* GPCHOL_TESTING_H */
