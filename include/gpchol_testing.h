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

#ifdef __cplusplus
}
#endif

#endif /* GPCHOL_TESTING_H */
