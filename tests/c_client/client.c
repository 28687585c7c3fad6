/*
 * A plain C client of libgpchol: compiles against include/gpchol.h alone (no
 * CUDA header, no C++), links libgpchol.so, and exercises the calls that need
 * no device -- version, status strings, workspace sizes and argument checks
 * that return before anything is enqueued.  Prints one line per check and
 * exits non-zero on the first failure.
 */
#include <stdio.h>
#include <stddef.h>

#include "gpchol.h"

#define CHECK(cond, what)                          \
  do {                                             \
    if (!(cond)) {                                 \
      printf("FAIL %s\n", what);                   \
      return 1;                                    \
    }                                              \
    printf("ok %s\n", what);                       \
  } while (0)

int main(void) {
  size_t bytes = 0;
  CHECK(gpc_version() > 0, "version");
  CHECK(gpc_status_string(GPC_ERR_NOT_PD) != NULL, "status string");
  CHECK(gpc_workspace_size(4096, GPC_FP64, &bytes) == GPC_OK && bytes > 0, "workspace size fp64");
  CHECK(gpc_workspace_size(4096, GPC_MIXED, &bytes) == GPC_OK && bytes > 0, "workspace size mixed");
  CHECK(gpc_workspace_size(-1, GPC_FP64, &bytes) == GPC_ERR_INVALID_ARG, "negative n rejected");
  CHECK(gpc_gemm_workspace_size(&bytes) == GPC_OK && bytes > 0, "gemm workspace size");
  CHECK(gpc_glm_workspace_size(512, &bytes) == GPC_OK && bytes > 0, "glm workspace size");
  CHECK(gpc_glm_workspace_size(GPC_GLM_MAX_K + 1, &bytes) == GPC_ERR_INVALID_ARG, "glm k limit");
  /* argument errors: nothing is dereferenced or enqueued */
  double *fake = (double *)(size_t)0x1000;
  CHECK(gpc_chol(10, fake, 9, fake + 4096, 10, GPC_FP64, fake + 8192, (size_t)1 << 30, (int *)fake, NULL) ==
            GPC_ERR_INVALID_ARG,
        "chol ld < n rejected");
  CHECK(gpc_tri_inverse(10, fake, 10, fake + 4, 10, NULL) == GPC_ERR_INVALID_ARG, "tri_inverse overlap rejected");
  CHECK(gpc_gemm(4, 3, 2, fake, 1, fake + 4096, 3, fake + 8192, 3, NULL, 0, NULL) == GPC_ERR_INVALID_ARG,
        "gemm lda < k rejected");
  /* zero sizes are no-ops */
  CHECK(gpc_tri_inverse(0, NULL, 0, NULL, 0, NULL) == GPC_OK, "tri_inverse n = 0");
  CHECK(gpc_gemm(0, 5, 5, NULL, 5, NULL, 5, NULL, 5, NULL, 0, NULL) == GPC_OK, "gemm m = 0");
  return 0;
}
