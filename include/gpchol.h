/*
 * gpchol.h -- C ABI of the GB300 (sm_103a) Cholesky / Cholesky-adjoint /
 * Gaussian-process likelihood library (libgpchol.so).
 *
 * The operations follow "GPU-based Parallel Computation Support for Stan"
 * (Cesnovar et al., 2019): the blocked Cholesky decomposition and its blocked
 * reverse mode (Section 3.3), the Gaussian-process log marginal likelihood
 * that the GP regression example of Section 4.2 evaluates on top of them,
 * triangular solves, the lower-triangular inverse and the solve's reverse
 * mode (Section 3.2), the general matrix product and its reverse mode
 * (Section 3.1), and fused GLM likelihoods with their gradients (Section 3.4).
 *
 * Conventions shared by every call
 * --------------------------------
 *  - Matrices are FP64, ROW-MAJOR: element (i, j) of an n x n matrix with
 *    leading dimension ld lives at ptr[i * ld + j], ld >= n.  Symmetric inputs
 *    are read from their LOWER triangle (i >= j) only.  Lower-triangular
 *    outputs (L, Kbar) have their strict upper triangle set to zero.
 *  - Every pointer argument is a DEVICE pointer unless stated otherwise, owned
 *    by the caller; the library never frees or retains it.  The library
 *    allocates no device memory: calls that need scratch take a workspace
 *    (ws, ws_bytes) sized by gpc_workspace_size().  Workspace contents are
 *    undefined on return; two calls in flight at the same time need two
 *    workspaces.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL = the
 *    legacy default stream) and returns a host status code once its kernels
 *    are enqueued.  Conditions found on the device (a failing pivot, NaN
 *    input) are written to the caller's device `info` array, which the caller
 *    reads after synchronising.
 *  - Sizes n = 0 are valid no-ops.  Negative sizes, ld < n, NULL pointers for
 *    n > 0, a too-small workspace or an unknown precision return
 *    GPC_ERR_INVALID_ARG without enqueuing anything.
 */
#ifndef GPCHOL_H
#define GPCHOL_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t, declared here so this header needs no CUDA one. */
typedef struct CUstream_st *gpc_stream_t;

/* Host status codes (return values), also used as info[1] on the device. */
#define GPC_OK 0
#define GPC_ERR_INVALID_ARG 1   /* bad size, leading dimension, pointer, flag or workspace */
#define GPC_ERR_NOT_PD 2        /* a pivot was <= 0: the matrix is not positive definite */
#define GPC_ERR_NAN 3           /* a pivot was NaN or infinite */
#define GPC_ERR_CUDA 4          /* a kernel launch or CUDA runtime call failed */
#define GPC_ERR_TIMEOUT 5       /* a bounded device-side wait gave up */
#define GPC_ERR_NO_CONVERGENCE 6 /* iterative refinement did not reach its tolerance */

/* Arithmetic of the O(n^3) products. */
#define GPC_FP64 0   /* every step in FP64 (DMMA tensor-core and FP64 ALU) */
#define GPC_MIXED 1  /* trailing/adjoint products as error-free split BF16 slices on tcgen05 */

/*
 * Device `info` arrays have two ints: info[0] = the 0-based index of the first
 * failing pivot, or -1; info[1] = GPC_OK, GPC_ERR_NOT_PD, GPC_ERR_NAN or
 * GPC_ERR_TIMEOUT.  Calls that take `info` reset it to {-1, GPC_OK} on the
 * stream before their first kernel.
 */

/*
 * Library error word (one per device).  Every kernel of this library that
 * waits on another thread block or on an asynchronous copy bounds the wait in
 * time; when a wait gives up, the kernel records GPC_ERR_TIMEOUT here (the
 * first status recorded since the last clear is kept) besides any per-call
 * info array, so calls that take no info (gpc_trsv, gpc_trsv_noalloc,
 * gpc_chol_adjoint, gpc_gp_lml_grad) still report it.  The outputs of a call
 * whose wait gave up are unspecified.
 * gpc_get_error synchronises `stream` (so call it after the calls of interest
 * were enqueued on that stream, or after the device was synchronised), then
 * copies the current device's word into *status (host pointer): GPC_OK or
 * GPC_ERR_TIMEOUT.  clear != 0 resets the word to GPC_OK afterwards.  The
 * first call on a device looks the word's device address up (a runtime query;
 * make it before any stream capture); the call itself cannot be captured.
 * Returns GPC_ERR_INVALID_ARG for a null status, GPC_ERR_CUDA if the copy or
 * the synchronisation fails.  No counterpart in the paper: the paper's OpenCL
 * framework reports device errors through exceptions on the host.
 */
int gpc_get_error(int *status, int clear, gpc_stream_t stream);

/* Human-readable text of a status code (static storage, never NULL). */
const char *gpc_status_string(int status);

/* Library ABI version (major * 10000 + minor * 100 + patch). */
int gpc_version(void);

/*
 * Workspace bytes that gpc_chol, gpc_chol_adjoint, gpc_gp_lml and
 * gpc_gp_lml_grad need for matrices of order n at `precision` with the
 * current tuning (gpc_set_tuning).  One workspace of this size serves any of
 * those calls with order <= n.  *bytes is a host pointer.
 */
int gpc_workspace_size(int n, int precision, size_t *bytes);

/*
 * Tuning knobs (host-side, process-wide; not thread-safe against concurrent
 * calls).  key: GPC_TUNE_BLOCK = block size b of the blocked factorisation and
 * adjoint (16..128, multiple of 16; default 128), GPC_TUNE_SLICES = number of
 * BF16 slices of the mixed path (read-only: the split kernels group their
 * products for 5 slices, so only 5 is accepted), GPC_TUNE_SPLITK_MIN = minimum K per
 * split of the split-K products.  Changing GPC_TUNE_BLOCK changes the
 * workspace size.  Returns GPC_ERR_INVALID_ARG for an unknown key or value.
 */
#define GPC_TUNE_BLOCK 0
#define GPC_TUNE_SLICES 1
#define GPC_TUNE_SPLITK_MIN 2
#define GPC_TUNE_BATCH_BLOCK 3  /* block size inside gpc_batched_gp_lml_grad: 32 or 64 */
/* Mixed factorisation (GPC_MIXED): block columns (128 wide) whose trailing
 * updates are merged into one product with K = 128 x value (1..8, default 6;
 * enters the mixed workspace size); SMs its background products leave to the
 * FP64 chain (0..32, default 2); work items per CTA of a background product
 * (0 = one persistent CTA per SM, else 1..1024, so CTAs retire and the
 * chain's kernels get SMs); and whether the chain's launches take the
 * device's greatest stream priority (0 or 1, default 1). */
#define GPC_TUNE_MIXED_DEFER 4
#define GPC_TUNE_MIXED_FREE_SMS 5
#define GPC_TUNE_MIXED_CTA_ITEMS 6
#define GPC_TUNE_MIXED_PRIORITY 7
/* Mixed adjoint: SMs its background products leave to the chain (0..64, default 16). */
#define GPC_TUNE_MIXED_ADJ_FREE_SMS 8
/* FP64 products (GEMM, factorisation and adjoint pieces): a single product
 * whose M and N are both at most this value takes 32 x 32 output tiles
 * instead of 64 x 64, so that it spreads over the part (0 = always 64 x 64;
 * 0..4096, default 256). */
#define GPC_TUNE_F64_SMALL_TILE 9
int gpc_set_tuning(int key, int value);
int gpc_get_tuning(int key, int *value);

/*
 * Squared-exponential covariance of the rows of X (n x d, row-major, ldx >= d):
 *   K_ij = alpha^2 exp(-|x_i - x_j|^2 / (2 rho^2)) + [i == j] (sigma^2 + jitter).
 * The paper's GP regression example (Section 4.2) builds this matrix; its
 * discussion lists covariance functions as GPU work to add (Section 5).
 * Writes the lower triangle of K (ldk >= n); full != 0 mirrors it into the
 * upper triangle, full == 0 leaves the upper triangle untouched.
 * precision GPC_FP64: FP64 arithmetic throughout.  GPC_MIXED: r^2 and the
 * exponential in double-float arithmetic (pairs of FP32 numbers, about 2^-46
 * relative error per entry, far below the mixed factorisation's own error),
 * one conversion to FP64 per entry; the diagonal is exact.
 * Requires rho > 0; 1 <= d <= 256.
 */
int gpc_se_cov(int n, int d, const double *X, int ldx, double alpha, double rho, double sigma,
               double jitter, double *K, int ldk, int full, int precision, gpc_stream_t stream);

/*
 * Cholesky factor L (lower, K = L L^T) of the SPD matrix whose lower triangle
 * is in K -- the blocked right-looking form of Section 3.3 (primitive
 * function): diagonal block factor and inverse, panel L21 = A21 L11^{-T} as a
 * product with the inverse, trailing update A22 -= L21 L21^T.
 * K == L (in place, same ld) is allowed; otherwise K is not modified.
 * On a failing pivot p, info = {p, GPC_ERR_NOT_PD or GPC_ERR_NAN}, rows >= p
 * of L are unspecified, and the call still returns GPC_OK (the failure is
 * only visible on the device).  info: 2 device ints.
 * precision GPC_MIXED computes the trailing updates with split-BF16 slices;
 * the diagonal blocks and panels stay FP64.
 */
int gpc_chol(int n, const double *K, int ldk, double *L, int ldl, int precision, void *ws,
             size_t ws_bytes, int *info, gpc_stream_t stream);

/*
 * Reverse mode of gpc_chol (Section 3.3, reverse mode function; the blocked
 * sweep after Murray 2016): given L and an adjoint Lbar (both lower), writes
 * Kbar = d f / d K restricted to the entries chol reads, i.e. for i >= j the
 * derivative with respect to the lower-triangle entry K_ij (lower output, zero
 * upper).  symmetric_out != 0 instead writes the full symmetric G with
 * G_ii = Kbar_ii and G_ij = G_ji = Kbar_ij / 2 (the gradient of f over a
 * symmetric K).  Kbar == Lbar (in place, same ld) is allowed; L must not
 * alias either.  L is not modified.
 */
int gpc_chol_adjoint(int n, const double *L, int ldl, const double *Lbar, int ldlb, double *Kbar,
                     int ldkb, int precision, int symmetric_out, void *ws, size_t ws_bytes,
                     gpc_stream_t stream);

/*
 * Triangular solve with the lower factor L (Section 3.2):
 *   trans == 0: x <- L^{-1} x      trans != 0: x <- L^{-T} x
 * x is a device vector of n doubles, overwritten.  ws/ws_bytes: scratch for
 * the solve's ready flags; gpc_workspace_size(n, GPC_FP64) bytes always
 * suffice.  Each 64-row block waits (bounded, 2 s) on the blocks before it; a
 * wait that gives up leaves x unspecified and records GPC_ERR_TIMEOUT in the
 * library error word (gpc_get_error).
 */
int gpc_trsv(int n, const double *L, int ldl, double *x, int trans, void *ws, size_t ws_bytes,
             gpc_stream_t stream);

/*
 * gpc_trsv without any caller-supplied scratch (the paper has no counterpart;
 * this is an addition for callers that cannot give the library device memory).
 * Callers that run under a device-memory budget owned by someone else (a
 * framework or sampler whose pool holds all device memory) or inside loops
 * that must not call cudaMalloc/cudaFree (cudaFree may synchronise the whole
 * device) pass only L and x; the solve's scratch -- a ticket counter and one
 * ready flag per 64-row block -- is a fixed 16.25 KiB array inside the library,
 * held by every GPU that loads the library until the process exits.
 *  - n must be <= GPC_TRSV_NOALLOC_MAX_N; larger n returns GPC_ERR_INVALID_ARG
 *    before anything is enqueued.  Other arguments as in gpc_trsv.  A bounded
 *    wait that gives up leaves x unspecified; the call still returns GPC_OK
 *    (it is asynchronous) and the timeout is recorded in the library error
 *    word, which the caller reads with gpc_get_error after a sync.
 *  - The first call on each device looks up the array's device address
 *    (cudaGetSymbolAddress, with that device current) and caches it with the
 *    device's current context; a later call in a new context (for example
 *    after cudaDeviceReset) looks it up again.  Make the first call in each
 *    context before any stream capture.  No call allocates memory.
 *  - All calls on a device share the one array, which keeps the last call's
 *    contents; each call clears the flags it uses on `stream` before its
 *    kernel.  Calls whose execution overlaps on the GPU (different streams
 *    without ordering between them) race on the array and give wrong results:
 *    serialise them.
 */
#define GPC_TRSV_NOALLOC_MAX_N 262144
int gpc_trsv_noalloc(int n, const double *L, int ldl, double *x, int trans, gpc_stream_t stream);

/*
 * Lower-triangular inverse Linv = L^{-1} (Section 3.2, solving triangular
 * systems, primitive function: the divide-and-conquer inverse with
 * C3 = -C2 A3 C1, run bottom-up from the b x b diagonal blocks).
 *  - L: n x n, row-major, leading dimension ldl >= n; only the lower triangle
 *    (diagonal included) is read.  The diagonal must be non-zero; a zero or
 *    non-finite diagonal entry is not detected and gives non-finite output.
 *  - Linv: n x n output, ldi >= n; lower triangle = L^{-1}, strict upper
 *    triangle = 0.  Linv == L (same ld) inverts in place; otherwise the two
 *    must not overlap.  The strict upper triangle of Linv is scratch during
 *    the call.
 *  - FP64 throughout (FP64 tensor-core products); needs no workspace and
 *    allocates nothing.  n == 0 returns GPC_OK without touching anything.
 *  - Returns GPC_ERR_INVALID_ARG (nothing enqueued) for n < 0, a null pointer
 *    or ld < n, or partially overlapping L and Linv; GPC_ERR_CUDA on a launch
 *    error.
 */
int gpc_tri_inverse(int n, const double *L, int ldl, double *Linv, int ldi, gpc_stream_t stream);

/*
 * Triangular solve with a matrix right-hand side, C = L^{-1} B (Section 3.2,
 * general solver: the inverse, then one product with it).
 *  - L: n x n lower (ldl >= n; lower triangle read).  B: n x m (ldb >= m).
 *  - Linv: n x n output (ldi >= n), written as by gpc_tri_inverse and kept for
 *    gpc_tri_solve_adjoint; Linv == L (same ld) is allowed.
 *  - C: n x m output (ldc >= m); must not overlap B, L or Linv.  B must not
 *    overlap Linv.
 *  - m == 0 computes only Linv.  FP64; no workspace.
 *  - Errors as gpc_tri_inverse (plus m < 0, ldb or ldc < m, overlaps above).
 */
int gpc_tri_solve(int n, int m, const double *L, int ldl, const double *B, int ldb, double *Linv, int ldi,
                  double *C, int ldc, gpc_stream_t stream);

/*
 * Reverse mode of C = L^{-1} B (Section 3.2, reverse mode function) for a
 * scalar f with Cbar = df/dC:
 *   Bbar = L^{-T} Cbar          (product with the kept inverse)
 *   Lbar = -tril(Bbar C^T)      (the derivative with respect to the lower
 *                                entries of L, the only ones the solve reads)
 *  - Linv: n x n, ldi >= n, lower with a zero strict upper triangle (as
 *    written by gpc_tri_inverse / gpc_tri_solve).  C, Cbar: n x m inputs.
 *  - Bbar: n x m output (ldbb >= m); Lbar: n x n output (ldlb >= n), strict
 *    upper triangle set to 0.  Both are overwritten, never read (a caller that
 *    accumulates adjoints adds the results itself).
 *  - Neither output may overlap any input or the other output.  FP64; no
 *    workspace.  Errors as gpc_tri_solve.
 */
int gpc_tri_solve_adjoint(int n, int m, const double *Linv, int ldi, const double *C, int ldc,
                          const double *Cbar, int ldcb, double *Bbar, int ldbb, double *Lbar, int ldlb,
                          gpc_stream_t stream);

/*
 * General matrix product C = A B (Section 3.1, primitive function) on the FP64
 * tensor path.  A: m x k (lda >= k), B: k x n (ldb >= n), C: m x n (ldc >= n),
 * all row-major device arrays; C must not overlap A or B.  ws/ws_bytes: NULL/0,
 * or at least gpc_gemm_workspace_size() bytes, which lets a product whose
 * output is too small to fill the GPU split its k range over CTAs (the
 * paper's large-k special case; partial products summed in a fixed order).
 * k == 0 writes C = 0; m == 0 or n == 0 does nothing.  Errors:
 * GPC_ERR_INVALID_ARG for negative sizes, null pointers, short leading
 * dimensions, overlaps or a short non-null workspace (nothing enqueued);
 * GPC_ERR_CUDA on a launch error.
 */
int gpc_gemm_workspace_size(size_t *bytes);
int gpc_gemm(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C, int ldc,
             void *ws, size_t ws_bytes, gpc_stream_t stream);

/*
 * Reverse mode of C = A B (Section 3.1, reverse mode function) for a scalar f
 * with Cbar = df/dC (m x n, ldcb >= n):
 *   Abar = Cbar B^T   (m x k, ldab >= k),    Bbar = A^T Cbar   (k x n, ldbb >= n).
 * Both outputs are overwritten and must not overlap any input or each other.
 * Workspace and errors as gpc_gemm.
 */
int gpc_gemm_adjoint(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                     const double *Cbar, int ldcb, double *Abar, int ldab, double *Bbar, int ldbb, void *ws,
                     size_t ws_bytes, gpc_stream_t stream);

/*
 * Fused GLM log likelihood with its gradient (Section 3.4): for n
 * observations with covariates X (n x k, row-major, ldx >= k) and targets y,
 * eta_i = alpha + X_i . beta and, by family,
 *   GPC_GLM_NORMAL_ID        y_i ~ Normal(eta_i, sigma)          (sigma > 0)
 *   GPC_GLM_BERNOULLI_LOGIT  y_i ~ Bernoulli(1 / (1 + e^-eta_i)) (y_i in {0, 1})
 *   GPC_GLM_POISSON_LOG      y_i ~ Poisson(e^eta_i)              (y_i = 0, 1, 2, ...)
 * Writes lp = sum_i log p(y_i), dalpha = d lp / d alpha, dbeta (k) = d lp / d beta,
 * and dsigma = d lp / d sigma (normal family; d lp / d phi for the negative
 * binomial below; 0 otherwise); all four are
 * device pointers.  alpha and sigma are host scalars; y and beta are device
 * vectors.  One pass over X; results are bitwise reproducible.  The family's
 * support of y is not checked.
 *  - k <= GPC_GLM_MAX_K.  ws: at least gpc_glm_workspace_size(k) bytes.
 *  - Errors: GPC_ERR_INVALID_ARG for an unknown family, n < 0, k < 0 or
 *    k > GPC_GLM_MAX_K, sigma <= 0 (normal family), null pointers, ldx < k or
 *    a short workspace (nothing enqueued); GPC_ERR_CUDA on a launch error.
 */
#define GPC_GLM_NORMAL_ID 0
#define GPC_GLM_BERNOULLI_LOGIT 1
#define GPC_GLM_POISSON_LOG 2
#define GPC_GLM_NEG_BINOMIAL_LOG 3
#define GPC_GLM_MAX_K 12288
int gpc_glm_workspace_size(int k, size_t *bytes);
int gpc_glm(int family, long long n, int k, const double *X, long long ldx, const double *y, double alpha,
            const double *beta, double sigma, double *lp, double *dalpha, double *dbeta, double *dsigma,
            void *ws, size_t ws_bytes, gpc_stream_t stream);

/*
 * GPC_GLM_NEG_BINOMIAL_LOG (gpc_glm above, Section 3.4): y_i ~ NegBinomial with
 * mean mu_i = e^eta_i and dispersion phi = sigma (> 0), variance mu + mu^2/phi:
 *   log p(y_i) = lgamma(y_i + phi) - lgamma(y_i + 1) - lgamma(phi)
 *                + phi (log phi - log(mu_i + phi)) + y_i (eta_i - log(mu_i + phi));
 * dsigma receives d lp / d phi (with the digamma function).
 *
 * Ordinal-logit GLM (Section 3.4, ordinal regression): C ordered classes,
 * y_i in {0, .., C - 1} (device vector of exact integers), eta_i = X_i . beta
 * (no intercept: the C - 1 increasing cut points c_m take its place) and
 *   P(y = m) = s(eta - c_{m-1}) - s(eta - c_m),  s(t) = 1 / (1 + e^-t),
 * with s(eta - c_{-1}) = 1 and s(eta - c_{C-1}) = 0.  Writes lp = sum log P(y_i),
 * dbeta (k) and dcuts (C - 1) = d lp / d c (device pointers).  2 <= C <=
 * GPC_GLM_MAX_CLASSES; a y_i outside the classes makes lp NaN.  Workspace:
 * gpc_glm_workspace_size(k).  One pass over X, bitwise reproducible.
 *
 * Categorical-logit GLM (Section 3.4, multinomial logistic regression): C
 * classes, scores eta_ic = alpha_c + X_i . beta_c with alpha (C) and beta
 * (k x C, row-major: beta[j * C + c]) device arrays; lp_i = eta_{i,y_i} -
 * log sum_c e^eta_ic.  Writes lp, dalpha (C) and dbeta (k x C, same layout).
 * 2 <= C <= GPC_GLM_MAX_CLASSES and k C <= GPC_GLM_MAX_KC; a y_i outside the
 * classes makes lp NaN.  Workspace: gpc_glm_categorical_workspace_size(k, C).
 *
 * Both: GPC_ERR_INVALID_ARG (nothing enqueued) for n < 0, k < 0, C outside
 * its range, null pointers, ldx < k or a short workspace; GPC_ERR_CUDA on a
 * launch error.
 */
#define GPC_GLM_MAX_CLASSES 16
#define GPC_GLM_MAX_KC 8192
int gpc_glm_ordinal(long long n, int k, int C, const double *X, long long ldx, const double *y,
                    const double *beta, const double *cuts, double *lp, double *dbeta, double *dcuts, void *ws,
                    size_t ws_bytes, gpc_stream_t stream);
int gpc_glm_categorical_workspace_size(int k, int C, size_t *bytes);
int gpc_glm_categorical(long long n, int k, int C, const double *X, long long ldx, const double *y,
                        const double *alpha, const double *beta, double *lp, double *dalpha, double *dbeta,
                        void *ws, size_t ws_bytes, gpc_stream_t stream);

/*
 * Gaussian-process log marginal likelihood of y ~ N(0, K), the likelihood of
 * the paper's GP regression example (Section 4.2), evaluated through the
 * Cholesky factor (Section 3.3, primitive function) and two triangular solves
 * (Section 3.2):
 *   L = chol(K), z = L^{-1} y, alpha = L^{-T} z, logdet = 2 sum log L_ii,
 *   value = -1/2 y^T alpha - 1/2 logdet - (n/2) log(2 pi).
 * Writes L (may alias K when precision == GPC_FP64), alpha (n doubles), and
 * the device scalars logdet and value.  With GPC_MIXED the solve is refined
 * in FP64 against K (r = y - K alpha, alpha += L^{-T} L^{-1} r) until
 * |r| <= 1e-14 |y| or 10 rounds; K must then not alias L, and a refinement
 * that stops above tolerance sets info = {-1, GPC_ERR_NO_CONVERGENCE}.
 */
int gpc_gp_lml(int n, const double *K, int ldk, const double *y, double *L, int ldl,
               int precision, double *logdet, double *alpha, double *value, void *ws,
               size_t ws_bytes, int *info, gpc_stream_t stream);

/*
 * Kbar = gbar * d value / d K for the likelihood of gpc_gp_lml -- the reverse
 * pass that the GP regression example of Section 4.2 needs for its sampler's
 * gradient -- through the Cholesky adjoint (Section 3.3, reverse mode
 * function): Lbar = gbar (tril(alpha z^T) - diag(1 / L_ii)) with
 * z = L^T alpha (the reverse of the solves and of logdet = 2 sum log L_ii),
 * then Kbar = chol_adjoint(L, Lbar) (lower convention).
 */
int gpc_gp_lml_grad(int n, const double *L, int ldl, const double *alpha, double gbar,
                    double *Kbar, int ldkb, int precision, void *ws, size_t ws_bytes,
                    gpc_stream_t stream);

/*
 * Hyperparameter gradient from Kbar (lower convention) for the covariance of
 * gpc_se_cov -- the last step of the gradient that the GP regression example
 * of Section 4.2 takes with respect to its covariance hyperparameters (the
 * reverse mode of the covariance build): grad3 = (d/d alpha, d/d rho,
 * d/d sigma) of f, with
 *   d K_ij/d alpha = 2 K^f_ij / alpha, d K_ij/d rho = K^f_ij r2_ij / rho^3,
 *   d K_ii/d sigma = 2 sigma   (K^f: the noise-free part; jitter is constant),
 * summed over i >= j.  K^f is recomputed from X; grad3: 3 device doubles.
 * precision as for gpc_se_cov (GPC_MIXED: K^f and the per-thread sums in
 * double-float arithmetic, the per-tile sums in FP64).
 * The sums are formed per tile and then added in a fixed order, so repeated
 * calls give bitwise-identical results.  ws/ws_bytes: at least
 * gpc_se_hyper_grad_workspace_size(n) bytes.  Requires alpha != 0, rho > 0.
 */
int gpc_se_hyper_grad(int n, int d, const double *X, int ldx, double alpha, double rho,
                      double sigma, const double *Kbar, int ldkb, double *grad3, int precision,
                      void *ws, size_t ws_bytes, gpc_stream_t stream);

/* Workspace bytes gpc_se_hyper_grad needs at order n (*bytes: host pointer). */
int gpc_se_hyper_grad_workspace_size(int n, size_t *bytes);

/*
 * Batched Gaussian-process likelihood and gradient for many independent GPs of
 * uneven size in one persistent launch.  The paper's batched diagonal
 * inverses (Section 3.2) give each small problem its own thread block; here
 * each thread block takes whole GPs from a device queue ordered by size,
 * largest first, and runs for each: the SE covariance of gpc_se_cov (jitter 0),
 * the Cholesky factorisation, the two solves, the log marginal likelihood of
 * gpc_gp_lml, Kbar of gpc_gp_lml_grad and the gradient of gpc_se_hyper_grad.
 * All arrays are device arrays:
 *   n[i]       order of GP i (1 <= n[i] <= nmax; larger sizes set info[i] to
 *              {-1, GPC_ERR_INVALID_ARG} on the device and skip the GP)
 *   offK[i]    element offset of GP i's n[i] x n[i] matrix in Kws (ld = n[i]);
 *              Kws receives the Cholesky factor (lower, zero upper)
 *   rowX[i]    first row of GP i in X (n x d, row-major, ld = d) and in y
 *   hyp[3i..]  (alpha, rho, sigma) of GP i
 *   value[i], grad3[3i..3i+2], info[2i..2i+1]  outputs per GP (info as for
 *              gpc_chol; a GP whose factorisation fails gets NaN outputs)
 * nmax: host int, at most 4096; workspace from gpc_batched_workspace_size
 * for the same precision (per SM room for Kbar, the kernel values, the
 * diagonal-block inverses and three vectors of order nmax; the mixed path
 * adds BF16 slice buffers of about 10 nmax^2 bytes, so an FP64 workspace is
 * too small for it).
 * The panel solves of the factorisation and of the adjoint are products with
 * the inverses of the diagonal blocks (formed once per block, right after it
 * is factored), and the forward and backward solves apply the same inverses.
 * precision GPC_FP64: every step in FP64.  GPC_MIXED: the O(n^3) products
 * (trailing updates of the factorisation and the adjoint's block products)
 * run on the tensor cores as split-BF16 slice products with FP32 group sums
 * folded into double-float accumulators (Section 3.3's blocked algorithms
 * with the products of Section 3.2 replaced); the diagonal blocks, the
 * solves and the log determinant stay FP64, and alpha is refined in FP64
 * against the FP64 covariance (residual K alpha - y) until the residual
 * stops shrinking.  Results do not depend on the order in which thread blocks
 * take GPs.  No counterpart of the API itself is in the paper.
 */
int gpc_batched_workspace_size(int batch, int nmax, int precision, size_t *bytes);
int gpc_batched_gp_lml_grad(int batch, int nmax, const int *n, const long long *offK, const long long *rowX, int d,
                            const double *X, const double *y, const double *hyp, int precision, double *Kws,
                            double *value, double *grad3, int *info, void *ws, size_t ws_bytes,
                            gpc_stream_t stream);

/*
 * Launch trace (no counterpart in the paper; measurement support).  The
 * library counts every kernel it launches; gpc_launch_count returns the
 * running total (host pointer *count).  gpc_trace_enable(1) clears the
 * per-class totals and starts recording a CUDA event pair around each launch
 * on the launching stream; gpc_trace_enable(2) does the same and also keeps a
 * timeline (one span per launch, cleared by this call); gpc_trace_enable(0)
 * stops and keeps what was recorded; other values return GPC_ERR_INVALID_ARG.
 * gpc_trace_summary synchronises the recorded events and returns, for one
 * class, the number of launches, their summed device time in ms and their
 * summed algorithmic flops and bytes (host pointers).
 * gpc_trace_timeline synchronises and copies up to max spans, in launch
 * order, into caller host arrays: class, kernel-name id, stream handle,
 * start (ms after the first traced launch began), device duration (ms) and
 * the launch's algorithmic flops;
 * *count receives the number of spans held (at most 2^21).  gpc_trace_name
 * writes the NUL-terminated kernel name of a name id into buf (truncated to
 * buf_bytes - 1 characters).  Not thread-safe; meant for benchmarks.
 */
#define GPC_TRACE_GEMM_F64 0   /* FP64 DMMA products (trailing update, adjoint) */
#define GPC_TRACE_DIAG 1       /* diagonal-block factor / inverse */
#define GPC_TRACE_TRSV 2       /* triangular solves */
#define GPC_TRACE_SECOV 3      /* covariance build */
#define GPC_TRACE_HYPER 4      /* hyperparameter gradient */
#define GPC_TRACE_ELEM 5       /* copies, reductions and other small kernels */
#define GPC_TRACE_GEMM_MIXED 6 /* split-BF16 tensor-core products */
#define GPC_TRACE_SPLIT 7      /* FP64 -> BF16 slice splitting */
#define GPC_TRACE_TRSM 8       /* FP64 panel solves against a diagonal block */
#define GPC_TRACE_GLM 9        /* fused GLM likelihood and gradient */
#define GPC_TRACE_CLASSES 10
int gpc_launch_count(long long *count);

/*
 * FP64 tensor-core throughput of the current device (measurement support, no
 * counterpart in the paper): runs an mma.sync m16n8k16 .f64 issue-rate kernel
 * (eight independent accumulator chains per warp, 32 warps per SM) three times
 * and returns the best rate in GFLOP/s in *gflops (host pointer).  ws: device
 * scratch of at least 8 * 128 * 8 * (SM count) bytes (4 MiB covers any
 * current device).  Synchronises
 * the stream.  Used as the roofline denominator of the FP64 products.
 */
int gpc_fp64_peak(void *ws, size_t ws_bytes, double *gflops, gpc_stream_t stream);
int gpc_trace_enable(int on);
int gpc_trace_summary(int cls, long long *launches, double *ms, double *flops, double *bytes);
int gpc_trace_timeline(long long max, int *cls, int *name, unsigned long long *stream, float *start_ms,
                       float *dur_ms, double *flops, long long *count);
int gpc_trace_name(int name, char *buf, size_t buf_bytes);

#ifdef __cplusplus
}
#endif

#endif /* GPCHOL_H */
