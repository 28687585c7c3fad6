// Mixed-precision blocked Cholesky and blocked adjoint (precision GPC_MIXED).
//
// Same block algorithms as the FP64 path (Section 3.3; see chol.cu), with the
// O(n^3) products moved to split-BF16 tensor-core products (ozaki.cu):
//   forward: the trailing update A22 -= L21 L21^T;
//   adjoint: Bbar -= Cbar R, Dbar -= Cbar^T C and Rbar -= [Dbar; Cbar]^T [R; B].
// The diagonal-block factors, their inverses, the panel solves and the Dbar
// symbolic step stay FP64.  Matrices that the split products update (the
// trailing part of L, the not-yet-final part of Lbar) are held in
// double-float storage (FP32 hi + lo in each 8-byte element); each block
// column is read as FP64 when it becomes current (the diagonal factor and the
// panel solves convert it as they load it), so every output is FP64 at the
// end.  The sweeps move by the 128-wide chunk of the split products so chunk
// boundaries line up with the blocks; within a block column the FP64 steps
// work on 64-wide halves (the blocked algorithm with b = 64 for its FP64
// steps, the updates of two consecutive 64-steps merged into one K = 128
// product), which halves the FP64 work of the panel solves and quarters that
// of the diagonal factors -- the FP64 pipe, not the tensor cores, bounds the
// critical path on this part.
#include "common.cuh"

#include <algorithm>
#include <mutex>

namespace gpc {
namespace {

constexpr int MB = 128;  // block size of the mixed path (== slice chunk)
constexpr int MH = 64;   // panel sub-block of the factorisation's FP64 steps
constexpr size_t kPartialCap = size_t(40) << 20;

#define TRY(x)                        \
  do {                                \
    cudaError_t e_ = (x);             \
    if (e_ != cudaSuccess) return e_; \
  } while (0)

struct MixWs {
  double *inv, *m, *t, *panel, *scratch;  // FP64 pieces (scratch doubles as the split-K partials)
  void *sc, *sdc, *lt;                    // slices: panel rows, block-column columns, L^T
};

size_t b2() { return align_up((size_t)MB * MB * sizeof(double), 256); }
constexpr int kSideSMs = 16;  // SMs left to the caller's stream while the adjoint's Bbar update runs

// Per-device auxiliary stream and events for the factorisation's lookahead.
struct Aux {
  cudaStream_t st = nullptr;
  cudaEvent_t ev_split = nullptr, ev_rest = nullptr;
};
std::mutex g_aux_mu;
Aux g_aux[64];

cudaError_t aux_for_device(Aux **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(g_aux_mu);
  Aux &a = g_aux[dev];
  if (!a.st) {
    if ((e = cudaStreamCreateWithFlags(&a.st, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&a.ev_split, cudaEventDisableTiming)) != cudaSuccess) return e;
    if ((e = cudaEventCreateWithFlags(&a.ev_rest, cudaEventDisableTiming)) != cudaSuccess) return e;
  }
  *out = &a;
  return cudaSuccess;
}
size_t scratch_bytes() { return std::max(gemm_f64_scratch_bytes(), kPartialCap); }
int nchunks(int n) { return std::max(1, (n + MB - 1) / MB); }

MixWs carve(void *ws, int n, bool adjoint) {
  char *p = (char *)ws;
  MixWs w{};
  w.inv = (double *)p; p += (size_t)nchunks(n) * b2();  // every diagonal-block inverse
  w.m = (double *)p; p += b2();
  w.t = (double *)p; p += b2();
  w.panel = (double *)p; p += align_up((size_t)n * MB * sizeof(double), 256);
  w.scratch = (double *)p; p += scratch_bytes();
  w.sc = p; p += 2 * slice_bytes(n, 1);  // two buffers: the next panel's slices while the last are in use
  if (adjoint) {
    w.sdc = p; p += slice_bytes(MB, nchunks(n));
    w.lt = p; p += slice_bytes(n, nchunks(n));
  }
  return w;
}

}  // namespace

size_t mixed_workspace_bytes(int n) {
  n = std::max(n, 1);
  return ((size_t)nchunks(n) + 2) * b2() + align_up((size_t)n * MB * sizeof(double), 256) + scratch_bytes() +
         2 * slice_bytes(n, 1) + slice_bytes(MB, nchunks(n)) + slice_bytes(n, nchunks(n)) + 1024;
}

// Lookahead: the trailing update of step k is split into the next block
// column (on the caller's stream, so step k+1 can start) and the rest (on an
// auxiliary stream, one SM left free).  Step k+1's conversion and diagonal
// factorisation then overlap the rest of step k's update; its panel solve,
// which needs the whole GPU's FP64 rate, waits for it.  Slices alternate
// between two buffers so a split never overwrites slices still being read.
cudaError_t chol_mixed(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s) {
  MixWs w = carve(ws, n, false);
  Aux *aux = nullptr;
  TRY(aux_for_device(&aux));
  bool rest_pending = false;
  int step = 0;
  for (int k0 = 0; k0 < n; k0 += MB, ++step) {
    const int nb = std::min(MB, n - k0), m = n - k0 - nb;
    double *A11 = L + (long long)k0 * ldl + k0;
    void *sbuf = (char *)w.sc + (size_t)(step & 1) * slice_bytes(n, 1);
    if (nb > MH) {
      // Two 64-wide steps: factor and solve the left half, update the right
      // half of the block column with it (split-BF16, K = 64), then factor and
      // solve the right half.  The FP64 work of the block column halves.  The
      // diagonal block's share of this (both halves' factors and the 64 x 64
      // update between them, a chain of small launches on a few SMs) runs
      // first, while the previous step's trailing update may still hold the
      // rest of the GPU; the panel rows below follow.
      const int hb = nb - MH;
      double *Aba = A11 + (long long)MH * ldl;  // right half's rows, left half's columns
      double *Ab = Aba + MH;                    // right half's diagonal block
      const size_t sb_small = slice_bytes(MH, 1);
      SliceBuf Sba = slice_view((char *)sbuf + slice_bytes(n, 1) - sb_small, hb, 1);
      TRY(potrf_diag(MH, A11, ldl, info, k0, s, true));
      TRY(trsm_rows(hb, MH, Aba, ldl, A11, ldl, 0, s, true));
      TRY(split_operand(Aba, ldl, 1, hb, MH, MH, Sba, s));
      TRY(ozaki_gemm(Sba, 0, 0, Sba, 0, 0, hb, hb, 1, true, -1.0f, (float2 *)Ab, ldl, 1, nullptr,
                     info ? info + 1 : nullptr, s, 0, MH));
      TRY(potrf_diag(hb, Ab, ldl, info, k0 + MH, s, true));
      if (rest_pending) {
        TRY(cudaStreamWaitEvent(s, aux->ev_rest, 0));
        rest_pending = false;
      }
      if (m <= 0) continue;
      double *Ca = A11 + (long long)nb * ldl;  // panel rows below the diagonal block, left half
      TRY(trsm_rows(m, MH, Ca, ldl, A11, ldl, 0, s, true));
      SliceBuf Sc = slice_view(sbuf, m, 1);
      TRY(split_operand(Ca, ldl, 1, m, MH, MH, Sc, s));
      TRY(ozaki_gemm(Sc, 0, 0, Sba, 0, 0, m, hb, 1, false, -1.0f, (float2 *)(Ca + MH), ldl, 1, nullptr,
                     info ? info + 1 : nullptr, s, 0, MH));
      TRY(trsm_rows(m, hb, Ca + MH, ldl, Ab, ldl, 0, s, true));
    } else {
      TRY(potrf_diag(nb, A11, ldl, info, k0, s, true));
      if (rest_pending) {
        TRY(cudaStreamWaitEvent(s, aux->ev_rest, 0));
        rest_pending = false;
      }
      if (m <= 0) continue;
      TRY(trsm_rows(m, nb, A11 + (long long)nb * ldl, ldl, A11, ldl, 0, s, true));  // L21 = A21 L11^{-T} (FP64)
    }
    double *A21 = L + (long long)(k0 + nb) * ldl + k0;
    // A22 -= L21 L21^T on split-BF16 slices, lower part, double-float storage
    SliceBuf S = slice_view(sbuf, m, 1);
    TRY(split_operand(A21, ldl, 1, m, nb, nb, S, s));
    const int nb2 = std::min(MB, m);
    float2 *T = (float2 *)(A21 + nb);
    TRY(ozaki_gemm(S, 0, 0, S, 0, 0, m, nb2, 1, true, -1.0f, T, ldl, 1, nullptr, info ? info + 1 : nullptr, s));
    if (m > nb2) {
      TRY(cudaEventRecord(aux->ev_split, s));
      TRY(cudaStreamWaitEvent(aux->st, aux->ev_split, 0));
      TRY(ozaki_gemm(S, nb2, 0, S, nb2, 0, m - nb2, m - nb2, 1, true, -1.0f,
                     (float2 *)(A21 + nb + (long long)nb2 * ldl + nb2), ldl, 1, nullptr,
                     info ? info + 1 : nullptr, aux->st, sm_count() - 1));
      TRY(cudaEventRecord(aux->ev_rest, aux->st));
      rest_pending = true;
    }
  }
  if (rest_pending) TRY(cudaStreamWaitEvent(s, aux->ev_rest, 0));
  // every diagonal-block inverse, for the solves that follow the factorisation
  return trtri_batched(n, L, ldl, std::min(MB, n), MB, w.inv, s);
}

cudaError_t chol_adjoint_mixed(int n, const double *L, long long ldl, double *A, long long lda, void *ws,
                               int *err, cudaStream_t s) {
  MixWs w = carve(ws, n, true);
  const int nblk = nchunks(n);
  const int first = n - (nblk - 1) * MB;  // rows in the top-left block
  // L^T slices: operand row t = column t of L, K = rows of L, chunked like the sweep's blocks.
  SliceBuf LT = slice_view(w.lt, n, nblk);
  TRY(split_operand(L, 1, ldl, n, n, first, LT, s));
  TRY(trtri_batched(n, L, ldl, first, MB, w.inv, s));  // independent of the sweep: one launch
  Aux *aux = nullptr;
  TRY(aux_for_device(&aux));
  // Within a step the Bbar update (rows below, columns left: the largest
  // product) runs on the auxiliary stream on all but kSideSMs SMs while the
  // caller's stream takes the rest of the Dbar chain (three small FP64
  // products that fill only a few SMs) on the others; Rbar follows the chain
  // and takes SMs as the Bbar update frees them, and the next step's Cbar,
  // which both updates write, waits for both.
  const int side = std::min(kSideSMs, sm_count() / 4);
  for (int ib = nblk - 1; ib >= 0; --ib) {
    const int j = (ib == 0) ? 0 : first + (ib - 1) * MB;
    const int k = first + ib * MB;
    const int nb = k - j, m = n - k;
    const int chunks = nblk - ib;  // K chunks of the block column, rows j..n
    const double *D = L + (long long)j * ldl + j;
    double *Dbar = A + (long long)j * lda + j;
    const double *dinv = w.inv + (size_t)ib * MB * MB;
    SliceBuf SDC = slice_view(w.sdc, nb, chunks);
    bool bbar_pending = false;
    if (m > 0) {
      double *Cbar = A + (long long)k * lda + j;
      if (nb > MH) {
        // Cbar <- Cbar D^{-1} as two 64-wide steps, right half first: with
        // D = [Da 0; Dba Db], Xb = Cb Db^{-1}, then Ca -= Xb Dba (split-BF16,
        // K = nb - 64) and Xa = Ca Da^{-1}.  The FP64 solves halve.
        const int hb = nb - MH;
        double *Cb = Cbar + MH;
        const double *Dba = D + (long long)MH * ldl;
        TRY(trsm_rows(m, hb, Cb, lda, Dba + MH, ldl, 1, s, true));
        SliceBuf SX = slice_view((char *)w.sc + slice_bytes(n, 1), m, 1);
        SliceBuf SD = slice_view(w.sdc, MH, 1);
        TRY(split_operand(Cb, lda, 1, m, hb, hb, SX, s));
        TRY(split_operand(Dba, 1, ldl, MH, hb, hb, SD, s));  // row c, K index t: Dba[t][c]
        TRY(ozaki_gemm(SX, 0, 0, SD, 0, 0, m, MH, 1, false, -1.0f, (float2 *)Cbar, lda, 1, nullptr, err, s, 0,
                       (hb + 31) / 32 * 32));
        TRY(trsm_rows(m, MH, Cbar, lda, D, ldl, 1, s, true));
      } else {
        TRY(trsm_rows(m, nb, Cbar, lda, D, ldl, 1, s, true));  // Cbar <- Cbar D^{-1} (FP64)
      }
      // Dbar -= Cbar^T C on slices, Dbar still in double-float storage: the
      // columns of Cbar (K = rows k..n) fill chunks 1.. of the block column's
      // slices; C^T is rows j..k of the L^T slices.
      TRY(split_operand(Cbar, 1, lda, nb, m, MB, SDC, s, 1));
      const int dch = chunks - 1;
      int dsplits = std::max(1, std::min(dch, (2 * sm_count() + 1) / 2));
      while (dsplits > 1 && ozaki_partial_bytes(nb, nb, dsplits) > kPartialCap) --dsplits;
      TRY(ozaki_gemm(SDC, 0, MB, LT, j, (ib + 1) * MB, nb, nb, dch, true, -1.0f, (float2 *)Dbar, lda, dsplits,
                     (float2 *)w.scratch, err, s));
      if (j > 0) {  // Bbar -= Cbar R on slices (Bbar in double-float storage)
        SliceBuf SC = slice_view(w.sc, m, 1);
        TRY(split_operand(Cbar, lda, 1, m, nb, nb, SC, s));
        TRY(cudaEventRecord(aux->ev_split, s));
        TRY(cudaStreamWaitEvent(aux->st, aux->ev_split, 0));
        TRY(ozaki_gemm(SC, 0, 0, LT, 0, ib * MB, m, j, 1, false, -1.0f, (float2 *)(A + (long long)k * lda),
                       lda, 1, nullptr, err, aux->st, sm_count() - side));
        TRY(cudaEventRecord(aux->ev_rest, aux->st));
        bbar_pending = true;
      }
    }
    TRY(from_df_rect(nb, nb, Dbar, lda, s));
    {
      Gemm p;  // M = sym(tril(D^T Dbar))
      p.M = nb; p.N = nb; p.K = nb;
      p.A = D; p.lda = ldl; p.transA = true;
      p.B = Dbar; p.ldb = lda;
      p.C = w.m; p.ldc = nb;
      p.uplo = UPLO_LOWER_MIRROR;
      p.kskip = KSKIP_ROWS;  // D^T upper triangular
      p.algo_flops = (double)nb * nb * nb / 3.0;
      TRY(gemm_f64(p, w.scratch, s));
      Gemm t;  // T = M D^{-1}
      t.M = nb; t.N = nb; t.K = nb;
      t.A = w.m; t.lda = nb;
      t.B = dinv; t.ldb = nb;
      t.C = w.t; t.ldc = nb;
      t.kskip = KSKIP_COLS;  // D^{-1} lower triangular
      t.algo_flops = (double)nb * nb * (nb + 1);
      TRY(gemm_f64(t, w.scratch, s));
      Gemm d;  // Dbar = D^{-T} T, symmetric
      d.M = nb; d.N = nb; d.K = nb;
      d.A = dinv; d.lda = nb; d.transA = true;
      d.B = w.t; d.ldb = nb;
      d.C = Dbar; d.ldc = lda;
      d.uplo = UPLO_LOWER_MIRROR;
      d.kskip = KSKIP_ROWS;  // D^{-T} upper triangular
      d.algo_flops = (double)nb * nb * nb / 3.0 * 2.0;
      TRY(gemm_f64(d, w.scratch, s));
    }
    if (j > 0) {  // Rbar -= [Dbar; Cbar]^T [R; B] on slices (Rbar in double-float storage)
      TRY(split_operand(Dbar, 1, lda, nb, nb, nb, SDC, s, 0));  // chunk 0: the finished Dbar
      const int tiles = (j + 63) / 64;
      int splits = std::max(1, std::min(chunks, (2 * sm_count() + tiles - 1) / tiles));
      while (splits > 1 && ozaki_partial_bytes(nb, j, splits) > kPartialCap) --splits;
      TRY(ozaki_gemm(SDC, 0, 0, LT, 0, ib * MB, nb, j, chunks, false, -1.0f, (float2 *)(A + (long long)j * lda),
                     lda, splits, (float2 *)w.scratch, err, s));
    }
    TRY(phi_block(nb, Dbar, lda, s));
    if (bbar_pending) {
      TRY(cudaStreamWaitEvent(s, aux->ev_rest, 0));
      bbar_pending = false;
    }
  }
  return cudaSuccess;
}

}  // namespace gpc
