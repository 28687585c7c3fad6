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
#include <cmath>
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
  void *grp, *tmp;                        // factorisation: two group buffers, per-step temporaries
};
constexpr int kMaxDefer = 8;
int defer_depth() { return std::max(1, std::min(tuning().mixed_defer, kMaxDefer)); }

size_t b2() { return align_up((size_t)MB * MB * sizeof(double), 256); }

// Per-device auxiliary stream and events for the factorisation's lookahead.
struct Aux {
  cudaStream_t st = nullptr;
  cudaEvent_t ev_split = nullptr, ev_rest = nullptr, ev_fork = nullptr;
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
    if ((e = cudaEventCreateWithFlags(&a.ev_fork, cudaEventDisableTiming)) != cudaSuccess) return e;
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
  } else {
    w.grp = p; p += 2 * slice_bytes(n, defer_depth());
    w.tmp = p; p += slice_bytes(n, 1);
  }
  return w;
}

}  // namespace

size_t mixed_workspace_bytes(int n) {
  n = std::max(n, 1);
  const size_t common = ((size_t)nchunks(n) + 2) * b2() + align_up((size_t)n * MB * sizeof(double), 256) +
                        scratch_bytes() + 2 * slice_bytes(n, 1) + 1024;
  const size_t adj = slice_bytes(MB, nchunks(n)) + slice_bytes(n, nchunks(n));
  const size_t fwd = 2 * slice_bytes(n, defer_depth()) + slice_bytes(n, 1);
  return common + std::max(adj, fwd);
}

// Factorisation with deferred trailing updates.  Block columns (128 wide)
// form groups of D = tuning().mixed_defer; the slices of a group's panels
// collect in one buffer (chunk t = the group's t-th block column, rows
// relative to the group's first column), and the group's update of the
// columns to its right is applied as products with K = 128 D:
//   * next-column update, after every block column (caller's stream): the
//     next block column minus the products of all of the group's block
//     columns so far (K = 128 (t + 1));
//   * after the group's last block column, on the auxiliary stream: the
//     strip (the next group's other block columns) and then the rest (every
//     column right of the next group), both with K = 128 D; the rest is cut
//     into D - 1 column slabs released one after each of the next group's
//     next-column updates.
// The background products leave tuning().mixed_free_sms SMs to the caller's
// stream, where the FP64 chain of the next group runs meanwhile (its panel
// solves also fit beside a product CTA on every SM: they use the FP64 pipes,
// the products the tensor cores).  The caller's stream waits for the strip
// before the first next-column update of the following group and for the
// rest before that group's last one -- the first writes into each update's
// region -- and group buffers alternate, so a split never overwrites slices
// still being read.  D = 1 is the one-block lookahead (rest of every step in
// the background).
cudaError_t chol_mixed(int n, double *L, long long ldl, void *ws, int *info, cudaStream_t s) {
  MixWs w = carve(ws, n, false);
  Aux *aux = nullptr;
  TRY(aux_for_device(&aux));
  const int D = defer_depth();
  const int nbc = nchunks(n);
  const int bg_ctas = std::max(1, sm_count() - std::max(0, std::min(tuning().mixed_free_sms, sm_count() / 2)));
  const int bg_items = std::max(0, tuning().mixed_cta_items);
  int *err = info ? info + 1 : nullptr;
  // the caller's stream carries the critical chain: its launches go first
  PriorityScope chain(tuning().mixed_priority ? greatest_priority() : 0);
  bool strip_pending = false, rest_pending = false;
  // The previous group's rest, cut into column slabs of about equal work: slab
  // i is released (by an event) after the i-th next-column update of the
  // current group, so the background work interleaves with the chain the way
  // a one-block lookahead does while every slab keeps K = 128 D.
  struct Slabs {
    SliceBuf G;
    int p0 = 0, chunks = 0, next = 0, count = 0;
    int cut[kMaxDefer + 1] = {};
  } slabs;
  auto launch_slab = [&]() -> cudaError_t {
    const int c0 = slabs.cut[slabs.next], c1 = slabs.cut[slabs.next + 1];
    ++slabs.next;
    cudaError_t e = cudaEventRecord(aux->ev_fork, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(aux->st, aux->ev_fork, 0);
    PriorityScope background(0);
    if (e == cudaSuccess && c1 > c0)
      e = ozaki_gemm(slabs.G, c0 - slabs.p0, 0, slabs.G, c0 - slabs.p0, 0, n - c0, c1 - c0, slabs.chunks, true,
                     -1.0f, (float2 *)(L + (long long)c0 * ldl + c0), ldl, 1, nullptr, err, aux->st, bg_ctas, 0,
                     bg_items);
    if (e == cudaSuccess && slabs.next == slabs.count) e = cudaEventRecord(aux->ev_rest, aux->st);
    return e;
  };
  for (int bc = 0; bc < nbc; ++bc) {
    const int g = bc / D, t = bc - g * D;
    const int p0 = g * D * MB, p1 = std::min(n, p0 + D * MB);
    const int k0 = bc * MB, nb = std::min(MB, n - k0), m = n - k0 - nb;
    double *A11 = L + (long long)k0 * ldl + k0;
    SliceBuf G = slice_view((char *)w.grp + (size_t)(g & 1) * slice_bytes(n, D), n - p0, D);
    // ---- FP64 steps of this block column (its updates are all applied)
    if (nb > MH) {
      // Two 64-wide steps: factor and solve the left half, update the right
      // half of the block column with it (split-BF16, K = 64), then factor and
      // solve the right half.  The diagonal block's share (both halves'
      // factors and the 64 x 64 update between them, a chain of small
      // launches) runs first; the panel rows below follow.
      const int hb = nb - MH;
      double *Aba = A11 + (long long)MH * ldl;  // right half's rows, left half's columns
      double *Ab = Aba + MH;                    // right half's diagonal block
      const size_t sb_small = slice_bytes(MH, 1);
      SliceBuf Sba = slice_view((char *)w.tmp + slice_bytes(n, 1) - sb_small, hb, 1);
      TRY(potrf_diag(MH, A11, ldl, info, k0, s, true));
      TRY(trsm_rows(hb, MH, Aba, ldl, A11, ldl, 0, s, true));
      TRY(split_operand(Aba, ldl, 1, hb, MH, MH, Sba, s));
      TRY(ozaki_gemm(Sba, 0, 0, Sba, 0, 0, hb, hb, 1, true, -1.0f, (float2 *)Ab, ldl, 1, nullptr, err, s, 0, MH));
      TRY(potrf_diag(hb, Ab, ldl, info, k0 + MH, s, true));
      if (m > 0) {
        double *Ca = A11 + (long long)nb * ldl;  // panel rows below the diagonal block, left half
        TRY(trsm_rows(m, MH, Ca, ldl, A11, ldl, 0, s, true));
        SliceBuf Sc = slice_view(w.tmp, m, 1);
        TRY(split_operand(Ca, ldl, 1, m, MH, MH, Sc, s));
        TRY(ozaki_gemm(Sc, 0, 0, Sba, 0, 0, m, hb, 1, false, -1.0f, (float2 *)(Ca + MH), ldl, 1, nullptr, err, s, 0,
                       MH));
        TRY(trsm_rows(m, hb, Ca + MH, ldl, Ab, ldl, 0, s, true));
      }
    } else {
      TRY(potrf_diag(nb, A11, ldl, info, k0, s, true));
      if (m > 0) TRY(trsm_rows(m, nb, A11 + (long long)nb * ldl, ldl, A11, ldl, 0, s, true));  // L21 = A21 L11^{-T}
    }
    if (m <= 0) continue;
    // ---- this block column's slices: chunk t of the group buffer, rows from k0 + nb
    const int r0 = k0 + nb - p0;  // first panel row, relative to the group
    TRY(split_operand(A11 + (long long)nb * ldl, ldl, 1, m, nb, nb, G, s, t, r0));
    // ---- next block column minus all of the group's block columns so far
    const int nb2 = std::min(MB, m);
    const bool last_in_group = (k0 + nb == p1);
    if (t == 0 && strip_pending) {  // the strip of the previous group writes this group's other columns
      TRY(cudaStreamWaitEvent(s, aux->ev_split, 0));
      strip_pending = false;
    }
    if (last_in_group && rest_pending) {  // the previous group's rest writes the next group's columns
      while (slabs.next < slabs.count) TRY(launch_slab());
      TRY(cudaStreamWaitEvent(s, aux->ev_rest, 0));
      rest_pending = false;
    }
    TRY(ozaki_gemm(G, r0, 0, G, r0, 0, m, nb2, t + 1, true, -1.0f, (float2 *)(A11 + (long long)nb * ldl + nb), ldl,
                   1, nullptr, err, s));
    if (rest_pending && slabs.next < slabs.count) TRY(launch_slab());
    if (!last_in_group || m <= nb2) continue;
    // ---- the group's deferred update of the columns right of the next block column
    const int q1 = p1 + nb2;                   // strip: [q1, p2) of the next group
    const int p2 = std::min(n, p1 + D * MB);   // the next group's end
    const int chunks = t + 1;
    TRY(cudaEventRecord(aux->ev_fork, s));
    TRY(cudaStreamWaitEvent(aux->st, aux->ev_fork, 0));
    PriorityScope background(0);
    if (p2 > q1) {
      TRY(ozaki_gemm(G, q1 - p0, 0, G, q1 - p0, 0, n - q1, p2 - q1, chunks, true, -1.0f,
                     (float2 *)(L + (long long)q1 * ldl + q1), ldl, 1, nullptr, err, aux->st, bg_ctas, 0,
                     bg_items));
      TRY(cudaEventRecord(aux->ev_split, aux->st));
      strip_pending = true;
    }
    if (n > p2) {
      slabs.G = G;
      slabs.p0 = p0;
      slabs.chunks = chunks;
      slabs.next = 0;
      // D - 1 slabs (one per next-column update before the next group's
      // last), cut where the remaining lower area falls by equal shares
      const int count = std::max(1, D - 1), width = n - p2;
      slabs.count = count;
      slabs.cut[0] = p2;
      for (int i = 1; i < count; ++i) {
        const double f = 1.0 - std::sqrt(1.0 - (double)i / count);
        const int c = p2 + (int)(f * width) / MB * MB;
        slabs.cut[i] = std::min(n, std::max(slabs.cut[i - 1], c));
      }
      slabs.cut[count] = n;
      rest_pending = true;
      if (D == 1) TRY(launch_slab());  // one-block lookahead: the rest goes at once
    }
  }
  while (rest_pending && slabs.next < slabs.count) TRY(launch_slab());
  if (strip_pending) TRY(cudaStreamWaitEvent(s, aux->ev_split, 0));
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
  // product) runs on the auxiliary stream on all but tuning().mixed_adj_free_sms
  // SMs (16 by default) while the
  // caller's stream takes the rest of the Dbar chain (three small FP64
  // products that fill only a few SMs) on the others; Rbar follows the chain
  // and takes SMs as the Bbar update frees them, and the next step's Cbar,
  // which both updates write, waits for both.
  const int side = std::min(tuning().mixed_adj_free_sms, sm_count() / 2);
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
