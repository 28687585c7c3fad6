// Mixed-precision products on the fifth-generation tensor cores (tcgen05).
//
// The O(n^3) products of the blocked Cholesky and of its blocked adjoint
// (Section 3.3) are evaluated with an error-free split of the FP64 operands
// into BF16 slices (the Ozaki scheme: Ozaki, Ogita, Oishi & Rump, 2012).
//
// Splitting.  The K index of an operand is cut into chunks of at most 128.
// For every (row, chunk) the exponent e with |x| < 2^e over the chunk is found
// and each element is rounded to the fixed-point integer X = rint(|x| 2^(40-e))
// (40 bits), written with five balanced base-256 digits: d_2..d_5 in
// [-128, 127] (a digit >= 128 becomes d - 256 with a carry upward) and
// d_1 in [0, 256].  The slices v_p = sign(x) d_p 2^(e - 8p) are exact in
// BF16.  The exponent is folded into the slice values, so no exponent arrays
// travel with them.
//
// Products.  For one output tile and one K chunk (K <= 128) the slice
// products A_p B_q^T are accumulated on tcgen05 into four FP32 TMEM
// accumulators, grouped by p + q (1-based):
//   G2: (1,1)                 |sum| <= 128 * 256 * 256          = 2^23
//   G3: (1,2) (2,1)           |sum| <= 128 * 2 * 256 * 128      = 2^23
//   G4: (1,3) (2,2) (3,1)     |sum| <= 128 * (2^15+2^14+2^15)   < 2^24
//   G56: the 9 pairs with p + q in {5, 6}
// G2, G3 and G4 are sums of integers (in units of their slice scales) whose
// partial sums all stay below 2^24, so the tensor core accumulates them
// exactly whatever its internal rounding; G56 is rounded but lies 2^-32
// below G2.  Pairs with p + q > 6 are dropped (2^-40 below G2 per term).  One
// chunk's contribution is good to about 2^-38 relative to max|a| max|b|.
//
// Accumulation across chunks and into the output.  The output lives in
// "double-float" storage: each 8-byte element holds an FP32 pair (hi, lo)
// with value hi + lo (about 48 significant bits).  After each chunk the
// epilogue warps read G2, G3, G4, G56 from TMEM and add them into (hi, lo)
// with error-free FP32 two-sums, two outputs per packed f32x2 instruction.
// This keeps the FP64 pipe -- a small fraction of the FP32 and tensor rates
// on this part -- out of the inner loop; the factorisation converts a block
// column to FP64 only when it becomes the current panel.  The fold is most of
// the epilogue's instructions, and the epilogue, not the tensor core, sets
// the pace of a deep-K product: the packed form and TMEM loads issued one
// 8-column slice ahead took an 8192^2 x 1024 product from 0.71 to 0.82 of the
// measured sustained BF16 rate with bit-identical results.
//
// Kernel structure: persistent CTAs (one per SM), 10 warps: warp 0 issues TMA
// loads of the slice tiles (64B-swizzled, K-major, 32 wide) into a 3-stage ring,
// warp 1 owns TMEM and issues the MMAs from one thread, warps 2..9 are the
// epilogue (two per TMEM lane quarter, 32 columns each); they fetch their C
// elements before waiting for the accumulators so the read-modify-write of
// the output overlaps the MMAs.  TMEM holds two accumulator sets, so
// the epilogue of one chunk overlaps the MMAs of the next (4 x 64 columns per set, 512 in all).  Every mbarrier
// wait is bounded in time; a timeout sets GPC_ERR_TIMEOUT in the error word,
// drains the copies and MMAs already issued, frees TMEM and returns.
#include "common.cuh"
#include "slices.cuh"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

namespace gpc {
namespace {

constexpr int OZ_BM = 128, OZ_BN = 64, OZ_BK = 32, OZ_CHUNK = 128, OZ_S = kSlices, OZ_STAGES = 3;
constexpr int OZ_EPI_WARPS = 8;                         // two per TMEM lane quarter
constexpr int OZ_THREADS = 64 + 32 * OZ_EPI_WARPS;
constexpr int OZ_A_PLANE = OZ_BM * OZ_BK * 2;            // 8 KiB
constexpr int OZ_B_PLANE = OZ_BN * OZ_BK * 2;            // 4 KiB
constexpr int OZ_A_STAGE = OZ_S * OZ_A_PLANE;            // 40 KiB
constexpr int OZ_B_STAGE = OZ_S * OZ_B_PLANE;            // 20 KiB
constexpr int OZ_ACCS = 4;                               // G2, G3, G4, G56
constexpr int OZ_ACC_COLS = OZ_ACCS * OZ_BN;             // one accumulator set
constexpr int OZ_TMEM_COLS = 512;
constexpr int OZ_EPI_LD = 17;                           // padded row of an epilogue transpose buffer (float2, 8-byte path)
constexpr int OZ_EPI_LD2 = 18;                          // the same for the 16-byte path (rows 16-byte aligned)
constexpr int OZ_EPI_BUF = 32 * OZ_EPI_LD2 * 8;          // 32 rows x 16 columns of double-floats per warp
constexpr int OZ_SMEM_BYTES = OZ_STAGES * (OZ_A_STAGE + OZ_B_STAGE) + OZ_EPI_WARPS * OZ_EPI_BUF +
                              1024 /*barriers*/ + 1024 /*align*/;
constexpr unsigned long long kDrainNs = 2000000000ull;  // 2 s: bound of the waits that drain the kernel's own work

struct OzParams {
  int M, N, chunks, qpc;  // qpc: 32-wide K stages used per chunk (chunks shorter than 128)
  int a_row0, b_row0, a_k0, b_k0;
  int lower, splits, tiles_m, tiles_n, num_work;
  float alpha;
  float2 *C;
  long long ldc;
  float2 *partial;
  int *err;                    // per-call status slot (may be null)
  int *gerr;                   // library error word (may be null)
  unsigned long long wait_ns;  // budget of each bounded wait
  int no_loads;                // test hook: the copy warp issues nothing
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// try_wait with a suspend-time hint: a waiting thread is parked until the
// phase completes or the hint (ns) runs out, instead of spinning and taking
// issue slots from the warps that do the work.
constexpr uint32_t kSuspendNs = 20000;
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred P;\n mbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2, %3;\n"
      " selp.b32 %0, 1, 0, P;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendNs)
      : "memory");
  return ok != 0;
}
// Bounded wait: false after wait_ns or when another role has aborted.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag,
                                          unsigned long long wait_ns) {
  if (mbar_try(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (unsigned it = 1;; ++it) {
    if (mbar_try(bar, parity)) return true;
    if ((it & 63) == 0) {
      if (*abort_flag) return false;
      if (global_ns() - t0 > wait_ns) return false;
    }
  }
}
// Wait that ignores the abort flag (used only to drain own work), bounded.
__device__ __forceinline__ bool mbar_wait_drain(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = global_ns();
  for (;;) {
    if (mbar_try(bar, parity)) return true;
    if (global_ns() - t0 > kDrainNs) return false;
  }
}
__device__ __forceinline__ void report_timeout(const OzParams &p) {
  if (p.err) atomicExch(p.err, GPC_ERR_TIMEOUT);
  record_error(p.gerr, GPC_ERR_TIMEOUT);
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int x, int y, int z,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 64B swizzle (rows of 32 BF16),
// 8-row groups 512 B apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
  uint64_t d = 0;
  d |= (uint64_t)((addr & 0x3FFFF) >> 4);       // start address
  d |= (uint64_t)1 << 16;                        // leading byte offset (16 B; unused for swizzled K-major)
  d |= (uint64_t)(512 >> 4) << 32;               // stride byte offset
  d |= (uint64_t)1 << 46;                        // descriptor version
  d |= (uint64_t)4 << 61;                        // 64B swizzle
  return d;
}
// Instruction descriptor: BF16 x BF16 -> FP32, both K-major, M = 128, N = n.
__host__ __device__ constexpr uint32_t idesc_n(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(OZ_BM >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The 15 slice products of one K = 16 step in 9 MMAs.  The B slice planes
// lie one after another in shared memory (64 rows each, same swizzle), so
// planes q..q+c-1 form one operand of N = 64 c rows, and a_p times that
// operand writes the products a_p b_q .. a_p b_{q+c-1} into consecutive
// 64-column accumulators.  With the accumulators G2 | G3 | G4 | G56 at
// columns 0, 64, 128, 192 of a set, a_p b_1.. lands in the group p + q
// wherever p + q <= 4, and every product with p + q in {5, 6} goes to G56:
//   a1 [b1 b2 b3 b4] -> G2 G3 G4 G56   a1 b5 -> G56
//   a2 [b1 b2 b3]    -> G3 G4 G56      a2 b4 -> G56
//   a3 [b1 b2]       -> G4 G56         a3 b3 -> G56
//   a4 b1, a4 b2, a5 b1                -> G56
// The first MMA of a chunk (first == 0) overwrites all four accumulators.
// da, db: descriptors of the first A and B plane of this K step; a plane
// further is a fixed increment of the 14-bit address field (shared-memory
// addresses stay below 2^18, so the field cannot carry into the next one).
__device__ __forceinline__ void ozaki_kstep(uint32_t tacc, uint64_t da, uint64_t db, uint32_t first) {
  constexpr uint32_t n64 = idesc_n(64), n128 = idesc_n(128), n192 = idesc_n(192), n256 = idesc_n(256);
  constexpr uint64_t pa = OZ_A_PLANE >> 4, pb = OZ_B_PLANE >> 4;
  const uint32_t g56 = tacc + 3 * OZ_BN;
  mma_bf16(tacc, da, db, n256, first);
  mma_bf16(g56, da, db + 4 * pb, n64, 1u);
  mma_bf16(tacc + OZ_BN, da + pa, db, n192, 1u);
  mma_bf16(g56, da + pa, db + 3 * pb, n64, 1u);
  mma_bf16(tacc + 2 * OZ_BN, da + 2 * pa, db, n128, 1u);
  mma_bf16(g56, da + 2 * pa, db + 2 * pb, n64, 1u);
  mma_bf16(g56, da + 3 * pa, db, n64, 1u);
  mma_bf16(g56, da + 3 * pa, db + pb, n64, 1u);
  mma_bf16(g56, da + 4 * pa, db, n64, 1u);
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
               : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// One 8-column slice of all four groups (G2, G3, G4, G56) of an accumulator
// set: g[grp][i] = column col0 + i of group grp.
__device__ __forceinline__ void tmem_ld_groups8(uint32_t taddr, float (&g)[4][8]) {
#pragma unroll
  for (int grp = 0; grp < 4; ++grp) {
    uint32_t r[8];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr + (uint32_t)(grp * OZ_BN)));
#pragma unroll
    for (int i = 0; i < 8; ++i) g[grp][i] = __uint_as_float(r[i]);
  }
}
// After tcgen05.wait::ld: pass the loaded registers through an empty asm so
// that no use of them can be scheduled above the wait.
__device__ __forceinline__ void tmem_pin(float (&g)[4][8]) {
#pragma unroll
  for (int grp = 0; grp < 4; ++grp)
#pragma unroll
    for (int i = 0; i < 8; ++i) asm volatile("" : "+f"(g[grp][i]));
}

// ------------------------------------------------------------------ double-float
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// Packed FP32 pairs: two values in one 64-bit register, added and subtracted
// lane by lane with the f32x2 instructions (IEEE round-to-nearest on each
// lane, so the results equal two scalar FADDs bit for bit at half the issue
// cost: the fold below is most of the epilogue's instruction stream).
typedef unsigned long long f2x;
__device__ __forceinline__ f2x pk2(float a, float b) {
  f2x d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void upk2(f2x d, float &a, float &b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(d));
}
__device__ __forceinline__ f2x add2(f2x a, f2x b) {
  f2x d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2x sub2(f2x a, f2x b) {
  f2x d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
// Knuth's two-sum on both lanes: s + e == a + b exactly.
__device__ __forceinline__ void two_sum2(f2x a, f2x b, f2x &s, f2x &e) {
  s = add2(a, b);
  const f2x bb = sub2(s, a);
  e = add2(sub2(a, sub2(s, bb)), sub2(b, bb));
}
// (hi, lo) += (g2 + g3 + g4 + g5) on two outputs at once, for one chunk's four
// slice groups (decreasing scale: each about 2^-8 of the one before): g2, g3
// and g4 enter the high part through exact two-sums, their errors and the
// rounded G56 group (whose own rounding sits near 2^-48 of g2) are added to
// the low part, then the pair is renormalised.  NEG subtracts instead (the
// sign bits are flipped first).
template <bool NEG>
__device__ __forceinline__ void df_acc2(f2x &hi, f2x &lo, f2x g2, f2x g3, f2x g4, f2x g5) {
  if (NEG) {
    constexpr f2x m = 0x8000000080000000ull;
    g2 ^= m;
    g3 ^= m;
    g4 ^= m;
    g5 ^= m;
  }
  f2x s, e1, e2, e3;
  two_sum2(hi, g2, s, e1);
  two_sum2(s, g3, s, e2);
  two_sum2(s, g4, s, e3);
  const f2x e = add2(add2(add2(lo, g5), add2(e1, e2)), e3);
  const f2x h = add2(s, e);
  lo = sub2(e, sub2(h, s));
  hi = h;
}
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, t;
  two_sum(a.x, b.x, s, t);
  const float e = __fadd_rn(__fadd_rn(a.y, b.y), t);
  const float hi = __fadd_rn(s, e);
  return make_float2(hi, __fsub_rn(e, __fsub_rn(hi, s)));
}

// ------------------------------------------------------------------ work list
__device__ __forceinline__ void work_coords(const OzParams &p, int w, int &tm, int &tn, int &c0, int &c1) {
  const int split = w % p.splits;
  int tile = w / p.splits;
  if (p.lower) {
    tm = 0;
    for (;;) {
      const int cnt = min(p.tiles_n, (tm * OZ_BM + OZ_BM - 1) / OZ_BN + 1);
      if (tile < cnt) break;
      tile -= cnt;
      ++tm;
    }
    tn = tile;
  } else {
    tm = tile / p.tiles_n;
    tn = tile - tm * p.tiles_n;
  }
  const int per = (p.chunks + p.splits - 1) / p.splits;
  c0 = split * per;
  c1 = min(p.chunks, c0 + per);
}

// ------------------------------------------------------------------ the GEMM
template <bool NEG>
__global__ void __launch_bounds__(OZ_THREADS, 1)
ozaki_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, OzParams p) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *smem = (unsigned char *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;
  unsigned char *sB = smem + OZ_STAGES * OZ_A_STAGE;
  float2 *epi_buf = (float2 *)(sB + OZ_STAGES * OZ_B_STAGE);
  uint64_t *bars = (uint64_t *)((unsigned char *)epi_buf + OZ_EPI_WARPS * OZ_EPI_BUF);
  // bars: full[3], empty[3], tfull[2], tempty[2], drain
  volatile int *abort_flag = (volatile int *)(bars + 16);
  uint32_t *tmem_slot = (uint32_t *)(bars + 17);
  const uint32_t full0 = smem_u32(bars + 0), empty0 = smem_u32(bars + OZ_STAGES);
  const uint32_t tfull0 = smem_u32(bars + 2 * OZ_STAGES), tempty0 = smem_u32(bars + 2 * OZ_STAGES + 2);
  const uint32_t drain = smem_u32(bars + 2 * OZ_STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < OZ_STAGES; ++i) {
      mbar_init(full0 + 8 * i, 1);
      mbar_init(empty0 + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(tfull0 + 8 * i, 1);
      mbar_init(tempty0 + 8 * i, OZ_EPI_WARPS);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(OZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tbase = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(&tmB) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      long long issued = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < p.num_work && ok && !p.no_loads; w += gridDim.x) {
        int tm, tn, c0, c1;
        work_coords(p, w, tm, tn, c0, c1);
        for (int c = c0; c < c1 && ok; ++c) {
          for (int h = 0; h < p.qpc; ++h) {
            if (!mbar_wait(empty0 + 8 * stage, phase ^ 1, abort_flag, p.wait_ns)) { ok = false; break; }
            mbar_expect_tx(full0 + 8 * stage, OZ_A_STAGE + OZ_B_STAGE);
            const int ka = p.a_k0 + c * OZ_CHUNK + h * OZ_BK;
            const int kb = p.b_k0 + c * OZ_CHUNK + h * OZ_BK;
            tma_load_3d(smem_u32(sA + stage * OZ_A_STAGE), &tmA, ka, p.a_row0 + tm * OZ_BM, 0, full0 + 8 * stage);
            tma_load_3d(smem_u32(sB + stage * OZ_B_STAGE), &tmB, kb, p.b_row0 + tn * OZ_BN, 0, full0 + 8 * stage);
            ++issued;
            if (++stage == OZ_STAGES) { stage = 0; phase ^= 1; }
          }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        report_timeout(p);
        // Drain: wait for the copies of the last (up to OZ_STAGES) issued loads.
        const long long first = issued > OZ_STAGES ? issued - OZ_STAGES : 0;
        for (long long i = first; i < issued; ++i) {
          const int st = (int)(i % OZ_STAGES);
          const uint32_t ph = (uint32_t)((i / OZ_STAGES) & 1);
          mbar_wait_drain(full0 + 8 * st, ph);
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int buf = 0;
      uint32_t tphase = 0;
      bool ok = true;
      bool any = false;
      for (int w = blockIdx.x; w < p.num_work && ok; w += gridDim.x) {
        int tm, tn, c0, c1;
        work_coords(p, w, tm, tn, c0, c1);
        for (int c = c0; c < c1 && ok; ++c) {
          if (!mbar_wait(tempty0 + 8 * buf, tphase ^ 1, abort_flag, p.wait_ns)) { ok = false; break; }
          fence_after();
          const uint32_t tacc = tbase + (uint32_t)(buf * OZ_ACC_COLS);
          for (int h = 0; h < p.qpc && ok; ++h) {
            if (!mbar_wait(full0 + 8 * stage, phase, abort_flag, p.wait_ns)) { ok = false; break; }
            fence_after();
            const uint64_t da = sdesc(smem_u32(sA + stage * OZ_A_STAGE));
            const uint64_t db = sdesc(smem_u32(sB + stage * OZ_B_STAGE));
#pragma unroll
            for (int k = 0; k < OZ_BK / 16; ++k)  // 16 BF16 = 32 bytes = 2 address units
              ozaki_kstep(tacc, da + 2 * k, db + 2 * k, (h == 0 && k == 0) ? 0u : 1u);
            mma_commit(empty0 + 8 * stage);
            any = true;
            if (++stage == OZ_STAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit(tfull0 + 8 * buf);
          if (++buf == 2) { buf = 0; tphase ^= 1; }
        }
      }
      if (!ok) {
        *abort_flag = 1;
        report_timeout(p);
      }
      // Drain: every MMA issued above completes before TMEM is released.
      if (any) {
        mma_commit(drain);
        mbar_wait_drain(drain, 0);
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9; lane quarter = warp % 4, column half by warp pair
    // Each warp owns a 32 x 32 block of the output: thread r holds row r's 32
    // columns (the TMEM lane layout).  C moves between global memory and the
    // registers through a padded shared-memory buffer, 16 columns at a time,
    // so that every global access of the warp covers two 128-byte row pieces.
    const int q = warp & 3, half = (warp - 2) >> 2;
    float2 *tb = epi_buf + (size_t)(warp - 2) * (OZ_EPI_BUF / 8);
    const int rl_lo = lane >> 4, cl = lane & 15;
    int buf = 0;
    uint32_t tphase = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < p.num_work && ok; w += gridDim.x) {
      int tm, tn, c0, c1;
      work_coords(p, w, tm, tn, c0, c1);
      const int split = w % p.splits;
      const int row0 = tm * OZ_BM + q * 32;
      const int colh = tn * OZ_BN + half * 32;
      float2 *base;
      long long ld;
      if (p.partial) {
        base = p.partial + (size_t)split * p.M * (size_t)p.N;
        ld = p.N;
      } else {
        base = p.C;
        ld = p.ldc;
      }
      // the double-float sum of this work item stays in registers across its
      // chunks: C is read once before the first chunk and written once after the last
      // (a split-K partial tile starts from zero and is written whole, so it is not read)
      float2 cv[32];
      // the warp's 32 x 32 block lies wholly inside the output (and below the
      // diagonal of a lower output): no per-element bounds tests
      const bool interior = row0 + 32 <= p.M && colh + 32 <= p.N && (!p.lower || colh + 31 < row0);
      // ... and its rows are 16-byte aligned: pairs of double-floats per access,
      // half the memory instructions
      const bool vec = interior && (ld & 1) == 0 && ((uintptr_t)base & 15) == 0;
      const int rq = lane >> 3, cp = lane & 7;  // 16-byte layout: 4 rows x 8 column pairs per access
      if (p.partial) {
#pragma unroll
        for (int i = 0; i < 32; ++i) cv[i] = make_float2(0.f, 0.f);
      } else if (vec) {
        const float2 *src = base + (long long)(row0 + rq) * ld + colh + 2 * cp;
#pragma unroll
        for (int hc = 0; hc < 2; ++hc)
#pragma unroll
          for (int it = 0; it < 8; ++it) {
            const float4 v = *reinterpret_cast<const float4 *>(src + (long long)(4 * it) * ld + hc * 16);
            cv[hc * 16 + 2 * it] = make_float2(v.x, v.y);
            cv[hc * 16 + 2 * it + 1] = make_float2(v.z, v.w);
          }
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
          for (int it = 0; it < 8; ++it)
            *reinterpret_cast<float4 *>(&tb[(4 * it + rq) * OZ_EPI_LD2 + 2 * cp]) =
                make_float4(cv[hc * 16 + 2 * it].x, cv[hc * 16 + 2 * it].y, cv[hc * 16 + 2 * it + 1].x,
                            cv[hc * 16 + 2 * it + 1].y);
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float4 v = *reinterpret_cast<const float4 *>(&tb[lane * OZ_EPI_LD2 + 2 * c]);
            cv[hc * 16 + 2 * c] = make_float2(v.x, v.y);
            cv[hc * 16 + 2 * c + 1] = make_float2(v.z, v.w);
          }
          __syncwarp();
        }
      } else {
        // all 32 loads in flight at once (cv holds them in the coalesced layout first)
        if (interior) {
          const float2 *src = base + (long long)(row0 + rl_lo) * ld + colh + cl;
#pragma unroll
          for (int hc = 0; hc < 2; ++hc)
#pragma unroll
            for (int it = 0; it < 16; ++it) cv[hc * 16 + it] = src[(long long)(2 * it) * ld + hc * 16];
        } else {
#pragma unroll
          for (int hc = 0; hc < 2; ++hc)
#pragma unroll
            for (int it = 0; it < 16; ++it) {
              const int rl = 2 * it + rl_lo, row = row0 + rl, col = colh + hc * 16 + cl;
              cv[hc * 16 + it] = (row < p.M && col < p.N && !(p.lower && col > row)) ? base[(long long)row * ld + col]
                                                                                     : make_float2(0.f, 0.f);
            }
        }
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
          for (int it = 0; it < 16; ++it) tb[(2 * it + rl_lo) * OZ_EPI_LD + cl] = cv[hc * 16 + it];
          __syncwarp();
#pragma unroll
          for (int c = 0; c < 16; ++c) cv[hc * 16 + c] = tb[lane * OZ_EPI_LD + c];
          __syncwarp();
        }
      }
      for (int c = c0; c < c1; ++c) {
        if (!mbar_wait(tfull0 + 8 * buf, tphase, abort_flag, p.wait_ns)) { ok = false; break; }
        fence_after();
        const uint32_t tacc = tbase + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * OZ_ACC_COLS) + half * 32;
        // Four 8-column slices, software-pipelined: the next slice's TMEM
        // loads are in flight while this slice is folded (two sets of group
        // registers, no more than one 16-column batch needed before).
        float ga[4][8], gb[4][8];
        auto fold8 = [&](int k, float(&g)[4][8]) {
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            float2 &c0 = cv[8 * k + i], &c1 = cv[8 * k + i + 1];
            f2x h = pk2(c0.x, c1.x), l = pk2(c0.y, c1.y);
            df_acc2<NEG>(h, l, pk2(g[0][i], g[0][i + 1]), pk2(g[1][i], g[1][i + 1]), pk2(g[2][i], g[2][i + 1]),
                         pk2(g[3][i], g[3][i + 1]));
            upk2(h, c0.x, c1.x);
            upk2(l, c0.y, c1.y);
          }
        };
        tmem_ld_groups8(tacc, ga);
        tmem_wait_ld();
        tmem_pin(ga);
        tmem_ld_groups8(tacc + 8, gb);
        fold8(0, ga);
        tmem_wait_ld();
        tmem_pin(gb);
        tmem_ld_groups8(tacc + 16, ga);
        fold8(1, gb);
        tmem_wait_ld();
        tmem_pin(ga);
        tmem_ld_groups8(tacc + 24, gb);
        fold8(2, ga);
        tmem_wait_ld();
        tmem_pin(gb);
        fold8(3, gb);
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(tempty0 + 8 * buf);
        if (++buf == 2) { buf = 0; tphase ^= 1; }
      }
      if (!ok) break;
      if (vec) {
        float2 *dst = base + (long long)(row0 + rq) * ld + colh + 2 * cp;
#pragma unroll
        for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
          for (int c = 0; c < 8; ++c)
            *reinterpret_cast<float4 *>(&tb[lane * OZ_EPI_LD2 + 2 * c]) =
                make_float4(cv[hc * 16 + 2 * c].x, cv[hc * 16 + 2 * c].y, cv[hc * 16 + 2 * c + 1].x,
                            cv[hc * 16 + 2 * c + 1].y);
          __syncwarp();
#pragma unroll
          for (int it = 0; it < 8; ++it)
            *reinterpret_cast<float4 *>(dst + (long long)(4 * it) * ld + hc * 16) =
                *reinterpret_cast<const float4 *>(&tb[(4 * it + rq) * OZ_EPI_LD2 + 2 * cp]);
          __syncwarp();
        }
        continue;
      }
#pragma unroll
      for (int hc = 0; hc < 2; ++hc) {
#pragma unroll
        for (int c = 0; c < 16; ++c) tb[lane * OZ_EPI_LD + c] = cv[hc * 16 + c];
        __syncwarp();
#pragma unroll
        for (int it = 0; it < 16; ++it) cv[hc * 16 + it] = tb[(2 * it + rl_lo) * OZ_EPI_LD + cl];
        __syncwarp();
      }
      if (interior) {
        float2 *dst = base + (long long)(row0 + rl_lo) * ld + colh + cl;
#pragma unroll
        for (int hc = 0; hc < 2; ++hc)
#pragma unroll
          for (int it = 0; it < 16; ++it) dst[(long long)(2 * it) * ld + hc * 16] = cv[hc * 16 + it];
      } else {
#pragma unroll
        for (int hc = 0; hc < 2; ++hc)
#pragma unroll
          for (int it = 0; it < 16; ++it) {
            const int rl = 2 * it + rl_lo, row = row0 + rl, col = colh + hc * 16 + cl;
            if (row < p.M && col < p.N && !(p.lower && col > row)) base[(long long)row * ld + col] = cv[hc * 16 + it];
          }
      }
    }
    if (!ok && lane == 0) {
      *abort_flag = 1;
      report_timeout(p);
    }
  }

  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(OZ_TMEM_COLS) : "memory");
  }
}

// ------------------------------------------------------------------ splitting
// Operand element (r, k) = src[r * rs + k * ks] for r < M, k < K.  Chunk 0
// covers k in [0, first), chunk c >= 1 covers [first + 128 (c - 1), + 128).
// Output planes: dst[p * plane + r * kpad + c * 128 + kk] (BF16), zero where
// the operand has no element; rows r >= row_end are not written.  Grid:
// (chunks, ceil(row_end / SPLIT_ROWS)), 256 threads, one row per warp.  The
// 8-row tile (8 KB of shared memory) lets a CTA run beside a product CTA on
// the same SM (which leaves about 11 KB free), so the splits of the chain do
// not wait for SMs while a product runs in the background.
constexpr int SPLIT_ROWS = 8;
__global__ void __launch_bounds__(256)
split_kernel(const double *src, long long rs, long long ks, int M, int K, int first, __nv_bfloat16 *dst,
             long long plane, int kpad, int row_end) {
  __shared__ double tile[SPLIT_ROWS][129];
  const int c = blockIdx.x, r0 = blockIdx.y * SPLIT_ROWS;
  const int kbeg = (c == 0) ? 0 : first + (c - 1) * OZ_CHUNK;
  const int klen = (c == 0) ? min(first, K) : min(OZ_CHUNK, K - kbeg);
  if (ks == 1) {
    for (int idx = threadIdx.x; idx < SPLIT_ROWS * 128; idx += blockDim.x) {
      const int rr = idx >> 7, kk = idx & 127;
      const int r = r0 + rr;
      tile[rr][kk] = (r < M && kk < klen) ? src[(long long)r * rs + (kbeg + kk)] : 0.0;
    }
  } else {
    for (int idx = threadIdx.x; idx < SPLIT_ROWS * 128; idx += blockDim.x) {
      const int kk = idx / SPLIT_ROWS, rr = idx % SPLIT_ROWS;
      const int r = r0 + rr;
      tile[rr][kk] = (r < M && kk < klen) ? src[(long long)r * rs + (long long)(kbeg + kk) * ks] : 0.0;
    }
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  static_assert(SPLIT_ROWS == 8, "one row per warp of 256 threads");
  {
    const int rr = warp;
    unsigned long long bits[4];
    int ex = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      bits[i] = (unsigned long long)__double_as_longlong(tile[rr][lane * 4 + i]);
      ex = max(ex, slice_exponent(bits[i]));
    }
    const int emax = __reduce_max_sync(0xffffffffu, ex);
    unsigned short out[OZ_S][4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      float v[OZ_S];
      split_value(bits[i], emax, v);
#pragma unroll
      for (int pp = 0; pp < OZ_S; ++pp) out[pp][i] = __bfloat16_as_ushort(__float2bfloat16_rn(v[pp]));
    }
    const int r = r0 + rr;
    if (r >= row_end) return;  // past the last barrier
#pragma unroll
    for (int pp = 0; pp < OZ_S; ++pp) {
      uint2 pack;
      pack.x = (unsigned)out[pp][0] | ((unsigned)out[pp][1] << 16);
      pack.y = (unsigned)out[pp][2] | ((unsigned)out[pp][3] << 16);
      *(uint2 *)(dst + pp * plane + (long long)r * kpad + c * OZ_CHUNK + lane * 4) = pack;
    }
  }
}

// ------------------------------------------------------------------ conversions
__global__ void to_df_lower_kernel(int n, const double *src, long long lds, float2 *dst, long long ldd) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)n * n) return;
  const int i = (int)(idx / n), j = (int)(idx - (long long)i * n);
  float2 v = make_float2(0.f, 0.f);
  if (j <= i) v = split_f64(src[(long long)i * lds + j]);
  dst[(long long)i * ldd + j] = v;
}

// lower triangle only: grid.y = row blocks of 4, 256 threads over the columns
__global__ void to_df_tri_kernel(int n, const double *src, long long lds, float2 *dst, long long ldd) {
  const int i = blockIdx.y * 4 + (threadIdx.x >> 6);
  if (i >= n) return;
  const double *row = src + (long long)i * lds;
  float2 *out = dst + (long long)i * ldd;
  for (int j = blockIdx.x * 64 + (threadIdx.x & 63); j <= i; j += gridDim.x * 64) out[j] = split_f64(row[j]);
}

__global__ void from_df_rect_kernel(int m, int c, double *p, long long ld) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)m * c) return;
  const int i = (int)(idx / c), j = (int)(idx - (long long)i * c);
  double *q = p + (long long)i * ld + j;
  const float2 v = *(const float2 *)q;
  *q = exact_f64(v.x) + exact_f64(v.y);
}

__global__ void df_reduce_kernel(int M, int N, int splits, const float2 *partial, float2 *C, long long ldc,
                                 int lower) {
  const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long long)M * N) return;
  const int row = (int)(idx / N), col = (int)(idx - (long long)row * N);
  if (lower && col > row) return;
  float2 acc = C[(long long)row * ldc + col];
  for (int s = 0; s < splits; ++s) acc = df_add(acc, partial[(size_t)s * M * N + idx]);
  C[(long long)row * ldc + col] = acc;
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

bool make_map(CUtensorMap *m, const SliceBuf &b, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)b.kpad, (cuuint64_t)b.rows_pad, (cuuint64_t)OZ_S};
  cuuint64_t strides[2] = {(cuuint64_t)b.kpad * 2, (cuuint64_t)b.rows_pad * b.kpad * 2};
  cuuint32_t box[3] = {(cuuint32_t)OZ_BK, (cuuint32_t)box_rows, (cuuint32_t)OZ_S};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void *)b.base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool g_oz_attr[64];

}  // namespace

int slices_count() { return OZ_S; }
int slice_chunk() { return OZ_CHUNK; }

size_t slice_bytes(int rows, int kchunks) {
  const size_t rp = align_up((size_t)std::max(rows, 1), OZ_BM);
  return align_up((size_t)OZ_S * rp * (size_t)kchunks * OZ_CHUNK * 2, 1024);
}

SliceBuf slice_view(void *base, int rows, int kchunks) {
  SliceBuf b;
  b.base = base;
  b.rows_pad = (int)align_up((size_t)std::max(rows, 1), OZ_BM);
  b.kpad = kchunks * OZ_CHUNK;
  return b;
}

cudaError_t split_operand(const double *src, long long rs, long long ks, int M, int K, int first,
                          const SliceBuf &out, cudaStream_t s, int chunk_offset, int row_offset) {
  if (M <= 0 || K <= 0) return cudaSuccess;
  const int op_chunks = (K <= first) ? 1 : 1 + (K - first + OZ_CHUNK - 1) / OZ_CHUNK;
  const int chunks = std::min(op_chunks, out.kpad / OZ_CHUNK - chunk_offset);
  if (chunks <= 0 || row_offset < 0 || row_offset + M > out.rows_pad) return cudaErrorInvalidValue;
  // rows written: the operand's M rows (at row_offset), or every row of the buffer when row_offset == 0
  const int row_end = row_offset > 0 ? M : out.rows_pad;
  static bool carveout_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !carveout_set[dev]) {  // the same shared-memory configuration as the products
    cudaError_t e = cudaFuncSetAttribute(split_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    carveout_set[dev] = true;
  }
  dim3 grid((unsigned)chunks, (unsigned)((row_end + SPLIT_ROWS - 1) / SPLIT_ROWS));
  const long long plane = (long long)out.rows_pad * out.kpad;
  GPC_LAUNCH(GPC_TRACE_SPLIT, 0.0, 8.0 * M * K + 2.0 * OZ_S * (double)row_end * chunks * OZ_CHUNK, s,
             launch_k(split_kernel, grid, 256, 0, s, src, rs, ks, M, K, first,
                      (__nv_bfloat16 *)out.base + (long long)row_offset * out.kpad + (long long)chunk_offset * OZ_CHUNK,
                      plane, out.kpad, row_end));
  return cudaGetLastError();
}

size_t ozaki_partial_bytes(int M, int N, int splits) {
  return splits > 1 ? align_up((size_t)splits * M * N * sizeof(float2), 256) : 0;
}

cudaError_t ozaki_gemm(const SliceBuf &A, int a_row0, int a_k0, const SliceBuf &B, int b_row0, int b_k0,
                       int M, int N, int chunks, bool lower, float alpha, float2 *C, long long ldc,
                       int splits, float2 *partial, int *err, cudaStream_t s, int max_ctas, int kdepth,
                       int max_items) {
  if (M <= 0 || N <= 0 || chunks <= 0) return cudaSuccess;
  if (kdepth <= 0) kdepth = OZ_CHUNK;
  if (kdepth > OZ_CHUNK || kdepth % OZ_BK) return cudaErrorInvalidValue;
  if (alpha != 1.0f && alpha != -1.0f) return cudaErrorInvalidValue;  // the epilogue applies a sign only
  CUtensorMap ma, mb;
  if (!make_map(&ma, A, OZ_BM) || !make_map(&mb, B, OZ_BN)) return cudaErrorInvalidValue;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_oz_attr[dev]) {
    cudaError_t e = cudaFuncSetAttribute(ozaki_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(ozaki_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, OZ_SMEM_BYTES);
    if (e != cudaSuccess) return e;
    g_oz_attr[dev] = true;
  }
  OzParams p;
  p.M = M;
  p.N = N;
  p.chunks = chunks;
  p.qpc = kdepth / OZ_BK;
  p.a_row0 = a_row0;
  p.b_row0 = b_row0;
  p.a_k0 = a_k0;
  p.b_k0 = b_k0;
  p.lower = lower ? 1 : 0;
  splits = std::max(1, std::min(splits, chunks));
  p.splits = splits;
  p.tiles_m = (M + OZ_BM - 1) / OZ_BM;
  p.tiles_n = (N + OZ_BN - 1) / OZ_BN;
  long long tiles = 0;
  if (lower) {
    for (int tm = 0; tm < p.tiles_m; ++tm) tiles += std::min(p.tiles_n, (tm * OZ_BM + OZ_BM - 1) / OZ_BN + 1);
  } else {
    tiles = (long long)p.tiles_m * p.tiles_n;
  }
  p.num_work = (int)(tiles * splits);
  p.alpha = alpha;
  p.C = C;
  p.ldc = ldc;
  p.partial = splits > 1 ? partial : nullptr;
  p.err = err;
  p.gerr = error_word();
  p.wait_ns = faults().wait_ns;
  p.no_loads = faults().ozaki_no_loads;
  const int ctas = max_ctas > 0 ? std::min(max_ctas, sm_count()) : sm_count();
  // output entries: the whole M x N block, or its lower part (col <= row)
  const double mn = !lower ? (double)M * N
                           : (M >= N ? 0.5 * (double)N * (N + 1) + (double)(M - N) * N : 0.5 * (double)M * (M + 1));
  const double flops = 2.0 * mn * (double)chunks * kdepth * 15.0;  // 15 slice products
  const double bytes = 16.0 * mn * chunks + (double)(M + N) * chunks * kdepth * 2 * OZ_S;
  int grid = std::min(p.num_work, ctas);
  if (max_items > 0) grid = std::max(grid, (p.num_work + max_items - 1) / max_items);
  if (alpha < 0.0f)
    GPC_LAUNCH(GPC_TRACE_GEMM_MIXED, flops, bytes, s,
               launch_k(ozaki_gemm_kernel<true>, grid, OZ_THREADS, OZ_SMEM_BYTES, s, ma, mb, p));
  else
    GPC_LAUNCH(GPC_TRACE_GEMM_MIXED, flops, bytes, s,
               launch_k(ozaki_gemm_kernel<false>, grid, OZ_THREADS, OZ_SMEM_BYTES, s, ma, mb, p));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  const long long total = (long long)M * N;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (splits + 2) * mn, s,
             df_reduce_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(M, N, splits, partial, C, ldc,
                                                                           lower ? 1 : 0));
  return cudaGetLastError();
}

cudaError_t to_df_tri(int n, const double *src, long long lds, float2 *dst, long long ldd, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const dim3 grid((unsigned)std::min((n + 63) / 64, 32), (unsigned)((n + 3) / 4));
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 8.0 * (double)n * (n + 1), s,
             to_df_tri_kernel<<<grid, 256, 0, s>>>(n, src, lds, dst, ldd));
  return cudaGetLastError();
}

cudaError_t to_df_lower(int n, const double *src, long long lds, double *dst, long long ldd, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  const long long total = (long long)n * n;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 12.0 * (double)total, s,
             to_df_lower_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(n, src, lds, (float2 *)dst, ldd));
  return cudaGetLastError();
}

cudaError_t from_df_rect(int m, int c, double *p, long long ld, cudaStream_t s) {
  if (m <= 0 || c <= 0) return cudaSuccess;
  const long long total = (long long)m * c;
  GPC_LAUNCH(GPC_TRACE_ELEM, 0.0, 16.0 * (double)total, s,
             from_df_rect_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m, c, p, ld));
  return cudaGetLastError();
}

}  // namespace gpc
