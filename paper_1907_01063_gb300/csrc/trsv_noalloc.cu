// gpc_trsv_noalloc: the triangular solve of gpc_trsv for callers that cannot
// hand the library any device memory of their own for scratch.
//
// Who needs it: code that runs under a fixed device-memory budget owned by
// someone else (a sampler or framework that reserved all device memory up
// front through its own pool, where an extra cudaMalloc fails or fragments the
// pool), and latency-critical loops that must not call cudaMalloc/cudaFree
// because cudaFree can synchronise the whole device and stall other streams.
// Those callers still own x and L; only the solve's small scratch (a ticket
// counter and one ready flag per 64-row block) comes from a fixed array that
// lives in this file.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library holds its 16.25 KiB until the process exits.  In host code its name
// is only a host-side stand-in for the symbol, not a device address, so the
// device address is looked up with cudaGetSymbolAddress (with the device
// current) on the first call made on that device, and cached together with
// the device's current context.  A call in a different context (the old one
// destroyed by cudaDeviceReset, say, which also reloads the module) looks the
// address up again instead of using a stale one.  The first call in a context
// therefore does one extra runtime query; make it before any stream capture.
// A bounded wait of the solve that gives up records GPC_ERR_TIMEOUT in the
// library error word (gpc_get_error).  No call here allocates device or pinned
// memory.
#include "common.cuh"

namespace gpc {
namespace {

constexpr int kSolveBlock = 64;  // rows per block of the solve kernel
constexpr int kMaxBlocks = GPC_TRSV_NOALLOC_MAX_N / kSolveBlock;

// [0] ticket counter, [1 + b] ready flag of block b.  Shared by every call on
// a device and never freed; zeroed by each call before its kernel runs.
// Rounded up to whole 256-byte units, the granularity the solve's scratch
// size is quoted in.
constexpr int kScratchInts = (kMaxBlocks + 1 + 63) / 64 * 64;
static __device__ __align__(256) int g_trsv_scratch[kScratchInts];

SymbolCache g_scratch_cache;

// Device address of g_trsv_scratch on the current device and context (looked
// up on first use in each context).
cudaError_t scratch_address(void **out) { return symbol_address(g_trsv_scratch, g_scratch_cache, out); }

}  // namespace
}  // namespace gpc

using namespace gpc;

extern "C" int gpc_trsv_noalloc(int n, const double *L, int ldl, double *x, int trans,
                                gpc_stream_t stream) {
  if (n < 0 || n > GPC_TRSV_NOALLOC_MAX_N) return GPC_ERR_INVALID_ARG;
  if (n == 0) return GPC_OK;
  if (!L || ldl < n || !x) return GPC_ERR_INVALID_ARG;
  // The solve's own scratch need must fit the fixed array.
  if (trsv_workspace_bytes(n) > sizeof(g_trsv_scratch)) return GPC_ERR_INVALID_ARG;
  void *scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return GPC_ERR_CUDA;
  // gpc::trsv clears the ticket and flags it uses (on the stream) and then
  // launches the same solve kernel as gpc_trsv, with this array as its scratch;
  // a timed-out wait is recorded in the library error word.
  return trsv(n, L, ldl, x, trans, scratch, nullptr, stream) == cudaSuccess ? GPC_OK : GPC_ERR_CUDA;
}
