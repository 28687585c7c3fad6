// Library error word (gpc_get_error), per-device symbol addresses and the
// fault-injection knobs of the test hooks.
//
// The error word is one int per device in a file-scope __device__ variable.
// Kernels whose bounded waits give up record GPC_ERR_TIMEOUT there (first
// status wins), next to any per-call info the caller passed, so a timed-out
// wait is visible even in calls that take no info array (gpc_trsv,
// gpc_trsv_noalloc, gpc_chol_adjoint).  Host code reaches the variable only
// through its device address, looked up with cudaGetSymbolAddress with the
// device current and cached per device together with the context it belongs
// to: a new context (after cudaDeviceReset, say) reloads the module and
// triggers a fresh lookup instead of reusing a stale address.
#include "../../include/gpchol_testing.h"
#include "common.cuh"

#include <cuda.h>

#include <mutex>

namespace gpc {
namespace {

static __device__ __align__(256) int g_error_word[64];  // [0] used; padded to one 256-byte unit

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);

CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  });
  return fn;
}

void *current_context() {
  CtxGetCurrentFn fn = ctx_get_current();
  CUcontext c = nullptr;
  if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
  return (void *)c;
}

SymbolCache g_error_cache;

}  // namespace

cudaError_t symbol_address(const void *symbol, SymbolCache &cache, void **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= SymbolCache::kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> g(cache.mu);
  void *ctx = current_context();
  if (!cache.addr[dev] || !ctx || ctx != cache.ctx[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, symbol);  // makes the device's primary context current if none is
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    cache.addr[dev] = p;
    cache.ctx[dev] = current_context();
  }
  *out = cache.addr[dev];
  return cudaSuccess;
}

int *error_word() {
  void *p = nullptr;
  return symbol_address(g_error_word, g_error_cache, &p) == cudaSuccess ? (int *)p : nullptr;
}

namespace {
thread_local int t_launch_priority = 0;
}

int launch_priority() { return t_launch_priority; }

PriorityScope::PriorityScope(int p) : saved(t_launch_priority) { t_launch_priority = p; }
PriorityScope::~PriorityScope() { t_launch_priority = saved; }

int greatest_priority() {
  static int cached[SymbolCache::kMaxDevices];
  static bool have[SymbolCache::kMaxDevices];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= SymbolCache::kMaxDevices) return 0;
  if (!have[dev]) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) greatest = 0;
    cached[dev] = greatest;
    have[dev] = true;
  }
  return cached[dev];
}

Faults &faults() {
  static Faults f;
  return f;
}

}  // namespace gpc

using namespace gpc;

extern "C" int gpc_get_error(int *status, int clear, gpc_stream_t stream) {
  if (!status) return GPC_ERR_INVALID_ARG;
  int *word = error_word();
  if (!word) return GPC_ERR_CUDA;
  cudaStream_t s = stream;
  int host = 0;
  cudaError_t e = cudaMemcpyAsync(&host, word, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess && clear) e = cudaMemsetAsync(word, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return GPC_ERR_CUDA;
  *status = host;
  return GPC_OK;
}

extern "C" int gpc_test_set_fault(int key, long long value) {
  Faults &f = faults();
  switch (key) {
    case GPC_TEST_WAIT_NS:
      if (value < 0 || value > 10000000000LL) return GPC_ERR_INVALID_ARG;
      f.wait_ns = value == 0 ? Faults::kDefaultWaitNs : (unsigned long long)value;
      return GPC_OK;
    case GPC_TEST_TRSV_WITHHOLD:
      if (value < -1 || value > (1LL << 30)) return GPC_ERR_INVALID_ARG;
      f.trsv_withhold = (int)value;
      return GPC_OK;
    case GPC_TEST_OZAKI_NO_LOADS:
      if (value != 0 && value != 1) return GPC_ERR_INVALID_ARG;
      f.ozaki_no_loads = (int)value;
      return GPC_OK;
    default:
      return GPC_ERR_INVALID_ARG;
  }
}
