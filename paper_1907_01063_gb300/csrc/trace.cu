// Launch counter and optional per-class CUDA-event timing of every launch.
#include "common.cuh"

#include <algorithm>
#include <deque>
#include <mutex>
#include <vector>

namespace gpc {
namespace {

struct Rec {
  int cls;
  cudaEvent_t e0, e1;
  double flops, bytes;
};

struct TraceState {
  std::mutex mu;
  long long launches = 0;
  bool on = false;
  std::deque<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t pending = nullptr;  // begin event of the launch in progress
  long long cls_launches[GPC_TRACE_CLASSES] = {};
  double cls_ms[GPC_TRACE_CLASSES] = {};
  double cls_flops[GPC_TRACE_CLASSES] = {};
  double cls_bytes[GPC_TRACE_CLASSES] = {};
};

TraceState &st() {
  static TraceState t;
  return t;
}

cudaEvent_t get_event(TraceState &t) {
  if (!t.pool.empty()) {
    cudaEvent_t e = t.pool.back();
    t.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Folds finished records into the per-class totals.  Non-blocking mode stops
// at the first record whose end event has not completed, so the host never
// waits on the device while a traced workload is being enqueued.
void drain(TraceState &t, bool block) {
  while (!t.recs.empty()) {
    Rec &r = t.recs.front();
    if (r.e1) {
      if (block) {
        cudaEventSynchronize(r.e1);
      } else if (cudaEventQuery(r.e1) != cudaSuccess) {
        break;
      }
    }
    float ms = 0.f;
    if (r.e0 && r.e1 && cudaEventElapsedTime(&ms, r.e0, r.e1) == cudaSuccess) t.cls_ms[r.cls] += ms;
    t.cls_launches[r.cls] += 1;
    t.cls_flops[r.cls] += r.flops;
    t.cls_bytes[r.cls] += r.bytes;
    if (r.e0) t.pool.push_back(r.e0);
    if (r.e1) t.pool.push_back(r.e1);
    t.recs.pop_front();
  }
}

}  // namespace

void trace_begin(int /*cls*/, cudaStream_t s) {
  TraceState &t = st();
  if (!t.on) return;
  std::lock_guard<std::mutex> g(t.mu);
  t.pending = get_event(t);
  if (t.pending) cudaEventRecord(t.pending, s);
}

void trace_end(int cls, double flops, double bytes, cudaStream_t s) {
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  t.launches += 1;
  if (!t.on) return;
  cudaEvent_t e1 = get_event(t);
  if (e1) cudaEventRecord(e1, s);
  t.recs.push_back(Rec{cls, t.pending, e1, flops, bytes});
  t.pending = nullptr;
  if (t.recs.size() >= 4096) drain(t, t.recs.size() >= (1u << 20));
}

namespace {

// Issue-rate kernel for the FP64 tensor peak: per warp, eight independent
// accumulator chains of mma.sync m16n8k16 .f64, each with its own A and B
// fragments so that no two chains compute the same values (identical chains
// could legally be merged by the compiler and would overstate the rate).
constexpr int kPeakIters = 512;
constexpr int kPeakChains = 8;
__global__ void __launch_bounds__(128) fp64_peak_kernel(double *sink, double av, double bv) {
  double a[kPeakChains][8], b[4], c[kPeakChains][4];
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[q][k] = av + q * 1e-3 + k * 1e-13 + threadIdx.x * 1e-12;
#pragma unroll
    for (int r = 0; r < 4; ++r) c[q][r] = 0.0;
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) b[k] = bv + k * 1e-13;
  for (int i = 0; i < kPeakIters; ++i) {
#pragma unroll
    for (int q = 0; q < kPeakChains; ++q)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f64.f64.f64.f64 {%0,%1,%2,%3}, "
          "{%4,%5,%6,%7,%8,%9,%10,%11}, {%12,%13,%14,%15}, {%0,%1,%2,%3};\n"
          : "+d"(c[q][0]), "+d"(c[q][1]), "+d"(c[q][2]), "+d"(c[q][3])
          : "d"(a[q][0]), "d"(a[q][1]), "d"(a[q][2]), "d"(a[q][3]), "d"(a[q][4]), "d"(a[q][5]),
            "d"(a[q][6]), "d"(a[q][7]), "d"(b[0]), "d"(b[1]), "d"(b[2]), "d"(b[3]));
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kPeakChains; ++q) s += c[q][0] + c[q][1] + c[q][2] + c[q][3];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace gpc

using namespace gpc;

extern "C" {

int gpc_fp64_peak(void *ws, size_t ws_bytes, double *gflops, gpc_stream_t stream) {
  const int blocks = sm_count() * 8, threads = 128;
  if (!ws || !gflops || ws_bytes < (size_t)blocks * threads * sizeof(double)) return GPC_ERR_INVALID_ARG;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return GPC_ERR_CUDA;
  double best = 0.0;
  cudaError_t err = cudaSuccess;
  for (int rep = 0; rep < 3 && err == cudaSuccess; ++rep) {
    cudaEventRecord(e0, stream);
    fp64_peak_kernel<<<blocks, threads, 0, stream>>>((double *)ws, 0.5, 0.25);
    cudaEventRecord(e1, stream);
    err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    const double flops = 2.0 * 16 * 8 * 16 * kPeakChains * (double)kPeakIters * blocks * (threads / 32);
    if (err == cudaSuccess && ms > 0.f) best = std::max(best, flops / (ms * 1e-3) / 1e9);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (err == cudaSuccess) err = cudaGetLastError();
  *gflops = best;
  return err == cudaSuccess ? GPC_OK : GPC_ERR_CUDA;
}

int gpc_launch_count(long long *count) {
  if (!count) return GPC_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> g(st().mu);
  *count = st().launches;
  return GPC_OK;
}

int gpc_trace_enable(int on) {
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  drain(t, true);
  if (on) {
    for (int c = 0; c < GPC_TRACE_CLASSES; ++c) {
      t.cls_launches[c] = 0;
      t.cls_ms[c] = t.cls_flops[c] = t.cls_bytes[c] = 0.0;
    }
  }
  t.on = on != 0;
  return GPC_OK;
}

int gpc_trace_summary(int cls, long long *launches, double *ms, double *flops, double *bytes) {
  if (cls < 0 || cls >= GPC_TRACE_CLASSES || !launches || !ms || !flops || !bytes)
    return GPC_ERR_INVALID_ARG;
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  drain(t, true);
  *launches = t.cls_launches[cls];
  *ms = t.cls_ms[cls];
  *flops = t.cls_flops[cls];
  *bytes = t.cls_bytes[cls];
  return GPC_OK;
}

}  // extern "C"
