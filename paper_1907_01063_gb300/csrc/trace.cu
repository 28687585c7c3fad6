// Launch counter and optional per-class CUDA-event timing of every launch.
#include "common.cuh"

#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

namespace gpc {
namespace {

struct Rec {
  int cls;
  int name;
  cudaStream_t stream;
  cudaEvent_t e0, e1;
  double flops, bytes;
};

struct Span {
  int cls, name;
  unsigned long long stream;
  float start_ms, dur_ms;
  double flops;
};

constexpr size_t kMaxSpans = 1u << 21;

struct TraceState {
  std::mutex mu;
  long long launches = 0;
  bool on = false;
  std::deque<Rec> recs;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t pending = nullptr;  // begin event of the launch in progress
  int pending_name = -1;
  cudaStream_t pending_stream = nullptr;
  // timeline mode: one span per launch, start relative to the first traced launch
  bool timeline = false;
  cudaEvent_t base = nullptr;
  std::vector<Span> spans;
  std::vector<std::string> names;
  std::unordered_map<const char *, int> name_ids;
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
    if (t.timeline && r.e0 && t.spans.size() < kMaxSpans) {
      float start = 0.f;
      if (t.base) cudaEventElapsedTime(&start, t.base, r.e0);
      t.spans.push_back(Span{r.cls, r.name, (unsigned long long)(uintptr_t)r.stream, start, ms, r.flops});
    }
    if (r.e0 && r.e0 != t.base) t.pool.push_back(r.e0);
    if (r.e1) t.pool.push_back(r.e1);
    t.recs.pop_front();
  }
}

}  // namespace

// The kernel's name is the launch expression's text up to "<<<", or, for a
// launch through launch_k(kernel, ...), its first argument (commas inside
// template brackets belong to the name).
int name_id(TraceState &t, const char *what) {
  auto it = t.name_ids.find(what);
  if (it != t.name_ids.end()) return it->second;
  std::string n(what);
  const std::string lk = "launch_k(";
  const size_t at = n.find(lk);
  if (at != std::string::npos && n.find("<<<") == std::string::npos) {
    size_t i = at + lk.size(), depth = 0, end = i;
    for (; end < n.size(); ++end) {
      const char ch = n[end];
      if (ch == '<') ++depth;
      else if (ch == '>' && depth > 0) --depth;
      else if (ch == ',' && depth == 0) break;
    }
    n = n.substr(i, end - i);
  } else {
    const size_t cut = n.find("<<<");
    if (cut != std::string::npos) n.resize(cut);
  }
  while (!n.empty() && (n.back() == ' ' || n.back() == '\n')) n.pop_back();
  while (!n.empty() && (n.front() == ' ' || n.front() == '\n' || n.front() == '{')) n.erase(0, 1);
  const int id = (int)t.names.size();
  t.names.push_back(n);
  t.name_ids.emplace(what, id);
  return id;
}

void trace_begin(int /*cls*/, const char *what, cudaStream_t s) {
  TraceState &t = st();
  if (!t.on) return;
  std::lock_guard<std::mutex> g(t.mu);
  t.pending = get_event(t);
  t.pending_name = name_id(t, what);
  t.pending_stream = s;
  if (t.pending) {
    cudaEventRecord(t.pending, s);
    if (t.timeline && !t.base) t.base = t.pending;
  }
}

void trace_end(int cls, double flops, double bytes, cudaStream_t s) {
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  t.launches += 1;
  if (!t.on) return;
  cudaEvent_t e1 = get_event(t);
  if (e1) cudaEventRecord(e1, s);
  t.recs.push_back(Rec{cls, t.pending_name, t.pending_stream, t.pending, e1, flops, bytes});
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
  if (on < 0 || on > 2) return GPC_ERR_INVALID_ARG;
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  drain(t, true);
  if (on) {
    for (int c = 0; c < GPC_TRACE_CLASSES; ++c) {
      t.cls_launches[c] = 0;
      t.cls_ms[c] = t.cls_flops[c] = t.cls_bytes[c] = 0.0;
    }
    if (on == 2) {
      if (t.base) t.pool.push_back(t.base);
      t.base = nullptr;
      t.spans.clear();
    }
  }
  if (on) t.timeline = on == 2;  // stopping keeps the spans recorded so far
  t.on = on != 0;
  return GPC_OK;
}

int gpc_trace_timeline(long long max, int *cls, int *name, unsigned long long *stream, float *start_ms,
                       float *dur_ms, double *flops, long long *count) {
  if (!count || max < 0 || (max > 0 && (!cls || !name || !stream || !start_ms || !dur_ms || !flops)))
    return GPC_ERR_INVALID_ARG;
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  drain(t, true);
  const long long n = (long long)t.spans.size();
  *count = n;
  for (long long i = 0; i < std::min(n, max); ++i) {
    const Span &sp = t.spans[(size_t)i];
    cls[i] = sp.cls;
    name[i] = sp.name;
    stream[i] = sp.stream;
    start_ms[i] = sp.start_ms;
    dur_ms[i] = sp.dur_ms;
    flops[i] = sp.flops;
  }
  return GPC_OK;
}

int gpc_trace_name(int name, char *buf, size_t buf_bytes) {
  if (!buf || buf_bytes == 0) return GPC_ERR_INVALID_ARG;
  TraceState &t = st();
  std::lock_guard<std::mutex> g(t.mu);
  if (name < 0 || name >= (int)t.names.size()) return GPC_ERR_INVALID_ARG;
  const std::string &n = t.names[(size_t)name];
  const size_t len = std::min(n.size(), buf_bytes - 1);
  std::memcpy(buf, n.data(), len);
  buf[len] = '\0';
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
