// Host runtime of the library: last-error state, per-device properties and
// the per-(device, stream) scratch cache used by the scan kernels.
#include <atomic>
#include <map>
#include <vector>
#include <mutex>
#include <utility>

#include "common.cuh"

namespace agg {

namespace {
thread_local std::string g_last_error;
std::mutex g_mu;
std::map<int, DeviceInfo> g_devices;

struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};
std::map<std::pair<int, cudaStream_t>, Scratch> g_scratch;
}  // namespace

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

void clear_error() { g_last_error.clear(); }

const DeviceInfo& device_info() {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_devices.find(dev);
  if (it != g_devices.end()) return it->second;
  DeviceInfo d;
  d.device = dev;
  cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d.smem_per_block_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&d.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev);
  cudaDeviceGetAttribute(&d.max_threads_per_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
  if (d.sm_count <= 0) d.sm_count = 1;
  // Keep freed stream-ordered allocations in this process's default pool
  // instead of unmapping them at every synchronisation: the GROUP BY paths
  // free and re-allocate large scratch on every call.
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
    uint64_t keep = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  return g_devices.emplace(dev, d).first->second;
}

// Scratch blocks only grow. A grown block replaces the old one in stream
// order (the old block is freed on the same stream), so work already queued
// on the stream keeps its memory until it has run.
void* stream_scratch(cudaStream_t s, size_t bytes, agg_status* st) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  Scratch& sc = g_scratch[{dev, s}];
  if (sc.bytes >= bytes) {
    *st = AGG_OK;
    return sc.ptr;
  }
  size_t want = bytes < (1u << 20) ? (1u << 20) : bytes;
  void* p = nullptr;
  cudaError_t e = dev_malloc_async(&p, want, s);
  if (e != cudaSuccess) {
    set_error("scratch allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    *st = e == cudaErrorMemoryAllocation ? AGG_ERR_OOM : AGG_ERR_CUDA;
    return nullptr;
  }
  e = cudaMemsetAsync(p, 0, want, s);
  if (e != cudaSuccess) {
    cudaFreeAsync(p, s);
    set_error("scratch clear failed: %s", cudaGetErrorString(e));
    *st = AGG_ERR_CUDA;
    return nullptr;
  }
  if (sc.ptr) cudaFreeAsync(sc.ptr, s);
  sc.ptr = p;
  sc.bytes = want;
  *st = AGG_OK;
  return p;
}

// ---------------------------------------------------------------------------
// Device allocations go through these two helpers so that a test can make the
// n-th one fail (agg_debug_fail_alloc) and check the error path.
// ---------------------------------------------------------------------------
namespace {
std::atomic<int64_t> g_fail_countdown{0};
bool injected_failure() {
  int64_t c = g_fail_countdown.load();
  while (c > 0) {
    if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 1;
  }
  return false;
}
}  // namespace

cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMallocAsync(p, bytes, s);
}

cudaError_t dev_malloc(void** p, size_t bytes) {
  if (injected_failure()) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  return cudaMalloc(p, bytes);
}

// A small pinned host buffer per (device, stream) for reading a few result
// words back without a pageable copy.
namespace {
std::map<std::pair<int, cudaStream_t>, Scratch> g_pinned;
}  // namespace

void* stream_pinned(cudaStream_t s, size_t bytes, agg_status* st) {
  auto& pinned = g_pinned;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_mu);
  Scratch& sc = pinned[{dev, s}];
  if (sc.bytes >= bytes) {
    *st = AGG_OK;
    return sc.ptr;
  }
  size_t want = bytes < 4096 ? 4096 : bytes;
  void* p = nullptr;
  cudaError_t e = cudaHostAlloc(&p, want, cudaHostAllocPortable);
  if (e != cudaSuccess) {
    set_error("pinned allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    *st = AGG_ERR_OOM;
    return nullptr;
  }
  if (sc.ptr) {
    cudaStreamSynchronize(s);
    cudaFreeHost(sc.ptr);
  }
  sc.ptr = p;
  sc.bytes = want;
  *st = AGG_OK;
  return p;
}

// ---------------------------------------------------------------------------
// Instrumentation.
// ---------------------------------------------------------------------------
namespace {
std::atomic<int64_t> g_launches{0};
std::atomic<bool> g_profile{false};
std::mutex g_prof_mu;
struct Pending {
  int phase;
  cudaEvent_t a, b;
};
std::vector<Pending> g_pending;
std::vector<cudaEvent_t> g_event_pool;
double g_ms[AGG_PHASES] = {0};
int64_t g_calls[AGG_PHASES] = {0};

cudaEvent_t take_event() {
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    if (!g_event_pool.empty()) {
      cudaEvent_t e = g_event_pool.back();
      g_event_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}
}  // namespace

void note_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

PhaseTimer::PhaseTimer(int ph, cudaStream_t st) : phase(ph), s(st) {
  if (!g_profile.load(std::memory_order_relaxed)) return;
  a = take_event();
  if (a) cudaEventRecord(a, s);
}

PhaseTimer::~PhaseTimer() {
  if (!a) return;
  cudaEvent_t b = take_event();
  if (!b) return;
  cudaEventRecord(b, s);
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_pending.push_back({phase, a, b});
}

}  // namespace agg

// Forget a stream: its device scratch is freed in stream order on the stream
// itself, its pinned read-back buffer once the stream has drained.
extern "C" agg_status agg_stream_release(void* stream) {
  using namespace agg;
  clear_error();
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0;
  AGG_CUDA_TRY(cudaGetDevice(&dev));
  Scratch sc, pin;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_scratch.find({dev, s});
    if (it != g_scratch.end()) {
      sc = it->second;
      g_scratch.erase(it);
    }
    auto jt = g_pinned.find({dev, s});
    if (jt != g_pinned.end()) {
      pin = jt->second;
      g_pinned.erase(jt);
    }
  }
  if (sc.ptr) AGG_CUDA_TRY(cudaFreeAsync(sc.ptr, s));
  if (pin.ptr) {
    AGG_CUDA_TRY(cudaStreamSynchronize(s));
    AGG_CUDA_TRY(cudaFreeHost(pin.ptr));
  }
  return AGG_OK;
}

extern "C" void agg_debug_fail_alloc(int64_t countdown) { agg::g_fail_countdown.store(countdown > 0 ? countdown : 0); }

extern "C" int64_t agg_launch_count(void) { return agg::g_launches.load(); }

extern "C" void agg_profile_enable(int on) { agg::g_profile.store(on != 0); }

extern "C" agg_status agg_profile_read(double* ms, int64_t* calls) {
  using namespace agg;
  std::vector<Pending> pend;
  {
    std::lock_guard<std::mutex> lk(g_prof_mu);
    pend.swap(g_pending);
  }
  agg_status st = AGG_OK;
  for (const Pending& p : pend) {
    float t = 0.f;
    if (cudaEventSynchronize(p.b) != cudaSuccess || cudaEventElapsedTime(&t, p.a, p.b) != cudaSuccess) {
      set_error("profile event failed");
      st = AGG_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_ms[p.phase] += t;
    g_calls[p.phase] += 1;
    g_event_pool.push_back(p.a);
    g_event_pool.push_back(p.b);
  }
  std::lock_guard<std::mutex> lk(g_prof_mu);
  for (int i = 0; i < AGG_PHASES; ++i) {
    if (ms) ms[i] = g_ms[i];
    if (calls) calls[i] = g_calls[i];
    g_ms[i] = 0;
    g_calls[i] = 0;
  }
  return st;
}

extern "C" const char* agg_last_error(void) { return agg::g_last_error.c_str(); }

extern "C" int agg_version(void) { return 101; }
