// Host runtime of the library: last-error state, per-device properties and
// the per-(device, stream) scratch cache used by the scan kernels.
#include <map>
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
  cudaError_t e = cudaMallocAsync(&p, want, s);
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

}  // namespace agg

extern "C" const char* agg_last_error(void) { return agg::g_last_error.c_str(); }

extern "C" int agg_version(void) { return 100; }
