// Internal helpers shared by the library's translation units: error state,
// dtype traits, order-preserving integer images of values, compensated
// floating-point addition and 128-bit read-only loads.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/agg.h"

namespace agg {

// ---------------------------------------------------------------------------
// Host-side error reporting (thread-local last error).
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

#define AGG_CUDA_TRY(call)                                                         \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      ::agg::set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),     \
                       __FILE__, __LINE__);                                        \
      (void)cudaGetLastError(); /* a later launch check must not see it again */   \
      return e_ == cudaErrorMemoryAllocation ? AGG_ERR_OOM : AGG_ERR_CUDA;         \
    }                                                                              \
  } while (0)

#define AGG_CHECK_ARG(cond, ...)                                                   \
  do {                                                                             \
    if (!(cond)) {                                                                 \
      ::agg::set_error(__VA_ARGS__);                                               \
      return AGG_ERR_INVALID;                                                      \
    }                                                                              \
  } while (0)

// Device properties, cached per device.
struct DeviceInfo {
  int device = -1;
  int sm_count = 0;
  int smem_per_block_optin = 0;
  int smem_per_sm = 0;
  int l2_bytes = 0;
  int max_threads_per_sm = 0;
};
const DeviceInfo& device_info();  // of the current device

// Stream-ordered scratch owned by the library, cached per (device, stream).
// The returned block is at least `bytes` long and was zeroed when it was
// (re)allocated; self-resetting counters kept there must be left zeroed by
// every user.
void* stream_scratch(cudaStream_t s, size_t bytes, agg_status* st);
void* stream_pinned(cudaStream_t s, size_t bytes, agg_status* st);

// Device allocation (stream-ordered / plain); both honour agg_debug_fail_alloc.
cudaError_t dev_malloc_async(void** p, size_t bytes, cudaStream_t s);
cudaError_t dev_malloc(void** p, size_t bytes);

// Kernel-launch counter and optional per-phase event timing.
void note_launch(int k = 1);
struct PhaseTimer {
  int phase;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  PhaseTimer(int phase, cudaStream_t s);
  ~PhaseTimer();
};

// MurmurHash3's 32-bit finaliser (Appleby), a published bijective mixer.
__host__ __device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

inline int64_t next_pow2(int64_t x) {
  int64_t p = 1;
  while (p < x) p <<= 1;
  return p;
}

inline size_t dtype_size(int dt) {
  switch (dt) {
    case AGG_I32: case AGG_U32: case AGG_F32: return 4;
    case AGG_I64: case AGG_F64: return 8;
    default: return 0;
  }
}
inline bool dtype_valid(int dt) { return dt >= AGG_I32 && dt <= AGG_F64; }
inline bool dtype_is_fp(int dt) { return dt == AGG_F32 || dt == AGG_F64; }

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------

// Order-preserving unsigned images: a < b (in the value order, with
// -0.0 < +0.0 for floats) iff img(a) < img(b) as unsigned integers.
__device__ __forceinline__ uint32_t img_f32(float x) {
  uint32_t b = __float_as_uint(x);
  return b ^ ((uint32_t)((int32_t)b >> 31) | 0x80000000u);
}
__device__ __forceinline__ float f32_of_img(uint32_t m) {
  uint32_t b = (m & 0x80000000u) ? (m ^ 0x80000000u) : ~m;
  return __uint_as_float(b);
}
__device__ __forceinline__ uint64_t img_f64(double x) {
  uint64_t b = (uint64_t)__double_as_longlong(x);
  return b ^ ((uint64_t)((int64_t)b >> 63) | 0x8000000000000000ull);
}
__device__ __forceinline__ double f64_of_img(uint64_t m) {
  uint64_t b = (m & 0x8000000000000000ull) ? (m ^ 0x8000000000000000ull) : ~m;
  return __longlong_as_double((long long)b);
}
__host__ __device__ __forceinline__ uint64_t img_i64(int64_t v) {
  return (uint64_t)v ^ 0x8000000000000000ull;
}
__host__ __device__ __forceinline__ int64_t i64_of_img(uint64_t m) {
  return (int64_t)(m ^ 0x8000000000000000ull);
}

// Knuth's TwoSum: s + e == a + b exactly, with s = fl(a + b).
template <class F>
__device__ __forceinline__ void two_sum(F a, F b, F& s, F& e) {
  s = a + b;
  F bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// 128-bit streaming read-only load (not kept in L1).
__device__ __forceinline__ uint4 ld_stream_v4(const void* p) {
  uint4 v;
  asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

}  // namespace agg
