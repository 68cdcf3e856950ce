// GPU side of the seeded input generators (see datagen/__init__.py for the
// NumPy side and the recipe). Holds no aggregation arithmetic: it only writes
// key and value columns, drawing the same SplitMix64 counter-based integers as
// the host generator, so integer columns are bit-identical on both sides.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr uint64_t kGamma = 0x9E3779B97F4A7C15ull;

__host__ __device__ inline uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ inline uint64_t stream_state(uint64_t seed, uint64_t stream) {
  return mix64(seed + kGamma * (stream + 1));
}
__device__ inline uint64_t draw(uint64_t st, int64_t i) { return mix64(st + kGamma * (uint64_t)(i + 1)); }
__device__ inline uint32_t perm32(uint32_t x) {
  x ^= x >> 16; x *= 0x7FEB352Du; x ^= x >> 15; x *= 0x846CA68Bu; x ^= x >> 16;
  return x;
}
__device__ inline uint64_t bounded(uint64_t u, uint64_t r) { return ((u >> 32) * r) >> 32; }

constexpr int kStreamKeys = 1, kStreamVals = 2, kStreamVals2 = 3, kStreamDomain = 7;

__global__ void keys_uniform(uint32_t* out, int64_t n, uint64_t st, uint32_t salt, uint64_t D, int64_t start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t idx = (uint32_t)bounded(draw(st, start + i), D);
    out[i] = perm32(idx ^ salt);
  }
}

__global__ void keys_zipf(uint32_t* out, int64_t n, uint64_t st, uint32_t salt, const uint64_t* t, int64_t D,
                          int64_t start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = draw(st, start + i);
    int64_t lo = 0, hi = D;  // first index with t[j] > u
    while (lo < hi) {
      int64_t mid = (lo + hi) >> 1;
      if (t[mid] <= u) lo = mid + 1; else hi = mid;
    }
    if (lo > D - 1) lo = D - 1;
    out[i] = perm32((uint32_t)lo ^ salt);
  }
}

__global__ void vals(void* out, int dt, int64_t n, uint64_t st, uint64_t st2, int64_t start) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t u = draw(st, start + i);
    switch (dt) {
      case 0: ((int32_t*)out)[i] = (int32_t)((int64_t)bounded(u, 1ull << 21) - (1 << 20)); break;
      case 1: ((int64_t*)out)[i] = (int64_t)(u >> 32); break;
      case 2: ((uint32_t*)out)[i] = (uint32_t)(u >> 32); break;
      default: {
        uint64_t u2 = draw(st2, start + i);
        double a = ((double)(u >> 11) + 0.5) * 0x1p-53;
        double b = (double)(u2 >> 11) * 0x1p-53;
        double z = sqrt(-2.0 * log(a)) * cos(2.0 * 3.141592653589793 * b) * 1e3;
        if (dt == 3) ((float*)out)[i] = (float)z; else ((double*)out)[i] = z;
      }
    }
  }
}

inline int grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" {

int dg_keys_uniform(uint32_t* out, int64_t n, uint64_t seed, uint64_t D, int64_t start, void* stream) {
  if (n <= 0) return 0;
  uint32_t salt = (uint32_t)stream_state(seed, kStreamDomain);
  keys_uniform<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, n, stream_state(seed, kStreamKeys), salt, D,
                                                              start);
  return (int)cudaGetLastError();
}

int dg_keys_zipf(uint32_t* out, int64_t n, uint64_t seed, const uint64_t* thresholds, int64_t D, int64_t start,
                 void* stream) {
  if (n <= 0) return 0;
  uint32_t salt = (uint32_t)stream_state(seed, kStreamDomain);
  keys_zipf<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, n, stream_state(seed, kStreamKeys), salt,
                                                           thresholds, D, start);
  return (int)cudaGetLastError();
}

int dg_values(void* out, int dtype, int64_t n, uint64_t seed, int64_t start, void* stream) {
  if (n <= 0) return 0;
  vals<<<grid_for(n), 256, 0, (cudaStream_t)stream>>>(out, dtype, n, stream_state(seed, kStreamVals),
                                                      stream_state(seed, kStreamVals2), start);
  return (int)cudaGetLastError();
}

}  // extern "C"
