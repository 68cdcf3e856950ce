// Key sketch: 16 features of a strided sample of m = min(n, 4096)
// keys, computed by one block. The strategy selectors (the rule and the MLP)
// read them; the global table is sized from the GEE distinct-count estimate
// (Charikar, Chaudhuri, Motwani and Narasayya, PODS 2000).
#include <cmath>
#include <cstdint>

#include "groupby.cuh"

namespace agg {

constexpr int kSketchThreads = 1024;
constexpr int kSketchSlots = 2 * kSketchSample;  // hash slots for the sample (load <= 1/2)
constexpr size_t kSketchSmem = (size_t)kSketchSlots * 8 + (size_t)kSketchSlots * 4 + (kSketchSample + 1) * 4 + 64 * 4;

// Block-wide sum in a fixed order (deterministic). One thread adds the warp
// sums: GB300's float64 pipe is narrow, so the block does not repeat that
// serial chain in every thread.
__device__ double block_sum_d(double v, double* red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  const double t = red[32];
  __syncthreads();
  return t;
}

// One block. The sample's keys are counted in a shared-memory hash table
// (64-bit slots holding key << 1 | 1, so every key value is representable),
// their counts histogrammed, and the 32 largest counts read off the histogram
// from the top by one warp.
// The sample: row p_j = (offset + j * (n / m)) mod n for j < m, and the row
// after it (for the adjacent-repeat feature).
__device__ __forceinline__ int64_t sample_row(int64_t n, int m, uint64_t offset, int j) {
  const int64_t stride = m > 0 ? n / m : 1;
  const uint64_t off = n > 0 ? offset % (uint64_t)n : 0;
  const uint64_t q = off + (uint64_t)j * (uint64_t)stride;  // < 2n
  return (int64_t)(q >= (uint64_t)n ? q - (uint64_t)n : q);
}

// Gathers the sampled keys (pre[j]) and their successors (pre[kSketchSample +
// j]) with many blocks: one block issuing 8192 scattered loads is bound by its
// own load queue.
__global__ void sketch_gather(const uint32_t* __restrict__ keys, int64_t n, uint64_t offset,
                              uint32_t* __restrict__ pre) {
  const int m = (int)(n < kSketchSample ? n : kSketchSample);
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int64_t p = sample_row(n, m, offset, j);
  pre[j] = keys[p];
  pre[kSketchSample + j] = p + 1 < n ? keys[p + 1] : 0u;
}

// pre: the gathered sample (sketch_gather), or null to load it here.
__device__ void sketch_block(const uint32_t* __restrict__ keys, int64_t n, int vbytes, int nops, int fp,
                             int slot_bytes, uint64_t offset, double smem_bytes, double l2_bytes,
                             float* __restrict__ feat, const uint32_t* __restrict__ pre) {
  extern __shared__ __align__(16) unsigned char sm[];
  unsigned long long* slot = (unsigned long long*)sm;            // kSketchSlots
  uint32_t* cnt = (uint32_t*)(slot + kSketchSlots);              // kSketchSlots
  uint32_t* hist = cnt + kSketchSlots;                           // kSketchSample + 1
  uint32_t* top = hist + kSketchSample + 1;                      // 32 (+ pad)
  __shared__ double red[33];
  __shared__ unsigned int s_d, s_f1, s_f2, s_adj, s_kmin, s_kmax, s_maxc, s_ntop;
  const int tid = threadIdx.x;
  for (int i = tid; i < kSketchSlots; i += kSketchThreads) {
    slot[i] = 0;
    cnt[i] = 0;
  }
  for (int i = tid; i <= kSketchSample; i += kSketchThreads) hist[i] = 0;
  if (tid == 0) {
    s_d = s_f1 = s_f2 = s_adj = s_maxc = s_ntop = 0;
    s_kmin = 0xFFFFFFFFu;
    s_kmax = 0;
  }
  const int m = (int)(n < kSketchSample ? n : kSketchSample);
  __syncthreads();
  constexpr int kPer = kSketchSample / kSketchThreads;  // sampled keys per thread
  uint32_t kk[kPer], nx[kPer];
  bool have[kPer], hasnx[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {  // issue every load before using any
    const int j = tid + u * kSketchThreads;
    have[u] = j < m;
    hasnx[u] = false;
    kk[u] = 0;
    nx[u] = 0;
    if (have[u]) {
      const int64_t p = sample_row(n, m, offset, j);
      hasnx[u] = p + 1 < n;
      if (pre) {
        kk[u] = pre[j];
        nx[u] = pre[kSketchSample + j];
      } else {
        kk[u] = keys[p];
        if (hasnx[u]) nx[u] = keys[p + 1];
      }
    }
  }
  {  // key range and adjacent repeats: reduced per warp, one atomic each per warp
    uint32_t lmin = 0xFFFFFFFFu, lmax = 0, ladj = 0;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      if (!have[u]) continue;
      lmin = min(lmin, kk[u]);
      lmax = max(lmax, kk[u]);
      ladj += (hasnx[u] && nx[u] == kk[u]) ? 1u : 0u;
    }
    lmin = __reduce_min_sync(0xffffffffu, lmin);
    lmax = __reduce_max_sync(0xffffffffu, lmax);
    ladj = __reduce_add_sync(0xffffffffu, ladj);
    if ((tid & 31) == 0) {
      atomicMin(&s_kmin, lmin);
      atomicMax(&s_kmax, lmax);
      if (ladj) atomicAdd(&s_adj, ladj);
    }
  }
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    if (!have[u]) continue;
    const uint32_t k = kk[u];
    const unsigned long long tag = ((unsigned long long)k << 1) | 1ull;
    uint32_t h = fmix32(k) & (kSketchSlots - 1);
    for (;;) {  // at most m < kSketchSlots occupied slots: an empty or matching one exists
      unsigned long long cur = *(volatile unsigned long long*)&slot[h];
      if (cur == 0) cur = atomicCAS(&slot[h], 0ull, tag);
      if (cur == 0 || cur == tag) break;
      h = (h + 1) & (kSketchSlots - 1);
    }
    atomicAdd(&cnt[h], 1u);
  }
  __syncthreads();
  float ent_t = 0.f;  // this thread's few entropy terms; the block sum is float64
  const float mf = (float)(m > 0 ? m : 1);
  {
    uint32_t ld = 0, lf1 = 0, lf2 = 0, lmaxc = 0;
    for (int i = tid; i < kSketchSlots; i += kSketchThreads) {  // same trip count in every thread
      const uint32_t c = cnt[i];
      if (c == 0) continue;
      ld += 1;
      lf1 += c == 1 ? 1u : 0u;
      lf2 += c == 2 ? 1u : 0u;
      lmaxc = max(lmaxc, c);
      atomicAdd(&hist[c], 1u);
      const float p = (float)c / mf;
      ent_t -= p * logf(p);
    }
    ld = __reduce_add_sync(0xffffffffu, ld);
    lf1 = __reduce_add_sync(0xffffffffu, lf1);
    lf2 = __reduce_add_sync(0xffffffffu, lf2);
    lmaxc = __reduce_max_sync(0xffffffffu, lmaxc);
    if ((tid & 31) == 0) {
      atomicAdd(&s_d, ld);
      atomicAdd(&s_f1, lf1);
      atomicAdd(&s_f2, lf2);
      atomicMax(&s_maxc, lmaxc);
    }
  }
  const double ent = block_sum_d((double)ent_t, red);
  const int R = (int)(s_d < 32 ? s_d : 32);
  if (tid < 32) {  // warp 0: the R largest counts, in descending order
    const int lane = tid;
    int got = 0;
    for (int base = (int)s_maxc; base >= 1 && got < R; base -= 32) {
      const int c = base - lane;
      const uint32_t v = c >= 1 ? hist[c] : 0u;
      uint32_t b = __ballot_sync(0xffffffffu, v != 0);
      while (b && got < R) {
        const int src = __ffs(b) - 1;
        b &= b - 1;
        const int mult = (int)__shfl_sync(0xffffffffu, v, src);
        const int take = mult < R - got ? mult : R - got;
        if (lane < take) top[got + lane] = (uint32_t)(base - src);
        got += take;
      }
    }
  }
  __syncthreads();
  // Least-squares slope of log(count) on log(rank) over the R largest counts:
  // lane r - 1 of warp 0 takes rank r, and the sums are warp reductions in a
  // fixed order (float64, few serial steps).
  __shared__ double s_slope;
  if (tid < 32) {
    const int r = tid + 1;
    const bool in = r <= R;
    const double x = in ? (double)logf((float)r) : 0.0, y = in ? (double)logf((float)top[r - 1]) : 0.0;
    double sx = x, sy = y, sxx = x * x, sxy = x * y;
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sxx += __shfl_xor_sync(0xffffffffu, sxx, o);
      sxy += __shfl_xor_sync(0xffffffffu, sxy, o);
    }
    if (tid == 0) s_slope = R >= 2 ? (R * sxy - sx * sy) / (R * sxx - sx * sx) : 0.0;
  }
  __syncthreads();
  if (tid != 0) return;
  const double md = m > 0 ? (double)m : 1.0;
  const double d = (double)s_d, f1 = (double)s_f1, f2 = (double)s_f2;
  float* f = feat;
  f[F_LOG2N] = n > 0 ? log2f((float)n) : 0.f;
  f[F_VBYTES] = (float)vbytes;
  f[F_NOPS] = (float)nops;
  f[F_FP] = (float)fp;
  if (m == 0) {
    for (int i = F_DISTINCT; i < F_COUNT; ++i) f[i] = 0.f;
    return;
  }
  f[F_DISTINCT] = (float)(d / md);
  f[F_F1] = (float)(f1 / md);
  f[F_F2] = (float)(f2 / md);
  f[F_TOP1] = (float)((double)top[0] / md);
  double top8 = 0;
  for (int r = 0; r < 8 && r < R; ++r) top8 += (double)top[r];
  f[F_TOP8] = (float)(top8 / md);
  f[F_SLOPE] = (float)s_slope;
  f[F_ENTROPY] = m > 1 ? (float)(ent / (double)logf(mf)) : 0.f;
  f[F_ADJ_EQ] = (float)((double)s_adj / md);
  // float32 from here on: the features are float32, and float64 library
  // calls on one thread are slow on GB300's narrow float64 pipe
  float gee = sqrtf((float)n / (float)md) * (float)f1 + (float)(d - f1);
  if (gee < 1.f) gee = 1.f;
  if (gee > (float)n) gee = (float)n;
  f[F_LOG2_GEE] = log2f(gee);
  const float tbytes = 2.f * gee * (float)slot_bytes;
  f[F_SMEM_RATIO] = log2f(1.f + tbytes / (float)smem_bytes);
  f[F_L2_RATIO] = log2f(1.f + tbytes / (float)l2_bytes);
  f[F_LOG2_RANGE] = log2f((float)(s_kmax - s_kmin) + 1.f);
}

__global__ void __launch_bounds__(kSketchThreads) sketch_kernel(const uint32_t* __restrict__ keys, int64_t n,
                                                                int vbytes, int nops, int fp, int slot_bytes,
                                                                uint64_t offset, double smem_bytes, double l2_bytes,
                                                                float* __restrict__ feat,
                                                                const uint32_t* __restrict__ pre) {
  sketch_block(keys, n, vbytes, nops, fp, slot_bytes, offset, smem_bytes, l2_bytes, feat, pre);
}

// One block per query of a batch.
__global__ void __launch_bounds__(kSketchThreads) sketch_batch_kernel(const SketchJob* __restrict__ jobs,
                                                                      double smem_bytes, double l2_bytes,
                                                                      float* __restrict__ feat) {
  const SketchJob j = jobs[blockIdx.x];
  sketch_block(j.keys, j.n, j.vbytes, j.nops, j.fp, j.slot_bytes, j.offset, smem_bytes, l2_bytes,
               feat + (size_t)blockIdx.x * F_COUNT, nullptr);
}

agg_status sketch_batch_launch(const SketchJob* jobs_dev, int nq, float* feat_dev, cudaStream_t s) {
  const DeviceInfo& di = device_info();
  static bool attr_set[64] = {};
  if (di.device >= 0 && di.device < 64 && !attr_set[di.device]) {
    AGG_CUDA_TRY(
        cudaFuncSetAttribute(sketch_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSketchSmem));
    attr_set[di.device] = true;
  }
  if (nq <= 0) return AGG_OK;
  PhaseTimer pt(AGG_PHASE_SKETCH, s);
  sketch_batch_kernel<<<nq, kSketchThreads, kSketchSmem, s>>>(jobs_dev, (double)di.smem_per_block_optin,
                                                              (double)di.l2_bytes, feat_dev);
  note_launch();
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

agg_status sketch_launch(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset, float* feat_dev,
                         cudaStream_t s) {
  const DeviceInfo& di = device_info();
  static bool attr_set[64] = {};
  if (di.device >= 0 && di.device < 64 && !attr_set[di.device]) {
    AGG_CUDA_TRY(cudaFuncSetAttribute(sketch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSketchSmem));
    attr_set[di.device] = true;
  }
  // the gathered sample sits at 64 KiB of the stream scratch (transient; the
  // scratch block is at least 1 MiB, so this request never moves it)
  agg_status st = AGG_OK;
  char* scr = (char*)stream_scratch(s, (size_t)96 << 10, &st);
  if (!scr) return st;
  uint32_t* pre = (uint32_t*)(scr + ((size_t)64 << 10));
  PhaseTimer pt(AGG_PHASE_SKETCH, s);
  const int m = (int)(n < kSketchSample ? n : kSketchSample);
  if (m > 0) {
    sketch_gather<<<(m + 255) / 256, 256, 0, s>>>(keys, n, offset, pre);
    note_launch();
  }
  note_launch();
  sketch_kernel<<<1, kSketchThreads, kSketchSmem, s>>>(keys, n, (int)dtype_size(vdt), __builtin_popcount(ops),
                                             dtype_is_fp(vdt) ? 1 : 0, gslot_bytes(ops_minmax(ops)), offset,
                                             (double)di.smem_per_block_optin, (double)di.l2_bytes, feat_dev, pre);
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

}  // namespace agg

using namespace agg;

extern "C" agg_status agg_sketch(const uint32_t* keys_dev, int64_t n, agg_dtype vdtype, uint32_t ops,
                                 uint64_t sample_offset, float* features_dev, void* stream) {
  clear_error();
  AGG_CHECK_ARG(dtype_valid(vdtype), "invalid dtype %d", (int)vdtype);
  AGG_CHECK_ARG(ops != 0 && (ops & ~(uint32_t)AGG_ALL) == 0, "invalid ops mask 0x%x", ops);
  AGG_CHECK_ARG(n >= 0, "invalid row count");
  AGG_CHECK_ARG(n == 0 || keys_dev != nullptr, "null key pointer");
  AGG_CHECK_ARG(features_dev != nullptr, "null features pointer");
  return sketch_launch(keys_dev, n, vdtype, ops, sample_offset, features_dev, (cudaStream_t)stream);
}
