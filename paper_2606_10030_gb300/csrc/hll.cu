// HyperLogLog estimate of the distinct keys of a column (Flajolet, Fusy,
// Gandouet and Meunier, AofA 2007), one pass over every key. The GROUP BY
// planner sizes its hash tables from it when the 4096-key sample does not
// cover a large column (a long tail of rare keys the sample cannot see).
//
// A key's hash is MurmurHash3's 32-bit finaliser (a bijection of uint32, so
// distinct keys never collide); its top 14 bits pick one of m = 2^14
// registers, which keeps the largest rank (position of the first one bit,
// from 1) of the remaining 18 bits (19 if they are all zero). Each block keeps its registers in shared memory (a rank
// is written only when it exceeds the register, so repeated keys cost a
// shared-memory read), merges them into the column's registers with atomicMax,
// and the last block to finish (fence plus ticket, no waiting) forms the
// estimate alpha_m m^2 / sum 2^-M_j (linear counting m ln(m / V) below 5m/2
// when V registers are zero; above 2^32/30, the correction for a 32-bit hash
// space). The registers and the ticket live in the
// stream's scratch and are cleared before every launch.
//
// The same pass can also count the rows of each of the 256 hash partitions
// that the one-level partition of the GROUP BY uses (the top 8 bits of the
// same hash), so that the partition does not read the keys once more for its
// histogram.
#include <cmath>
#include <cstring>

#include "groupby.cuh"

namespace agg {

constexpr int kHllP = 14;
constexpr int kHllM = 1 << kHllP;
constexpr int kHllThreads = 512;
constexpr size_t kHllScratchOff = 8192;  // in the stream scratch, past the scan ticket
// State: registers (kHllM x u32), ticket (+0 past them), estimate (+8, double),
// partition counts (+256, 256 x u64).
constexpr size_t kHllTicketOff = (size_t)kHllM * 4;
constexpr size_t kHllEstOff = kHllTicketOff + 8;
constexpr size_t kHllHistOff = kHllTicketOff + 256;
constexpr size_t kHllStateBytes = kHllHistOff + 256 * 8;
constexpr size_t kHllScratchBytes = kHllScratchOff + kHllStateBytes;
constexpr int kHllWarps = kHllThreads / 32;
constexpr int kHllLoads = 4;  // 16-byte key loads a thread keeps in flight

// whist: the warp's 256 partition counters (HIST only).
template <bool HIST>
__device__ __forceinline__ void hll_add(uint32_t* sreg, uint32_t* whist, uint32_t key) {
  const uint32_t h = fmix32(key);
  const uint32_t idx = h >> (32 - kHllP);
  const uint32_t rank = (uint32_t)__clz((int)((h << kHllP) | (1u << (kHllP - 1)))) + 1u;  // 1..19
  if (rank > *(volatile uint32_t*)&sreg[idx]) atomicMax(&sreg[idx], rank);
  if (HIST) atomicAdd(&whist[h >> 24], 1u);
}

template <bool HIST>
__global__ void __launch_bounds__(kHllThreads) hll_kernel(const uint32_t* __restrict__ keys, int64_t n, int64_t head,
                                                          uint32_t* __restrict__ regs) {
  extern __shared__ uint32_t sreg[];  // kHllM registers, then (HIST) kHllWarps x 256 counters
  __shared__ double red[33];
  __shared__ int s_last;
  unsigned* ticket = (unsigned*)((char*)regs + kHllTicketOff);
  double* est = (double*)((char*)regs + kHllEstOff);
  uint32_t* whist = sreg + kHllM + (threadIdx.x >> 5) * 256;
  for (int i = threadIdx.x; i < kHllM + (HIST ? kHllWarps * 256 : 0); i += blockDim.x) sreg[i] = 0;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t nq = (n - head) / 4;
  const int64_t tail0 = head + nq * 4;
  if (g < head) hll_add<HIST>(sreg, whist, keys[g]);
  if (g < n - tail0) hll_add<HIST>(sreg, whist, keys[tail0 + g]);
  const uint4* kq = (const uint4*)(keys + head);
  for (int64_t q = g; q < nq; q += kHllLoads * nthreads) {  // kHllLoads 16-byte loads in flight per thread
    uint4 x[kHllLoads];
#pragma unroll
    for (int u = 0; u < kHllLoads; ++u)
      x[u] = q + u * nthreads < nq ? ld_stream_v4(kq + q + u * nthreads) : make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < kHllLoads; ++u) {
      if (q + u * nthreads < nq) {
        hll_add<HIST>(sreg, whist, x[u].x);
        hll_add<HIST>(sreg, whist, x[u].y);
        hll_add<HIST>(sreg, whist, x[u].z);
        hll_add<HIST>(sreg, whist, x[u].w);
      }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kHllM; i += blockDim.x) {
    const uint32_t r = sreg[i];
    if (r != 0 && r > __ldcg(&regs[i])) atomicMax(&regs[i], r);
  }
  if (HIST && threadIdx.x < 256) {
    unsigned long long* hist = (unsigned long long*)((char*)regs + kHllHistOff);
    uint32_t t = 0;
    for (int w = 0; w < kHllWarps; ++w) t += sreg[kHllM + w * 256 + threadIdx.x];
    if (t) atomicAdd(&hist[threadIdx.x], (unsigned long long)t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double sum = 0.0, zeros = 0.0;
  for (int i = threadIdx.x; i < kHllM; i += blockDim.x) {
    const uint32_t r = __ldcg(&regs[i]);
    sum += ldexp(1.0, -(int)r);
    zeros += r == 0 ? 1.0 : 0.0;
  }
  // block sums in a fixed order
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    sum += __shfl_xor_sync(0xffffffffu, sum, o);
    zeros += __shfl_xor_sync(0xffffffffu, zeros, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    red[32] = t;
  }
  __syncthreads();
  const double tot = red[32];
  __syncthreads();
  if (l == 0) red[w] = zeros;
  __syncthreads();
  if (threadIdx.x == 0) {
    double v = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) v += red[i];
    const double m = (double)kHllM;
    const double alpha = 0.7213 / (1.0 + 1.079 / m);
    double e = alpha * m * m / tot;
    if (e <= 2.5 * m && v > 0.0) e = m * log(m / v);                               // linear counting
    else if (e > 4294967296.0 / 30.0) e = -4294967296.0 * log(1.0 - e / 4294967296.0);  // 32-bit hash space
    *est = e;
  }
}

size_t hll_state_bytes() { return kHllStateBytes; }

agg_status hll_add_chunk(const uint32_t* keys, int64_t n, uint32_t* regs, bool first, cudaStream_t s, bool hist) {
  if (first) AGG_CUDA_TRY(cudaMemsetAsync(regs, 0, kHllStateBytes, s));  // registers, ticket, estimate, counts
  if (n <= 0) return AGG_OK;
  static bool attr_set[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  const int smem0 = kHllM * 4, smem1 = (kHllM + kHllWarps * 256) * 4;
  if (dev < 64 && !attr_set[dev]) {
    AGG_CUDA_TRY(cudaFuncSetAttribute(hll_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem0));
    AGG_CUDA_TRY(cudaFuncSetAttribute(hll_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem1));
    attr_set[dev] = true;
  }
  const void* kern = hist ? (const void*)hll_kernel<true> : (const void*)hll_kernel<false>;
  const int smem = hist ? smem1 : smem0;
  int64_t head = (int64_t)(((16 - ((uintptr_t)keys & 15)) & 15) / 4);
  if (head > n) head = n;
  int bps = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, kHllThreads, smem) != cudaSuccess || bps < 1) bps = 1;
  int64_t grid = (int64_t)device_info().sm_count * bps;
  const int64_t need = ((n - head) / 4 + kHllLoads * kHllThreads - 1) / (kHllLoads * kHllThreads);
  if (need < grid) grid = std::max<int64_t>(1, need);
  if (!first) AGG_CUDA_TRY(cudaMemsetAsync((char*)regs + kHllTicketOff, 0, 8, s));  // the ticket
  {
    PhaseTimer pt(AGG_PHASE_SKETCH, s);
    if (hist) hll_kernel<true><<<(unsigned)grid, kHllThreads, smem, s>>>(keys, n, head, regs);
    else hll_kernel<false><<<(unsigned)grid, kHllThreads, smem, s>>>(keys, n, head, regs);
    note_launch();
    AGG_CUDA_TRY(cudaGetLastError());
  }
  return AGG_OK;
}

agg_status hll_read(const uint32_t* regs, cudaStream_t s, double* est, unsigned long long* hist) {
  agg_status st = AGG_OK;
  constexpr size_t kBytes = kHllStateBytes - kHllEstOff;  // the estimate through the counts
  char* hb = (char*)stream_pinned(s, kBytes, &st);
  if (!hb) return st;
  AGG_CUDA_TRY(cudaMemcpyAsync(hb, (const char*)regs + kHllEstOff, hist ? kBytes : sizeof(double),
                               cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(est, hb, sizeof(double));
  if (hist) std::memcpy(hist, hb + (kHllHistOff - kHllEstOff), 256 * sizeof(unsigned long long));
  return AGG_OK;
}

agg_status hll_estimate(const uint32_t* keys, int64_t n, cudaStream_t s, double* est, unsigned long long* hist) {
  *est = 0.0;
  if (n <= 0) return AGG_OK;
  agg_status st = AGG_OK;
  char* scr = (char*)stream_scratch(s, kHllScratchBytes, &st);
  if (!scr) return st;
  uint32_t* regs = (uint32_t*)(scr + kHllScratchOff);
  st = hll_add_chunk(keys, n, regs, true, s, hist != nullptr);
  if (st != AGG_OK) return st;
  return hll_read(regs, s, est, hist);
}

}  // namespace agg

extern "C" agg_status agg_distinct_estimate(const uint32_t* keys_dev, int64_t n, double* estimate_host, void* stream) {
  using namespace agg;
  clear_error();
  AGG_CHECK_ARG(estimate_host != nullptr, "null output pointer");
  AGG_CHECK_ARG(n >= 0 && n < (int64_t(1) << 62), "invalid row count %lld", (long long)n);
  AGG_CHECK_ARG(n == 0 || keys_dev != nullptr, "null key pointer");
  AGG_CHECK_ARG(((uintptr_t)keys_dev & 3) == 0, "key pointer not 4-byte aligned");
  return hll_estimate(keys_dev, n, (cudaStream_t)stream, estimate_host);
}
