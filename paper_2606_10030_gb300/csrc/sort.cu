// Exclusive scan and stable LSD radix sort (8-bit digits) for GROUP BY.
//
// One radix pass = three launches:
//   radix_hist     per 4096-row tile, a 256-bin digit histogram, stored
//                  digit-major (digit * ntiles + tile) so that one exclusive
//                  scan of the whole array gives every (digit, tile) its
//                  global output offset;
//   scan           device-wide exclusive scan of those counts;
//   radix_scatter  per tile: stable rank of every row among rows with the
//                  same digit (ballots + per-warp running counts), staging
//                  of the tile in shared memory in digit order, then coalesced
//                  writes of each digit's run to its global offset.
#include <algorithm>
#include <vector>

#include "sort.cuh"

namespace agg {

// ---------------------------------------------------------------------------
// Exclusive scan of uint32.
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Block-wide exclusive scan for blocks of up to 1024 threads (a multiple of 32).
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
  __shared__ uint32_t warp_sums[32];
  const int nw = blockDim.x >> 5;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < nw ? warp_sums[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) warp_sums[lane] = s;
  }
  __syncthreads();
  uint32_t base = w ? warp_sums[w - 1] : 0;
  if (total) *total = warp_sums[nw - 1];
  uint32_t r = base + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce(const uint32_t* in, int64_t n, uint32_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t j = base + (int64_t)i * kScanThreads + threadIdx.x;
    if (j < n) s += in[j];
  }
  uint32_t tot;
  block_exclusive_scan(s, &tot);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Single block: exclusive scan of the block sums (any count), total to *total.
__global__ void __launch_bounds__(kScanThreads) scan_sums(uint32_t* sums, int64_t nb, uint32_t* total) {
  uint32_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += kScanThreads) {
    int64_t j = b0 + threadIdx.x;
    uint32_t v = j < nb ? sums[j] : 0;
    uint32_t t;
    uint32_t e = block_exclusive_scan(v, &t);
    if (j < nb) sums[j] = carry + e;
    carry += t;
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// Per tile: exclusive scan of kScanItems consecutive values per thread (blocked).
__global__ void __launch_bounds__(kScanThreads) scan_apply(const uint32_t* in, uint32_t* out, int64_t n,
                                                           const uint32_t* sums) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t j = base + i;
    v[i] = j < n ? in[j] : 0;
    s += v[i];
  }
  uint32_t e = block_exclusive_scan(s, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    int64_t j = base + i;
    if (j < n) out[j] = e;
    e += v[i];
  }
}

size_t scan_tmp_bytes(int64_t n) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  return (size_t)(nb > 0 ? nb : 1) * sizeof(uint32_t) + 256;
}

agg_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, void* tmp,
                              cudaStream_t s) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  uint32_t* sums = (uint32_t*)tmp;
  if (nb == 0) {
    if (total_dev) AGG_CUDA_TRY(cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s));
    return AGG_OK;
  }
  scan_reduce<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, sums);
  scan_sums<<<1, kScanThreads, 0, s>>>(sums, nb, total_dev);
  scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, sums);
  note_launch(3);
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

// ---------------------------------------------------------------------------
// Radix sort.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int64_t rows_of(int64_t n_cap, const int64_t* n_dev) {
  if (!n_dev) return n_cap;
  int64_t n = *n_dev;
  return n < n_cap ? n : n_cap;
}

// Digit of a key: 8 bits of key - kbase (kbase <= every key, so the order is
// the keys' order).
__device__ __forceinline__ uint32_t digit_of(uint32_t key, int shift, uint32_t kbase) {
  return ((key - kbase) >> shift) & 0xFFu;
}

__global__ void __launch_bounds__(kSortThreads) radix_hist(const uint32_t* __restrict__ keys, int64_t n_cap,
                                                           const int64_t* n_dev, int shift, uint32_t kbase,
                                                           int64_t ntiles, uint32_t* __restrict__ counts) {
  __shared__ uint32_t h[256];
  const int64_t n = rows_of(n_cap, n_dev);
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  uint32_t k[kSortItems];  // every load of the tile is issued before the first count
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t j = base + (int64_t)i * kSortThreads + threadIdx.x;
    k[i] = j < n ? keys[j] : 0u;
  }
  if (threadIdx.x < 256) h[threadIdx.x] = 0;
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const int64_t j = base + (int64_t)i * kSortThreads + threadIdx.x;
    if (j < n) atomicAdd(&h[digit_of(k[i], shift, kbase)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 256) counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

// Per tile (512 threads x 8 rows, each warp owning 256 consecutive rows;
// three blocks per SM, so at most 40 registers a thread):
// 0. the warp's keys are loaded into registers up front;
// 1. each warp ranks its rows among equal digits, round by round, with
//    digit-bit ballots and a per-warp running digit count (ranks stay in
//    registers);
// 2. digit totals are scanned across warps and digits, and the tile's digit
//    starts folded into the per-warp offsets and the global offsets;
// 3. values are loaded (keys are in registers) and rows staged in shared
//    memory in digit order;
// 4. each digit's run is written to its global offset with coalesced stores.
template <class P>
__global__ void __launch_bounds__(kSortThreads, 3) radix_scatter(const uint32_t* __restrict__ keys,
                                                              const P* __restrict__ vals, uint32_t* __restrict__ okeys,
                                                              P* __restrict__ ovals, int64_t n_cap,
                                                              const int64_t* n_dev, int shift, uint32_t kbase,
                                                              int64_t ntiles, const uint32_t* __restrict__ offsets) {
  constexpr int kWarps = kSortThreads / 32;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  P* stage_v = (P*)sm_raw;                                // kSortTile
  uint32_t* stage_k = (uint32_t*)(stage_v + kSortTile);  // kSortTile
  uint32_t* whist = stage_k + kSortTile;                 // kWarps x 256
  uint32_t* gbase = whist + kWarps * 256;                // 256

  const int64_t n = rows_of(n_cap, n_dev);
  const int64_t tile0 = (int64_t)blockIdx.x * kSortTile;
  if (tile0 >= n) return;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kSortThreads) whist[i] = 0;
  // the tile's global digit offsets are needed only from step 2 on: their
  // load is issued now and waited for there
  const uint32_t goff = threadIdx.x < 256 ? offsets[(int64_t)threadIdx.x * ntiles + blockIdx.x] : 0u;
  __syncthreads();

  uint32_t lr[kSortItems];
  uint32_t kr[kSortItems];
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t wbase = tile0 + (int64_t)w * (kSortItems * 32);
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t j = wbase + r * 32 + lane;
    kr[r] = j < n ? keys[j] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t j = wbase + r * 32 + lane;
    const bool ok = j < n;
    const uint32_t d = ok ? digit_of(kr[r], shift, kbase) : 0u;
    // lanes holding the same digit: one ballot per digit bit
    uint32_t peers = __ballot_sync(0xffffffffu, ok);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const uint32_t bit = (d >> b) & 1u;
      const uint32_t m = __ballot_sync(0xffffffffu, bit != 0u);
      peers &= bit ? m : ~m;
    }
    const uint32_t before = ok ? whist[w * 256 + d] : 0u;
    lr[r] = before + __popc(peers & lt);
    __syncwarp();
    if (ok && (peers & lt) == 0) whist[w * 256 + d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {  // per digit: exclusive prefix over warps, then over digits
    uint32_t run = 0;
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = whist[ww * 256 + d];
        whist[ww * 256 + d] = run;
        run += c;
      }
    }
    const uint32_t e = block_exclusive_scan(threadIdx.x < 256 ? run : 0u, nullptr);
    if (threadIdx.x < 256) {
      // fold the digit's tile start into its per-warp offsets, and its global
      // offset minus the tile start into gbase (mod 2^32: positions are < 2^32)
      const int d = threadIdx.x;
#pragma unroll
      for (int ww = 0; ww < kWarps; ++ww) whist[ww * 256 + d] += e;
      gbase[d] = goff - e;
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t j = wbase + r * 32 + lane;
    if (j < n) {
      const uint32_t key = kr[r];
      const uint32_t d = digit_of(key, shift, kbase);
      const uint32_t lp = whist[w * 256 + d] + lr[r];
      stage_k[lp] = key;
      stage_v[lp] = vals[j];
    }
  }
  __syncthreads();
  const int cnt = (int)(n - tile0 < kSortTile ? n - tile0 : kSortTile);
  for (int i = threadIdx.x; i < cnt; i += kSortThreads) {
    const uint32_t key = stage_k[i];
    const uint32_t d = digit_of(key, shift, kbase);
    const int64_t pos = (int64_t)(uint32_t)(gbase[d] + (uint32_t)i);
    okeys[pos] = key;
    ovals[pos] = stage_v[i];
  }
}

template <class P>
static size_t scatter_smem() {
  return (size_t)kSortTile * (sizeof(P) + 4) + ((kSortThreads / 32) * 256 + 256) * 4;
}

size_t radix_tmp_bytes(int64_t n_cap) {
  int64_t ntiles = (n_cap + kSortTile - 1) / kSortTile;
  if (ntiles < 1) ntiles = 1;
  size_t counts = (size_t)256 * ntiles * sizeof(uint32_t);
  return ((counts + 255) & ~size_t(255)) + scan_tmp_bytes(256 * ntiles);
}

template <class P>
agg_status radix_sort_pairs(const uint32_t* kin, const P* vin, uint32_t* ka, P* va, uint32_t* kb, P* vb,
                            int64_t n_cap, const int64_t* n_dev, int bits, void* tmp, cudaStream_t s,
                            uint32_t** kout, P** vout, uint32_t kbase) {
  *kout = const_cast<uint32_t*>(kin);
  *vout = const_cast<P*>(vin);
  const int64_t ntiles = (n_cap + kSortTile - 1) / kSortTile;
  if (ntiles == 0) return AGG_OK;
  uint32_t* counts = (uint32_t*)tmp;
  size_t cbytes = ((size_t)256 * ntiles * sizeof(uint32_t) + 255) & ~size_t(255);
  void* stmp = (char*)tmp + cbytes;
  const size_t sm = scatter_smem<P>();
  agg_status pst = radix_prepare();  // a no-op once done on this device
  if (pst != AGG_OK) return pst;
  const uint32_t* ki = kin;
  const P* vi = vin;
  int pass = 0;
  for (int shift = 0; shift < bits; shift += 8, ++pass) {
    uint32_t* ko = (pass & 1) ? kb : ka;
    P* vo = (pass & 1) ? vb : va;
    radix_hist<<<(unsigned)ntiles, kSortThreads, 0, s>>>(ki, n_cap, n_dev, shift, kbase, ntiles, counts);
    agg_status st = scan_exclusive_u32(counts, counts, 256 * ntiles, nullptr, stmp, s);
    if (st != AGG_OK) return st;
    radix_scatter<P><<<(unsigned)ntiles, kSortThreads, sm, s>>>(ki, vi, ko, vo, n_cap, n_dev, shift, kbase,
                                                                        ntiles, counts);
    note_launch(2);
    AGG_CUDA_TRY(cudaGetLastError());
    ki = ko;
    vi = vo;
    *kout = ko;
    *vout = vo;
  }
  return AGG_OK;
}

agg_status radix_prepare() {
  int dev = 0;
  cudaGetDevice(&dev);
  static bool done[64] = {};
  if (dev < 64 && done[dev]) return AGG_OK;
  AGG_CUDA_TRY(cudaFuncSetAttribute(radix_scatter<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)scatter_smem<uint32_t>()));
  AGG_CUDA_TRY(cudaFuncSetAttribute(radix_scatter<uint64_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)scatter_smem<uint64_t>()));
  if (dev < 64) done[dev] = true;
  return AGG_OK;
}

// ---------------------------------------------------------------------------
// One-level hash partition without a stable order (the hash build needs rows
// grouped by partition, in any order within one). Two kernels:
//   part_hist     256-bin histogram of the partition digit (top 8 bits of
//                 fmix32(key)) in per-warp shared counters, merged with one
//                 global atomic per bin and block; the last block to finish
//                 turns the totals into each partition's start;
//   part_scatter  per tile of 6144 or 8192 rows (a block of 512 threads, 12 or
//                 16 rows a thread, the next tile's keys and values loaded
//                 while the current one is written out): each row's place
//                 among its warp's rows of the same digit from a per-warp
//                 shared counter (a plain atomic: order within a partition is
//                 free), the warps' counts scanned per digit, the tile's runs
//                 reserved in the output with one global atomic per digit
//                 (whose latency overlaps the scan and the staging), the
//                 rows staged in shared memory in digit order and written out
//                 run by run.
// Reads 4 + 12 B and writes 12 B per row (uint32 key, 8-byte value); no per-tile
// count array and no ranking rounds. The histogram pass is skipped when the
// caller already holds the counts (the GROUP BY planner's HyperLogLog pass
// counts them from the same hash).
//
// A second level (65536 partitions) splits each of the 256 partitions by the
// next 8 hash bits with the same scatter over tiles that never straddle a
// partition (seg_hist counts per (partition, digit), seg_starts scans each
// partition's counts from its start).
// ---------------------------------------------------------------------------
constexpr int kPartHistThreads = 512;
constexpr int kPartThreads = 512;
// Rows per scatter tile and blocks per SM by payload: 8-byte values take
// 8192-row tiles, one block a SM (112 KB of stage); 4-byte values 6144-row
// tiles, two blocks a SM (longer runs per partition and fewer per-tile scans
// than 4096-row tiles; measured on the 2^30-row partition: 5.6 vs 6.1 ms).
template <class P>
struct PartCfg {
  static constexpr int kTile = sizeof(P) == 8 ? 8192 : 6144;
  static constexpr int kBlocks = sizeof(P) == 8 ? 1 : 2;
};
constexpr int kFillStride = 32;  // global fill counters 256 B apart (different L2 lines)

__device__ __forceinline__ uint32_t part_digit(uint32_t key, int shift) { return (fmix32(key) >> shift) & 255u; }

// fill[d * kFillStride]: partition starts (written by the last block), fill[256 * kFillStride]: ticket.
// Starts count from row_base; with starts_out, they are also saved there (and
// row_base + n at [256]).
__global__ void __launch_bounds__(kPartHistThreads) part_hist(const uint32_t* __restrict__ keys, int64_t n,
                                                              int64_t head, unsigned long long* __restrict__ fill,
                                                              int64_t row_base,
                                                              unsigned long long* __restrict__ starts_out, int shift) {
  constexpr int kWarps = kPartHistThreads / 32;
  __shared__ uint32_t h[kWarps][256];
  __shared__ unsigned long long tot[256];
  __shared__ int s_last;
  const int w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kWarps * 256; i += kPartHistThreads) (&h[0][0])[i] = 0;
  __syncthreads();
  const int64_t g = (int64_t)blockIdx.x * kPartHistThreads + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kPartHistThreads;
  const int64_t nq = (n - head) / 4;
  const int64_t tail0 = head + nq * 4;
  if (g < head) atomicAdd(&h[w][part_digit(keys[g], shift)], 1u);
  if (g < n - tail0) atomicAdd(&h[w][part_digit(keys[tail0 + g], shift)], 1u);
  const uint4* kq = (const uint4*)(keys + head);
  for (int64_t q = g; q < nq; q += 2 * nthreads) {  // two 16-byte loads in flight per thread
    const uint4 a = ld_stream_v4(kq + q);
    const bool two = q + nthreads < nq;
    const uint4 b = two ? ld_stream_v4(kq + q + nthreads) : make_uint4(0, 0, 0, 0);
    atomicAdd(&h[w][part_digit(a.x, shift)], 1u);
    atomicAdd(&h[w][part_digit(a.y, shift)], 1u);
    atomicAdd(&h[w][part_digit(a.z, shift)], 1u);
    atomicAdd(&h[w][part_digit(a.w, shift)], 1u);
    if (two) {
      atomicAdd(&h[w][part_digit(b.x, shift)], 1u);
      atomicAdd(&h[w][part_digit(b.y, shift)], 1u);
      atomicAdd(&h[w][part_digit(b.z, shift)], 1u);
      atomicAdd(&h[w][part_digit(b.w, shift)], 1u);
    }
  }
  __syncthreads();
  if (threadIdx.x < 256) {
    uint32_t t = 0;
    for (int ww = 0; ww < kWarps; ++ww) t += h[ww][threadIdx.x];
    if (t) atomicAdd(&fill[threadIdx.x * kFillStride], (unsigned long long)t);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(&fill[256 * kFillStride], 1ull) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;  // the whole block leaves together
  __threadfence();
  if (threadIdx.x < 256) tot[threadIdx.x] = __ldcg(&fill[threadIdx.x * kFillStride]);
  __syncthreads();
  if (threadIdx.x < 32) {  // exclusive scan of the 256 totals: one warp, 8 chunks of 32
    const int lane = threadIdx.x;
    unsigned long long run = 0;
    for (int j = 0; j < 8; ++j) {
      unsigned long long x = tot[j * 32 + lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      const unsigned long long start = (unsigned long long)row_base + run + x - tot[j * 32 + lane];
      fill[(j * 32 + lane) * kFillStride] = start;
      if (starts_out) starts_out[j * 32 + lane] = start;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (starts_out && lane == 0) starts_out[256] = (unsigned long long)row_base + run;
  }
}

// Partition starts from counts the host already holds (one warp).
struct PartCounts {
  unsigned long long c[256];
};
__global__ void __launch_bounds__(32) part_starts(const __grid_constant__ PartCounts h,
                                                  unsigned long long* __restrict__ fill, int64_t row_base,
                                                  unsigned long long* __restrict__ starts_out) {
  const int lane = threadIdx.x;
  unsigned long long run = 0;
  for (int j = 0; j < 8; ++j) {
    const unsigned long long c = h.c[j * 32 + lane];
    unsigned long long x = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    const unsigned long long start = (unsigned long long)row_base + run + x - c;
    fill[(j * 32 + lane) * kFillStride] = start;
    if (starts_out) starts_out[j * 32 + lane] = start;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  if (starts_out && lane == 0) starts_out[256] = (unsigned long long)row_base + run;
}

// Tiles of a segmented pass (rows grouped into 256 partitions, starts[0..256]):
// first[p] = the tiles of partitions before p (TILE rows each, no tile
// straddling two partitions), first[256] = all tiles. One warp computes them.
template <int TILE>
__device__ __forceinline__ void seg_first_tiles(const unsigned long long* __restrict__ starts, int64_t* first) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int64_t run = 0;
    for (int j = 0; j < 8; ++j) {
      const int p = j * 32 + lane;
      const int64_t len = (int64_t)(starts[p + 1] - starts[p]);
      const int64_t c = (len + TILE - 1) / TILE;
      int64_t x = c;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      first[p] = run + x - c;
      run += __shfl_sync(0xffffffffu, x, 31);
    }
    if (lane == 0) first[256] = run;
  }
}

// The partition of tile t < first[256]: the last p with first[p] <= t (it has
// a tile, so first[p + 1] > t).
__device__ __forceinline__ int seg_of_tile(const int64_t* first, int64_t t) {
  int lo = 0, hi = 256;  // first[lo] <= t < first[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (first[mid] <= t) lo = mid;
    else hi = mid;
  }
  return lo;
}

// SEG = false: tile t covers rows [t kTile, ...) of the column, fill
// holds one counter per digit (kFillStride apart). SEG = true: tiles follow
// the partitions of starts (see seg_first_tiles) and fill holds one counter
// per (partition, digit), partition-major.
template <class P, bool SEG>
__global__ void __launch_bounds__(kPartThreads, PartCfg<P>::kBlocks) part_scatter(const uint32_t* __restrict__ keys,
                                                                const P* __restrict__ vals,
                                                                uint32_t* __restrict__ okeys, P* __restrict__ ovals,
                                                                int64_t n, unsigned long long* __restrict__ fill,
                                                                int shift,
                                                                const unsigned long long* __restrict__ starts) {
  constexpr int kTile = PartCfg<P>::kTile;
  constexpr int kRows = kTile / kPartThreads;  // rows per thread and tile
  constexpr int kWarps = kPartThreads / 32;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  P* stage_v = (P*)sm_raw;                            // kTile
  uint32_t* stage_k = (uint32_t*)(stage_v + kTile);  // kTile
  uint32_t* whist = stage_k + kTile;                 // kWarps x 256
  __shared__ uint32_t off[256];
  __shared__ unsigned long long base[256];
  __shared__ int64_t first[SEG ? 257 : 1];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t ntiles;
  if (SEG) {
    seg_first_tiles<kTile>(starts, first);
    __syncthreads();
    ntiles = first[256];
  } else {
    ntiles = (n + kTile - 1) / kTile;
  }
  // tile t: its first row, its rows, and where its digits' counters are
  auto tile_of = [&](int64_t t, int64_t& r0, int& rows, int& fbase) {
    if (SEG) {
      const int p = seg_of_tile(first, t);
      r0 = (int64_t)starts[p] + (t - first[p]) * kTile;
      rows = (int)min((int64_t)kTile, (int64_t)starts[p + 1] - r0);
      fbase = p * 256;
    } else {
      r0 = t * kTile;
      rows = (int)min((int64_t)kTile, n - r0);
      fbase = 0;
    }
  };
  constexpr int kStride = SEG ? 1 : kFillStride;
  // each warp owns kRows * 32 consecutive rows of a tile; the next tile's keys
  // and values are loaded while the current one is written out
  uint32_t kr[kRows];
  P vr[kRows];
  const int wbase = w * kRows * 32;
  auto load = [&](int64_t r0, int rows) {
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = wbase + r * 32 + lane;
      kr[r] = j < rows ? keys[r0 + j] : 0u;
      vr[r] = j < rows ? vals[r0 + j] : P(0);
    }
  };
  int64_t t = blockIdx.x, r0 = 0;
  int rows = 0, fbase = 0;
  if (t < ntiles) {
    tile_of(t, r0, rows, fbase);
    load(r0, rows);
  }
  for (int i = threadIdx.x; i < kWarps * 256; i += kPartThreads) whist[i] = 0;
  __syncthreads();
  for (; t < ntiles; t += gridDim.x) {
    uint32_t pr[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = wbase + r * 32 + lane;
      if (j < rows) pr[r] = atomicAdd(&whist[w * 256 + part_digit(kr[r], shift)], 1u);
    }
    __syncthreads();
    // per digit: the warps' runs and the tile's count; the tile's run in the
    // output is reserved now, its offset stored only after the staging (the
    // atomic's latency overlaps the scan and the staging)
    unsigned long long my_base = 0;
    if (threadIdx.x < 256) {
      const int d = threadIdx.x;
      uint32_t run = 0;
      for (int ww = 0; ww < kWarps; ++ww) {
        const uint32_t c = whist[ww * 256 + d];
        whist[ww * 256 + d] = run;
        run += c;
      }
      off[d] = run;  // the tile's count of digit d, until the scan below
      if (run) my_base = atomicAdd(&fill[fbase + d * kStride], (unsigned long long)run);
    }
    __syncthreads();
    if (threadIdx.x < 32) {  // exclusive scan of the counts over digits
      uint32_t run = 0;
      for (int j = 0; j < 8; ++j) {
        const uint32_t c = off[j * 32 + lane];
        uint32_t x = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
          if (lane >= o) x += y;
        }
        off[j * 32 + lane] = run + x - c;
        run += __shfl_sync(0xffffffffu, x, 31);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = wbase + r * 32 + lane;
      if (j < rows) {
        const uint32_t d = part_digit(kr[r], shift);
        const uint32_t p = off[d] + whist[w * 256 + d] + pr[r];
        stage_k[p] = kr[r];
        stage_v[p] = vr[r];
      }
    }
    // a row at stage position p goes to base[d] + p (mod 2^64)
    if (threadIdx.x < 256) base[threadIdx.x] = my_base - (unsigned long long)off[threadIdx.x];
    const int rows_now = rows;
    if (t + gridDim.x < ntiles) {
      tile_of(t + gridDim.x, r0, rows, fbase);
      load(r0, rows);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kWarps * 256; i += kPartThreads) whist[i] = 0;  // for the next tile
    for (int p = threadIdx.x; p < rows_now; p += kPartThreads) {
      const uint32_t key = stage_k[p];
      const uint32_t d = part_digit(key, shift);
      const unsigned long long q = base[d] + (unsigned long long)p;
      okeys[q] = key;
      ovals[q] = stage_v[p];
    }
    __syncthreads();  // the stage and base are reused by the next tile
  }
}

// Second-level counts: per tile of a segmented pass, the rows of each digit
// (per-warp shared counters), added to counts[partition * 256 + digit].
template <int TILE>
__global__ void __launch_bounds__(kPartThreads) seg_hist(const uint32_t* __restrict__ keys,
                                                         const unsigned long long* __restrict__ starts,
                                                         unsigned long long* __restrict__ counts, int shift) {
  constexpr int kRows = TILE / kPartThreads;
  constexpr int kWarps = kPartThreads / 32;
  __shared__ uint32_t h[kWarps][256];
  __shared__ int64_t first[257];
  const int w = threadIdx.x >> 5;
  seg_first_tiles<TILE>(starts, first);
  __syncthreads();
  const int64_t ntiles = first[256];
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    for (int i = threadIdx.x; i < kWarps * 256; i += kPartThreads) (&h[0][0])[i] = 0;
    const int p = seg_of_tile(first, t);
    const int64_t r0 = (int64_t)starts[p] + (t - first[p]) * TILE;
    const int rows = (int)min((int64_t)TILE, (int64_t)starts[p + 1] - r0);
    uint32_t kr[kRows];
#pragma unroll
    for (int r = 0; r < kRows; ++r) {
      const int j = r * kPartThreads + (int)threadIdx.x;
      kr[r] = j < rows ? keys[r0 + j] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRows; ++r)
      if (r * kPartThreads + (int)threadIdx.x < rows) atomicAdd(&h[w][part_digit(kr[r], shift)], 1u);
    __syncthreads();
    if (threadIdx.x < 256) {
      uint32_t c = 0;
      for (int ww = 0; ww < kWarps; ++ww) c += h[ww][threadIdx.x];
      if (c) atomicAdd(&counts[p * 256 + threadIdx.x], (unsigned long long)c);
    }
    __syncthreads();
  }
}

// The 65536 (partition, digit) counts become the first output row of each
// run, in place: block p scans partition p's 256 counts (one per thread) and
// adds the partition's start (its rows are starts[p] .. starts[p + 1]).
__global__ void __launch_bounds__(256) seg_starts(unsigned long long* __restrict__ counts,
                                                  const unsigned long long* __restrict__ starts) {
  __shared__ unsigned long long warp_tot[8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  unsigned long long* c = counts + (size_t)blockIdx.x * 256;
  const unsigned long long own = c[threadIdx.x];
  unsigned long long x = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_tot[w] = x;
  __syncthreads();
  unsigned long long before = starts[blockIdx.x];
  for (int k = 0; k < w; ++k) before += warp_tot[k];
  c[threadIdx.x] = before + x - own;
}

template <class P>
static size_t part_smem() {
  return (size_t)PartCfg<P>::kTile * (sizeof(P) + 4) + (size_t)(kPartThreads / 32) * 256 * 4;
}

size_t partition_tmp_bytes() { return (257 * kFillStride) * sizeof(unsigned long long) + 256; }

template <class P>
agg_status partition_hashed(const uint32_t* kin, const P* vin, uint32_t* kout, P* vout, int64_t n, void* tmp,
                            cudaStream_t s, int64_t row_base, unsigned long long* starts_out,
                            const unsigned long long* hist, int shift) {
  if (n <= 0) {
    if (starts_out) {
      std::vector<unsigned long long> st(257, (unsigned long long)row_base);
      AGG_CUDA_TRY(cudaMemcpyAsync(starts_out, st.data(), sizeof(unsigned long long) * 257, cudaMemcpyHostToDevice, s));
      AGG_CUDA_TRY(cudaStreamSynchronize(s));  // the host vector goes out of scope
    }
    return AGG_OK;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  static bool attr[64] = {};
  if (dev < 64 && !attr[dev]) {
    AGG_CUDA_TRY(cudaFuncSetAttribute(part_scatter<uint32_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)part_smem<uint32_t>()));
    AGG_CUDA_TRY(cudaFuncSetAttribute(part_scatter<uint64_t, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)part_smem<uint64_t>()));
    AGG_CUDA_TRY(cudaFuncSetAttribute(part_scatter<uint32_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)part_smem<uint32_t>()));
    AGG_CUDA_TRY(cudaFuncSetAttribute(part_scatter<uint64_t, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)part_smem<uint64_t>()));
    attr[dev] = true;
  }
  unsigned long long* fill = (unsigned long long*)tmp;
  PartCounts pc;
  if (shift < 0 || shift > 24 || (hist && shift != 24)) {
    set_error("partition digit shift %d (counts given: %d)", shift, hist != nullptr);
    return AGG_ERR_INVALID;
  }
  if (hist) {
    unsigned long long tot = 0;
    for (int d = 0; d < 256; ++d) tot += (pc.c[d] = hist[d]);
    if (tot != (unsigned long long)n) {
      set_error("partition counts sum to %llu, not %lld rows", tot, (long long)n);
      return AGG_ERR_INVALID;
    }
  } else {
    AGG_CUDA_TRY(cudaMemsetAsync(fill, 0, (257 * kFillStride) * sizeof(unsigned long long), s));
  }
  const DeviceInfo& di = device_info();
  int bh = 1, bs = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bh, part_hist, kPartHistThreads, 0) != cudaSuccess || bh < 1)
    bh = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, part_scatter<P, false>, kPartThreads, part_smem<P>()) !=
          cudaSuccess ||
      bs < 1)
    bs = 1;
  int64_t head = (int64_t)(((16 - ((uintptr_t)kin & 15)) & 15) / 4);
  if (head > n) head = n;
  const int64_t ntiles = (n + PartCfg<P>::kTile - 1) / PartCfg<P>::kTile;
  const int64_t gh = std::max<int64_t>(
      1, std::min<int64_t>((int64_t)di.sm_count * bh, ((n - head) / 4 + 2 * kPartHistThreads - 1) / (2 * kPartHistThreads)));
  const int64_t gs = std::max<int64_t>(1, std::min<int64_t>((int64_t)di.sm_count * bs, ntiles));
  if (hist) part_starts<<<1, 32, 0, s>>>(pc, fill, row_base, starts_out);
  else part_hist<<<(unsigned)gh, kPartHistThreads, 0, s>>>(kin, n, head, fill, row_base, starts_out, shift);
  part_scatter<P, false><<<(unsigned)gs, kPartThreads, part_smem<P>(), s>>>(kin, vin, kout, vout, n, fill, shift,
                                                                            nullptr);
  note_launch(2);
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

size_t partition2_tmp_bytes() {  // level-1 counters, level-1 starts, (partition, digit) counts
  return ((partition_tmp_bytes() + 255) & ~size_t(255)) + ((257 * 8 + 255) & ~size_t(255)) + 65536 * 8;
}

template <class P>
agg_status partition_hashed2(const uint32_t* kin, const P* vin, uint32_t* kmid, P* vmid, uint32_t* kout, P* vout,
                             int64_t n, void* tmp, cudaStream_t s, const unsigned long long* hist) {
  if (n <= 0) return AGG_OK;
  char* t = (char*)tmp;
  const size_t off1 = (partition_tmp_bytes() + 255) & ~size_t(255);
  unsigned long long* starts1 = (unsigned long long*)(t + off1);                  // 257 level-1 starts
  unsigned long long* counts = (unsigned long long*)(t + off1 + ((257 * 8 + 255) & ~size_t(255)));  // 65536
  agg_status st = partition_hashed<P>(kin, vin, kmid, vmid, n, tmp, s, 0, starts1, hist, 24);
  if (st != AGG_OK) return st;
  AGG_CUDA_TRY(cudaMemsetAsync(counts, 0, 65536 * sizeof(unsigned long long), s));
  const DeviceInfo& di = device_info();
  int bh = 1, bs = 1;
  constexpr int kTile = PartCfg<P>::kTile;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bh, seg_hist<kTile>, kPartThreads, 0) != cudaSuccess || bh < 1)
    bh = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bs, part_scatter<P, true>, kPartThreads, part_smem<P>()) !=
          cudaSuccess ||
      bs < 1)
    bs = 1;
  const int64_t tiles_max = n / kTile + 256;  // tiles of the segmented passes, at most
  const int64_t gh = std::max<int64_t>(1, std::min<int64_t>((int64_t)di.sm_count * bh, tiles_max));
  const int64_t gs = std::max<int64_t>(1, std::min<int64_t>((int64_t)di.sm_count * bs, tiles_max));
  seg_hist<kTile><<<(unsigned)gh, kPartThreads, 0, s>>>(kmid, starts1, counts, 16);
  seg_starts<<<256, 256, 0, s>>>(counts, starts1);
  part_scatter<P, true><<<(unsigned)gs, kPartThreads, part_smem<P>(), s>>>(kmid, vmid, kout, vout, n, counts, 16,
                                                                           starts1);
  note_launch(3);
  AGG_CUDA_TRY(cudaGetLastError());
  return AGG_OK;
}

template agg_status partition_hashed2<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                                uint32_t*, int64_t, void*, cudaStream_t, const unsigned long long*);
template agg_status partition_hashed2<uint64_t>(const uint32_t*, const uint64_t*, uint32_t*, uint64_t*, uint32_t*,
                                                uint64_t*, int64_t, void*, cudaStream_t, const unsigned long long*);

template agg_status partition_hashed<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, int64_t, void*,
                                               cudaStream_t, int64_t, unsigned long long*, const unsigned long long*, int);
template agg_status partition_hashed<uint64_t>(const uint32_t*, const uint64_t*, uint32_t*, uint64_t*, int64_t, void*,
                                               cudaStream_t, int64_t, unsigned long long*, const unsigned long long*, int);


template agg_status radix_sort_pairs<uint32_t>(const uint32_t*, const uint32_t*, uint32_t*, uint32_t*, uint32_t*,
                                               uint32_t*, int64_t, const int64_t*, int, void*, cudaStream_t,
                                               uint32_t**, uint32_t**, uint32_t);
template agg_status radix_sort_pairs<uint64_t>(const uint32_t*, const uint64_t*, uint32_t*, uint64_t*, uint32_t*,
                                               uint64_t*, int64_t, const int64_t*, int, void*, cudaStream_t,
                                               uint32_t**, uint64_t**, uint32_t);

}  // namespace agg
