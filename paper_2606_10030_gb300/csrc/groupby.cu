// GROUP BY driver: sketch, strategy choice,
// table sizing and regrowth, the single-query hash path, the host-fed
// (end-to-end) path and the C entry points. The device code of the hash
// strategies is in hashtab.cuh; the sort strategy in sortagg.cu.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

#include "hashtab.cuh"
#include "sort.cuh"

namespace agg {

// The tile list of a column partitioned chunk by chunk: starts[k * 257 + p] is
// where partition p of chunk k begins (starts[k * 257 + 256] the chunk's end);
// piece (p, k) becomes ceil(rows / tile_rows) tiles, listed partition by
// partition (chunk order within a partition), so that neighbouring tiles
// update one region of the global table. One block.
__global__ void __launch_bounds__(1024) gb_piece_tiles(const unsigned long long* __restrict__ starts, int nchunks,
                                                       int64_t tile_rows, longlong2* __restrict__ tiles,
                                                       unsigned long long* __restrict__ ntiles) {
  __shared__ unsigned long long warp_tot[32];
  __shared__ unsigned long long carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int64_t npieces = (int64_t)nchunks * 256;
  for (int64_t q0 = 0; q0 < npieces; q0 += blockDim.x) {
    const int64_t q = q0 + threadIdx.x;
    int64_t a = 0, len = 0;
    if (q < npieces) {
      const int p = (int)(q / nchunks), k = (int)(q % nchunks);
      a = (int64_t)starts[(int64_t)k * 257 + p];
      len = (int64_t)starts[(int64_t)k * 257 + p + 1] - a;
    }
    const unsigned long long nt = (unsigned long long)((len + tile_rows - 1) / tile_rows);
    unsigned long long x = nt;  // inclusive scan over the block
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[w] = x;
    __syncthreads();
    if (w == 0) {
      unsigned long long v = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0ull;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += y;
      }
      if (lane < (int)(blockDim.x >> 5)) warp_tot[lane] = v;
    }
    __syncthreads();
    unsigned long long first = carry + (w ? warp_tot[w - 1] : 0ull) + x - nt;
    for (unsigned long long i = 0; i < nt; ++i) {
      const int64_t r = a + (int64_t)i * tile_rows;
      tiles[first + i] = make_longlong2(r, min(tile_rows, a + len - r));
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[(blockDim.x >> 5) - 1];
    __syncthreads();
  }
  if (threadIdx.x == 0) *ntiles = carry;
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
using KernelPtr = const void*;

// qpi: quads (4 rows) a thread folds per iteration of the vector loop, 1 or 2.
template <int DT, bool MM, bool SMEM, bool MULTI>
static KernelPtr build_vec(int qpi) {
  return qpi == 2 ? (KernelPtr)gb_build<DT, MM, SMEM, true, MULTI, 2> : (KernelPtr)gb_build<DT, MM, SMEM, true, MULTI, 1>;
}

template <int DT, bool MM>
static KernelPtr build_kernel(bool smem, bool vec, bool multi, int qpi) {
  if (smem) {
    if (!vec) return (KernelPtr)gb_build<DT, MM, true, false, false>;
    return multi ? build_vec<DT, MM, true, true>(qpi) : build_vec<DT, MM, true, false>(qpi);
  }
  if (!vec) return (KernelPtr)gb_build<DT, MM, false, false, false>;
  return multi ? build_vec<DT, MM, false, true>(qpi) : build_vec<DT, MM, false, false>(qpi);
}

static KernelPtr pick_build(int dt, bool mm, bool smem, bool vec, bool multi, int qpi) {
#define AGG_B(D) \
  case D: return mm ? build_kernel<D, true>(smem, vec, multi, qpi) : build_kernel<D, false>(smem, vec, multi, qpi);
  switch (dt) { AGG_B(AGG_I32) AGG_B(AGG_I64) AGG_B(AGG_U32) AGG_B(AGG_F32) AGG_B(AGG_F64) }
#undef AGG_B
  return nullptr;
}

template <int DT, bool MM>
static KernelPtr tiles_kernel(int qpi, bool home) {
  if (home)
    return qpi == 2 ? (KernelPtr)gb_build_tiles<DT, MM, true, 2, true> : (KernelPtr)gb_build_tiles<DT, MM, true, 1, true>;
  return qpi == 2 ? (KernelPtr)gb_build_tiles<DT, MM, true, 2> : (KernelPtr)gb_build_tiles<DT, MM, true, 1>;
}

// home: the tiles' shared tables are lightly loaded (see s_find_home).
static KernelPtr pick_tiles(int dt, bool mm, int qpi, bool home) {
#define AGG_T(D) \
  case D: return mm ? tiles_kernel<D, true>(qpi, home) : tiles_kernel<D, false>(qpi, home);
  switch (dt) { AGG_T(AGG_I32) AGG_T(AGG_I64) AGG_T(AGG_U32) AGG_T(AGG_F32) AGG_T(AGG_F64) }
#undef AGG_T
  return nullptr;
}

template <int DT>
static KernelPtr fin_small(bool mm) {
  return mm ? (KernelPtr)gb_rank_gather<DT, true> : (KernelPtr)gb_rank_gather<DT, false>;
}
template <int DT>
static KernelPtr fin_gather(bool mm) {
  return mm ? (KernelPtr)gb_gather<DT, true> : (KernelPtr)gb_gather<DT, false>;
}
static KernelPtr pick_small(int dt, bool mm) {
  switch (dt) {
    case AGG_I32: return fin_small<AGG_I32>(mm);
    case AGG_I64: return fin_small<AGG_I64>(mm);
    case AGG_U32: return fin_small<AGG_U32>(mm);
    case AGG_F32: return fin_small<AGG_F32>(mm);
    case AGG_F64: return fin_small<AGG_F64>(mm);
  }
  return nullptr;
}
static KernelPtr pick_gather(int dt, bool mm) {
  switch (dt) {
    case AGG_I32: return fin_gather<AGG_I32>(mm);
    case AGG_I64: return fin_gather<AGG_I64>(mm);
    case AGG_U32: return fin_gather<AGG_U32>(mm);
    case AGG_F32: return fin_gather<AGG_F32>(mm);
    case AGG_F64: return fin_gather<AGG_F64>(mm);
  }
  return nullptr;
}

static size_t stab_bytes_dt(int dt, bool mm, int S) {
#define AGG_SB(D) \
  case D: return mm ? stab_bytes<D, true>(S) : stab_bytes<D, false>(S);
  switch (dt) { AGG_SB(AGG_I32) AGG_SB(AGG_I64) AGG_SB(AGG_U32) AGG_SB(AGG_F32) AGG_SB(AGG_F64) }
#undef AGG_SB
  return 0;
}

static size_t tile_smem_bytes_dt(int dt, bool mm, int S) {
#define AGG_SB(D) \
  case D: return mm ? tile_smem_bytes<D, true>(S) : tile_smem_bytes<D, false>(S);
  switch (dt) { AGG_SB(AGG_I32) AGG_SB(AGG_I64) AGG_SB(AGG_U32) AGG_SB(AGG_F32) AGG_SB(AGG_F64) }
#undef AGG_SB
  return 0;
}

// Resident blocks per SM of a kernel for (threads, dynamic smem), cached.
static int occupancy(KernelPtr fn, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, KernelPtr, int, size_t>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, fn, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (smem > 48 * 1024) cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, threads, smem) != cudaSuccess || b < 1) b = 1;
  cache[key] = b;
  return b;
}

// Distinct-key estimates from the sketch of m sampled keys (d distinct, f1
// seen once, f2 seen twice).
//  coverage = 1 - f1/m, Good's estimate of the probability mass of the keys
//  seen in the sample;
//  Chao1 = d + f1 (f1 - 1) / (2 (f2 + 1)), the bias-corrected lower-bound
//  estimator (Chao, Scand. J. Stat. 1984), close for near-uniform keys;
//  GEE = sqrt(n/m) f1 + (d - f1) (Charikar et al., PODS 2000), which errs high
//  on flat columns and is the safer bound for skewed ones.
// A sample is flat when its top-8 keys hold at most twice what the largest
// counts of a uniform column of Chao1 keys would hold (Poisson, mean m/Chao1,
// largest counts about mean + 3 sd + 3); Chao1 of a flat sample is reliable
// once f2 >= 2 (below, the column has about m^2/4 or more keys, and Chao1 can
// be off by several times).
KeyEstimate key_estimate(const float* f) {
  KeyEstimate e;
  const double m = std::min(std::exp2((double)f[F_LOG2N]), (double)kSketchSample);
  const double d = (double)f[F_DISTINCT] * m, f1 = (double)f[F_F1] * m, f2 = (double)f[F_F2] * m;
  e.chao1 = std::max(1.0, d + f1 * (f1 - 1.0) / (2.0 * (f2 + 1.0)));
  e.gee = std::exp2((double)f[F_LOG2_GEE]);
  e.covered = m <= 0 || 1.0 - f1 / m >= 0.9;
  const double lam = m / e.chao1;
  const double top8_flat = m > 0 ? 8.0 * (lam + 3.0 * std::sqrt(lam) + 3.0) / m : 1.0;
  e.flat = (double)f[F_TOP8] <= 2.0 * top8_flat;
  e.reliable = e.covered || (e.flat && f2 >= 1.5);
  if (e.covered) e.plan = e.chao1;
  else if (e.flat) e.plan = (e.reliable ? 1.0 : 2.0) * e.chao1;
  else e.plan = std::max(e.chao1, 8.0 * e.gee);
  return e;
}

double distinct_estimate(const float* f, bool* covered) {
  const KeyEstimate e = key_estimate(f);
  *covered = e.covered;
  return e.plan;
}

// Global-table slots for a column of n rows from its sketch: a power of two
// at least twice a sizing estimate, within [1024, 2^31] and at most 2n.
//  - covered: 1.25 x Chao1;
//  - flat: 2 x Chao1 (4 x while Chao1 is unreliable);
//  - skewed and not covered: max(2 x Chao1, 16 x GEE), as the long tail of
//    rare keys is barely seen in the sample.
// A table that still overflows is regrown (4x) and the build redone.
int64_t table_slots_from_sketch(const float* f, int64_t n) {
  const KeyEstimate e = key_estimate(f);
  double est;
  if (e.covered) est = 1.25 * e.chao1;
  else if (e.flat) est = (e.reliable ? 2.0 : 4.0) * e.chao1;
  else est = std::max(2.0 * e.chao1, 16.0 * e.gee);
  double want = 2.0 * est;
  if (want > 2.0 * (double)n) want = 2.0 * (double)n;
  int64_t p = next_pow2((int64_t)std::ceil(std::max(want, 1.0)));
  if (p < 1024) p = 1024;
  if (p > (int64_t(1) << 31)) p = int64_t(1) << 31;
  return p;
}

// The AUTO rule (thresholds from the autotuner's timings of 5000 labelled
// queries; m = 4096 sampled keys, coverage = 1 - f1 / m):
//  - the sample covers >= 97% of the mass: SMEM (partitioned when the keys
//    overflow a shared table);
//  - columns under 2^20 rows: SMEM for few keys or a skewed sample, else one
//    global table;
//  - a skewed sample covering 90-97% whose singletons suggest at least half
//    as many unseen keys as seen ones (f1^2 / 2 f2 >= d / 2: a hot head and a
//    long tail of rare keys): SORT, which needs no key count;
//  - few keys: SMEM;
//  - a flat sample: SMEM on hash-partitioned rows while Chao1 is reliable and
//    below 10^5 keys (any reliable Chao1 from 2^28 rows on); otherwise SORT (a
//    flat sample of a large key domain often hides a mildly skewed column with
//    many more keys than Chao1);
//  - a skewed sample far from covering the column: SMEM on hash-partitioned
//    rows from 2^25 rows on, SORT below.
int rule_strategy(const float* f, uint32_t ops, double hll) {
  const KeyEstimate e = key_estimate(f);
  const int cap = ops_minmax(ops) ? 1536 : 3072;  // 3/4 of the largest shared tables
  const double coverage = 1.0 - (double)f[F_F1];  // F_F1 = f1 / m
  const float log2n = f[F_LOG2N];
  if (coverage >= 0.97) return AGG_STRAT_SMEM;
  // with the column's HyperLogLog count: a hot head that shared tables absorb
  // (the rest spilling to a right-sized table), or a flat column of up to 2^25
  // keys (hash-partitioned shared tables); larger flat columns sort (on 2^30
  // rows: 2^24 uniform keys 31 ms partitioned vs 43 ms sorted, 2^26 keys 59
  // vs 45 ms)
  if (hll > 0.0) {
    if (hot_sample(f, cap) || hll <= cap) return AGG_STRAT_SMEM;
    if (e.flat) return hll <= 33554432.0 ? AGG_STRAT_SMEM : AGG_STRAT_SORT;
  }
  if (log2n < 20.0f) return (e.plan <= cap || !e.flat) ? AGG_STRAT_SMEM : AGG_STRAT_GLOBAL;
  const double m = std::min(std::exp2((double)log2n), (double)kSketchSample);
  const double d = (double)f[F_DISTINCT] * m, f1 = (double)f[F_F1] * m, f2 = (double)f[F_F2] * m;
  const double unseen = f1 * (f1 - 1.0) / (2.0 * (f2 + 1.0));  // Chao1's unseen keys
  if (!e.flat && coverage >= 0.9 && unseen >= 0.5 * d) return AGG_STRAT_SORT;
  if (e.plan <= cap) return AGG_STRAT_SMEM;
  if (e.flat) return (e.reliable && (e.chao1 < 1e5 || log2n >= 28.0f)) ? AGG_STRAT_SMEM : AGG_STRAT_SORT;
  return log2n >= 25.0f ? AGG_STRAT_SMEM : AGG_STRAT_SORT;
}

agg_status groups_alloc(int64_t cap, int vdt, uint32_t ops, cudaStream_t s, agg_groups** out) {
  if (cap < 1) cap = 1;
  const size_t a8 = (size_t)cap * 8;
  const size_t kbytes = ((size_t)cap * 4 + 255) & ~size_t(255);
  const size_t bytes = kbytes + 5 * ((a8 + 255) & ~size_t(255)) + 256;
  void* blk = nullptr;
  cudaError_t e = dev_malloc_async(&blk, bytes, s);
  if (e != cudaSuccess) {
    set_error("result allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return AGG_ERR_OOM;
  }
  agg_groups* g = new agg_groups();
  std::memset(g, 0, sizeof(*g));
  GroupsPriv* p = new GroupsPriv();
  p->block = blk;
  p->stream = s;
  cudaGetDevice(&p->device);
  char* c = (char*)blk;
  g->keys = (uint32_t*)c;
  c += kbytes;
  const size_t a8r = (a8 + 255) & ~size_t(255);
  g->count = (int64_t*)c; c += a8r;
  g->sum = c; c += a8r;
  g->min = c; c += a8r;
  g->max = c; c += a8r;
  g->avg = (double*)c;
  g->dtype = vdt;
  g->ops = ops;
  g->priv = p;
  *out = g;
  return AGG_OK;
}

struct HashPlan {
  int strategy;     // AGG_STRAT_SMEM or AGG_STRAT_GLOBAL
  bool partition = false;  // hash-partition the rows first (table larger than L2)
  int partition_passes = 1;  // 1: 256 partitions; 2: 65536 partitions
  int64_t slots;    // global main slots (power of two)
  int smem_slots;   // shared slots (power of two) for SMEM
  int threads;
  int blocks_per_sm;
  bool multi_keys = true;  // per-warp reduction of several frequent keys (see build_rows)
  // quads (4 rows) a thread folds per iteration: items per thread / 4; 0 = the
  // default: 2 for the plain shared-memory build of integer columns without
  // the frequent-key step (2^26 rows over 64-1024 uniform keys: up to 3 %
  // faster; int64, 1024 keys: 0.401 vs 0.409 ms), else 1 (float columns
  // measured up to 2 % slower with 2, the tile builds 1.5x slower)
  int qpi = 0;
  int64_t tile_rows = 0;   // rows per tile of the partitioned build (0: from the column)
  // Rows of each one-level partition of the column (host memory, counted by
  // the HyperLogLog pass), or null: the partition then counts them itself.
  const unsigned long long* part_hist = nullptr;
  double est_keys = 0.0;  // the planner's distinct-key estimate of the column
};

// Whether a partitioned build's shared tables stay lightly loaded (at most a
// quarter of the slots): about est / P keys per tile when a tile lies within
// one of the P partitions, proportionally more when it spans several.
static bool tiles_lightly_loaded(double est, int64_t n, int passes, int64_t tile_rows, int smem_slots) {
  const double parts = passes == 2 ? 65536.0 : 256.0;
  const double span = std::max(1.0, (double)tile_rows * parts / (double)std::max<int64_t>(n, 1));
  return est > 0.0 && (est / parts) * span <= 0.25 * (double)smem_slots;
}

// One hash aggregation: a zeroed global table, any number of build launches
// over row ranges (one for a device column, one per chunk for a host-fed
// column), then one finalise into a result.
class HashRun {
 public:
  HashRun(int vdt, uint32_t ops, const HashPlan& plan, cudaStream_t s)
      : vdt_(vdt), ops_(ops), mm_(ops_minmax(ops)), plan_(plan), s_(s) {}
  ~HashRun() {
    if (mem_) cudaFreeAsync(mem_, s_);
  }

  agg_status init() {
    const size_t slot = (size_t)gslot_bytes(mm_);
    nslots_ = plan_.slots + 1;
    small_ = nslots_ <= kSmallRank;
    const size_t tbytes = (size_t)(nslots_ + 1) * slot;
    status_off_ = (tbytes + 255) & ~size_t(255);
    aux_off_ = status_off_ + 256;
    size_t aux_bytes = small_ ? 2 * (size_t)nslots_ * 4 + 1024 : 4 * (size_t)nslots_ * 4 + 1024 + radix_tmp_bytes(nslots_);
    AGG_CUDA_TRY(dev_malloc_async(&mem_, aux_off_ + aux_bytes, s_));
    AGG_CUDA_TRY(cudaMemsetAsync(mem_, 0, aux_off_, s_));
    status_ = (int*)((char*)mem_ + status_off_);
    counter_ = (unsigned long long*)((char*)mem_ + status_off_ + 64);
    progress_ = (unsigned long long*)((char*)mem_ + status_off_ + 192);
    return AGG_OK;
  }

  // After finish returned TABLE_FULL: rows the build went through, and rows
  // that found no slot.
  uint64_t rows_seen() const { return rows_seen_; }
  uint64_t rows_failed() const { return rows_failed_; }

  // Enqueue the build over rows [0, n) of (keys, vals).
  agg_status build(const uint32_t* keys, const void* vals, int64_t n) {
    if (n <= 0) return AGG_OK;
    const size_t es = dtype_size(vdt_);
    const uintptr_t ka = (uintptr_t)keys, va = (uintptr_t)vals;
    int64_t head = (int64_t)(((16 - (ka & 15)) & 15) / 4);
    if (head > n) head = n;
    const bool vec = ((va + (uintptr_t)head * es) & 15) == 0;
    if (!vec) head = 0;
    const bool use_smem = plan_.strategy == AGG_STRAT_SMEM;
    BuildArgs a;
    a.keys = keys;
    a.vals = vals;
    a.n = n;
    a.head = head;
    a.table = mem_;
    a.mask = (uint32_t)(plan_.slots - 1);
    a.gshift = 32 - (63 - __builtin_clzll((unsigned long long)plan_.slots));
    a.smem_slots = use_smem ? plan_.smem_slots : 0;
    a.smem_cap = use_smem ? (plan_.smem_slots * 3) / 4 : 0;
    a.status = status_;
    a.progress = progress_;
    if (plan_.partition && n >= kPartTileRows) return build_partitioned(a, use_smem);
    const bool int_col = vdt_ == AGG_I32 || vdt_ == AGG_I64 || vdt_ == AGG_U32;
    const int qpi = plan_.qpi ? plan_.qpi : (use_smem && !plan_.multi_keys && int_col ? 2 : 1);
    KernelPtr bk = pick_build(vdt_, mm_, use_smem, vec, plan_.multi_keys, qpi);
    const size_t smem = use_smem ? tile_smem_bytes_dt(vdt_, mm_, plan_.smem_slots) : 0;  // table + 32-bit pairs
    const int threads = plan_.threads;
    int bps = occupancy(bk, threads, smem);
    if (plan_.blocks_per_sm > 0 && plan_.blocks_per_sm < bps) bps = plan_.blocks_per_sm;
    const DeviceInfo& di = device_info();
    const int64_t work = vec ? (n + 3) / 4 : n;
    int64_t grid = (int64_t)di.sm_count * bps;
    const int64_t need = (work + threads - 1) / threads;
    if (need < grid) grid = need < 1 ? 1 : need;
    void* args[] = {&a};
    PhaseTimer pt(AGG_PHASE_BUILD, s_);
    cudaError_t e = cudaLaunchKernel(bk, dim3((unsigned)grid), dim3(threads), args, smem, s_);
    note_launch();
    if (e != cudaSuccess) {
      set_error("group-by build launch failed: %s", cudaGetErrorString(e));
      return AGG_ERR_CUDA;
    }
    return AGG_OK;
  }

  // Hash-partition the rows (one radix pass on the top 8 hash bits) into
  // scratch, then build over the partitioned rows: a tile queue with a
  // per-tile shared table (SMEM) or grid-stride global updates (GLOBAL).
  agg_status build_partitioned(BuildArgs a, bool use_smem) {
    const int64_t n = a.n;
    const size_t es = dtype_size(vdt_);
    const size_t kb = ((size_t)n * 4 + 255) & ~size_t(255), vb = ((size_t)n * es + 255) & ~size_t(255);
    const int passes = plan_.partition_passes;
    void* tmp = nullptr;
    AGG_CUDA_TRY(dev_malloc_async(&tmp, passes * (kb + vb) + partition2_tmp_bytes(), s_));
    uint32_t* kp = (uint32_t*)tmp;
    char* vp = (char*)tmp + kb;
    uint32_t* kq = (uint32_t*)((char*)tmp + kb + vb);
    char* vq = (char*)tmp + 2 * kb + vb;
    void* rt = (char*)tmp + passes * (kb + vb);
    agg_status st;
    {
      PhaseTimer pt(AGG_PHASE_SORT, s_);
      if (passes == 1) {  // rows only need grouping by partition: no stable order
        st = es == 4 ? partition_hashed<uint32_t>(a.keys, (const uint32_t*)a.vals, kp, (uint32_t*)vp, n, rt, s_, 0,
                                                  nullptr, plan_.part_hist)
                     : partition_hashed<uint64_t>(a.keys, (const uint64_t*)a.vals, kp, (uint64_t*)vp, n, rt, s_, 0,
                                                  nullptr, plan_.part_hist);
      } else {  // by the top 8 bits, then each partition by bits 16..23: ordered by the top 16 bits
        st = es == 4 ? partition_hashed2<uint32_t>(a.keys, (const uint32_t*)a.vals, kq, (uint32_t*)vq, kp,
                                                   (uint32_t*)vp, n, rt, s_, plan_.part_hist)
                     : partition_hashed2<uint64_t>(a.keys, (const uint64_t*)a.vals, kq, (uint64_t*)vq, kp,
                                                   (uint64_t*)vp, n, rt, s_, plan_.part_hist);
      }
    }
    if (st != AGG_OK) {
      cudaFreeAsync(tmp, s_);
      return st;
    }
    a.keys = kp;
    a.vals = vp;
    a.head = 0;
    const DeviceInfo& di = device_info();
    cudaError_t e;
    {
      PhaseTimer pt(AGG_PHASE_BUILD, s_);
      if (use_smem) {
        unsigned long long* next_tile = (unsigned long long*)((char*)mem_ + status_off_ + 128);
        e = cudaMemsetAsync(next_tile, 0, 8, s_);
        if (e != cudaSuccess) {
          cudaFreeAsync(tmp, s_);
          set_error("partitioned build: %s", cudaGetErrorString(e));
          return AGG_ERR_CUDA;
        }
        const size_t smem = tile_smem_bytes_dt(vdt_, mm_, plan_.smem_slots);
        const int threads = plan_.threads;
        // both variants have the same resources: occupancy from either
        int bps = occupancy(pick_tiles(vdt_, mm_, plan_.qpi, false), threads, smem);
        if (plan_.blocks_per_sm > 0 && plan_.blocks_per_sm < bps) bps = plan_.blocks_per_sm;
        int64_t grid = (int64_t)di.sm_count * bps;
        // tiles of up to 65532 rows (32 Ki after two levels), smaller (down to
        // 4 Ki) when the column would give each resident block fewer than two
        int64_t tile_rows = plan_.tile_rows;
        if (tile_rows == 0) {
          tile_rows = plan_.partition_passes == 2 ? kPartTileRows / 2 : kPartTileRows;
          while (tile_rows > 4096 && n < 2 * grid * tile_rows) tile_rows >>= 1;
        }
        tile_rows = std::min(tile_rows, kTileRowsMax);
        KernelPtr bk = pick_tiles(vdt_, mm_, plan_.qpi,
                                  tiles_lightly_loaded(plan_.est_keys, n, passes, tile_rows, plan_.smem_slots));
        (void)occupancy(bk, threads, smem);  // sets the kernel's shared-memory limit
        const int64_t tiles = (n + tile_rows - 1) / tile_rows;
        if (tiles < grid) grid = tiles;
        const longlong2* no_tiles = nullptr;
        const unsigned long long* no_count = nullptr;
        void* args[] = {&a, &next_tile, &tile_rows, &no_tiles, &no_count};
        e = cudaLaunchKernel(bk, dim3((unsigned)grid), dim3(threads), args, smem, s_);
      } else {
        KernelPtr bk = pick_build(vdt_, mm_, false, true, true, plan_.qpi);
        const int threads = plan_.threads;
        int bps = occupancy(bk, threads, 0);
        if (plan_.blocks_per_sm > 0 && plan_.blocks_per_sm < bps) bps = plan_.blocks_per_sm;
        int64_t grid = (int64_t)di.sm_count * bps;
        const int64_t need = ((n + 3) / 4 + threads - 1) / threads;
        if (need < grid) grid = need;
        void* args[] = {&a};
        e = cudaLaunchKernel(bk, dim3((unsigned)grid), dim3(threads), args, 0, s_);
      }
      note_launch();
    }
    cudaFreeAsync(tmp, s_);
    if (e != cudaSuccess) {
      set_error("partitioned build launch failed: %s", cudaGetErrorString(e));
      return AGG_ERR_CUDA;
    }
    return AGG_OK;
  }

  // Build over a column hash-partitioned chunk by chunk (starts: nchunks x 257
  // partition starts, device memory): a tile list in partition order, then the
  // tile-queue build. tiles / ntiles: device scratch for the list.
  agg_status build_pieces(const uint32_t* keys, const void* vals, int64_t n, const unsigned long long* starts,
                          int nchunks, longlong2* tiles, unsigned long long* ntiles) {
    if (n <= 0) return AGG_OK;
    BuildArgs a;
    a.keys = keys;
    a.vals = vals;
    a.n = n;
    a.head = 0;
    a.table = mem_;
    a.mask = (uint32_t)(plan_.slots - 1);
    a.gshift = 32 - (63 - __builtin_clzll((unsigned long long)plan_.slots));
    a.smem_slots = plan_.smem_slots;
    a.smem_cap = (plan_.smem_slots * 3) / 4;
    a.status = status_;
    a.progress = progress_;
    int64_t tile_rows = std::min(plan_.tile_rows ? (int64_t)plan_.tile_rows : kPartTileRows / 2, kTileRowsMax);
    PhaseTimer pt(AGG_PHASE_BUILD, s_);
    gb_piece_tiles<<<1, 1024, 0, s_>>>(starts, nchunks, tile_rows, tiles, ntiles);
    note_launch();
    unsigned long long* next_tile = (unsigned long long*)((char*)mem_ + status_off_ + 128);
    AGG_CUDA_TRY(cudaMemsetAsync(next_tile, 0, 8, s_));
    KernelPtr bk = pick_tiles(vdt_, mm_, plan_.qpi, tiles_lightly_loaded(plan_.est_keys, n, 1, 1, plan_.smem_slots));
    const size_t smem = tile_smem_bytes_dt(vdt_, mm_, plan_.smem_slots);
    int bps = occupancy(bk, plan_.threads, smem);
    if (plan_.blocks_per_sm > 0 && plan_.blocks_per_sm < bps) bps = plan_.blocks_per_sm;
    const int64_t grid = (int64_t)device_info().sm_count * bps;
    const longlong2* tl = tiles;
    const unsigned long long* nt = ntiles;
    void* args[] = {&a, &next_tile, &tile_rows, &tl, &nt};
    cudaError_t e = cudaLaunchKernel(bk, dim3((unsigned)grid), dim3(plan_.threads), args, smem, s_);
    note_launch();
    if (e != cudaSuccess) {
      set_error("piecewise build launch failed: %s", cudaGetErrorString(e));
      return AGG_ERR_CUDA;
    }
    return AGG_OK;
  }

  // Finalise into a new result; TABLE_FULL (and no result) if the table overflowed.
  agg_status finish(agg_groups** gout) {
    *gout = nullptr;
    agg_groups* g = nullptr;
    agg_status st = groups_alloc(nslots_, vdt_, ops_, s_, &g);
    if (st != AGG_OK) return st;
    OutArrays o;
    o.keys = g->keys;
    o.count = g->count;
    o.sum = (unsigned long long*)g->sum;
    o.min = (unsigned long long*)g->min;
    o.max = (unsigned long long*)g->max;
    o.avg = g->avg;
    o.d = (int64_t*)counter_;
    uint32_t mask = (uint32_t)(plan_.slots - 1);
    const DeviceInfo& di = device_info();
    cudaError_t e;
    PhaseTimer pt(AGG_PHASE_FINALIZE, s_);
    if (small_) {
      char* aux = (char*)mem_ + aux_off_;
      uint32_t* ck = (uint32_t*)aux;
      uint32_t* cs = ck + nslots_;
      const int cgrid = (int)((nslots_ + 255) / 256);
      if (mm_) gb_compact<true, 1><<<cgrid, 256, 0, s_>>>((const GSlot<true>*)mem_, mask, ck, cs, counter_);
      else gb_compact<false, 1><<<cgrid, 256, 0, s_>>>((const GSlot<false>*)mem_, mask, ck, cs, counter_);
      note_launch();
      const int rgrid = (int)((nslots_ + kRankKeys - 1) / kRankKeys);
      void* args[] = {&mem_, &ck, &cs, &o};
      e = cudaLaunchKernel(pick_small(vdt_, mm_), dim3(rgrid), dim3(kRankThreads), args, 0, s_);
      note_launch();
    } else {
      char* aux = (char*)mem_ + aux_off_;
      uint32_t* k0 = (uint32_t*)aux;
      uint32_t* s0 = k0 + nslots_;
      uint32_t* k1 = s0 + nslots_;
      uint32_t* s1 = k1 + nslots_;
      void* rtmp = (void*)(((uintptr_t)(s1 + nslots_) + 255) & ~(uintptr_t)255);
      int64_t cgrid = (nslots_ + 255) / 256;
      if (cgrid > (int64_t)di.sm_count * 8) cgrid = (int64_t)di.sm_count * 8;
      if (mm_) gb_compact<true><<<(unsigned)cgrid, 256, 0, s_>>>((const GSlot<true>*)mem_, mask, k0, s0, counter_);
      else gb_compact<false><<<(unsigned)cgrid, 256, 0, s_>>>((const GSlot<false>*)mem_, mask, k0, s0, counter_);
      note_launch();
      uint32_t *sk = nullptr, *ss = nullptr;
      st = radix_sort_pairs<uint32_t>(k0, s0, k1, s1, k0, s0, nslots_, (const int64_t*)counter_, 32, rtmp, s_,
                                      &sk, &ss);
      if (st != AGG_OK) {
        agg_groups_free(g);
        return st;
      }
      int64_t ggrid = cgrid;
      int64_t cap = nslots_;
      void* args[] = {&mem_, &sk, &ss, &o, &cap};
      e = cudaLaunchKernel(pick_gather(vdt_, mm_), dim3((unsigned)ggrid), dim3(256), args, 0, s_);
      note_launch();
    }
    if (e != cudaSuccess) {
      set_error("group-by finalize launch failed: %s", cudaGetErrorString(e));
      agg_groups_free(g);
      return AGG_ERR_CUDA;
    }
    // one copy of the status block: status (+0), group count (+64), and the
    // rows seen / failed of a build stopped by a full table (+192, +200)
    unsigned char* hb = (unsigned char*)stream_pinned(s_, 256, &st);
    if (!hb) {
      agg_groups_free(g);
      return st;
    }
    const cudaError_t e1 = cudaMemcpyAsync(hb, status_, 208, cudaMemcpyDeviceToHost, s_);
    const cudaError_t e3 = cudaStreamSynchronize(s_);
    if (e1 != cudaSuccess || e3 != cudaSuccess) {
      set_error("group-by read-back failed: %s", cudaGetErrorString(e3 != cudaSuccess ? e3 : e1));
      agg_groups_free(g);
      return AGG_ERR_CUDA;
    }
    const int64_t groups = *(const int64_t*)(hb + 64);
    if (*(const int*)hb != 0) {
      rows_seen_ = *(const uint64_t*)(hb + 192);
      rows_failed_ = *(const uint64_t*)(hb + 200);
      agg_groups_free(g);
      set_error("global hash table of %lld slots is full", (long long)plan_.slots);
      return AGG_ERR_TABLE_FULL;
    }
    g->num_groups = groups;
    g->table_slots = plan_.slots;
    g->smem_slots = plan_.strategy == AGG_STRAT_SMEM ? plan_.smem_slots : 0;
    g->strategy = plan_.strategy;
    *gout = g;
    return AGG_OK;
  }

 private:
  int vdt_;
  uint32_t ops_;
  bool mm_;
  HashPlan plan_;
  cudaStream_t s_;
  void* mem_ = nullptr;
  int64_t nslots_ = 0;
  bool small_ = true;
  size_t status_off_ = 0, aux_off_ = 0;
  int* status_ = nullptr;
  unsigned long long* progress_ = nullptr;
  uint64_t rows_seen_ = 0, rows_failed_ = 0;
  unsigned long long* counter_ = nullptr;
};

// Sort-based GROUP BY; feat (nullable) is the column's sketch, whose sampled
// key range can spare the exact range pass.
agg_status sort_groupby(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops, cudaStream_t s,
                        agg_groups** gout, const float* feat);

static int smem_slots_for(double est, bool mm) {
  const int maxs = mm ? 2048 : 4096;
  int64_t s = next_pow2((int64_t)std::ceil(2.0 * est));
  if (s < 256) s = 256;
  if (s > maxs) s = maxs;
  return (int)s;
}

// Selector hooks (the learned selector and the autotuner live in their own units).
int select_learned(const float* feat, bool* ok);
agg_status sketch_and_select(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset,
                             cudaStream_t s, float* feat, int* strategy);
agg_status autotune_pick(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                         const float* feat, double hll, cudaStream_t s, int* strategy, int* smem_slots,
                         int64_t* table_slots, int* items, int* tile_rows);

// Sketch the keys on the device and read the features back (one sync).
agg_status sketch_features(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset,
                                 cudaStream_t s, float* feat) {
  agg_status st = AGG_OK;
  float* fd = (float*)stream_scratch(s, 4096, &st);
  if (!fd) return st;
  float* fdev = fd + 512;  // past the reduce ticket area
  st = sketch_launch(keys, n, vdt, ops, offset, fdev, s);
  if (st != AGG_OK) return st;
  float* hb = (float*)stream_pinned(s, 256, &st);
  if (!hb) return st;
  AGG_CUDA_TRY(cudaMemcpyAsync(hb, fdev, F_COUNT * sizeof(float), cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  std::memcpy(feat, hb, F_COUNT * sizeof(float));
  return AGG_OK;
}

// Rescale the size-dependent features of a sketch taken over the first
// n_part rows to the whole column of n_total rows.
static void rescale_features(float* f, int64_t n_part, int64_t n_total, uint32_t ops) {
  const double m = (double)(n_part < kSketchSample ? n_part : kSketchSample);
  if (m <= 0) return;
  const DeviceInfo& di = device_info();
  const double f1 = (double)f[F_F1] * m, d = (double)f[F_DISTINCT] * m;
  double gee = std::sqrt((double)n_total / m) * f1 + (d - f1);
  if (gee < 1.0) gee = 1.0;
  if (gee > (double)n_total) gee = (double)n_total;
  const double tb = 2.0 * gee * gslot_bytes(ops_minmax(ops));
  f[F_LOG2N] = (float)std::log2((double)n_total);
  f[F_LOG2_GEE] = (float)std::log2(gee);
  f[F_SMEM_RATIO] = (float)std::log2(1.0 + tb / (double)di.smem_per_block_optin);
  f[F_L2_RATIO] = (float)std::log2(1.0 + tb / (double)di.l2_bytes);
}

struct Choice {
  int strategy;
  HashPlan plan;
};

bool wants_hll(const float* f, int64_t n) {
  return n >= (int64_t(1) << 22) && 1.0 - (double)f[F_F1] < 0.97;
}

bool hot_sample(const float* f, int cap) {
  const double m = std::min(std::exp2((double)f[F_LOG2N]), (double)kSketchSample);
  return 1.0 - (double)f[F_F1] >= 0.9 && (double)f[F_DISTINCT] * m <= (double)cap;
}

// Global-table slots for a column with about `keys` distinct keys (a
// HyperLogLog count, relative error about 1%): load at most about 1/2.
static int64_t slots_for_count(double keys, int64_t n) {
  const int64_t cap = std::min<int64_t>(int64_t(1) << 31, next_pow2(std::max<int64_t>(2 * n, 1024)));
  return std::min<int64_t>(cap, std::max<int64_t>(1024, next_pow2((int64_t)std::ceil(2.2 * keys))));
}

int64_t table_slots_for(const float* feat, int64_t n, double hll) {
  return hll > 0.0 ? slots_for_count(hll, n) : table_slots_from_sketch(feat, n);
}

static agg_status choose(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                         const agg_options& o, const float* feat, bool have_feat, double hll, cudaStream_t s,
                         Choice* c) {
  bool covered = false;
  double est = have_feat ? distinct_estimate(feat, &covered) : 1024.0;
  if (hll > 0.0) est = hll;
  int strategy = o.strategy;
  int64_t tslots = o.table_slots;
  int sslots = o.smem_slots;
  int items = o.items_per_thread;
  int tile = o.tile_rows;
  if (strategy == AGG_STRAT_LEARNED) {
    bool ok = false;
    strategy = select_learned(feat, &ok);
    if (!ok) strategy = rule_strategy(feat, ops, hll);
  } else if (strategy == AGG_STRAT_AUTOTUNE) {
    agg_status st = autotune_pick(keys, vals, n, vdt, ops, feat, hll, s, &strategy, &sslots, &tslots, &items, &tile);
    if (st != AGG_OK) return st;
  } else if (strategy == AGG_STRAT_AUTO) {
    strategy = have_feat ? rule_strategy(feat, ops, hll) : AGG_STRAT_GLOBAL;
  }
  c->strategy = strategy;
  c->plan.strategy = strategy;
  c->plan.slots = tslots ? tslots
                         : hll > 0.0 ? slots_for_count(hll, n) : (have_feat ? table_slots_from_sketch(feat, n) : 2048);
  c->plan.smem_slots = sslots ? sslots : smem_slots_for(est, ops_minmax(ops));
  c->plan.threads = o.block_threads ? o.block_threads : (strategy == AGG_STRAT_SMEM ? 512 : 256);
  // frequent keys (a key with >= 3% of the sample, or a handful of keys) make
  // the warp-level reduction of several keys pay; without a sketch, assume so
  c->plan.multi_keys = !have_feat || feat[F_TOP1] >= 0.03f || est <= 32.0;
  c->plan.blocks_per_sm = o.blocks_per_sm;
  c->plan.qpi = items == 8 ? 2 : items == 4 ? 1 : 0;
  c->plan.tile_rows = tile;
  c->plan.est_keys = est;
  // Partition the rows by hash first when the shared tables would spill (more
  // distinct keys than a shared table admits) or the global table exceeds
  // half of L2; each partition then has about 1/256 of the keys.
  const double table_bytes = (double)(c->plan.slots + 2) * gslot_bytes(ops_minmax(ops));
  // a hot head that the shared tables absorb needs no partitioning: the few
  // rows of rarer keys spill to the (right-sized) global table
  const bool hot = hll > 0.0 && hot_sample(feat, (c->plan.smem_slots * 3) / 4);
  const bool spills = strategy == AGG_STRAT_SMEM && est > 0.75 * c->plan.smem_slots && !hot;
  const bool big_table = table_bytes > 0.5 * device_info().l2_bytes;
  c->plan.partition = o.partition > 0 || (o.partition == 0 && n >= (int64_t(1) << 20) && (spills || big_table));
  // two levels (65536 partitions) when 256 partitions would still spill
  c->plan.partition_passes =
      (o.partition == 2 ||
       (o.partition == 0 && strategy == AGG_STRAT_SMEM && est > 256.0 * 0.75 * c->plan.smem_slots))
          ? 2
          : 1;
  return AGG_OK;
}

static bool needs_sketch(const agg_options& o) {
  return o.strategy == AGG_STRAT_AUTO || o.strategy == AGG_STRAT_LEARNED || o.strategy == AGG_STRAT_AUTOTUNE ||
         (o.strategy != AGG_STRAT_SORT && o.table_slots == 0) || (o.strategy == AGG_STRAT_SMEM && o.smem_slots == 0);
}

// Run the hash plan over a device column, regrowing the table on overflow.
// Slots for the next table after a table of `slots` slots filled: the build
// went through `seen` rows, of which `failed` found no slot, so those rows had
// at most slots + failed distinct keys; that bound is scaled to all n rows and
// doubled (load <= 1/2). At least 4x the old table, at most 2n (a table of 2n
// slots holds any key set of n rows) and 2^31. Columns of up to 2^22 rows go
// straight to 2n slots (at most 256 MB): a further retry would cost more.
static int64_t regrow_slots(int64_t slots, int64_t n, uint64_t seen, uint64_t failed) {
  const double nn = (double)std::max<int64_t>(n, 1);
  double keys = (double)slots + (double)failed;
  if (seen > 0 && (double)seen < nn) keys *= nn / (double)seen;
  double want = std::max(4.0 * (double)slots, 2.0 * std::min(keys, nn));
  if (n <= (int64_t(1) << 22)) want = std::max(want, 2.0 * nn);
  const double cap = std::min(2.0 * nn, (double)(int64_t(1) << 31));
  if (want > cap) want = std::max(cap, 4.0 * (double)slots);
  const int64_t p = next_pow2((int64_t)std::ceil(want));
  return std::min<int64_t>(p, int64_t(1) << 31);
}

static agg_status hash_device(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                              HashPlan plan, cudaStream_t s, agg_groups** g) {
  int retries = 0;
  for (;;) {
    agg_status st;
    uint64_t seen = 0, failed = 0;
    {
      HashRun run(vdt, ops, plan, s);
      st = run.init();
      if (st == AGG_OK) st = run.build(keys, vals, n);
      if (st == AGG_OK) st = run.finish(g);
      seen = run.rows_seen();
      failed = run.rows_failed();
    }
    if (st == AGG_OK) {
      (*g)->retries = retries;
      return AGG_OK;
    }
    if (st != AGG_ERR_TABLE_FULL || plan.slots >= (int64_t(1) << 31) || plan.slots >= 4 * std::max<int64_t>(n, 1))
      return st;
    ++retries;
    plan.slots = regrow_slots(plan.slots, n, seen, failed);
  }
}

}  // namespace agg

using namespace agg;

namespace agg {

// GROUP BY of a device column with explicit options. known_feat, when not
// null, is the column's sketch (the autotuner passes it, so that its timed
// candidates plan partitioning exactly as the untuned call would).
agg_status groupby_with(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                        const agg_options& o, cudaStream_t s, agg_groups** out, const float* known_feat,
                        double known_hll) {
  float feat[F_COUNT] = {0};
  bool have = false;
  double hll = 0.0;
  unsigned long long part_counts[256];  // rows per one-level partition, from the HyperLogLog pass
  bool have_counts = false;
  agg_status st = AGG_OK;
  if (known_feat && n > 0) {
    std::memcpy(feat, known_feat, sizeof(feat));
    have = true;
    hll = known_hll;
  } else if (needs_sketch(o) && n > 0) {
    if (o.strategy == AGG_STRAT_LEARNED) {
      int learned = -1;
      st = sketch_and_select(keys, n, vdt, ops, o.sample_offset, s, feat, &learned);
      if (st != AGG_OK) return st;
      have = true;
      if (wants_hll(feat, n)) {
        st = hll_estimate(keys, n, s, &hll, part_counts);
        if (st != AGG_OK) return st;
        have_counts = true;
      }
      agg_options o2 = o;
      o2.strategy = learned >= 0 ? learned : rule_strategy(feat, ops, hll);
      Choice c;
      st = choose(keys, vals, n, vdt, ops, o2, feat, have, hll, s, &c);
      if (st != AGG_OK) return st;
      if (have_counts) c.plan.part_hist = part_counts;
      agg_groups* g = nullptr;
      if (c.strategy == AGG_STRAT_SORT) st = sort_groupby(keys, vals, n, vdt, ops, s, &g, feat);
      else st = hash_device(keys, vals, n, vdt, ops, c.plan, s, &g);
      if (st != AGG_OK) return st;
      std::memcpy(g->features, feat, sizeof(feat));
      *out = g;
      return AGG_OK;
    }
    st = sketch_features(keys, n, vdt, ops, o.sample_offset, s, feat);
    if (st != AGG_OK) return st;
    have = true;
    if (wants_hll(feat, n)) {
      st = hll_estimate(keys, n, s, &hll, part_counts);
      if (st != AGG_OK) return st;
      have_counts = true;
    }
  }
  Choice c;
  st = choose(keys, vals, n, vdt, ops, o, feat, have, hll, s, &c);
  if (st != AGG_OK) return st;
  if (have_counts) c.plan.part_hist = part_counts;
  agg_groups* g = nullptr;
  if (c.strategy == AGG_STRAT_SORT) st = sort_groupby(keys, vals, n, vdt, ops, s, &g, have ? feat : nullptr);
  else st = hash_device(keys, vals, n, vdt, ops, c.plan, s, &g);
  if (st != AGG_OK) return st;
  std::memcpy(g->features, feat, sizeof(feat));
  *out = g;
  return AGG_OK;
}

}  // namespace agg

namespace agg {
agg_status exact_fp_sums(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                         agg_groups* g, cudaStream_t s, bool replace, bool report);
}

static agg_status groupby_impl(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                               const agg_options* opt, cudaStream_t s, agg_groups** out) {
  agg_options o{};
  if (opt) o = *opt;
  agg_status st = groupby_with(keys, vals, n, vdt, ops, o, s, out, nullptr, 0.0);
  const bool exact = o.flags & AGG_FLAG_EXACT_SUM, report = o.flags & AGG_FLAG_SUM_ERROR;
  if (st == AGG_OK && (exact || report) && dtype_is_fp(vdt) && (ops & (AGG_SUM | AGG_AVG))) {
    st = exact_fp_sums(keys, vals, n, vdt, ops, *out, s, exact, report);
    if (st != AGG_OK) {
      agg_groups_free(*out);
      *out = nullptr;
    }
  }
  return st;
}

// ---------------------------------------------------------------------------
// Host-fed GROUP BY: chunks of keys and values are copied on a copy stream
// into a ring of device buffers while the build of the previous chunk runs.
// ---------------------------------------------------------------------------
namespace agg {

struct GbPipe {
  static constexpr int kRing = 3;
  cudaStream_t copy = nullptr;
  cudaEvent_t ready[kRing] = {};
  cudaEvent_t freed[kRing] = {};
  bool ok = false;
  std::mutex call_mu;
};

static GbPipe* gb_pipe(agg_status* st) {
  static std::mutex mu;
  static std::map<int, GbPipe*> pipes;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  GbPipe*& p = pipes[dev];
  if (!p) p = new GbPipe();
  *st = AGG_OK;
  if (!p->ok) {
    if (cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cannot create copy stream");
      *st = AGG_ERR_CUDA;
      return p;
    }
    for (int i = 0; i < GbPipe::kRing; ++i) {
      cudaEventCreateWithFlags(&p->ready[i], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&p->freed[i], cudaEventDisableTiming);
    }
    p->ok = true;
  }
  return p;
}

constexpr int64_t kHostChunkRows = int64_t(1) << 23;  // 8 Mi rows per chunk

}  // namespace agg

static agg_status groupby_host_impl(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                                    const agg_options* opt, cudaStream_t s, agg_groups** out) {
  agg_options o{};
  if (opt) o = *opt;
  agg_status st = AGG_OK;
  GbPipe* pipe = gb_pipe(&st);
  if (st != AGG_OK) return st;
  std::lock_guard<std::mutex> lk(pipe->call_mu);
  const size_t es = dtype_size(vdt);
  const int64_t chunk = kHostChunkRows;
  const size_t kbytes = (size_t)chunk * 4, vbytes = (size_t)chunk * es;
  const size_t slot_bytes = ((kbytes + 255) & ~size_t(255)) + ((vbytes + 255) & ~size_t(255));
  void* ring = nullptr;
  AGG_CUDA_TRY(dev_malloc_async(&ring, (size_t)GbPipe::kRing * slot_bytes, s));
  struct Free {
    void* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } ring_free{ring, s};
  auto kbuf = [&](int b) { return (uint32_t*)((char*)ring + (size_t)b * slot_bytes); };
  auto vbuf = [&](int b) { return (void*)((char*)ring + (size_t)b * slot_bytes + ((kbytes + 255) & ~size_t(255))); };
  const int64_t nchunks = (n + chunk - 1) / chunk;
  cudaEvent_t start_ev;
  AGG_CUDA_TRY(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  struct EvFree {
    cudaEvent_t e;
    ~EvFree() { cudaEventDestroy(e); }
  } ev_free{start_ev};

  // Enqueue the copy of chunk k into ring slot k % kRing (after its last use).
  auto copy_chunk = [&](int64_t k, bool first_round) -> agg_status {
    const int b = (int)(k % GbPipe::kRing);
    const int64_t r0 = k * chunk;
    const int64_t rows = std::min<int64_t>(chunk, n - r0);
    if (!first_round || k >= GbPipe::kRing) cudaStreamWaitEvent(pipe->copy, pipe->freed[b], 0);  // slot reused
    AGG_CUDA_TRY(cudaMemcpyAsync(kbuf(b), keys + r0, (size_t)rows * 4, cudaMemcpyHostToDevice, pipe->copy));
    AGG_CUDA_TRY(cudaMemcpyAsync(vbuf(b), (const char*)vals + (size_t)r0 * es, (size_t)rows * es,
                                 cudaMemcpyHostToDevice, pipe->copy));
    cudaEventRecord(pipe->ready[b], pipe->copy);
    return AGG_OK;
  };

  cudaEventRecord(start_ev, s);
  cudaStreamWaitEvent(pipe->copy, start_ev, 0);  // the ring is ours once prior work on s is done
  // The copy engine runs up to kRing chunks ahead of the builds; the first
  // kRing copies are queued before the sketch's host synchronisation.
  int64_t next_copy = 0;
  bool fresh_ring = true;
  auto ensure_copied = [&](int64_t upto) -> agg_status {
    for (; next_copy <= upto && next_copy < nchunks; ++next_copy) {
      agg_status e = copy_chunk(next_copy, fresh_ring);
      if (e != AGG_OK) return e;
    }
    return AGG_OK;
  };
  float feat[F_COUNT] = {0};
  bool have = false;
  double hll0 = 0.0;  // distinct keys of the first chunk
  const int64_t r0 = std::min<int64_t>(chunk, n);
  if (n > 0) {
    st = ensure_copied(GbPipe::kRing - 1);
    if (st != AGG_OK) return st;
    if (needs_sketch(o)) {
      cudaStreamWaitEvent(s, pipe->ready[0], 0);
      st = sketch_features(kbuf(0), r0, vdt, ops, o.sample_offset, s, feat);
      if (st != AGG_OK) return st;
      rescale_features(feat, r0, n, ops);
      have = true;
      if (wants_hll(feat, n)) {
        st = hll_estimate(kbuf(0), r0, s, &hll0);
        if (st != AGG_OK) return st;
      }
    }
  }
  // The first chunk's count plans a column whose keys recur (far fewer distinct
  // keys than rows in the chunk); one with a long tail keeps the sketch's plan.
  const double hll_plan = hll0 > 0.0 && hll0 < 0.25 * (double)r0 ? hll0 : 0.0;
  Choice c;
  // the autotuner times candidates on a device column: give it the first chunk
  cudaStreamWaitEvent(s, pipe->ready[0], 0);
  st = choose(kbuf(0), vbuf(0), r0, vdt, ops, o, feat, have, hll_plan, s, &c);
  if (st != AGG_OK) return st;
  agg_groups* g = nullptr;
  // The sort, and hash plans that partition the rows, work on the whole
  // column: it is copied once (the prefetched chunks device to device, the
  // rest from the host at link speed) and the device path runs on it. Plans
  // that partition fall back to per-chunk builds when the device lacks room.
  const size_t kb = ((size_t)n * 4 + 255) & ~size_t(255);
  const size_t col_bytes = kb + (size_t)n * es + 256;
  bool whole = c.strategy == AGG_STRAT_SORT;
  bool room = false;
  if (c.plan.partition && n > chunk) {
    size_t free_b = 0, total_b = 0;
    const double table_b = (double)(c.plan.slots + 2) * gslot_bytes(ops_minmax(ops));
    room = cudaMemGetInfo(&free_b, &total_b) == cudaSuccess && (double)free_b > 4.0 * col_bytes + 2.0 * table_b;
  }
  // Streamed: a one-level hash partition of each chunk as it arrives into its
  // own region of a column-sized buffer and a build of its pieces, both
  // overlapped with the copies of the next chunks; a HyperLogLog count over
  // every chunk sizes the table again if the first chunk's count undersized it.
  const bool streamed = room && hll_plan > 0.0 && c.strategy == AGG_STRAT_SMEM && c.plan.partition_passes == 1;
  if (!whole && !streamed && c.plan.partition && n > chunk) whole = room;
  if (streamed) {
    const size_t starts_b = ((size_t)nchunks * 257 * 8 + 255) & ~size_t(255);
    const int64_t max_tiles = (int64_t)nchunks * 256 + n / 4096 + 1;
    const size_t tiles_b = ((size_t)max_tiles * 16 + 255) & ~size_t(255);
    const size_t extra = starts_b + tiles_b + 256 + ((partition_tmp_bytes() + 255) & ~size_t(255)) + hll_state_bytes();
    void* full = nullptr;
    const size_t col_r = (col_bytes + 255) & ~size_t(255);
    AGG_CUDA_TRY(dev_malloc_async(&full, col_r + extra, s));
    Free full_free{full, s};
    uint32_t* fk = (uint32_t*)full;
    char* fv = (char*)full + kb;
    char* x = (char*)full + col_r;
    unsigned long long* starts = (unsigned long long*)x;
    longlong2* tiles = (longlong2*)(x + starts_b);
    unsigned long long* ntiles = (unsigned long long*)(x + starts_b + tiles_b);
    void* ptmp = x + starts_b + tiles_b + 256;
    uint32_t* regs = (uint32_t*)(x + starts_b + tiles_b + 256 + ((partition_tmp_bytes() + 255) & ~size_t(255)));
    // Each chunk's pieces are built as soon as it is partitioned (overlapped
    // with the copies of the next chunks), into a table sized from the first
    // chunk's count with room for twice as many keys. A table that fills is
    // rebuilt after the last chunk over every piece, sized from the count of
    // all chunks.
    HashPlan plan = c.plan;
    plan.slots = o.table_slots ? o.table_slots : table_slots_for(feat, n, 2.0 * hll_plan);
    uint64_t seen = 0, failed = 0;
    {
      HashRun early(vdt, ops, plan, s);
      st = early.init();
      if (st != AGG_OK) return st;
      for (int64_t k = 0; k < nchunks; ++k) {
        st = ensure_copied(k + GbPipe::kRing - 1);
        if (st != AGG_OK) return st;
        const int b = (int)(k % GbPipe::kRing);
        cudaStreamWaitEvent(s, pipe->ready[b], 0);
        const int64_t rows = std::min<int64_t>(chunk, n - k * chunk);
        {
          PhaseTimer pt(AGG_PHASE_SORT, s);
          st = hll_add_chunk(kbuf(b), rows, regs, k == 0, s);
          if (st == AGG_OK)
            st = es == 4 ? partition_hashed<uint32_t>(kbuf(b), (const uint32_t*)vbuf(b), fk, (uint32_t*)fv, rows,
                                                      ptmp, s, k * chunk, starts + k * 257)
                         : partition_hashed<uint64_t>(kbuf(b), (const uint64_t*)vbuf(b), fk, (uint64_t*)fv, rows,
                                                      ptmp, s, k * chunk, starts + k * 257);
        }
        cudaEventRecord(pipe->freed[b], s);
        if (st == AGG_OK) st = early.build_pieces(fk, fv, n, starts + k * 257, 1, tiles, ntiles);
        if (st != AGG_OK) return st;
      }
      st = early.finish(&g);
      seen = early.rows_seen();
      failed = early.rows_failed();
    }
    if (st == AGG_OK) {
      g->retries = 0;
    } else if (st != AGG_ERR_TABLE_FULL) {
      return st;
    } else {
      double hll_all = 0.0;
      st = hll_read(regs, s, &hll_all);
      if (st != AGG_OK) return st;
      const int64_t grown = regrow_slots(plan.slots, n, seen, failed);
      plan.slots = o.table_slots ? grown : std::max(table_slots_for(feat, n, hll_all), grown);
      int retries = 1;
      for (;;) {
        {
          HashRun run(vdt, ops, plan, s);
          st = run.init();
          if (st == AGG_OK) st = run.build_pieces(fk, fv, n, starts, (int)nchunks, tiles, ntiles);
          if (st == AGG_OK) st = run.finish(&g);
          seen = run.rows_seen();
          failed = run.rows_failed();
        }
        if (st == AGG_OK) {
          g->retries = retries;
          break;
        }
        if (st != AGG_ERR_TABLE_FULL || plan.slots >= (int64_t(1) << 31) || plan.slots >= 4 * std::max<int64_t>(n, 1))
          return st;
        ++retries;
        plan.slots = regrow_slots(plan.slots, n, seen, failed);
      }
    }
  } else if (whole) {
    void* full = nullptr;
    AGG_CUDA_TRY(dev_malloc_async(&full, col_bytes, s));
    Free full_free{full, s};
    uint32_t* fk = (uint32_t*)full;
    char* fv = (char*)full + kb;
    const int64_t pre = std::min<int64_t>(next_copy, nchunks);  // chunks already queued into the ring
    if (n > pre * chunk) {
      const int64_t r0 = pre * chunk;
      AGG_CUDA_TRY(cudaMemcpyAsync(fk + r0, keys + r0, (size_t)(n - r0) * 4, cudaMemcpyHostToDevice, pipe->copy));
      AGG_CUDA_TRY(cudaMemcpyAsync(fv + (size_t)r0 * es, (const char*)vals + (size_t)r0 * es, (size_t)(n - r0) * es,
                                   cudaMemcpyHostToDevice, pipe->copy));
    }
    cudaEvent_t done_ev;
    AGG_CUDA_TRY(cudaEventCreateWithFlags(&done_ev, cudaEventDisableTiming));
    EvFree done_free{done_ev};
    cudaEventRecord(done_ev, pipe->copy);
    for (int64_t k = 0; k < pre; ++k) {
      const int b = (int)(k % GbPipe::kRing);
      const int64_t r0 = k * chunk, rows = std::min<int64_t>(chunk, n - r0);
      cudaStreamWaitEvent(s, pipe->ready[b], 0);
      AGG_CUDA_TRY(cudaMemcpyAsync(fk + r0, kbuf(b), (size_t)rows * 4, cudaMemcpyDeviceToDevice, s));
      AGG_CUDA_TRY(cudaMemcpyAsync(fv + (size_t)r0 * es, vbuf(b), (size_t)rows * es, cudaMemcpyDeviceToDevice, s));
    }
    cudaStreamWaitEvent(s, done_ev, 0);
    if (c.strategy == AGG_STRAT_SORT) st = sort_groupby(fk, fv, n, vdt, ops, s, &g, have ? feat : nullptr);
    else st = hash_device(fk, fv, n, vdt, ops, c.plan, s, &g);
    if (st != AGG_OK) return st;
  } else {
    HashPlan plan = c.plan;
    int retries = 0;
    for (;;) {
      uint64_t seen = 0, failed = 0;
      {
        HashRun run(vdt, ops, plan, s);
        st = run.init();
        for (int64_t k = 0; st == AGG_OK && k < nchunks; ++k) {
          st = ensure_copied(k + GbPipe::kRing - 1);
          if (st != AGG_OK) break;
          const int b = (int)(k % GbPipe::kRing);
          cudaStreamWaitEvent(s, pipe->ready[b], 0);
          const int64_t rows = std::min<int64_t>(chunk, n - k * chunk);
          st = run.build(kbuf(b), vbuf(b), rows);
          cudaEventRecord(pipe->freed[b], s);
        }
        if (st == AGG_OK) st = run.finish(&g);
        seen = run.rows_seen();  // rough: chunks enqueued after the table filled count too
        failed = run.rows_failed();
      }
      if (st == AGG_OK) {
        g->retries = retries;
        break;
      }
      if (st != AGG_ERR_TABLE_FULL || plan.slots >= (int64_t(1) << 31) || plan.slots >= 4 * std::max<int64_t>(n, 1))
        return st;
      ++retries;
      plan.slots = regrow_slots(plan.slots, n, seen, failed);
      next_copy = 0;  // copy the column again
      fresh_ring = false;
    }
  }
  std::memcpy(g->features, feat, sizeof(feat));
  *out = g;
  return AGG_OK;
}

static agg_status check_groupby_args(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                                     const agg_options* opt, agg_groups** out) {
  AGG_CHECK_ARG(dtype_valid(vdt), "invalid dtype %d", vdt);
  AGG_CHECK_ARG(ops != 0 && (ops & ~(uint32_t)AGG_ALL) == 0, "invalid ops mask 0x%x", ops);
  AGG_CHECK_ARG(n >= 0 && n <= 0xFFFFFFFFll, "invalid row count %lld (group-by needs n < 2^32)", (long long)n);
  AGG_CHECK_ARG(n == 0 || (keys && vals), "null key or value pointer");
  AGG_CHECK_ARG(out != nullptr, "null result pointer");
  AGG_CHECK_ARG(((uintptr_t)keys & 3) == 0, "key pointer not 4-byte aligned");
  AGG_CHECK_ARG(((uintptr_t)vals % dtype_size(vdt)) == 0, "value pointer not aligned to its element size");
  if (opt) {
    AGG_CHECK_ARG(opt->strategy >= AGG_STRAT_AUTO && opt->strategy <= AGG_STRAT_AUTOTUNE, "invalid strategy %d",
                  opt->strategy);
    AGG_CHECK_ARG(opt->table_slots == 0 || (opt->table_slots >= 2 && (opt->table_slots & (opt->table_slots - 1)) == 0 &&
                                             opt->table_slots <= (int64_t(1) << 31)),
                  "table_slots must be 0 or a power of two <= 2^31");
    AGG_CHECK_ARG(opt->smem_slots == 0 || (opt->smem_slots >= 64 && opt->smem_slots <= 8192 &&
                                            (opt->smem_slots & (opt->smem_slots - 1)) == 0),
                  "smem_slots must be 0 or a power of two in [64, 8192]");
    AGG_CHECK_ARG(opt->block_threads == 0 || (opt->block_threads >= 64 && opt->block_threads <= 1024 &&
                                               opt->block_threads % 32 == 0),
                  "block_threads must be 0 or a multiple of 32 in [64, 1024]");
    AGG_CHECK_ARG(opt->blocks_per_sm >= 0, "blocks_per_sm must be >= 0");
    AGG_CHECK_ARG(opt->items_per_thread == 0 || opt->items_per_thread == 4 || opt->items_per_thread == 8,
                  "items_per_thread must be 0, 4 or 8");
    AGG_CHECK_ARG(opt->tile_rows == 0 || (opt->tile_rows >= 4096 && opt->tile_rows <= 65536 &&
                                          (opt->tile_rows & (opt->tile_rows - 1)) == 0),
                  "tile_rows must be 0 or a power of two in [4096, 65536]");
    AGG_CHECK_ARG((opt->flags & ~(AGG_FLAG_EXACT_SUM | AGG_FLAG_SUM_ERROR)) == 0, "unknown flags 0x%x",
                  (unsigned)opt->flags);
  }
  return AGG_OK;
}

extern "C" agg_status agg_groupby(const uint32_t* keys_dev, const void* vals_dev, int64_t n, agg_dtype vdtype,
                                  uint32_t ops, const agg_options* opt, agg_groups** out, void* stream) {
  clear_error();
  agg_status st = check_groupby_args(keys_dev, vals_dev, n, vdtype, ops, opt, out);
  if (st != AGG_OK) return st;
  *out = nullptr;
  return groupby_impl(keys_dev, vals_dev, n, vdtype, ops, opt, (cudaStream_t)stream, out);
}

extern "C" agg_status agg_groups_to_host(const agg_groups* g, uint32_t* keys, int64_t* count, void* sum, void* min,
                                         void* max, double* avg, double* sum_err) {
  clear_error();
  AGG_CHECK_ARG(g != nullptr, "null result");
  const int64_t d = g->num_groups;
  if (d == 0) return AGG_OK;
  if (keys) AGG_CUDA_TRY(cudaMemcpy(keys, g->keys, (size_t)d * 4, cudaMemcpyDeviceToHost));
  if (count) AGG_CUDA_TRY(cudaMemcpy(count, g->count, (size_t)d * 8, cudaMemcpyDeviceToHost));
  if (sum) AGG_CUDA_TRY(cudaMemcpy(sum, g->sum, (size_t)d * 8, cudaMemcpyDeviceToHost));
  if (min) AGG_CUDA_TRY(cudaMemcpy(min, g->min, (size_t)d * 8, cudaMemcpyDeviceToHost));
  if (max) AGG_CUDA_TRY(cudaMemcpy(max, g->max, (size_t)d * 8, cudaMemcpyDeviceToHost));
  if (avg) AGG_CUDA_TRY(cudaMemcpy(avg, g->avg, (size_t)d * 8, cudaMemcpyDeviceToHost));
  if (sum_err && g->sum_err) AGG_CUDA_TRY(cudaMemcpy(sum_err, g->sum_err, (size_t)d * 8, cudaMemcpyDeviceToHost));
  return AGG_OK;
}

extern "C" void agg_groups_free(agg_groups* g) {
  if (!g) return;
  GroupsPriv* p = (GroupsPriv*)g->priv;
  if (p && p->shared) {
    shared_block_release(p->shared);
    delete p;
    p = nullptr;
  }
  if (p) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    // stream-ordered: work queued on the producing stream finishes first, and
    // no other stream or the host has to wait
    cudaFreeAsync(p->block, p->stream);
    if (p->extra) cudaFreeAsync(p->extra, p->stream);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
  }
  delete g;
}

extern "C" agg_status agg_groupby_host(const uint32_t* keys_host, const void* vals_host, int64_t n, agg_dtype vdtype,
                                       uint32_t ops, const agg_options* opt, agg_groups** out, void* stream) {
  clear_error();
  agg_status st = check_groupby_args(keys_host, vals_host, n, vdtype, ops, opt, out);
  if (st != AGG_OK) return st;
  AGG_CHECK_ARG(!opt || !(opt->flags & (AGG_FLAG_EXACT_SUM | AGG_FLAG_SUM_ERROR)),
                "AGG_FLAG_EXACT_SUM and AGG_FLAG_SUM_ERROR need device columns (agg_groupby)");
  *out = nullptr;
  return groupby_host_impl(keys_host, vals_host, n, vdtype, ops, opt, (cudaStream_t)stream, out);
}

extern "C" int agg_rule_strategy(const float* features_host, uint32_t ops) {
  if (!features_host) return AGG_STRAT_GLOBAL;
  return rule_strategy(features_host, ops);
}
