// Batched GROUP BY: many queries of uneven sizes, key
// distributions and value types in one persistent kernel, captured in a CUDA
// graph.
//
// Plan (once per batch, one host synchronisation): a batched sketch launch
// (one block per query) and, with a selector installed, one batched network
// inference give every query its strategy (shared-memory or global hash) and
// table sizes; tables, outputs and scratch are allocated in one block.
//
// Run (device only; captured into a CUDA graph on the first run, replayed
// after): zero the tables; one persistent build kernel whose blocks pull
// (query, 64 Ki-row tile) work items from a device counter, so large and small
// queries share the GPU without per-query launches; a per-tile shared table
// is cleared before and merged into the query's global table after each
// tile. Finalise: queries whose table has at most 4097 slots are each
// compacted and rank-sorted by one block of a single batched launch; the
// others are compacted together, radix-sorted by (query, key) in two stable
// LSD stages (key, then query) and gathered into their outputs. One read-back
// of the group counts and table status follows the graph.
//
// The sort strategy needs whole-column passes that a tile queue cannot
// interleave; in a batch, a query for which SORT is chosen runs on
// shared-memory tables that spill to its global table (identical results).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <vector>

#include "hashtab.cuh"
#include "sort.cuh"

namespace agg {

constexpr int64_t kTileRows = int64_t(1) << 16;  // default rows per work item (agg_batch_tune may change it)
constexpr int kBatchThreads = 512;

struct BQ {  // one query of a batch, on the device
  const uint32_t* keys;
  const void* vals;
  int64_t n;
  int64_t tile0;  // first tile of this query in the batch's tile space
  void* table;
  int* status;
  int64_t slot0;  // first slot of this query in the concatenated large-table slot space (-1: small)
  OutArrays out;
  uint32_t mask;
  int dt, mm, smem, vec;
  int smem_slots, smem_cap;
  int gshift;
};

template <int DT, bool MM, bool SMEM>
__device__ void batch_tile(const BQ& q, int64_t r0, int64_t r1, unsigned char* smem) {
  BuildArgs a;
  const size_t es = (DT == AGG_I64 || DT == AGG_F64) ? 8 : 4;
  a.keys = q.keys + r0;
  a.vals = (const char*)q.vals + (size_t)r0 * es;
  a.n = r1 - r0;
  a.head = 0;
  a.table = q.table;
  a.mask = q.mask;
  a.gshift = q.gshift;
  a.smem_slots = SMEM ? q.smem_slots : 0;
  a.smem_cap = SMEM ? q.smem_cap : 0;
  a.status = q.status;
  a.progress = nullptr;  // the plan regrows a full table 4x
  a.block_fails = nullptr;
  STab<DT, MM> st;
  if (SMEM) {
    st.carve(smem, a.smem_slots);
    st.clear(a.smem_slots);
    __syncthreads();
  }
  if (q.vec) build_rows<DT, MM, SMEM, true>(a, st, threadIdx.x, blockDim.x);
  else build_rows<DT, MM, SMEM, false>(a, st, threadIdx.x, blockDim.x);
  if (SMEM) {
    __syncthreads();
    flush_smem<DT, MM>(a, st);
  }
}

template <int DT>
__device__ void batch_tile_dt(const BQ& q, int64_t r0, int64_t r1, unsigned char* smem) {
  if (q.mm) {
    if (q.smem) batch_tile<DT, true, true>(q, r0, r1, smem);
    else batch_tile<DT, true, false>(q, r0, r1, smem);
  } else {
    if (q.smem) batch_tile<DT, false, true>(q, r0, r1, smem);
    else batch_tile<DT, false, false>(q, r0, r1, smem);
  }
}

__global__ void __launch_bounds__(kBatchThreads) batch_build(const BQ* __restrict__ qs, int nq,
                                                             const int64_t* __restrict__ tile_prefix,
                                                             int64_t total_tiles, unsigned long long* next_tile,
                                                             int64_t tile_rows) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_tile;
  __shared__ int s_q;
  for (;;) {
    if (threadIdx.x == 0) {
      const int64_t t = (int64_t)atomicAdd(next_tile, 1ull);
      int lo = 0, hi = nq;  // last query with tile_prefix[q] <= t
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_prefix[mid] <= t) lo = mid; else hi = mid;
      }
      s_tile = t;
      s_q = lo;
    }
    __syncthreads();
    const int64_t t = s_tile;
    const int qi = s_q;
    __syncthreads();  // everyone has read s_tile before the next pull overwrites it
    if (t >= total_tiles) return;
    const BQ& q = qs[qi];
    const int64_t r0 = (t - q.tile0) * tile_rows;
    const int64_t r1 = min(r0 + tile_rows, q.n);
    switch (q.dt) {
      case AGG_I32: batch_tile_dt<AGG_I32>(q, r0, r1, smem); break;
      case AGG_I64: batch_tile_dt<AGG_I64>(q, r0, r1, smem); break;
      case AGG_U32: batch_tile_dt<AGG_U32>(q, r0, r1, smem); break;
      case AGG_F32: batch_tile_dt<AGG_F32>(q, r0, r1, smem); break;
      default: batch_tile_dt<AGG_F64>(q, r0, r1, smem); break;
    }
    __syncthreads();  // shared table free before the next tile
  }
}

// ---------------------------------------------------------------------------
// Finalise: small tables, one block per query (compaction + rank sort).
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 1024;

template <int DT, bool MM>
__device__ void small_finalize(const BQ& q, uint32_t* ck, uint32_t* cs, int* s_d) {
  const GSlot<MM>* tab = (const GSlot<MM>*)q.table;
  const int nslots = (int)q.mask + 2;
  for (int j = threadIdx.x; j < nslots; j += kFinThreads) {
    if (occupied<MM>(tab, q.mask, j)) {
      const int pos = atomicAdd(s_d, 1);
      ck[pos] = key_of<MM>(tab, q.mask, j);
      cs[pos] = (uint32_t)j;
    }
  }
  __syncthreads();
  const int d = *s_d;
  for (int i = threadIdx.x; i < d; i += kFinThreads) {
    const uint32_t key = ck[i];
    int rank = 0;
#pragma unroll 8
    for (int t = 0; t < d; ++t) rank += ck[t] < key ? 1 : 0;
    write_group<DT, MM>(q.out, rank, key, tab[cs[i]]);
  }
  if (threadIdx.x == 0) *q.out.d = d;
}

__global__ void __launch_bounds__(kFinThreads) batch_finalize_small(const BQ* __restrict__ qs,
                                                                    const int* __restrict__ small_ids) {
  __shared__ uint32_t ck[kSmallRank];
  __shared__ uint32_t cs[kSmallRank];
  __shared__ int s_d;
  if (threadIdx.x == 0) s_d = 0;
  __syncthreads();
  const BQ& q = qs[small_ids[blockIdx.x]];
#define AGG_SF(D)                                                   \
  case D:                                                           \
    if (q.mm) small_finalize<D, true>(q, ck, cs, &s_d);             \
    else small_finalize<D, false>(q, ck, cs, &s_d);                 \
    break;
  switch (q.dt) { AGG_SF(AGG_I32) AGG_SF(AGG_I64) AGG_SF(AGG_U32) AGG_SF(AGG_F32) AGG_SF(AGG_F64) }
#undef AGG_SF
}

// ---------------------------------------------------------------------------
// Finalise: large tables, all together.
// ---------------------------------------------------------------------------
// Compact the occupied slots of every large table into (key, (query << 32) |
// slot) pairs and count the groups of each query.
__global__ void batch_compact(const BQ* __restrict__ qs, const int* __restrict__ large_ids, int nlarge,
                              const int64_t* __restrict__ slot_prefix, int64_t total_slots, uint32_t* okeys,
                              unsigned long long* opay, unsigned long long* counter) {
  const int lane = threadIdx.x & 31;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < total_slots; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t gs = base + threadIdx.x;
    bool occ = false;
    uint32_t key = 0;
    int qi = 0;
    int64_t local = 0;
    if (gs < total_slots) {
      int lo = 0, hi = nlarge;
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (slot_prefix[mid] <= gs) lo = mid; else hi = mid;
      }
      qi = large_ids[lo];
      const BQ& q = qs[qi];
      local = gs - slot_prefix[lo];
      if (q.mm) {
        occ = occupied<true>((const GSlot<true>*)q.table, q.mask, local);
        if (occ) key = key_of<true>((const GSlot<true>*)q.table, q.mask, local);
      } else {
        occ = occupied<false>((const GSlot<false>*)q.table, q.mask, local);
        if (occ) key = key_of<false>((const GSlot<false>*)q.table, q.mask, local);
      }
    }
    const uint32_t b = __ballot_sync(0xffffffffu, occ);
    if (occ) {  // one count update per query present in the warp
      const uint32_t peers = __match_any_sync(b, qi);
      if ((peers & ((1u << lane) - 1u)) == 0)
        atomicAdd((unsigned long long*)qs[qi].out.d, (unsigned long long)__popc(peers));
    }
    unsigned long long w0 = 0;
    if (lane == 0 && b) w0 = atomicAdd(counter, (unsigned long long)__popc(b));
    w0 = __shfl_sync(0xffffffffu, w0, 0);
    if (occ) {
      const unsigned long long pos = w0 + __popc(b & ((1u << lane) - 1u));
      okeys[pos] = key;
      opay[pos] = ((unsigned long long)qi << 32) | (unsigned long long)local;
    }
  }
}

// After the key stage: query id as the key of the second stage, (key, slot) as its payload.
__global__ void batch_restage(const uint32_t* __restrict__ k, const unsigned long long* __restrict__ p,
                              const unsigned long long* __restrict__ counter, uint32_t* __restrict__ k2,
                              unsigned long long* __restrict__ p2, int64_t cap) {
  const int64_t n = (int64_t)*counter;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n && i < cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long v = p[i];
    k2[i] = (uint32_t)(v >> 32);
    p2[i] = ((unsigned long long)k[i] << 32) | (v & 0xFFFFFFFFull);
  }
}

// Sorted by (query, key): element i goes to position i - first[query] of its query.
__global__ void batch_gather(const BQ* __restrict__ qs, const uint32_t* __restrict__ qid,
                             const unsigned long long* __restrict__ p2, const unsigned long long* __restrict__ counter,
                             const int64_t* __restrict__ first, int64_t cap) {
  const int64_t n = (int64_t)*counter;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n && i < cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int qi = (int)qid[i];
    const BQ& q = qs[qi];
    const uint32_t key = (uint32_t)(p2[i] >> 32);
    const int64_t slot = (int64_t)(p2[i] & 0xFFFFFFFFull);
    const int64_t pos = i - first[qi];
#define AGG_G(D)                                                                                           \
  case D:                                                                                                  \
    if (q.mm) write_group<D, true>(q.out, pos, key, ((const GSlot<true>*)q.table)[slot]);                 \
    else write_group<D, false>(q.out, pos, key, ((const GSlot<false>*)q.table)[slot]);                   \
    break;
    switch (q.dt) { AGG_G(AGG_I32) AGG_G(AGG_I64) AGG_G(AGG_U32) AGG_G(AGG_F32) AGG_G(AGG_F64) }
#undef AGG_G
  }
}

// first[q] = number of large-table groups of queries before q (queries in id order).
__global__ void batch_first(const BQ* __restrict__ qs, int nq, const int* __restrict__ is_large,
                            int64_t* __restrict__ first) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int64_t run = 0;
  for (int q = 0; q < nq; ++q) {
    first[q] = run;
    if (is_large[q]) run += *qs[q].out.d;
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
int select_learned(const float* feat, bool* ok);
double distinct_estimate(const float* feat, bool* covered);
int64_t table_slots_from_sketch(const float* feat, int64_t n);

struct SharedBlock {
  void* p = nullptr;
  int device = 0;
  int refs = 0;
};
static std::mutex g_blk_mu;

static void block_release(SharedBlock* b) {
  bool last = false;
  {
    std::lock_guard<std::mutex> lk(g_blk_mu);
    last = --b->refs == 0;
  }
  if (!last) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != b->device) cudaSetDevice(b->device);
  cudaFree(b->p);
  if (cur != b->device) cudaSetDevice(cur);
  delete b;
}

struct QueryPlan {
  int strategy;  // SMEM or GLOBAL
  int64_t slots;
  int smem_slots;
  bool mm, large;
  size_t table_off, out_off;
  int64_t cap;  // output rows = slots + 1
};

}  // namespace agg

struct agg_batch_plan {
  int device = 0;
  int nq = 0;
  std::vector<agg_query> q;
  std::vector<agg::QueryPlan> qp;
  std::vector<agg::BQ> hq;
  std::vector<float> features;       // nq x 16
  agg::SharedBlock* outs = nullptr;  // output arrays (shared with returned results)
  void* work = nullptr;              // tables, descriptors and scratch
  size_t zero_bytes = 0;             // prefix of `work` cleared by every run
  agg::BQ* dq = nullptr;
  int64_t* tile_prefix = nullptr;
  int64_t total_tiles = 0;
  unsigned long long* next_tile = nullptr;
  unsigned long long* ccount = nullptr;
  int* status = nullptr;
  int64_t* dcount = nullptr;
  int* small_ids = nullptr;
  int* large_ids = nullptr;
  int* is_large = nullptr;
  int nsmall = 0, nlarge = 0;
  int64_t* slot_prefix = nullptr;
  int64_t total_large_slots = 0;
  uint32_t *ck = nullptr, *ck2 = nullptr;
  unsigned long long *cp = nullptr, *cp2 = nullptr;
  int64_t* first = nullptr;
  void* rtmp = nullptr;
  size_t build_smem = 0;
  int build_grid = 0;
  void* pinned = nullptr;  // group counts and status words read back after a run
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t graph_kernels = 0;
  std::vector<int64_t> groups;
  int64_t tile_rows = agg::kTileRows;  // rows per (query, tile) work item
};

namespace agg {

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

static agg_status plan_alloc(agg_batch_plan* P, cudaStream_t s) {
  const int nq = P->nq;
  // outputs, shared with the caller's results
  size_t out_bytes = 0;
  for (int i = 0; i < nq; ++i) {
    QueryPlan& qp = P->qp[i];
    qp.out_off = out_bytes;
    out_bytes += align256((size_t)qp.cap * 4) + 5 * align256((size_t)qp.cap * 8);
  }
  P->outs = new SharedBlock();
  P->outs->refs = 1;
  cudaGetDevice(&P->outs->device);
  AGG_CUDA_TRY(dev_malloc(&P->outs->p, std::max<size_t>(out_bytes, 256)));
  // tables and the small / large split
  size_t tb = 0;
  std::vector<int> small_ids, large_ids, is_large(nq, 0);
  std::vector<int64_t> slot_prefix;
  P->total_large_slots = 0;
  for (int i = 0; i < nq; ++i) {
    QueryPlan& qp = P->qp[i];
    qp.table_off = tb;
    tb += align256((size_t)(qp.slots + 2) * gslot_bytes(qp.mm));
    if (qp.large) {
      is_large[i] = 1;
      large_ids.push_back(i);
      slot_prefix.push_back(P->total_large_slots);
      P->total_large_slots += qp.slots + 1;
    } else {
      small_ids.push_back(i);
    }
  }
  slot_prefix.push_back(P->total_large_slots);
  P->nsmall = (int)small_ids.size();
  P->nlarge = (int)large_ids.size();
  // work block: [tables | status | group counts | counters] (cleared by every
  // run), then descriptors, tile prefix, id lists, slot prefix, first offsets,
  // compaction buffers and radix scratch
  const int64_t L = std::max<int64_t>(P->total_large_slots, 1);
  const size_t ids_stride = align256(sizeof(int) * (nq + 1));
  size_t off = align256(tb);
  const size_t status_off = off;
  off += align256((size_t)nq * 4);
  const size_t dcount_off = off;
  off += align256((size_t)nq * 8);
  const size_t ctr_off = off;
  off += 256;
  const size_t zero_end = off;
  const size_t dq_off = off;
  off += align256(sizeof(BQ) * nq);
  const size_t tp_off = off;
  off += align256(sizeof(int64_t) * (nq + 1));
  const size_t ids_off = off;
  off += 3 * ids_stride;
  const size_t sp_off = off;
  off += align256(sizeof(int64_t) * slot_prefix.size());
  const size_t first_off = off;
  off += align256(sizeof(int64_t) * nq);
  const size_t ck_off = off;
  off += 2 * align256((size_t)L * 4) + 2 * align256((size_t)L * 8);
  const size_t rt_off = off;
  off += align256(radix_tmp_bytes(L));
  AGG_CUDA_TRY(dev_malloc(&P->work, off));
  char* w = (char*)P->work;
  P->zero_bytes = zero_end;
  P->status = (int*)(w + status_off);
  P->dcount = (int64_t*)(w + dcount_off);
  P->next_tile = (unsigned long long*)(w + ctr_off);
  P->ccount = (unsigned long long*)(w + ctr_off + 64);
  P->dq = (BQ*)(w + dq_off);
  P->tile_prefix = (int64_t*)(w + tp_off);
  P->small_ids = (int*)(w + ids_off);
  P->large_ids = (int*)(w + ids_off + ids_stride);
  P->is_large = (int*)(w + ids_off + 2 * ids_stride);
  P->slot_prefix = (int64_t*)(w + sp_off);
  P->first = (int64_t*)(w + first_off);
  P->ck = (uint32_t*)(w + ck_off);
  P->ck2 = (uint32_t*)(w + ck_off + align256((size_t)L * 4));
  P->cp = (unsigned long long*)(w + ck_off + 2 * align256((size_t)L * 4));
  P->cp2 = (unsigned long long*)(w + ck_off + 2 * align256((size_t)L * 4) + align256((size_t)L * 8));
  P->rtmp = w + rt_off;
  // descriptors
  P->hq.assign(nq, BQ{});
  std::vector<int64_t> tile_prefix(nq + 1, 0);
  P->build_smem = 0;
  char* ob = (char*)P->outs->p;
  int li = 0;
  for (int i = 0; i < nq; ++i) {
    const agg_query& q = P->q[i];
    const QueryPlan& qp = P->qp[i];
    BQ& b = P->hq[i];
    b.keys = q.keys;
    b.vals = q.vals;
    b.n = q.n;
    b.tile0 = tile_prefix[i];
    tile_prefix[i + 1] = tile_prefix[i] + (q.n + P->tile_rows - 1) / P->tile_rows;
    b.table = w + qp.table_off;
    b.status = P->status + i;
    b.slot0 = qp.large ? slot_prefix[li++] : -1;
    b.mask = (uint32_t)(qp.slots - 1);
    b.gshift = 32 - (63 - __builtin_clzll((unsigned long long)qp.slots));
    b.dt = q.dtype;
    b.mm = qp.mm ? 1 : 0;
    b.smem = qp.strategy == AGG_STRAT_SMEM ? 1 : 0;
    b.vec = (((uintptr_t)q.keys & 15) == 0 && ((uintptr_t)q.vals & 15) == 0) ? 1 : 0;
    b.smem_slots = b.smem ? qp.smem_slots : 0;
    b.smem_cap = b.smem ? (qp.smem_slots * 3) / 4 : 0;
    char* o = ob + qp.out_off;
    const int64_t cap = qp.cap;
    b.out.keys = (uint32_t*)o;
    o += align256((size_t)cap * 4);
    b.out.count = (int64_t*)o;
    o += align256((size_t)cap * 8);
    b.out.sum = (unsigned long long*)o;
    o += align256((size_t)cap * 8);
    b.out.min = (unsigned long long*)o;
    o += align256((size_t)cap * 8);
    b.out.max = (unsigned long long*)o;
    o += align256((size_t)cap * 8);
    b.out.avg = (double*)o;
    b.out.d = P->dcount + i;
    if (b.smem) {
      const bool wide = b.dt == AGG_I64 || b.dt == AGG_F64;
      const size_t sb = wide ? (b.mm ? stab_bytes<AGG_I64, true>(b.smem_slots) : stab_bytes<AGG_I64, false>(b.smem_slots))
                             : (b.mm ? stab_bytes<AGG_I32, true>(b.smem_slots) : stab_bytes<AGG_I32, false>(b.smem_slots));
      P->build_smem = std::max(P->build_smem, sb);
    }
  }
  P->total_tiles = tile_prefix[nq];
  const size_t st = ids_stride / sizeof(int);
  std::vector<int> ids(3 * st, 0);
  for (int i = 0; i < P->nsmall; ++i) ids[i] = small_ids[i];
  for (int i = 0; i < P->nlarge; ++i) ids[st + i] = large_ids[i];
  for (int i = 0; i < nq; ++i) ids[2 * st + i] = is_large[i];
  if (nq > 0) {
    AGG_CUDA_TRY(cudaMemcpyAsync(P->dq, P->hq.data(), sizeof(BQ) * nq, cudaMemcpyHostToDevice, s));
    AGG_CUDA_TRY(cudaMemcpyAsync(P->tile_prefix, tile_prefix.data(), sizeof(int64_t) * (nq + 1),
                                 cudaMemcpyHostToDevice, s));
    AGG_CUDA_TRY(cudaMemcpyAsync(P->small_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s));
    AGG_CUDA_TRY(cudaMemcpyAsync(P->slot_prefix, slot_prefix.data(), sizeof(int64_t) * slot_prefix.size(),
                                 cudaMemcpyHostToDevice, s));
  }
  AGG_CUDA_TRY(cudaMallocHost(&P->pinned, (size_t)nq * 12 + 64));
  // build grid: blocks resident per SM for the shared table size
  if (P->build_smem > 48 * 1024)
    AGG_CUDA_TRY(cudaFuncSetAttribute(batch_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)P->build_smem));
  int bps = 0;
  AGG_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, batch_build, kBatchThreads, P->build_smem));
  if (bps < 1) bps = 1;
  P->build_grid = device_info().sm_count * bps;
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  return AGG_OK;
}

// The device work of a run (what the graph holds).
static agg_status plan_enqueue(agg_batch_plan* P, cudaStream_t s, int64_t* kernels) {
  int64_t k = 0;
  AGG_CUDA_TRY(cudaMemsetAsync(P->work, 0, P->zero_bytes, s));
  if (P->total_tiles > 0) {
    batch_build<<<P->build_grid, kBatchThreads, P->build_smem, s>>>(P->dq, P->nq, P->tile_prefix, P->total_tiles,
                                                                     P->next_tile, P->tile_rows);
    ++k;
  }
  if (P->nsmall > 0) {
    batch_finalize_small<<<P->nsmall, kFinThreads, 0, s>>>(P->dq, P->small_ids);
    ++k;
  }
  if (P->nlarge > 0) {
    const DeviceInfo& di = device_info();
    int64_t g = (P->total_large_slots + 255) / 256;
    g = std::min<int64_t>(g, (int64_t)di.sm_count * 8);
    batch_compact<<<(unsigned)g, 256, 0, s>>>(P->dq, P->large_ids, P->nlarge, P->slot_prefix,
                                              P->total_large_slots, P->ck, P->cp, P->ccount);
    ++k;
    const int64_t L = P->total_large_slots;
    uint32_t* kout = nullptr;
    uint64_t* pout = nullptr;
    // stage 1: by key (32 bits)
    agg_status st = radix_sort_pairs<uint64_t>(P->ck, (const uint64_t*)P->cp, P->ck2, (uint64_t*)P->cp2, P->ck,
                                               (uint64_t*)P->cp, L, (const int64_t*)P->ccount, 32, P->rtmp, s, &kout,
                                               &pout);
    if (st != AGG_OK) return st;
    k += 4 * 5;
    // stage 2: stably by query id (16 bits), (key, slot) as the payload
    uint32_t* k2 = kout == P->ck ? P->ck2 : P->ck;
    uint64_t* p2 = pout == (uint64_t*)P->cp ? (uint64_t*)P->cp2 : (uint64_t*)P->cp;
    batch_restage<<<(unsigned)g, 256, 0, s>>>(kout, (const unsigned long long*)pout, P->ccount, k2,
                                              (unsigned long long*)p2, L);
    ++k;
    uint32_t* kfin = nullptr;
    uint64_t* pfin = nullptr;
    st = radix_sort_pairs<uint64_t>(k2, p2, kout, pout, k2, p2, L, (const int64_t*)P->ccount, 16, P->rtmp, s, &kfin,
                                    &pfin);
    if (st != AGG_OK) return st;
    k += 2 * 5;
    batch_first<<<1, 32, 0, s>>>(P->dq, P->nq, P->is_large, P->first);
    batch_gather<<<(unsigned)g, 256, 0, s>>>(P->dq, kfin, (const unsigned long long*)pfin, P->ccount, P->first, L);
    k += 2;
  }
  // group counts and status words to the host
  AGG_CUDA_TRY(cudaMemcpyAsync(P->pinned, P->dcount, (size_t)P->nq * 8, cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaMemcpyAsync((char*)P->pinned + (size_t)P->nq * 8, P->status, (size_t)P->nq * 4,
                               cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaGetLastError());
  *kernels = k;
  return AGG_OK;
}

static void plan_release(agg_batch_plan* P) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
  if (P->work) cudaFree(P->work);
  P->work = nullptr;
  if (P->pinned) cudaFreeHost(P->pinned);
  P->pinned = nullptr;
  if (P->outs) block_release(P->outs);
  P->outs = nullptr;
}

// Strategy and table sizes of every query from the batch sketch.
static void plan_sizes(agg_batch_plan* P, const std::vector<int>& learned) {
  const int nq = P->nq;
  P->qp.assign(nq, QueryPlan{});
  for (int i = 0; i < nq; ++i) {
    const agg_query& q = P->q[i];
    const float* f = &P->features[(size_t)i * F_COUNT];
    QueryPlan& qp = P->qp[i];
    qp.mm = ops_minmax(q.ops);
    int strat = q.strategy;
    if (strat == AGG_STRAT_LEARNED) strat = learned[i] >= 0 ? learned[i] : rule_strategy(f, q.ops);
    else if (strat == AGG_STRAT_AUTOTUNE) {
      int sslots = 0;  // the autotuner's cached choice for this signature, else the rule
      if (!autotune_cached(q.dtype, q.ops, f, &strat, &sslots)) strat = rule_strategy(f, q.ops);
    } else if (strat == AGG_STRAT_AUTO) {
      strat = rule_strategy(f, q.ops);
    }
    // the batch runs hash strategies only: a query the selector would sort gets
    // shared-memory tables (hot keys stay in shared memory; a global table
    // alone would serialize their atomics)
    qp.strategy = strat == AGG_STRAT_GLOBAL ? AGG_STRAT_GLOBAL : AGG_STRAT_SMEM;
    bool covered = false;
    const double est = q.n > 0 ? distinct_estimate(f, &covered) : 1.0;
    const int64_t slots = q.n > 0 ? table_slots_from_sketch(f, q.n) : 1024;
    qp.slots = slots;
    const int maxs = qp.mm ? 2048 : 4096;
    const int64_t ss = next_pow2((int64_t)std::ceil(2.0 * est));
    qp.smem_slots = (int)std::max<int64_t>(256, std::min<int64_t>(ss, maxs));
    qp.cap = slots + 1;
    qp.large = qp.cap > kSmallRank;
  }
}

// Batched sketch and, with a selector installed, batched network inference.
agg_status batch_select(const SketchJob* jobs_dev, int nq, float* feat_dev, float* probs_dev, cudaStream_t s,
                        bool* have_probs);

}  // namespace agg

using namespace agg;

extern "C" agg_status agg_batch_plan_create(const agg_query* queries, int nq, agg_batch_plan** out, void* stream) {
  clear_error();
  AGG_CHECK_ARG(out != nullptr && nq >= 0 && (nq == 0 || queries != nullptr), "invalid arguments");
  AGG_CHECK_ARG(nq < 65536, "a batch holds at most 65535 queries");
  for (int i = 0; i < nq; ++i) {
    const agg_query& q = queries[i];
    AGG_CHECK_ARG(dtype_valid(q.dtype), "query %d: invalid dtype", i);
    AGG_CHECK_ARG(q.ops != 0 && (q.ops & ~(uint32_t)AGG_ALL) == 0, "query %d: invalid ops", i);
    AGG_CHECK_ARG(q.n >= 0 && q.n <= 0xFFFFFFFFll, "query %d: invalid row count", i);
    AGG_CHECK_ARG(q.n == 0 || (q.keys && q.vals), "query %d: null column", i);
    AGG_CHECK_ARG(((uintptr_t)q.keys & 3) == 0 && ((uintptr_t)q.vals % dtype_size(q.dtype)) == 0,
                  "query %d: misaligned column", i);
    AGG_CHECK_ARG(q.strategy >= AGG_STRAT_AUTO && q.strategy <= AGG_STRAT_AUTOTUNE, "query %d: invalid strategy", i);
  }
  cudaStream_t s = (cudaStream_t)stream;
  auto* P = new agg_batch_plan();
  cudaGetDevice(&P->device);
  P->nq = nq;
  P->q.assign(queries, queries + nq);
  P->features.assign((size_t)nq * F_COUNT, 0.f);
  std::vector<int> learned(nq, -1);
  if (nq > 0) {
    std::vector<SketchJob> jobs(nq);
    for (int i = 0; i < nq; ++i) {
      jobs[i] = SketchJob{queries[i].keys, queries[i].n, 0, (int)dtype_size(queries[i].dtype),
                          __builtin_popcount(queries[i].ops), dtype_is_fp(queries[i].dtype) ? 1 : 0,
                          gslot_bytes(ops_minmax(queries[i].ops))};
    }
    void* tmp = nullptr;
    const size_t jb = align256(sizeof(SketchJob) * nq), fb = align256(sizeof(float) * F_COUNT * nq);
    if (dev_malloc(&tmp, jb + fb + align256(sizeof(float) * 3 * nq)) != cudaSuccess) {
      delete P;
      set_error("batch plan: allocation failed");
      return AGG_ERR_OOM;
    }
    float* fdev = (float*)((char*)tmp + jb);
    float* pdev = (float*)((char*)tmp + jb + fb);
    agg_status st = AGG_OK;
    bool have_probs = false;
    if (cudaMemcpyAsync(tmp, jobs.data(), sizeof(SketchJob) * nq, cudaMemcpyHostToDevice, s) != cudaSuccess)
      st = AGG_ERR_CUDA;
    if (st == AGG_OK) st = batch_select((const SketchJob*)tmp, nq, fdev, pdev, s, &have_probs);
    std::vector<float> probs((size_t)nq * 3, 0.f);
    if (st == AGG_OK) {
      cudaMemcpyAsync(P->features.data(), fdev, sizeof(float) * F_COUNT * nq, cudaMemcpyDeviceToHost, s);
      if (have_probs) cudaMemcpyAsync(probs.data(), pdev, sizeof(float) * 3 * nq, cudaMemcpyDeviceToHost, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) st = AGG_ERR_CUDA;
    }
    cudaFree(tmp);
    if (st != AGG_OK) {
      delete P;
      if (st == AGG_ERR_CUDA) set_error("batch sketch failed");
      return st;
    }
    if (have_probs) {
      for (int i = 0; i < nq; ++i) {
        const float* p = &probs[(size_t)i * 3];
        int b = 0;
        for (int o = 1; o < 3; ++o)
          if (p[o] > p[b]) b = o;
        learned[i] = b == 0 ? AGG_STRAT_SMEM : b == 1 ? AGG_STRAT_GLOBAL : AGG_STRAT_SORT;
      }
    }
  }
  plan_sizes(P, learned);
  agg_status st = plan_alloc(P, s);
  if (st != AGG_OK) {
    plan_release(P);
    delete P;
    return st;
  }
  P->groups.assign(nq, 0);
  *out = P;
  return AGG_OK;
}

extern "C" agg_status agg_batch_run(agg_batch_plan* P, void* stream) {
  clear_error();
  AGG_CHECK_ARG(P != nullptr, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  for (int attempt = 0;; ++attempt) {
    if (!P->exec) {
      // kernel attributes are set outside the capture; then the run is captured
      agg_status st = radix_prepare();
      if (st != AGG_OK) return st;
      cudaStream_t cs = nullptr;
      AGG_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) {
        cudaStreamDestroy(cs);
        AGG_CUDA_TRY(e);
      }
      int64_t kernels = 0;
      st = plan_enqueue(P, cs, &kernels);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(cs, &g);
      cudaStreamDestroy(cs);
      if (st != AGG_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      AGG_CUDA_TRY(e);
      P->graph = g;
      AGG_CUDA_TRY(cudaGraphInstantiate(&P->exec, g, 0));
      P->graph_kernels = kernels;
    }
    {
      PhaseTimer pt(AGG_PHASE_BATCH, s);
      AGG_CUDA_TRY(cudaGraphLaunch(P->exec, s));
    }
    note_launch((int)P->graph_kernels);
    AGG_CUDA_TRY(cudaStreamSynchronize(s));
    const int64_t* d = (const int64_t*)P->pinned;
    const int* status = (const int*)((const char*)P->pinned + (size_t)P->nq * 8);
    bool any_full = false;
    for (int i = 0; i < P->nq; ++i) {
      P->groups[i] = d[i];
      if (status[i]) {
        any_full = true;
        P->qp[i].slots = std::min<int64_t>(P->qp[i].slots * 4, int64_t(1) << 31);
        P->qp[i].cap = P->qp[i].slots + 1;
        P->qp[i].large = P->qp[i].cap > kSmallRank;
      }
    }
    if (!any_full) return AGG_OK;
    if (attempt >= 10) {
      set_error("batch: a table stayed full after regrowth");
      return AGG_ERR_TABLE_FULL;
    }
    // regrow the full tables: new allocations and a new graph
    plan_release(P);
    agg_status st = plan_alloc(P, s);
    if (st != AGG_OK) return st;
  }
}

// Re-tile a plan: the per-query tile prefix is rebuilt and the graph
// re-captured at the next run; tables and outputs stay.
static agg_status plan_retile(agg_batch_plan* P, int64_t tile_rows, cudaStream_t s) {
  if (P->exec) cudaGraphExecDestroy(P->exec);
  if (P->graph) cudaGraphDestroy(P->graph);
  P->exec = nullptr;
  P->graph = nullptr;
  P->tile_rows = tile_rows;
  std::vector<int64_t> tp(P->nq + 1, 0);
  for (int i = 0; i < P->nq; ++i) {
    P->hq[i].tile0 = tp[i];
    tp[i + 1] = tp[i] + (P->q[i].n + tile_rows - 1) / tile_rows;
  }
  P->total_tiles = tp[P->nq];
  if (P->nq > 0) {
    AGG_CUDA_TRY(cudaMemcpyAsync(P->dq, P->hq.data(), sizeof(BQ) * P->nq, cudaMemcpyHostToDevice, s));
    AGG_CUDA_TRY(cudaMemcpyAsync(P->tile_prefix, tp.data(), sizeof(int64_t) * (P->nq + 1), cudaMemcpyHostToDevice, s));
  }
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  return AGG_OK;
}

extern "C" agg_status agg_batch_tune(agg_batch_plan* P, int reps, int32_t* tile_rows_out, void* stream) {
  clear_error();
  AGG_CHECK_ARG(P != nullptr, "null plan");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t cand[] = {16384, 32768, 65536};
  float best_ms = INFINITY;
  int64_t best = P->tile_rows;
  cudaEvent_t a, b;
  AGG_CUDA_TRY(cudaEventCreate(&a));
  AGG_CUDA_TRY(cudaEventCreate(&b));
  agg_status st = AGG_OK;
  for (int64_t t : cand) {
    st = plan_retile(P, t, s);
    if (st == AGG_OK) st = agg_batch_run(P, stream);  // capture (and regrow if needed)
    if (st != AGG_OK) break;
    float ms = INFINITY;
    for (int r = 0; r < std::max(1, reps) && st == AGG_OK; ++r) {
      cudaEventRecord(a, s);
      st = agg_batch_run(P, stream);
      cudaEventRecord(b, s);
      cudaEventSynchronize(b);
      float m = 0.f;
      cudaEventElapsedTime(&m, a, b);
      ms = std::min(ms, m);
    }
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != AGG_OK) return st;
  if (P->tile_rows != best) {
    st = plan_retile(P, best, s);
    if (st != AGG_OK) return st;
  }
  if (tile_rows_out) *tile_rows_out = (int32_t)best;
  return AGG_OK;
}

extern "C" agg_status agg_batch_result(const agg_batch_plan* P, int i, agg_groups** out) {
  clear_error();
  AGG_CHECK_ARG(P != nullptr && out != nullptr && i >= 0 && i < P->nq, "invalid arguments");
  const BQ& b = P->hq[i];
  agg_groups* g = new agg_groups();
  std::memset(g, 0, sizeof(*g));
  g->num_groups = P->groups[i];
  g->dtype = P->q[i].dtype;
  g->ops = P->q[i].ops;
  g->strategy = P->qp[i].strategy;
  g->table_slots = P->qp[i].slots;
  g->smem_slots = P->qp[i].strategy == AGG_STRAT_SMEM ? P->qp[i].smem_slots : 0;
  g->keys = b.out.keys;
  g->count = b.out.count;
  g->sum = b.out.sum;
  g->min = b.out.min;
  g->max = b.out.max;
  g->avg = b.out.avg;
  std::memcpy(g->features, &P->features[(size_t)i * F_COUNT], sizeof(float) * F_COUNT);
  auto* priv = new GroupsPriv();
  priv->block = nullptr;
  priv->shared = P->outs;
  priv->device = P->device;
  {
    std::lock_guard<std::mutex> lk(g_blk_mu);
    ++P->outs->refs;
  }
  g->priv = priv;
  *out = g;
  return AGG_OK;
}

extern "C" int agg_batch_size(const agg_batch_plan* P) { return P ? P->nq : 0; }

extern "C" void agg_batch_plan_free(agg_batch_plan* P) {
  if (!P) return;
  plan_release(P);
  delete P;
}

extern "C" agg_status agg_batch(const agg_query* queries, int nq, agg_groups** outs, void* stream) {
  clear_error();
  AGG_CHECK_ARG(outs != nullptr || nq == 0, "null result array");
  agg_batch_plan* P = nullptr;
  agg_status st = agg_batch_plan_create(queries, nq, &P, stream);
  if (st != AGG_OK) return st;
  st = agg_batch_run(P, stream);
  for (int i = 0; st == AGG_OK && i < nq; ++i) st = agg_batch_result(P, i, &outs[i]);
  agg_batch_plan_free(P);
  return st;
}

namespace agg {
void shared_block_release(SharedBlock* b) { block_release(b); }
}  // namespace agg
