// GROUP BY by sorting (step a5s; the sort-based group-by of Sec. 7).
//
// 1. Stable LSD radix sort of the (key, value) pairs by key.
// 2. seg_heads: per 4096-row tile, the number of run heads (rows whose key
//    differs from the previous row's); an exclusive scan gives each tile the
//    index of its first run, and the total is the number of groups d.
// 3. seg_reduce: each thread folds 16 consecutive sorted rows. A run that
//    starts and ends inside one thread is complete and stored directly; a run
//    piece that crosses a thread boundary is combined with the other pieces of
//    the same run in the warp (match on the run index) and added to the output
//    with one set of atomics per warp.
// 4. seg_finalize: decode MIN/MAX images and compute AVG.
// Runs come out in ascending key order by construction.
#include <type_traits>

#include "groupby.cuh"
#include "sort.cuh"

namespace agg {

constexpr int kSegThreads = 256;
constexpr int kSegItems = 16;
constexpr int kSegTile = kSegThreads * kSegItems;

template <int DT> struct SV;
template <> struct SV<AGG_I32> { using T = int32_t; using P = uint32_t; };
template <> struct SV<AGG_I64> { using T = int64_t; using P = uint64_t; };
template <> struct SV<AGG_U32> { using T = uint32_t; using P = uint32_t; };
template <> struct SV<AGG_F32> { using T = float; using P = uint32_t; };
template <> struct SV<AGG_F64> { using T = double; using P = uint64_t; };

template <int DT>
__device__ __forceinline__ typename SV<DT>::T sv_val(typename SV<DT>::P p) {
  typename SV<DT>::T t;
  memcpy(&t, &p, sizeof(t));
  return t;
}

template <int DT>
__device__ __forceinline__ uint64_t sv_img(typename SV<DT>::T v) {
  if (DT == AGG_F32) return (uint64_t)img_f32((float)v);
  if (DT == AGG_F64) return img_f64((double)v);
  return img_i64((int64_t)v);
}

__device__ __forceinline__ uint32_t block_excl_scan256(uint32_t v) {
  __shared__ uint32_t ws[kSegThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < kSegThreads / 32 ? ws[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < kSegThreads / 32) ws[lane] = s;
  }
  __syncthreads();
  uint32_t r = (w ? ws[w - 1] : 0) + x - v;
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kSegThreads) seg_heads(const uint32_t* __restrict__ sk, int64_t n,
                                                         uint32_t* __restrict__ tile_counts) {
  const int64_t r0 = (int64_t)blockIdx.x * kSegTile + (int64_t)threadIdx.x * kSegItems;
  uint32_t prev = r0 > 0 && r0 - 1 < n ? sk[r0 - 1] : 0;
  uint32_t c = 0;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    const int64_t r = r0 + i;
    if (r < n) {
      const uint32_t k = sk[r];
      c += (r == 0 || k != prev) ? 1u : 0u;
      prev = k;
    }
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  __shared__ uint32_t ws[kSegThreads / 32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int i = 0; i < kSegThreads / 32; ++i) t += ws[i];
    tile_counts[blockIdx.x] = t;
  }
}

struct SegOut {
  uint32_t* keys;
  unsigned long long* count;
  unsigned long long* sum;
  unsigned long long* minc;  // complement of the min image (atomicMax)
  unsigned long long* mx;    // max image
  double* avg;
};

struct Piece {
  uint32_t cnt;
  unsigned long long sum;  // int64 bits or double bits
  unsigned long long mn, mx;
};

template <int DT>
__device__ __forceinline__ unsigned long long sum_add(unsigned long long a, unsigned long long b) {
  if (DT == AGG_F32 || DT == AGG_F64)
    return (unsigned long long)__double_as_longlong(__longlong_as_double((long long)a) +
                                                    __longlong_as_double((long long)b));
  return a + b;
}

template <int DT, bool MM>
__device__ __forceinline__ void store_run(const SegOut& o, uint32_t run, uint32_t key, const Piece& p) {
  o.keys[run] = key;
  o.count[run] = p.cnt;
  o.sum[run] = p.sum;
  if (MM) {
    o.minc[run] = ~p.mn;
    o.mx[run] = p.mx;
  }
}

template <int DT, bool MM>
__device__ __forceinline__ void add_run(const SegOut& o, uint32_t run, uint32_t key, const Piece& p) {
  o.keys[run] = key;
  atomicAdd(&o.count[run], (unsigned long long)p.cnt);
  if (DT == AGG_F32 || DT == AGG_F64) atomicAdd((double*)&o.sum[run], __longlong_as_double((long long)p.sum));
  else atomicAdd(&o.sum[run], p.sum);
  if (MM) {
    atomicMax(&o.minc[run], ~p.mn);
    atomicMax(&o.mx[run], p.mx);
  }
}

// Warp-combine boundary pieces with equal run index, then one atomic set per run.
template <int DT, bool MM>
__device__ __forceinline__ void warp_emit(const SegOut& o, bool has, uint32_t run, uint32_t key, Piece p) {
  const int lane = threadIdx.x & 31;
  // lanes without a piece get a tag no run index can take
  const unsigned long long tag = has ? (unsigned long long)run : ((1ull << 32) | (unsigned long long)lane);
  const uint32_t peers = __match_any_sync(0xffffffffu, tag);
  const bool leader = has && (peers & ((1u << lane) - 1u)) == 0;
  for (int src = 0; src < 32; ++src) {
    const uint32_t c2 = __shfl_sync(0xffffffffu, p.cnt, src);
    const unsigned long long s2 = __shfl_sync(0xffffffffu, p.sum, src);
    unsigned long long n2 = 0, x2 = 0;
    if (MM) {
      n2 = __shfl_sync(0xffffffffu, p.mn, src);
      x2 = __shfl_sync(0xffffffffu, p.mx, src);
    }
    if (leader && src != lane && ((peers >> src) & 1u)) {
      p.cnt += c2;
      p.sum = sum_add<DT>(p.sum, s2);
      if (MM) {
        p.mn = min(p.mn, n2);
        p.mx = max(p.mx, x2);
      }
    }
  }
  if (leader) add_run<DT, MM>(o, run, key, p);
}

template <int DT, bool MM>
__global__ void __launch_bounds__(kSegThreads) seg_reduce(const uint32_t* __restrict__ sk,
                                                          const typename SV<DT>::P* __restrict__ sv, int64_t n,
                                                          const uint32_t* __restrict__ tile_first_run, SegOut o) {
  using T = typename SV<DT>::T;
  using F = typename std::conditional<DT == AGG_F32, float, double>::type;
  const int64_t r0 = (int64_t)blockIdx.x * kSegTile + (int64_t)threadIdx.x * kSegItems;
  uint32_t k[kSegItems];
  T v[kSegItems];
  uint32_t heads = 0;
  const uint32_t prev0 = (r0 > 0 && r0 - 1 < n) ? sk[r0 - 1] : 0;
  {
    uint32_t prev = prev0;
#pragma unroll
    for (int i = 0; i < kSegItems; ++i) {
      const int64_t r = r0 + i;
      k[i] = r < n ? sk[r] : 0;
      v[i] = r < n ? sv_val<DT>(sv[r]) : T(0);
      if (r < n && (r == 0 || k[i] != prev)) heads |= 1u << i;
      prev = k[i];
    }
  }
  const uint32_t excl = block_excl_scan256((uint32_t)__popc(heads));
  const int nv = (int)(r0 < n ? (n - r0 < kSegItems ? n - r0 : kSegItems) : 0);
  const bool next_is_head = (r0 + kSegItems >= n) || (nv == kSegItems && sk[r0 + kSegItems] != k[kSegItems - 1]);
  // run index of the run holding row r0 (the run continuing from the left, or the first head's)
  uint32_t run = tile_first_run[blockIdx.x] + excl - ((heads & 1u) ? 0u : 1u);
  Piece first{}, last{};
  bool have_first = false, have_last = false;
  uint32_t first_key = 0, last_key = 0, first_run = 0, last_run = 0;
  // current piece
  bool open = false, open_at_head = false;
  uint32_t pk = 0;
  Piece cur{};
  F cs = 0, cc = 0;  // compensated float sum of the current piece
  long long isum = 0;
  auto close_piece = [&](bool ends_here) {
    cur.sum = (DT == AGG_F32 || DT == AGG_F64) ? (unsigned long long)__double_as_longlong((double)cs + (double)cc)
                                               : (unsigned long long)isum;
    const bool complete = open_at_head && ends_here;
    if (complete) {
      store_run<DT, MM>(o, run, pk, cur);
    } else if (!open_at_head) {
      first = cur; first_key = pk; first_run = run; have_first = true;
    } else {
      last = cur; last_key = pk; last_run = run; have_last = true;
    }
  };
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    if (i >= nv) break;
    const bool h = (heads >> i) & 1u;
    if (h && open) {
      close_piece(true);
      ++run;
    }
    if (!open || h) {
      open = true;
      open_at_head = h;
      pk = k[i];
      cur.cnt = 0;
      cur.mn = ~0ull;
      cur.mx = 0;
      cs = 0; cc = 0; isum = 0;
    }
    cur.cnt += 1;
    if (DT == AGG_F32 || DT == AGG_F64) {
      F t, e;
      two_sum(cs, (F)v[i], t, e);
      cs = t;
      cc += e;
    } else {
      isum += (long long)v[i];
    }
    if (MM) {
      const uint64_t m = sv_img<DT>(v[i]);
      cur.mn = min(cur.mn, (unsigned long long)m);
      cur.mx = max(cur.mx, (unsigned long long)m);
    }
  }
  if (open) close_piece(next_is_head);
  // A piece that neither starts at a head nor ends here is both first and last.
  warp_emit<DT, MM>(o, have_first, first_run, first_key, first);
  warp_emit<DT, MM>(o, have_last, last_run, last_key, last);
}

template <int DT, bool MM>
__global__ void seg_finalize(SegOut o, int64_t d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long c = o.count[i];
    const unsigned long long s = o.sum[i];
    double fs = (DT == AGG_F32 || DT == AGG_F64) ? __longlong_as_double((long long)s) : (double)(long long)s;
    o.avg[i] = fs / (double)c;
    if (MM) {
      const uint64_t mn = ~o.minc[i], mx = o.mx[i];
      double dmn, dmx;
      if (DT == AGG_F32) {
        dmn = (double)f32_of_img((uint32_t)mn);
        dmx = (double)f32_of_img((uint32_t)mx);
        o.minc[i] = (unsigned long long)__double_as_longlong(dmn);
        o.mx[i] = (unsigned long long)__double_as_longlong(dmx);
      } else if (DT == AGG_F64) {
        o.minc[i] = (unsigned long long)__double_as_longlong(f64_of_img(mn));
        o.mx[i] = (unsigned long long)__double_as_longlong(f64_of_img(mx));
      } else {
        o.minc[i] = (unsigned long long)i64_of_img(mn);
        o.mx[i] = (unsigned long long)i64_of_img(mx);
      }
    }
  }
}

template <int DT, bool MM>
static agg_status sort_groupby_t(const uint32_t* keys, const void* vals, int64_t n, uint32_t ops, cudaStream_t s,
                                 agg_groups** gout) {
  using P = typename SV<DT>::P;
  if (n == 0) {
    agg_groups* g = nullptr;
    agg_status st0 = groups_alloc(0, DT, ops, s, &g);
    if (st0 != AGG_OK) return st0;
    g->num_groups = 0;
    g->strategy = AGG_STRAT_SORT;
    *gout = g;
    return AGG_OK;
  }
  const int64_t ntiles = (n + kSegTile - 1) / kSegTile;
  const size_t kb = ((size_t)n * 4 + 255) & ~size_t(255);
  const size_t vb = ((size_t)n * sizeof(P) + 255) & ~size_t(255);
  const size_t rt = (radix_tmp_bytes(n) + 255) & ~size_t(255);
  const size_t tc = ((size_t)(ntiles + 1) * 4 + 255) & ~size_t(255);
  const size_t st_b = (scan_tmp_bytes(ntiles) + 255) & ~size_t(255);
  void* tmp = nullptr;
  AGG_CUDA_TRY(dev_malloc_async(&tmp, 2 * kb + 2 * vb + rt + tc + st_b + 256, s));
  char* c = (char*)tmp;
  uint32_t* kA = (uint32_t*)c; c += kb;
  uint32_t* kB = (uint32_t*)c; c += kb;
  P* vA = (P*)c; c += vb;
  P* vB = (P*)c; c += vb;
  void* rtmp = c; c += rt;
  uint32_t* tile_counts = (uint32_t*)c; c += tc;
  void* stmp = c; c += st_b;
  uint32_t* total = (uint32_t*)c;
  auto release = [&]() { cudaFreeAsync(tmp, s); };
  uint32_t* sk = nullptr;
  P* sv = nullptr;
  agg_status st;
  {
    PhaseTimer pt(AGG_PHASE_SORT, s);
    st = radix_sort_pairs<P>(keys, (const P*)vals, kA, vA, kB, vB, n, nullptr, 32, rtmp, s, &sk, &sv);
  }
  if (st != AGG_OK) { release(); return st; }
  PhaseTimer pt_seg(AGG_PHASE_SEGREDUCE, s);
  seg_heads<<<(unsigned)ntiles, kSegThreads, 0, s>>>(sk, n, tile_counts);
  note_launch();
  st = scan_exclusive_u32(tile_counts, tile_counts, ntiles, total, stmp, s);
  if (st != AGG_OK) { release(); return st; }
  uint32_t* hb = (uint32_t*)stream_pinned(s, 64, &st);
  if (!hb) { release(); return st; }
  cudaMemcpyAsync(hb, total, 4, cudaMemcpyDeviceToHost, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error("sort group-by: %s", cudaGetErrorString(e));
    release();
    return AGG_ERR_CUDA;
  }
  const int64_t d = *hb;
  agg_groups* g = nullptr;
  st = groups_alloc(d, DT, ops, s, &g);
  if (st != AGG_OK) { release(); return st; }
  SegOut o;
  o.keys = g->keys;
  o.count = (unsigned long long*)g->count;
  o.sum = (unsigned long long*)g->sum;
  o.minc = (unsigned long long*)g->min;
  o.mx = (unsigned long long*)g->max;
  o.avg = g->avg;
  // count, sum, min, max are contiguous 256-aligned arrays of d 8-byte words: clear them
  const size_t a8r = ((size_t)(d > 0 ? d : 1) * 8 + 255) & ~size_t(255);
  cudaMemsetAsync(g->count, 0, 4 * a8r, s);
  seg_reduce<DT, MM><<<(unsigned)ntiles, kSegThreads, 0, s>>>(sk, sv, n, tile_counts, o);
  const DeviceInfo& di = device_info();
  int64_t fg = (d + 255) / 256;
  if (fg > (int64_t)di.sm_count * 8) fg = (int64_t)di.sm_count * 8;
  if (fg < 1) fg = 1;
  seg_finalize<DT, MM><<<(unsigned)fg, 256, 0, s>>>(o, d);
  note_launch(2);
  e = cudaGetLastError();
  release();
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    set_error("sort group-by: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    agg_groups_free(g);
    return AGG_ERR_CUDA;
  }
  g->num_groups = d;
  g->strategy = AGG_STRAT_SORT;
  *gout = g;
  return AGG_OK;
}

agg_status sort_groupby(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops, cudaStream_t s,
                        agg_groups** gout) {
  const bool mm = ops_minmax(ops);
#define AGG_S(D) \
  case D: return mm ? sort_groupby_t<D, true>(keys, vals, n, ops, s, gout) : sort_groupby_t<D, false>(keys, vals, n, ops, s, gout);
  switch (vdt) { AGG_S(AGG_I32) AGG_S(AGG_I64) AGG_S(AGG_U32) AGG_S(AGG_F32) AGG_S(AGG_F64) }
#undef AGG_S
  set_error("invalid dtype");
  return AGG_ERR_INVALID;
}

}  // namespace agg
