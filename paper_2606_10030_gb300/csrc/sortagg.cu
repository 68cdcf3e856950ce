// GROUP BY by sorting (the sort-based group-by of Sec. 7).
//
// 1. Stable LSD radix sort of the (key, value) pairs by key.
// 2. seg_count: each warp owns a chunk of 512 consecutive sorted rows and
//    counts its run heads (rows whose key differs from the previous row's);
//    an exclusive scan gives every chunk the index of the first run starting
//    in it, and the total is the number of groups d.
// 3. seg_reduce: each lane folds 16 consecutive rows of its warp's chunk in
//    order (16-byte vector loads); a run begun and ended in the lane is
//    written in its final form. The parts of runs that cross lanes are joined
//    with one segmented scan over the warp, and the run a lane's first head
//    ends is written by that lane. The part of a run that crosses the chunk's
//    start or end is written as a piece (at most two per chunk).
// 4. The pieces of one run are consecutive in chunk order: their targets are
//    cleared, the pieces added with atomics (one set per run per warp), and
//    the targets brought to the raw form of the finished runs.
// 5. seg_finalize converts every group to the output encodings and computes
//    AVG in float64 with converged warps (GB300's float64 pipe is narrow; in
//    the divergent per-run code it was the bottleneck).
// Runs come out in ascending key order by construction.
#include <type_traits>

#include "groupby.cuh"
#include "sort.cuh"

namespace agg {

constexpr int kSegThreads = 256;
constexpr int kSegItems = 16;                // consecutive sorted rows per lane
constexpr int kSegRounds = kSegItems;        // rounds of 32 rows when counting heads
constexpr int kSegChunk = 32 * kSegItems;    // sorted rows per warp
constexpr int kSegChunksPerBlock = kSegThreads / 32;
constexpr uint32_t kNoRun = 0xFFFFFFFFu;

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

constexpr bool is_fp(int dt) { return dt == AGG_F32 || dt == AGG_F64; }

// Partial aggregate of rows of one run: count, sum (compensated pair in the
// input precision for floats, wrapping 64-bit integer otherwise) and the
// order-preserving images of MIN and MAX.
template <int DT>
struct SAcc {
  using F = typename std::conditional<DT == AGG_F32, float, double>::type;
  uint32_t cnt;
  F s, c;
  unsigned long long is;
  unsigned long long mn, mx;
};

template <int DT, bool MM>
__device__ __forceinline__ SAcc<DT> acc_of(bool valid, typename SV<DT>::T v) {
  using F = typename SAcc<DT>::F;
  SAcc<DT> a;
  a.cnt = valid ? 1u : 0u;
  a.s = valid && is_fp(DT) ? (F)v : F(0);
  a.c = F(0);
  a.is = valid && !is_fp(DT) ? (unsigned long long)(int64_t)v : 0ull;
  if (MM) {
    const unsigned long long m = sv_img<DT>(v);
    a.mn = valid ? m : ~0ull;
    a.mx = valid ? m : 0ull;
  }
  return a;
}

// a holds earlier rows of the run than b.
template <int DT, bool MM>
__device__ __forceinline__ SAcc<DT> acc_combine(const SAcc<DT>& a, const SAcc<DT>& b) {
  using F = typename SAcc<DT>::F;
  SAcc<DT> r;
  r.cnt = a.cnt + b.cnt;
  if (DT == AGG_F32) {
    F t, e;
    two_sum(a.s, b.s, t, e);
    r.s = t;
    r.c = a.c + b.c + e;
  } else if (DT == AGG_F64) {  // plain float64 additions: GB300's FP64 pipe is narrow
    r.s = a.s + b.s;
    r.c = F(0);
  } else {
    r.s = F(0);
    r.c = F(0);
  }
  r.is = is_fp(DT) ? 0ull : a.is + b.is;
  if (MM) {
    r.mn = min(a.mn, b.mn);
    r.mx = max(a.mx, b.mx);
  }
  return r;
}

template <int DT, bool MM, bool UP>
__device__ __forceinline__ SAcc<DT> acc_shfl(const SAcc<DT>& a, int arg) {
  SAcc<DT> r;
  r.cnt = UP ? __shfl_up_sync(0xffffffffu, a.cnt, arg) : __shfl_sync(0xffffffffu, a.cnt, arg);
  if (is_fp(DT)) {
    r.s = UP ? __shfl_up_sync(0xffffffffu, a.s, arg) : __shfl_sync(0xffffffffu, a.s, arg);
    r.c = UP ? __shfl_up_sync(0xffffffffu, a.c, arg) : __shfl_sync(0xffffffffu, a.c, arg);
    r.is = 0ull;
  } else {
    r.s = 0;
    r.c = 0;
    r.is = UP ? __shfl_up_sync(0xffffffffu, a.is, arg) : __shfl_sync(0xffffffffu, a.is, arg);
  }
  if (MM) {
    r.mn = UP ? __shfl_up_sync(0xffffffffu, a.mn, arg) : __shfl_sync(0xffffffffu, a.mn, arg);
    r.mx = UP ? __shfl_up_sync(0xffffffffu, a.mx, arg) : __shfl_sync(0xffffffffu, a.mx, arg);
  }
  return r;
}

// Sum of a piece (added with atomics): int64 bits or float64 bits.
template <int DT>
__device__ __forceinline__ unsigned long long sum_bits(const SAcc<DT>& a) {
  if (DT == AGG_F32) return (unsigned long long)__double_as_longlong((double)a.s + (double)a.c);
  if (DT == AGG_F64) return (unsigned long long)__double_as_longlong(a.s);
  return a.is;
}

// Sum as first stored, before seg_finalize: int64 bits, float64 bits, or for
// float32 the compensated pair (s in the low word, c in the high word), so
// that no float64 instruction runs in the divergent per-run code.
template <int DT>
__device__ __forceinline__ unsigned long long raw_sum(const SAcc<DT>& a) {
  if (DT == AGG_F32)
    return ((unsigned long long)__float_as_uint((float)a.c) << 32) | (unsigned long long)__float_as_uint((float)a.s);
  if (DT == AGG_F64) return (unsigned long long)__double_as_longlong((double)a.s);
  return a.is;
}

template <int DT>
__device__ __forceinline__ double fsum_of_raw(unsigned long long r) {
  if (DT == AGG_F32)
    return (double)__uint_as_float((uint32_t)r) + (double)__uint_as_float((uint32_t)(r >> 32));
  if (DT == AGG_F64) return __longlong_as_double((long long)r);
  return (double)(long long)r;
}

struct SegOut {
  uint32_t* keys;
  unsigned long long* count;
  unsigned long long* sum;
  unsigned long long* min;
  unsigned long long* max;
  double* avg;
};

// Part of a run cut by a chunk boundary.
struct SegPiece {
  uint32_t run, key;
  uint32_t cnt, pad;
  unsigned long long sum;  // int64 bits or float64 bits
  unsigned long long mn, mx;
};

// MIN/MAX image -> the output encoding (float64 bits for floats, int64 otherwise).
template <int DT>
__device__ __forceinline__ unsigned long long out_of_img(unsigned long long m) {
  if (DT == AGG_F32) return (unsigned long long)__double_as_longlong((double)f32_of_img((uint32_t)m));
  if (DT == AGG_F64) return (unsigned long long)__double_as_longlong(f64_of_img(m));
  return (unsigned long long)i64_of_img(m);
}

// A finished run in raw form (count, raw sum, MIN/MAX images); seg_finalize
// converts every group afterwards with converged warps.
template <int DT, bool MM>
__device__ __forceinline__ void store_final(const SegOut& o, uint32_t run, uint32_t key, const SAcc<DT>& a) {
  o.keys[run] = key;
  o.count[run] = a.cnt;
  o.sum[run] = raw_sum<DT>(a);
  if (MM) {
    o.min[run] = a.mn;
    o.max[run] = a.mx;
  }
}

template <int DT, bool MM>
__device__ __forceinline__ void store_piece(SegPiece* p, uint32_t run, uint32_t key, const SAcc<DT>& a) {
  SegPiece q;
  q.run = run;
  q.key = key;
  q.cnt = a.cnt;
  q.pad = 0;
  q.sum = sum_bits<DT>(a);
  q.mn = MM ? a.mn : 0ull;
  q.mx = MM ? a.mx : 0ull;
  *p = q;
}

// Run heads per chunk of kSegChunk sorted rows (one warp per chunk).
__global__ void __launch_bounds__(kSegThreads) seg_count(const uint32_t* __restrict__ sk, int64_t n,
                                                         uint32_t* __restrict__ chunk_heads) {
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * kSegChunksPerBlock + (threadIdx.x >> 5);
  const int64_t r0 = chunk * kSegChunk;
  if (r0 >= n) return;
  uint32_t k[kSegRounds];
#pragma unroll
  for (int r = 0; r < kSegRounds; ++r) {
    const int64_t row = r0 + r * 32 + lane;
    k[r] = row < n ? sk[row] : 0u;
  }
  uint32_t prev = r0 > 0 ? sk[r0 - 1] : 0u;
  uint32_t heads = 0;
#pragma unroll
  for (int r = 0; r < kSegRounds; ++r) {
    const int64_t row = r0 + r * 32 + lane;
    uint32_t pk = __shfl_up_sync(0xffffffffu, k[r], 1);
    if (lane == 0) pk = prev;
    prev = __shfl_sync(0xffffffffu, k[r], 31);
    heads += __popc(__ballot_sync(0xffffffffu, row < n && (row == 0 || k[r] != pk)));
  }
  if (lane == 0) chunk_heads[chunk] = heads;
}

template <int DT, bool MM>
__global__ void __launch_bounds__(kSegThreads) seg_reduce(const uint32_t* __restrict__ sk,
                                                          const typename SV<DT>::P* __restrict__ sv, int64_t n,
                                                          const uint32_t* __restrict__ chunk_first, SegOut o,
                                                          SegPiece* __restrict__ pieces) {
  using P = typename SV<DT>::P;
  const int lane = threadIdx.x & 31;
  const int64_t chunk = (int64_t)blockIdx.x * kSegChunksPerBlock + (threadIdx.x >> 5);
  const int64_t r0 = chunk * kSegChunk;
  if (r0 >= n) return;
  // this lane's kSegItems consecutive rows, loaded with 16-byte vectors when whole
  const int64_t l0 = r0 + (int64_t)lane * kSegItems;
  const int nv = l0 >= n ? 0 : (int)(n - l0 < kSegItems ? n - l0 : kSegItems);
  uint32_t k[kSegItems];
  P v[kSegItems];
  if (nv == kSegItems) {
    const uint4* kq = (const uint4*)(sk + l0);
    const uint4* vq = (const uint4*)(sv + l0);
#pragma unroll
    for (int q = 0; q < kSegItems / 4; ++q) {
      const uint4 a = kq[q];
      k[4 * q] = a.x;
      k[4 * q + 1] = a.y;
      k[4 * q + 2] = a.z;
      k[4 * q + 3] = a.w;
    }
    constexpr int VQ = kSegItems * (int)sizeof(P) / 16;
#pragma unroll
    for (int q = 0; q < VQ; ++q) {
      const uint4 a = vq[q];
      const uint32_t w[4] = {a.x, a.y, a.z, a.w};
      memcpy((char*)v + 16 * q, w, 16);
    }
  } else {
#pragma unroll
    for (int i = 0; i < kSegItems; ++i) {
      k[i] = i < nv ? sk[l0 + i] : 0u;
      v[i] = i < nv ? sv[l0 + i] : P(0);
    }
  }
  uint32_t before = __shfl_up_sync(0xffffffffu, k[kSegItems - 1], 1);  // key of the row before this lane's first
  if (lane == 0) before = r0 > 0 ? sk[r0 - 1] : 0u;
  uint32_t hb = 0;  // run heads among this lane's rows
#pragma unroll
  for (int i = 0; i < kSegItems; ++i)
    if (i < nv && (l0 + i == 0 || k[i] != (i ? k[i - 1] : before))) hb |= 1u << i;
  const uint32_t nh = (uint32_t)__popc(hb);
  uint32_t hin = nh;  // inclusive scan of head counts over the warp's lanes
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, hin, d);
    if (lane >= d) hin += y;
  }
  const uint32_t hx = hin - nh;  // heads in earlier lanes of the chunk
  const uint32_t heads_in_chunk = __shfl_sync(0xffffffffu, hin, 31);
  const uint32_t cf = chunk_first[chunk];
  // Fold the lane's rows: rows before its first head form the prefix (the end
  // of a run begun earlier); a run begun and ended in the lane is final here;
  // the run begun at its last head stays open.
  SAcc<DT> pre = acc_of<DT, MM>(false, sv_val<DT>(P(0)));
  SAcc<DT> cur = pre;
  bool open = false;
  uint32_t next_run = cf + hx, cur_run = 0, cur_key = 0;
#pragma unroll
  for (int i = 0; i < kSegItems; ++i) {
    if (i < nv) {
      const SAcc<DT> a = acc_of<DT, MM>(true, sv_val<DT>(v[i]));
      if ((hb >> i) & 1u) {
        if (open) store_final<DT, MM>(o, cur_run, cur_key, cur);
        open = true;
        cur = a;
        cur_run = next_run++;
        cur_key = k[i];
      } else if (open) {
        cur = acc_combine<DT, MM>(cur, a);
      } else {
        pre = acc_combine<DT, MM>(pre, a);
      }
    }
  }
  // Segmented inclusive scan over the lanes of the open parts: a lane with a
  // head starts a new run; a lane without one extends the run open before it.
  SAcc<DT> x = open ? cur : pre;
  const uint32_t fm = __ballot_sync(0xffffffffu, open);
  const uint32_t le = lane == 31 ? 0xffffffffu : ((2u << lane) - 1u);
  const uint32_t fle = fm & le;
  const int seg0 = fle ? 31 - __clz(fle) : 0;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const SAcc<DT> b = acc_shfl<DT, MM, true>(x, d);
    if (lane - d >= seg0) x = acc_combine<DT, MM>(b, x);
  }
  SAcc<DT> left = acc_shfl<DT, MM, true>(x, 1);  // the run open at the end of the previous lane
  if (lane == 0) left = acc_of<DT, MM>(false, sv_val<DT>(P(0)));
  // A lane with a head ends, with its prefix, the run open before it.
  bool wrote_first = false;
  if (open) {
    const SAcc<DT> tot = acc_combine<DT, MM>(left, pre);
    if (tot.cnt > 0) {
      if (hx == 0) {  // begun before the chunk: a piece
        store_piece<DT, MM>(&pieces[2 * chunk], cf - 1, before, tot);
        wrote_first = true;
      } else {
        store_final<DT, MM>(o, cf + hx - 1, before, tot);
      }
    }
  }
  wrote_first = __any_sync(0xffffffffu, wrote_first);
  // The run open at the end of the chunk.
  const SAcc<DT> xl = acc_shfl<DT, MM, false>(x, 31);
  if (lane == 0) {
    const int64_t last = (r0 + kSegChunk < n ? r0 + kSegChunk : n) - 1;
    const uint32_t last_key = sk[last];
    const bool ends = last + 1 >= n || sk[last + 1] != last_key;
    const uint32_t run = cf + heads_in_chunk - 1;
    if (ends && heads_in_chunk > 0) {
      store_final<DT, MM>(o, run, last_key, xl);
      pieces[2 * chunk + 1].run = kNoRun;
    } else {
      store_piece<DT, MM>(&pieces[2 * chunk + 1], run, last_key, xl);
    }
    if (!wrote_first) pieces[2 * chunk].run = kNoRun;
  }
}

// Targets of pieces: clear count and sum, set MIN/MAX accumulators (the
// complement of the MIN image and the MAX image, both combined with atomicMax).
template <bool MM>
__global__ void seg_piece_clear(const SegPiece* __restrict__ pieces, int64_t np, SegOut o) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t run = pieces[p].run;
    if (run == kNoRun) continue;
    o.count[run] = 0;
    o.sum[run] = 0;
    if (MM) {
      o.min[run] = 0;
      o.max[run] = 0;
    }
  }
}

// Add the pieces; pieces of one run in a warp are combined first.
template <int DT, bool MM>
__global__ void seg_piece_add(const SegPiece* __restrict__ pieces, int64_t np, SegOut o) {
  const int lane = threadIdx.x & 31;
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x; b < np; b += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = b + threadIdx.x;
    SegPiece q;
    q.run = kNoRun;
    if (p < np) q = pieces[p];
    const bool has = q.run != kNoRun;
    const uint32_t vm = __ballot_sync(0xffffffffu, has);
    if (has) {
    const uint32_t peers = __match_any_sync(vm, q.run);
    const bool leader = (peers & ((1u << lane) - 1u)) == 0;
    unsigned long long cnt = q.cnt, sum = q.sum, mn = q.mn, mx = q.mx;
    // gather the peers' parts into the leader (peers form one set per run)
    for (int src = 0; src < 32; ++src) {
      if (!((vm >> src) & 1u)) continue;
      const unsigned long long c2 = __shfl_sync(vm, cnt, src);
      const unsigned long long s2 = __shfl_sync(vm, sum, src);
      const unsigned long long n2 = MM ? __shfl_sync(vm, mn, src) : 0ull;
      const unsigned long long x2 = MM ? __shfl_sync(vm, mx, src) : 0ull;
      if (leader && src != lane && ((peers >> src) & 1u)) {
        cnt += c2;
        if (is_fp(DT))
          sum = (unsigned long long)__double_as_longlong(__longlong_as_double((long long)sum) +
                                                         __longlong_as_double((long long)s2));
        else
          sum += s2;
        if (MM) {
          mn = min(mn, n2);
          mx = max(mx, x2);
        }
      }
    }
    if (leader) {
      o.keys[q.run] = q.key;
      atomicAdd(&o.count[q.run], cnt);
      if (is_fp(DT)) atomicAdd((double*)&o.sum[q.run], __longlong_as_double((long long)sum));
      else atomicAdd(&o.sum[q.run], sum);
      if (MM) {
        atomicMax(&o.min[q.run], ~mn);
        atomicMax(&o.max[q.run], mx);
      }
    }
    }
  }
}

// Bring each piece target to the raw form of store_final, once per run: from
// the first piece slot of its run (the previous valid slot, one or two back,
// holds another run or none).
template <int DT, bool MM>
__global__ void seg_piece_finish(const SegPiece* __restrict__ pieces, int64_t np, SegOut o) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t run = pieces[p].run;
    if (run == kNoRun) continue;
    uint32_t prev = kNoRun;
    if (p >= 1) prev = pieces[p - 1].run;
    if (prev == kNoRun && p >= 2) prev = pieces[p - 2].run;
    if (prev == run) continue;
    if (DT == AGG_F32) {  // float64 total -> (s, c) float pair
      const double d = __longlong_as_double((long long)o.sum[run]);
      const float hi = (float)d;
      const float lo = (float)(d - (double)hi);
      o.sum[run] = ((unsigned long long)__float_as_uint(lo) << 32) | (unsigned long long)__float_as_uint(hi);
    }
    if (MM) o.min[run] = ~o.min[run];
  }
}

// Every group: the output encodings and AVG = SUM / COUNT in float64.
template <int DT, bool MM>
__global__ void seg_finalize(SegOut o, int64_t d) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long c = o.count[i];
    const double fs = fsum_of_raw<DT>(o.sum[i]);
    if (DT == AGG_F32) o.sum[i] = (unsigned long long)__double_as_longlong(fs);
    o.avg[i] = fs / (double)c;
    if (MM) {
      o.min[i] = out_of_img<DT>(o.min[i]);
      o.max[i] = out_of_img<DT>(o.max[i]);
    }
  }
}

// Exact key range for the sort: grid-stride min and max, one atomic pair per
// warp into mm[0] (min) and mm[1] (max).
__global__ void __launch_bounds__(256) key_range(const uint32_t* __restrict__ k, int64_t n, uint32_t* mm) {
  uint32_t lo = 0xFFFFFFFFu, hi = 0u;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i + 3 * stride < n; i += 4 * stride) {  // four loads in flight per thread
    const uint32_t a = k[i], b = k[i + stride], c = k[i + 2 * stride], d = k[i + 3 * stride];
    lo = min(min(lo, a), min(b, min(c, d)));
    hi = max(max(hi, a), max(b, max(c, d)));
  }
  for (; i < n; i += stride) {
    lo = min(lo, k[i]);
    hi = max(hi, k[i]);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(&mm[0], lo);
    atomicMax(&mm[1], hi);
  }
}

// Columns of at least this many rows sort only the bits their key range needs
// (one pass fewer per 8 bits; the range costs one read of the keys and a sync).
constexpr int64_t kRangeRows = int64_t(1) << 16;

template <int DT, bool MM>
static agg_status sort_groupby_t(const uint32_t* keys, const void* vals, int64_t n, uint32_t ops, cudaStream_t s,
                                 agg_groups** gout, const float* feat) {
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
  const int64_t nchunks = (n + kSegChunk - 1) / kSegChunk;
  const int64_t nblocks = (nchunks + kSegChunksPerBlock - 1) / kSegChunksPerBlock;
  const int64_t np = 2 * nchunks;
  const size_t kb = ((size_t)n * 4 + 255) & ~size_t(255);
  const size_t vb = ((size_t)n * sizeof(P) + 255) & ~size_t(255);
  const size_t rt = (radix_tmp_bytes(n) + 255) & ~size_t(255);
  const size_t tc = ((size_t)(nchunks + 1) * 4 + 255) & ~size_t(255);
  const size_t st_b = (scan_tmp_bytes(nchunks) + 255) & ~size_t(255);
  const size_t pb = ((size_t)np * sizeof(SegPiece) + 255) & ~size_t(255);
  void* tmp = nullptr;
  AGG_CUDA_TRY(dev_malloc_async(&tmp, 2 * kb + 2 * vb + rt + tc + st_b + pb + 256, s));
  char* c = (char*)tmp;
  uint32_t* kA = (uint32_t*)c; c += kb;
  uint32_t* kB = (uint32_t*)c; c += kb;
  P* vA = (P*)c; c += vb;
  P* vB = (P*)c; c += vb;
  void* rtmp = c; c += rt;
  uint32_t* chunk_first = (uint32_t*)c; c += tc;
  void* stmp = c; c += st_b;
  SegPiece* pieces = (SegPiece*)c; c += pb;
  uint32_t* total = (uint32_t*)c;
  auto release = [&]() { cudaFreeAsync(tmp, s); };
  uint32_t* sk = nullptr;
  P* sv = nullptr;
  agg_status st;
  {
    PhaseTimer pt(AGG_PHASE_SORT, s);
    int bits = 32;
    uint32_t kbase = 0;
    // a sampled key range already wider than 2^24 needs all four passes
    const bool wide = feat != nullptr && feat[F_LOG2_RANGE] > 24.5f;
    if (n >= kRangeRows && !wide) {  // digits of key - min cover max - min: the passes that range needs
      uint32_t* mm = total + 2;
      cudaMemsetAsync(mm, 0xFF, 4, s);
      cudaMemsetAsync(mm + 1, 0, 4, s);
      const DeviceInfo& di = device_info();
      key_range<<<(unsigned)(di.sm_count * 8), 256, 0, s>>>(keys, n, mm);
      note_launch();
      uint32_t* hr = (uint32_t*)stream_pinned(s, 64, &st);
      if (!hr) { release(); return st; }
      cudaMemcpyAsync(hr, mm, 8, cudaMemcpyDeviceToHost, s);
      const cudaError_t er = cudaStreamSynchronize(s);
      if (er != cudaSuccess) {
        set_error("sort group-by: %s", cudaGetErrorString(er));
        release();
        return AGG_ERR_CUDA;
      }
      kbase = hr[0];
      const uint32_t span = hr[1] - hr[0];
      const int need = span ? 32 - __builtin_clz(span) : 1;  // bits of the largest key - kbase
      bits = ((need + 7) / 8) * 8;  // at least one pass, so the result lands in aligned scratch
    }
    st = radix_sort_pairs<P>(keys, (const P*)vals, kA, vA, kB, vB, n, nullptr, bits, rtmp, s, &sk, &sv, kbase);
  }
  if (st != AGG_OK) { release(); return st; }
  PhaseTimer pt_seg(AGG_PHASE_SEGREDUCE, s);
  seg_count<<<(unsigned)nblocks, kSegThreads, 0, s>>>(sk, n, chunk_first);
  note_launch();
  st = scan_exclusive_u32(chunk_first, chunk_first, nchunks, total, stmp, s);
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
  o.min = (unsigned long long*)g->min;
  o.max = (unsigned long long*)g->max;
  o.avg = g->avg;
  seg_reduce<DT, MM><<<(unsigned)nblocks, kSegThreads, 0, s>>>(sk, sv, n, chunk_first, o, pieces);
  const DeviceInfo& di = device_info();
  int64_t pg = (np + 255) / 256;
  if (pg > (int64_t)di.sm_count * 8) pg = (int64_t)di.sm_count * 8;
  if (pg < 1) pg = 1;
  seg_piece_clear<MM><<<(unsigned)pg, 256, 0, s>>>(pieces, np, o);
  seg_piece_add<DT, MM><<<(unsigned)pg, 256, 0, s>>>(pieces, np, o);
  seg_piece_finish<DT, MM><<<(unsigned)pg, 256, 0, s>>>(pieces, np, o);
  int64_t fg = (d + 255) / 256;
  if (fg > (int64_t)di.sm_count * 8) fg = (int64_t)di.sm_count * 8;
  if (fg < 1) fg = 1;
  seg_finalize<DT, MM><<<(unsigned)fg, 256, 0, s>>>(o, d);
  note_launch(5);
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
                        agg_groups** gout, const float* feat) {
  const bool mm = ops_minmax(ops);
#define AGG_S(D) \
  case D:        \
    return mm ? sort_groupby_t<D, true>(keys, vals, n, ops, s, gout, feat) : sort_groupby_t<D, false>(keys, vals, n, ops, s, gout, feat);
  switch (vdt) { AGG_S(AGG_I32) AGG_S(AGG_I64) AGG_S(AGG_U32) AGG_S(AGG_F32) AGG_S(AGG_F64) }
#undef AGG_S
  set_error("invalid dtype");
  return AGG_ERR_INVALID;
}

}  // namespace agg
