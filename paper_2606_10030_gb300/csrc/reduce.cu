// Ungrouped aggregation: the column scan, per-thread fold, block tree and grid merge.
//
// One fused kernel in the spirit of the paper's specialised GPU design
// (Sec. 3.2, "GPU Optimizations"): the grid is a multiple of the SM count,
// each thread walks the column with a grid-stride loop of coalesced 128-bit
// read-only loads (several in flight per thread), folds the items into
// register accumulators, the block reduces them with warp shuffles and shared
// memory, and the block partials are merged once for the whole grid. The
// paper merges with a cooperative-groups grid synchronisation; here the last
// block to finish (a fence plus an atomic ticket) does the merge, so no block
// ever waits on another and no cooperative launch is needed.
//
// Accumulators per thread:
//   integers  int64 sum (wraps mod 2^64), min and max in the value type;
//   float32   TwoSum-compensated float32 pair (s, c), order-preserving
//             uint32 images for min/max;
//   float64   a 128-bit fixed-point integer at the scale of the largest
//             exponent seen (integer operations only: GB300 issues few
//             float64 operations), uint64 images for min/max.
// Block partials carry the sum as a float64 pair (hi, lo); the final merge is
// a float64 double-double sum in a fixed order, so the result is
// deterministic for a given grid.
//
// Error bound of a float SUM. Every partial also carries eb, a bound on
// |hi + lo - (exact sum of its rows)|, built from the roundings that can
// occur: per thread, those of the compensation word of a float32 pair (each
// at most 2^-24 of the word's new value, tracked as the word's largest
// magnitude) or the truncations of the float64 fixed-point sum (less than one
// unit each, at most two per row); per merge, the two float64 roundings of
// the low words. The result's err_bound adds the final rounding of hi + lo
// and the oracle's own rounding of the exact sum, so that
// |sum_f - (exact sum rounded to float64)| <= err_bound.
#include <cfloat>
#include <climits>
#include <cmath>
#include <map>
#include <mutex>

#include "common.cuh"

namespace agg {

struct Partial {  // one block's partial aggregate
  int64_t si;     // integer sum
  double hi, lo;  // float sum, unevaluated hi + lo
  uint64_t mn, mx;  // order-preserving images of min / max
  double eb;      // bound on |hi + lo - exact sum of the rows| (float columns)
};

template <int DT> struct Traits;
template <> struct Traits<AGG_I32> { using T = int32_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_I64> { using T = int64_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_U32> { using T = uint32_t; static constexpr bool FP = false; };
template <> struct Traits<AGG_F32> { using T = float; static constexpr bool FP = true; };
template <> struct Traits<AGG_F64> { using T = double; static constexpr bool FP = true; };

// ---------------------------------------------------------------------------
// Per-thread accumulators. fold() is the aggregate() of Fig. 4.
// ---------------------------------------------------------------------------
template <int DT, bool SUM, bool MM, bool FP = Traits<DT>::FP>
struct Acc;

template <int DT, bool SUM, bool MM>
struct Acc<DT, SUM, MM, false> {
  using T = typename Traits<DT>::T;
  int64_t s;
  T mn, mx;
  __device__ void init() {
    s = 0;
    if (DT == AGG_I32) { mn = (T)INT_MAX; mx = (T)INT_MIN; }
    if (DT == AGG_U32) { mn = (T)UINT_MAX; mx = (T)0; }
    if (DT == AGG_I64) { mn = (T)LLONG_MAX; mx = (T)LLONG_MIN; }
  }
  __device__ __forceinline__ void fold(T v) {
    if (SUM) s += (int64_t)v;
    if (MM) { mn = min(mn, v); mx = max(mx, v); }
  }
  __device__ __forceinline__ void fold_vec(const uint4& r) {
    if (sizeof(T) == 4) {
      fold((T)r.x); fold((T)r.y); fold((T)r.z); fold((T)r.w);
    } else {
      fold((T)(((uint64_t)r.y << 32) | r.x));
      fold((T)(((uint64_t)r.w << 32) | r.z));
    }
  }
  __device__ void to_partial(Partial& p, uint32_t) const {
    p.si = s;
    p.hi = 0.0;
    p.lo = 0.0;
    p.mn = img_i64((int64_t)mn);
    p.mx = img_i64((int64_t)mx);
    p.eb = 0.0;
  }
};

template <class F> struct FpImg;
template <> struct FpImg<float> {
  using U = uint32_t;
  __device__ static U img(float x) { return img_f32(x); }
  __device__ static uint64_t widen(U m) {  // f32 image -> image of the same value as f64
    if (m == 0xFFFFFFFFu) return ~0ull;    // identity of min
    if (m == 0u) return 0ull;              // identity of max
    return img_f64((double)f32_of_img(m));
  }
};
template <> struct FpImg<double> {
  using U = uint64_t;
  __device__ static U img(double x) { return img_f64(x); }
  __device__ static uint64_t widen(U m) { return m; }
};

// float64 SUM on the integer pipes: a 128-bit two's-complement fixed-point
// number (hi:lo) scaled to the largest exponent field E seen so far, worth
// (hi:lo) x 2^(E - 1075 - kFixGuard). A row with significand m (53 bits,
// implicit bit included) and exponent field e >= 1 is worth m x 2^(e - 1075),
// i.e. m shifted left by kFixGuard - (E - e) units. Rows more than kFixGuard
// binades below E keep their bits above the unit (each loses less than
// 2^(E - 1075 - kFixGuard)); a row with a larger exponent shifts the sum right
// (again less than a unit lost). Sums of up to 2^27 rows per thread cannot
// overflow (|m x 2^kFixGuard| < 2^100). Infinities and NaNs are added in
// float64 on the side, so that a column holding one sums to a non-finite
// value (which one is unspecified, as for the other float paths).
// GB300 issues few float64 operations per clock (a TwoSum per row held the
// float64 scan to 0.6 TB/s); this takes only integer operations per row.
constexpr int kFixGuard = 47;

struct Fix128 {
  uint64_t lo, hi;
  int E;
  double special;
  __device__ void init() {
    lo = 0;
    hi = 0;
    E = 0;
    special = 0.0;
  }
  __device__ __forceinline__ void rescale(int e) {  // e > E
    const int k = e - E;
    if (k >= 127) {
      lo = (int64_t)hi < 0 ? ~0ull : 0ull;
      hi = lo;
    } else if (k >= 64) {
      lo = (uint64_t)((int64_t)hi >> (k - 64));
      hi = (uint64_t)((int64_t)hi >> 63);
    } else {
      lo = (lo >> k) | (hi << (64 - k));
      hi = (uint64_t)((int64_t)hi >> k);
    }
    E = e;
  }
  __device__ __forceinline__ void add(uint64_t u) {
    const int ef = (int)(u >> 52) & 0x7FF;
    if (ef == 0x7FF) {  // infinity or NaN
      special += __longlong_as_double((long long)u);
      return;
    }
    const int e = ef > 0 ? ef : 1;  // subnormals: exponent 1, no implicit bit
    const uint64_t m = (u & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(ef > 0) << 52);
    if (e > E) rescale(e);
    const int d = E - e;
    uint64_t vlo, vhi;
    if (d <= kFixGuard) {
      const int sh = kFixGuard - d;  // 0 .. kFixGuard
      vlo = m << sh;
      vhi = sh > 0 ? m >> (64 - sh) : 0ull;
    } else {
      const int r = d - kFixGuard;
      vlo = r < 64 ? m >> r : 0ull;
      vhi = 0ull;
    }
    if ((int64_t)u < 0) {  // two's-complement negation of vhi:vlo
      vlo = ~vlo + 1ull;
      vhi = ~vhi + (vlo == 0ull ? 1ull : 0ull);
    }
    lo += vlo;
    hi += vhi + (lo < vlo ? 1ull : 0ull);
  }
  // The sum as an unevaluated float64 pair (rel. error about 2^-106 before
  // scaling): the 128-bit integer in three chunks that float64 holds exactly,
  // added with TwoSum, then scaled by 2^(E - 1075 - kFixGuard).
  __device__ void to_pair(double& h, double& l) const {
    const uint64_t m43 = (1ull << 43) - 1ull;
    const double q0 = (double)(lo & m43);
    const double q1 = (double)(((lo >> 43) | (hi << 21)) & m43);
    const double q2 = (double)((int64_t)hi >> 22);
    double s1, e1, s2, e2;
    two_sum(ldexp(q2, 86), ldexp(q1, 43), s1, e1);
    two_sum(s1, q0, s2, e2);
    double t, f;
    two_sum(s2, e1 + e2, t, f);
    const int sc = E - 1075 - kFixGuard;
    h = ldexp(t, sc) + special;
    l = special == 0.0 ? ldexp(f, sc) : 0.0;
  }
  // Bound on |h + l - exact sum| after `rows` adds: each add loses less than
  // one unit 2^(E - 1075 - kFixGuard) (a row far below E), each rescale less
  // than one unit of the new scale; to_pair rounds e1 + e2 (under 2^-104 of
  // the sum) and may round h and l into the subnormal range.
  __device__ double error_bound(uint32_t rows, double h, double l) const {
    if (special != 0.0) return __longlong_as_double(0x7ff0000000000000ll);
    if (E == 0) return 0.0;
    return ldexp(2.0 * (double)rows, E - 1075 - kFixGuard) + (fabs(h) + fabs(l)) * 0x1p-100 + 0x1p-1072;
  }
};

template <int DT, bool SUM, bool MM>
struct Acc<DT, SUM, MM, true> {
  using T = typename Traits<DT>::T;
  using U = typename FpImg<T>::U;
  static constexpr bool F64 = sizeof(T) == 8;
  T s, c;       // float32: TwoSum-compensated pair
  T cmax;       // float32: largest |c| so far (bounds the roundings of c)
  Fix128 fx;    // float64
  U mn, mx;
  __device__ void init() {
    s = 0; c = 0; cmax = 0;
    if (F64) fx.init();
    mn = (U)~(U)0; mx = 0;
  }
  __device__ __forceinline__ void fold(T v) {
    if (SUM) {
      if (F64) {
        fx.add((uint64_t)__double_as_longlong((double)v));
      } else {
        T t, e;
        two_sum(s, v, t, e);
        s = t;
        c += e;
        cmax = fmaxf(cmax, fabsf(c));
      }
    }
    if (MM) {
      U m = FpImg<T>::img(v);
      mn = min(mn, m);
      mx = max(mx, m);
    }
  }
  __device__ __forceinline__ void fold_vec(const uint4& r) {
    if (sizeof(T) == 4) {
      fold(__uint_as_float(r.x)); fold(__uint_as_float(r.y));
      fold(__uint_as_float(r.z)); fold(__uint_as_float(r.w));
    } else {
      fold(__longlong_as_double((long long)(((uint64_t)r.y << 32) | r.x)));
      fold(__longlong_as_double((long long)(((uint64_t)r.w << 32) | r.z)));
    }
  }
  // rows: the number of values this thread folded.
  __device__ void to_partial(Partial& p, uint32_t rows) const {
    p.si = 0;
    p.eb = 0.0;
    if (F64 && SUM) {
      fx.to_pair(p.hi, p.lo);
      p.eb = fx.error_bound(rows, p.hi, p.lo);
    } else {
      p.hi = (double)s;
      p.lo = (double)c;
      // TwoSum leaves s + c short only by the roundings of c: each at most
      // 2^-24 of |c| after the add (2^-150 when c is subnormal)
      if (SUM && !F64) {
        p.eb = (isfinite(p.hi) && isfinite(p.lo))
                   ? (double)rows * ((double)cmax * (0x1p-24 * (1.0 + 0x1p-23)) + 0x1p-150)
                   : __longlong_as_double(0x7ff0000000000000ll);
      }
    }
    p.mn = FpImg<T>::widen(mn);
    p.mx = FpImg<T>::widen(mx);
  }
};

// ---------------------------------------------------------------------------
// Warp / block reduction of Partial values (fixed shuffle tree).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void combine(Partial& a, const Partial& b) {
  a.si += b.si;
  double s, e;
  two_sum(a.hi, b.hi, s, e);
  a.hi = s;
  const double r1 = e + b.lo;  // rounded: at most 2^-53 |r1| (+ 2^-1075)
  a.lo += r1;                  // rounded: at most 2^-53 |a.lo| (+ 2^-1075)
  a.eb = a.eb + b.eb + (fabs(r1) + fabs(a.lo)) * 0x1p-53 + 0x1p-1074;
  a.mn = min(a.mn, b.mn);
  a.mx = max(a.mx, b.mx);
}

__device__ __forceinline__ Partial shfl_xor(const Partial& p, int m) {
  Partial q;
  q.si = __shfl_xor_sync(0xffffffffu, p.si, m);
  q.hi = __shfl_xor_sync(0xffffffffu, p.hi, m);
  q.lo = __shfl_xor_sync(0xffffffffu, p.lo, m);
  q.mn = __shfl_xor_sync(0xffffffffu, p.mn, m);
  q.mx = __shfl_xor_sync(0xffffffffu, p.mx, m);
  q.eb = __shfl_xor_sync(0xffffffffu, p.eb, m);
  return q;
}

// Block-wide reduction; the result is valid in thread 0.
template <int BLOCK>
__device__ Partial block_reduce(Partial p) {
  __shared__ Partial sm[BLOCK / 32];
#pragma unroll
  for (int m = 16; m >= 1; m >>= 1) combine(p, shfl_xor(p, m));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sm[w] = p;
  __syncthreads();
  if (w == 0) {
    if (l < BLOCK / 32) p = sm[l];
    else p = Partial{0, 0.0, 0.0, ~0ull, 0ull, 0.0};
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) combine(p, shfl_xor(p, m));
  }
  return p;
}

// Merge np partials (written by other blocks or launches) into *out.
// Called by one whole block; thread 0 writes.
template <int DT, int BLOCK>
__device__ void merge_partials(const Partial* parts, int np, agg_scalar* out, uint32_t ops,
                               int64_t count) {
  Partial acc{0, 0.0, 0.0, ~0ull, 0ull, 0.0};
  for (int i = threadIdx.x; i < np; i += BLOCK) {
    Partial q;
    q.si = __ldcg(&parts[i].si);
    q.hi = __ldcg(&parts[i].hi);
    q.lo = __ldcg(&parts[i].lo);
    q.mn = __ldcg(&parts[i].mn);
    q.mx = __ldcg(&parts[i].mx);
    q.eb = __ldcg(&parts[i].eb);
    combine(acc, q);
  }
  __syncthreads();
  acc = block_reduce<BLOCK>(acc);
  if (threadIdx.x != 0) return;
  agg_scalar r;
  r.count = count;
  r.dtype = DT;
  r.ops = ops;
  r.err_bound = 0.0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  if (Traits<DT>::FP) {
    double s = acc.hi + acc.lo;
    r.sum_i = 0;
    r.sum_f = s;
    // the partials' bound, plus the rounding of hi + lo and the oracle's own
    // rounding of the exact sum (each at most 2^-53 of the value), plus a
    // margin for the roundings of the bound's own sums
    if (ops & (AGG_SUM | AGG_AVG)) {
      r.err_bound = (acc.eb + fabs(s) * 0x1p-52 + 0x1p-1073) * (1.0 + 0x1p-40);
      // a column holding an infinity or a NaN has no finite bound
      if (!isfinite(s) || !isfinite(r.err_bound)) r.err_bound = __longlong_as_double(0x7ff0000000000000ll);
    }
    r.avg = count ? s / (double)count : nan;
    r.min_f = count ? f64_of_img(acc.mn) : __longlong_as_double(0x7ff0000000000000ll);
    r.max_f = count ? f64_of_img(acc.mx) : __longlong_as_double((long long)0xfff0000000000000ull);
    r.min_i = 0;
    r.max_i = 0;
  } else {
    r.sum_i = acc.si;
    r.sum_f = (double)acc.si;
    r.avg = count ? (double)acc.si / (double)count : nan;
    r.min_i = count ? i64_of_img(acc.mn) : LLONG_MAX;
    r.max_i = count ? i64_of_img(acc.mx) : LLONG_MIN;
    r.min_f = 0.0;
    r.max_f = 0.0;
  }
  *out = r;
}

constexpr int kBlock = 256;
constexpr int kUnroll = 4;

// The scan. Rows [0, head) and the ragged tail are folded with scalar loads by
// the first threads of the grid; the 16-byte-aligned body with vector loads.
template <int DT, bool SUM, bool MM>
__global__ void __launch_bounds__(kBlock) reduce_scan(const typename Traits<DT>::T* __restrict__ col,
                                                      int64_t n, int64_t head, Partial* __restrict__ parts,
                                                      int part_base, unsigned* ticket, agg_scalar* out,
                                                      uint32_t ops, int64_t count_total, int finalize) {
  using T = typename Traits<DT>::T;
  constexpr int EPV = 16 / sizeof(T);
  Acc<DT, SUM, MM> a;
  a.init();
  uint32_t rows = 0;  // values this thread folds
  if (SUM || MM) {
    const int64_t nv = (n - head) / EPV;
    const int64_t tail0 = head + nv * EPV;
    const int64_t g = (int64_t)blockIdx.x * kBlock + threadIdx.x;
    if (g < head) { a.fold(col[g]); ++rows; }
    if (g < n - tail0) { a.fold(col[tail0 + g]); ++rows; }
    const uint4* v = reinterpret_cast<const uint4*>(col + head);
    const int64_t stride = (int64_t)gridDim.x * kBlock * kUnroll;
    for (int64_t base = (int64_t)blockIdx.x * kBlock * kUnroll + threadIdx.x; base < nv; base += stride) {
      uint4 r[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t i = base + (int64_t)u * kBlock;
        r[u] = i < nv ? ld_stream_v4(v + i) : make_uint4(0, 0, 0, 0);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        if (base + (int64_t)u * kBlock < nv) {
          a.fold_vec(r[u]);
          rows += EPV;
        }
      }
    }
  }
  Partial p;
  a.to_partial(p, rows);
  p = block_reduce<kBlock>(p);
  __shared__ int s_last;
  if (threadIdx.x == 0) {
    parts[part_base + blockIdx.x] = p;
    if (finalize) {
      __threadfence();
      unsigned t = atomicAdd(ticket, 1u);
      s_last = (t == gridDim.x - 1);
    }
  }
  if (!finalize) return;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  merge_partials<DT, kBlock>(parts + part_base, gridDim.x, out, ops, count_total);
  if (threadIdx.x == 0) *ticket = 0;  // leave the ticket zeroed for the next call
}

template <int DT>
__global__ void __launch_bounds__(kBlock) reduce_merge(const Partial* parts, int np, agg_scalar* out,
                                                       uint32_t ops, int64_t count_total) {
  merge_partials<DT, kBlock>(parts, np, out, ops, count_total);
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
template <int DT, bool SUM, bool MM>
static void* scan_kernel_ptr() {
  return (void*)reduce_scan<DT, SUM, MM>;
}

static void* pick_scan(int dt, bool sum, bool mm) {
#define AGG_PICK(D)                                                               \
  case D:                                                                         \
    return sum ? (mm ? scan_kernel_ptr<D, true, true>() : scan_kernel_ptr<D, true, false>()) \
               : (mm ? scan_kernel_ptr<D, false, true>() : scan_kernel_ptr<D, false, false>());
  switch (dt) {
    AGG_PICK(AGG_I32)
    AGG_PICK(AGG_I64)
    AGG_PICK(AGG_U32)
    AGG_PICK(AGG_F32)
    AGG_PICK(AGG_F64)
  }
#undef AGG_PICK
  return nullptr;
}

static void* pick_merge(int dt) {
  switch (dt) {
    case AGG_I32: return (void*)reduce_merge<AGG_I32>;
    case AGG_I64: return (void*)reduce_merge<AGG_I64>;
    case AGG_U32: return (void*)reduce_merge<AGG_U32>;
    case AGG_F32: return (void*)reduce_merge<AGG_F32>;
    case AGG_F64: return (void*)reduce_merge<AGG_F64>;
  }
  return nullptr;
}

// Resident blocks of the scan kernel per SM (occupancy-limited), cached.
static int scan_blocks_per_sm(void* fn) {
  static std::mutex mu;
  static std::map<std::pair<int, void*>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find({dev, fn});
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, fn, kBlock, 0) != cudaSuccess || b <= 0) b = 1;
  cache[{dev, fn}] = b;
  return b;
}

// Grid for a scan over n rows of dt: a multiple of the SM count, no larger
// than the number of 16-byte vector tiles.
static int scan_grid(void* fn, int64_t n, int dt) {
  const DeviceInfo& di = device_info();
  const int64_t epv = 16 / (int64_t)dtype_size(dt);
  const int64_t tiles = (n / epv + (int64_t)kBlock * kUnroll - 1) / ((int64_t)kBlock * kUnroll);
  int64_t g = (int64_t)di.sm_count * scan_blocks_per_sm(fn);
  if (tiles < g) g = tiles;
  return g < 1 ? 1 : (int)g;
}

static agg_status check_reduce_args(const void* col, int64_t n, int dt, uint32_t ops, const void* out) {
  AGG_CHECK_ARG(dtype_valid(dt), "invalid dtype %d", dt);
  AGG_CHECK_ARG(ops != 0 && (ops & ~(uint32_t)AGG_ALL) == 0, "invalid ops mask 0x%x", ops);
  AGG_CHECK_ARG(n >= 0 && n < (int64_t(1) << 62), "invalid row count %lld", (long long)n);
  AGG_CHECK_ARG(n == 0 || col != nullptr, "null column pointer");
  AGG_CHECK_ARG(out != nullptr, "null output pointer");
  AGG_CHECK_ARG(((uintptr_t)col % dtype_size(dt)) == 0, "column pointer not aligned to its element size");
  return AGG_OK;
}

static inline bool need_sum(uint32_t ops) { return ops & (AGG_SUM | AGG_AVG); }
static inline bool need_mm(uint32_t ops) { return ops & (AGG_MIN | AGG_MAX); }

static constexpr size_t kTicketBytes = 256;

}  // namespace agg

using namespace agg;

extern "C" agg_status agg_reduce(const void* col_dev, int64_t n, agg_dtype dtype, uint32_t ops,
                                 agg_scalar* out_dev, void* stream) {
  clear_error();
  agg_status st = check_reduce_args(col_dev, n, dtype, ops, out_dev);
  if (st != AGG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  void* fn = pick_scan(dtype, need_sum(ops), need_mm(ops));
  const size_t es = dtype_size(dtype);
  int64_t head = (int64_t)(((16 - ((uintptr_t)col_dev & 15)) & 15) / es);
  if (head > n) head = n;
  const int grid = scan_grid(fn, n - head, dtype);
  char* scratch = (char*)stream_scratch(s, kTicketBytes + (size_t)grid * sizeof(Partial), &st);
  if (!scratch) return st;
  unsigned* ticket = (unsigned*)scratch;
  Partial* parts = (Partial*)(scratch + kTicketBytes);
  int part_base = 0, finalize = 1;
  int64_t count = n;
  void* args[] = {(void*)&col_dev, (void*)&n, (void*)&head, (void*)&parts, (void*)&part_base,
                  (void*)&ticket, (void*)&out_dev, (void*)&ops, (void*)&count, (void*)&finalize};
  PhaseTimer pt(AGG_PHASE_SCAN, s);
  AGG_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, 0, s));
  note_launch();
  return AGG_OK;
}

// ---------------------------------------------------------------------------
// End-to-end from host memory: chunked copies on a copy stream overlapped with
// the scans of earlier chunks; one merge of all chunk partials at the end.
// ---------------------------------------------------------------------------
namespace agg {

struct HostPipe {
  cudaStream_t copy = nullptr;
  static constexpr int kRing = 3;
  cudaEvent_t ready[kRing] = {};
  cudaEvent_t freed[kRing] = {};
  bool ok = false;
};

static HostPipe& host_pipe(agg_status* st) {
  static std::mutex mu;
  static std::map<int, HostPipe> pipes;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  HostPipe& p = pipes[dev];
  *st = AGG_OK;
  if (!p.ok) {
    if (cudaStreamCreateWithFlags(&p.copy, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cannot create copy stream");
      *st = AGG_ERR_CUDA;
      return p;
    }
    for (int i = 0; i < HostPipe::kRing; ++i) {
      cudaEventCreateWithFlags(&p.ready[i], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&p.freed[i], cudaEventDisableTiming);
    }
    p.ok = true;
  }
  return p;
}

// Bytes per chunk of the end-to-end pipelines (a multiple of 16).
size_t host_chunk_bytes() { return size_t(64) << 20; }

}  // namespace agg

extern "C" agg_status agg_reduce_host(const void* col_host, int64_t n, agg_dtype dtype, uint32_t ops,
                                      agg_scalar* out_host, void* stream) {
  clear_error();
  agg_status st = check_reduce_args(col_host, n, dtype, ops, out_host);
  if (st != AGG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  static std::mutex call_mu;  // one pipeline per device; serialise its users
  std::lock_guard<std::mutex> lk(call_mu);
  HostPipe& pipe = host_pipe(&st);
  if (st != AGG_OK) return st;
  const size_t es = dtype_size(dtype);
  const int64_t chunk_rows = (int64_t)(host_chunk_bytes() / es);
  const int64_t nchunks = n == 0 ? 0 : (n + chunk_rows - 1) / chunk_rows;
  const bool scan = need_sum(ops) || need_mm(ops);
  void* fn = pick_scan(dtype, need_sum(ops), need_mm(ops));
  const int grid = scan_grid(fn, chunk_rows, dtype);
  const int64_t nparts = nchunks * (int64_t)grid;
  const size_t ring_bytes = scan ? (size_t)HostPipe::kRing * host_chunk_bytes() : 0;
  char* scratch = (char*)stream_scratch(
      s, kTicketBytes + sizeof(agg_scalar) + (size_t)(nparts > 0 ? nparts : 1) * sizeof(Partial) + 256 +
             ring_bytes,
      &st);
  if (!scratch) return st;
  agg_scalar* out_dev = (agg_scalar*)(scratch + kTicketBytes);
  Partial* parts = (Partial*)(scratch + kTicketBytes + sizeof(agg_scalar));
  char* ring = scratch + (((kTicketBytes + sizeof(agg_scalar) + (size_t)(nparts > 0 ? nparts : 1) *
                                                                    sizeof(Partial)) + 255) & ~size_t(255));
  cudaEvent_t start_ev;
  AGG_CUDA_TRY(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  cudaEventRecord(start_ev, s);
  cudaStreamWaitEvent(pipe.copy, start_ev, 0);  // the ring is free once prior work on s is done
  int64_t zero = 0;
  int fin = 0;
  unsigned* no_ticket = nullptr;
  agg_scalar* no_out = nullptr;
  for (int64_t k = 0; scan && k < nchunks; ++k) {
    const int b = (int)(k % HostPipe::kRing);
    const int64_t r0 = k * chunk_rows;
    int64_t rows = n - r0 < chunk_rows ? n - r0 : chunk_rows;
    char* buf = ring + (size_t)b * host_chunk_bytes();
    if (k >= HostPipe::kRing) cudaStreamWaitEvent(pipe.copy, pipe.freed[b], 0);
    AGG_CUDA_TRY(cudaMemcpyAsync(buf, (const char*)col_host + (size_t)r0 * es, (size_t)rows * es,
                                 cudaMemcpyHostToDevice, pipe.copy));
    cudaEventRecord(pipe.ready[b], pipe.copy);
    cudaStreamWaitEvent(s, pipe.ready[b], 0);
    int g = grid;
    int base = (int)(k * grid);
    void* args[] = {(void*)&buf, (void*)&rows, (void*)&zero, (void*)&parts, (void*)&base,
                    (void*)&no_ticket, (void*)&no_out, (void*)&ops, (void*)&n, (void*)&fin};
    AGG_CUDA_TRY(cudaLaunchKernel(fn, dim3(g), dim3(kBlock), args, 0, s));
    note_launch();
    cudaEventRecord(pipe.freed[b], s);
  }
  int np = scan ? (int)nparts : 0;
  void* margs[] = {(void*)&parts, (void*)&np, (void*)&out_dev, (void*)&ops, (void*)&n};
  AGG_CUDA_TRY(cudaLaunchKernel(pick_merge(dtype), dim3(1), dim3(kBlock), margs, 0, s));
  note_launch();
  AGG_CUDA_TRY(cudaMemcpyAsync(out_host, out_dev, sizeof(agg_scalar), cudaMemcpyDeviceToHost, s));
  cudaError_t e = cudaStreamSynchronize(s);
  cudaEventDestroy(start_ev);
  if (e != cudaSuccess) {
    set_error("agg_reduce_host: %s", cudaGetErrorString(e));
    return AGG_ERR_CUDA;
  }
  return AGG_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of agg_reduce.
//
// Its scratch (the ticket and one Partial per block) lives in a file-scope
// __device__ array instead of library-allocated memory, so a call performs no
// device allocation at all. Host code must not pass the array's name to a
// kernel (on the host it names a stand-in object, not device memory); the
// device address is looked up once per device with cudaGetSymbolAddress and
// cached.
// ---------------------------------------------------------------------------
namespace agg {

constexpr int kNoAllocMaxBlocks = 2048;
constexpr size_t kNoAllocScratchBytes = kTicketBytes + (size_t)kNoAllocMaxBlocks * sizeof(Partial);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch on the current device (set up on first use).
static void* noalloc_scratch_address(agg_status* st) {
  static std::mutex mu;
  static std::map<int, void*> addr;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_error("agg_reduce_noalloc: cudaGetDevice failed: %s", cudaGetErrorString(e));
    *st = AGG_ERR_CUDA;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  auto it = addr.find(dev);
  if (it != addr.end()) {
    *st = AGG_OK;
    return it->second;
  }
  void* p = nullptr;
  e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    set_error("agg_reduce_noalloc: cudaGetSymbolAddress of the static scratch failed on device %d: %s", dev,
              cudaGetErrorString(e));
    *st = AGG_ERR_CUDA;
    return nullptr;
  }
  addr[dev] = p;
  *st = AGG_OK;
  return p;
}

}  // namespace agg

extern "C" agg_status agg_reduce_noalloc(const void* col_dev, int64_t n, agg_dtype dtype, uint32_t ops,
                                         agg_scalar* out_dev, void* stream) {
  clear_error();
  agg_status st = check_reduce_args(col_dev, n, dtype, ops, out_dev);
  if (st != AGG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  void* fn = pick_scan(dtype, need_sum(ops), need_mm(ops));
  const size_t es = dtype_size(dtype);
  int64_t head = (int64_t)(((16 - ((uintptr_t)col_dev & 15)) & 15) / es);
  if (head > n) head = n;
  const int grid = scan_grid(fn, n - head, dtype);
  const size_t need = kTicketBytes + (size_t)grid * sizeof(Partial);
  if (need > kNoAllocScratchBytes) {
    set_error("agg_reduce_noalloc: this launch needs %zu bytes of scratch (%d blocks) but the static scratch "
              "holds %zu bytes (%d blocks)",
              need, grid, kNoAllocScratchBytes, kNoAllocMaxBlocks);
    return AGG_ERR_INVALID;
  }
  char* scratch = (char*)noalloc_scratch_address(&st);
  if (!scratch) return st;
  unsigned* ticket = (unsigned*)scratch;
  Partial* parts = (Partial*)(scratch + kTicketBytes);
  // The array keeps the previous call's contents; the ticket must start at zero.
  AGG_CUDA_TRY(cudaMemsetAsync(ticket, 0, sizeof(unsigned), s));
  int part_base = 0, finalize = 1;
  int64_t count = n;
  void* args[] = {(void*)&col_dev, (void*)&n, (void*)&head, (void*)&parts, (void*)&part_base,
                  (void*)&ticket, (void*)&out_dev, (void*)&ops, (void*)&count, (void*)&finalize};
  AGG_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, 0, s));
  note_launch();
  return AGG_OK;
}
