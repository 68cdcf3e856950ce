// GROUP BY over a composite 64-bit key with several value columns and a range
// filter, fused into one scan: the selection feeding an aggregation that the
// paper names as operator fusion for future work (Sec. 8). A row takes part
// iff lo <= f[i] <= hi in the filter column's type; its group is the key
// (key_hi[i] << 32) | key_lo[i].
//
// One pass over the rows (multi_build): the filter is tested first and a row
// that fails it is dropped before any other column is read; a passing row
// finds (or inserts) its key in an open-addressing table of 64-bit keys in
// HBM (SplitMix64's finaliser as the hash, linear probing, bounded probes) and
// that slot's index is its group: every value column is folded into
// accumulator arrays indexed by the slot, in shared memory when every block
// can hold one accumulator per slot (a dense block-local copy, merged once at
// the end of the block), else directly in HBM with L2 atomics. The
// accumulators are those of the hash GROUP BY: 32-bit count; integer sums
// mod 2^64 (two 32-bit words with an explicit carry in shared memory); float32
// sums as a TwoSum-compensated float32 pair in shared memory, float64 in HBM;
// MIN/MAX as order-preserving 64-bit images. Finalise: the occupied slots are
// compacted, sorted by their 64-bit key (a stable radix sort on the low word,
// then on the high word) and gathered into the outputs.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "groupby.cuh"
#include "sort.cuh"

namespace agg {

constexpr int kMultiThreads = 512;
constexpr int kMultiProbe = 128;
constexpr unsigned long long kEmpty64 = ~0ull;
constexpr int kMultiFull = 1;  // status: a key found no slot

// SplitMix64's output function (Steele, Lea and Flood 2014), a bijective mixer.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

struct MultiArgs {
  const uint32_t* klo;
  const uint32_t* khi;  // null: high word 0
  int64_t n;
  int ncols;
  const void* col[AGG_MAX_COLUMNS];
  int dt[AGG_MAX_COLUMNS];
  bool mm[AGG_MAX_COLUMNS];
  const void* fcol;  // null: no filter
  int fdt;
  int64_t flo_i, fhi_i;
  double flo_f, fhi_f;
  unsigned long long* keys;  // S main slots (kEmpty64 = empty) + side slot S for the key ~0
  uint32_t mask;             // S - 1
  int shift;                 // home slot = mix64(key) >> shift
  uint32_t* cnt;             // [S + 1]
  unsigned long long* sum[AGG_MAX_COLUMNS];   // [S + 1] integer sum / float64 sum
  unsigned long long* minc[AGG_MAX_COLUMNS];  // [S + 1] complement of the MIN image
  unsigned long long* mx[AGG_MAX_COLUMNS];    // [S + 1] MAX image
  int dense;                 // accumulate in shared memory (S + 1 slots per block)
  int* status;               // kMultiFull when a key found no slot
};

__device__ __forceinline__ bool multi_pass(const MultiArgs& a, int64_t i) {
  if (!a.fcol) return true;
  switch (a.fdt) {
    case AGG_I32: { const int64_t x = ((const int32_t*)a.fcol)[i]; return a.flo_i <= x && x <= a.fhi_i; }
    case AGG_I64: { const int64_t x = ((const int64_t*)a.fcol)[i]; return a.flo_i <= x && x <= a.fhi_i; }
    case AGG_U32: { const int64_t x = ((const uint32_t*)a.fcol)[i]; return a.flo_i <= x && x <= a.fhi_i; }
    case AGG_F32: { const double x = ((const float*)a.fcol)[i]; return a.flo_f <= x && x <= a.fhi_f; }
    default: { const double x = ((const double*)a.fcol)[i]; return a.flo_f <= x && x <= a.fhi_f; }
  }
}

// Slot of a 64-bit key (inserted if absent), or -1 after kMultiProbe probes.
__device__ __forceinline__ int64_t multi_slot(const MultiArgs& a, uint64_t key) {
  if (key == kEmpty64) return (int64_t)a.mask + 1;
  uint32_t h = (uint32_t)(mix64(key) >> a.shift);
#pragma unroll 1
  for (int p = 0; p < kMultiProbe; ++p) {
    const unsigned long long cur = *(volatile unsigned long long*)&a.keys[h];
    if (cur == key) return h;
    if (cur == kEmpty64) {
      const unsigned long long old = atomicCAS(&a.keys[h], kEmpty64, (unsigned long long)key);
      if (old == kEmpty64 || old == key) return h;
    }
    h = (h + 1) & a.mask;
  }
  return -1;
}

// A value as (integer or float64 sum term, float32 value, order-preserving image).
struct MVal {
  int64_t i;
  double d;
  float f;
  uint64_t img;
};

__device__ __forceinline__ MVal multi_val(const void* col, int dt, int64_t r) {
  MVal v;
  v.i = 0;
  v.d = 0.0;
  v.f = 0.f;
  switch (dt) {
    case AGG_I32: v.i = ((const int32_t*)col)[r]; v.img = img_i64(v.i); break;
    case AGG_I64: v.i = ((const int64_t*)col)[r]; v.img = img_i64(v.i); break;
    case AGG_U32: v.i = ((const uint32_t*)col)[r]; v.img = img_i64(v.i); break;
    case AGG_F32: v.f = ((const float*)col)[r]; v.d = v.f; v.img = img_f64(v.d); break;
    default: v.d = ((const double*)col)[r]; v.img = img_f64(v.d); break;
  }
  return v;
}

// Shared-memory layout for S1 = S + 1 slots: cnt u32[S1], then per column a
// 64-bit sum word and, with MIN/MAX, a (min, max) pair of 64-bit images.
struct MultiSmem {
  uint32_t* cnt;
  unsigned long long* sum[AGG_MAX_COLUMNS];
  unsigned long long* mm[AGG_MAX_COLUMNS];
};

__host__ __device__ inline size_t multi_smem_bytes(int S1, int ncols, const bool* mm) {
  size_t b = ((size_t)S1 * 4 + 15) & ~size_t(15);
  for (int c = 0; c < ncols; ++c) b += (size_t)S1 * 8 + (mm[c] ? (size_t)S1 * 16 : 0);
  return b;
}

__device__ __forceinline__ MultiSmem multi_carve(unsigned char* base, int S1, const MultiArgs& a) {
  MultiSmem m;
  m.cnt = (uint32_t*)base;
  unsigned char* p = base + (((size_t)S1 * 4 + 15) & ~size_t(15));
  for (int c = 0; c < AGG_MAX_COLUMNS; ++c) {
    m.sum[c] = nullptr;
    m.mm[c] = nullptr;
    if (c >= a.ncols) continue;
    m.sum[c] = (unsigned long long*)p;
    p += (size_t)S1 * 8;
    if (a.mm[c]) {
      m.mm[c] = (unsigned long long*)p;
      p += (size_t)S1 * 16;
    }
  }
  return m;
}

__device__ __forceinline__ void multi_fold_smem(const MultiSmem& m, int c, int dt, bool mm, int64_t j, const MVal& v) {
  uint32_t* w = (uint32_t*)&m.sum[c][j];
  if (dt == AGG_F32) {
    const float old = atomicAdd((float*)&w[0], v.f);
    float t, e;
    two_sum(old, v.f, t, e);  // t is what the atomic stored, e its rounding error
    if (e != 0.f) atomicAdd((float*)&w[1], e);
  } else if (dt == AGG_F64) {
    atomicAdd((double*)&m.sum[c][j], v.d);
  } else {
    const uint64_t u = (uint64_t)v.i;
    const uint32_t lo = (uint32_t)u;
    const uint32_t old = atomicAdd(&w[0], lo);
    const uint32_t hi = (uint32_t)(u >> 32) + ((uint32_t)(old + lo) < old ? 1u : 0u);
    if (hi) atomicAdd(&w[1], hi);
  }
  if (mm) {
    unsigned long long* q = &m.mm[c][2 * j];
    if (v.img < *(volatile unsigned long long*)&q[0]) atomicMin(&q[0], (unsigned long long)v.img);
    if (v.img > *(volatile unsigned long long*)&q[1]) atomicMax(&q[1], (unsigned long long)v.img);
  }
}

__device__ __forceinline__ void multi_fold_global(const MultiArgs& a, int c, int64_t j, const MVal& v) {
  if (a.dt[c] == AGG_F32 || a.dt[c] == AGG_F64) atomicAdd((double*)&a.sum[c][j], v.d);
  else atomicAdd(&a.sum[c][j], (unsigned long long)v.i);
  if (a.mm[c]) {
    if (~v.img > *(volatile unsigned long long*)&a.minc[c][j]) atomicMax(&a.minc[c][j], (unsigned long long)~v.img);
    if (v.img > *(volatile unsigned long long*)&a.mx[c][j]) atomicMax(&a.mx[c][j], (unsigned long long)v.img);
  }
}

__global__ void __launch_bounds__(kMultiThreads) multi_build(MultiArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int S1 = (int)a.mask + 2;
  MultiSmem m;
  if (a.dense) {
    m = multi_carve(smem, S1, a);
    for (int j = threadIdx.x; j < S1; j += blockDim.x) {
      m.cnt[j] = 0;
      for (int c = 0; c < a.ncols; ++c) {
        m.sum[c][j] = 0;
        if (a.mm[c]) {
          m.mm[c][2 * j] = ~0ull;
          m.mm[c][2 * j + 1] = 0;
        }
      }
    }
    __syncthreads();
  }
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  int it = 0;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < a.n; r += stride) {
    if ((++it & 63) == 0 && *(volatile int*)a.status) break;  // a full table: the build is redone
    if (!multi_pass(a, r)) continue;
    const uint64_t key = ((uint64_t)(a.khi ? a.khi[r] : 0u) << 32) | a.klo[r];
    const int64_t j = multi_slot(a, key);
    if (j < 0) {
      *(volatile int*)a.status = kMultiFull;
      continue;
    }
    if (a.dense) atomicAdd(&m.cnt[j], 1u);
    else atomicAdd(&a.cnt[j], 1u);
    for (int c = 0; c < a.ncols; ++c) {
      const MVal v = multi_val(a.col[c], a.dt[c], r);
      if (a.dense) multi_fold_smem(m, c, a.dt[c], a.mm[c], j, v);
      else multi_fold_global(a, c, j, v);
    }
  }
  if (!a.dense) return;
  __syncthreads();
  for (int j = threadIdx.x; j < S1; j += blockDim.x) {  // merge the block's accumulators
    const uint32_t k = m.cnt[j];
    if (k == 0) continue;
    atomicAdd(&a.cnt[j], k);
    for (int c = 0; c < a.ncols; ++c) {
      const unsigned long long sv = m.sum[c][j];
      if (a.dt[c] == AGG_F32) {
        atomicAdd((double*)&a.sum[c][j],
                  (double)__uint_as_float((uint32_t)sv) + (double)__uint_as_float((uint32_t)(sv >> 32)));
      } else {
        if (a.dt[c] == AGG_F64) atomicAdd((double*)&a.sum[c][j], __longlong_as_double((long long)sv));
        else atomicAdd(&a.sum[c][j], sv);
      }
      if (a.mm[c]) {
        const unsigned long long mn = m.mm[c][2 * j], mx = m.mm[c][2 * j + 1];
        if (~mn > a.minc[c][j]) atomicMax(&a.minc[c][j], ~mn);
        if (mx > a.mx[c][j]) atomicMax(&a.mx[c][j], mx);
      }
    }
  }
}

// Occupied slots -> (low word, high word, slot) triples; the count of groups into *d.
__global__ void __launch_bounds__(kMultiThreads) multi_compact(const unsigned long long* keys, const uint32_t* cnt,
                                                                int64_t S1, uint32_t mask, uint32_t* klo,
                                                                uint32_t* khi, uint32_t* slot,
                                                                unsigned long long* d) {
  // the loop runs per warp (all lanes take every iteration) for the ballot
  const int lane = threadIdx.x & 31;
  for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); w0 < S1;
       w0 += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = w0 + lane;
    const bool occ = j < S1 && cnt[j] != 0;
    const uint32_t b = __ballot_sync(0xffffffffu, occ);
    if (b == 0) continue;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(d, (unsigned long long)__popc(b));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (occ) {
      const uint64_t key = j <= (int64_t)mask ? keys[j] : kEmpty64;
      const unsigned long long p = base + __popc(b & ((1u << lane) - 1u));
      klo[p] = (uint32_t)key;
      khi[p] = (uint32_t)(key >> 32);
      slot[p] = (uint32_t)j;
    }
  }
}

// dst[i] = src[perm[i]] for i < *d (perm null: dst[i] = i).
__global__ void multi_permute_u32(const uint32_t* src, const uint32_t* perm, uint32_t* dst, const int64_t* d) {
  const int64_t n = *d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = perm ? src[perm[i]] : (uint32_t)i;
}

struct MultiOut {
  uint64_t* keys;
  int64_t* count;
  unsigned long long* sum[AGG_MAX_COLUMNS];
  unsigned long long* min[AGG_MAX_COLUMNS];
  unsigned long long* max[AGG_MAX_COLUMNS];
  double* avg[AGG_MAX_COLUMNS];
};

__global__ void multi_gather(MultiArgs a, const uint32_t* slot, const uint32_t* order, const int64_t* d, MultiOut o) {
  const int64_t n = *d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t j = slot[order[i]];
    const uint32_t c0 = a.cnt[j];
    o.keys[i] = j <= a.mask ? a.keys[j] : kEmpty64;
    o.count[i] = c0;
    for (int c = 0; c < a.ncols; ++c) {
      const unsigned long long sv = a.sum[c][j];
      const bool fp = a.dt[c] == AGG_F32 || a.dt[c] == AGG_F64;
      o.sum[c][i] = sv;
      const double s = fp ? __longlong_as_double((long long)sv) : (double)(long long)sv;
      o.avg[c][i] = s / (double)c0;
      if (a.mm[c]) {
        const uint64_t mn = ~a.minc[c][j], mx = a.mx[c][j];
        if (fp) {
          o.min[c][i] = (unsigned long long)__double_as_longlong(f64_of_img(mn));
          o.max[c][i] = (unsigned long long)__double_as_longlong(f64_of_img(mx));
        } else {
          o.min[c][i] = (unsigned long long)i64_of_img(mn);
          o.max[c][i] = (unsigned long long)i64_of_img(mx);
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
struct MultiPriv {
  void* block = nullptr;
  int device = 0;
  cudaStream_t stream = nullptr;
};

static agg_status multi_alloc(int64_t cap, int ncols, cudaStream_t s, agg_multi** out) {
  if (cap < 1) cap = 1;
  const size_t a8 = ((size_t)cap * 8 + 255) & ~size_t(255);
  const size_t bytes = a8 * (2 + 4 * (size_t)ncols) + 256;
  void* blk = nullptr;
  cudaError_t e = dev_malloc_async(&blk, bytes, s);
  if (e != cudaSuccess) {
    set_error("multi-column result allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    return AGG_ERR_OOM;
  }
  agg_multi* m = new agg_multi();
  std::memset(m, 0, sizeof(*m));
  MultiPriv* p = new MultiPriv();
  p->block = blk;
  p->stream = s;
  cudaGetDevice(&p->device);
  char* c = (char*)blk;
  m->keys = (uint64_t*)c; c += a8;
  m->count = (int64_t*)c; c += a8;
  for (int k = 0; k < ncols; ++k) {
    m->sum[k] = c; c += a8;
    m->min[k] = c; c += a8;
    m->max[k] = c; c += a8;
    m->avg[k] = (double*)c; c += a8;
  }
  m->ncols = ncols;
  m->priv = p;
  *out = m;
  return AGG_OK;
}

// One build and finalise with S main slots; TABLE_FULL if a key found no slot.
static agg_status multi_run(MultiArgs a, int64_t S, cudaStream_t s, agg_multi** out) {
  const DeviceInfo& di = device_info();
  const int64_t S1 = S + 1;
  // table: keys [S1] u64, cnt [S1] u32, per column sum/minc/max [S1] u64; status; finalise scratch
  const size_t k8 = ((size_t)S1 * 8 + 255) & ~size_t(255), k4 = ((size_t)S1 * 4 + 255) & ~size_t(255);
  size_t bytes = k8 + k4;
  for (int c = 0; c < a.ncols; ++c) bytes += k8 * (a.mm[c] ? 3 : 1);
  const size_t status_off = bytes;
  bytes += 256;
  const size_t fin_off = bytes;
  bytes += 6 * k4 + radix_tmp_bytes(S1) + 256;
  char* mem = nullptr;
  AGG_CUDA_TRY(dev_malloc_async((void**)&mem, bytes, s));
  struct Free {
    void* p;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(p, s); }
  } mem_free{mem, s};
  AGG_CUDA_TRY(cudaMemsetAsync(mem, 0xFF, k8, s));                         // keys empty
  AGG_CUDA_TRY(cudaMemsetAsync(mem + k8, 0, fin_off - k8, s));             // accumulators, status
  char* p = mem;
  a.keys = (unsigned long long*)p; p += k8;
  a.cnt = (uint32_t*)p; p += k4;
  for (int c = 0; c < a.ncols; ++c) {
    a.sum[c] = (unsigned long long*)p; p += k8;
    if (a.mm[c]) {
      a.minc[c] = (unsigned long long*)p; p += k8;
      a.mx[c] = (unsigned long long*)p; p += k8;
    }
  }
  a.status = (int*)(mem + status_off);
  unsigned long long* dcount = (unsigned long long*)(mem + status_off + 64);
  a.mask = (uint32_t)(S - 1);
  a.shift = 64 - (63 - __builtin_clzll((unsigned long long)S));
  const size_t sm = multi_smem_bytes((int)std::min<int64_t>(S1, INT32_MAX), a.ncols, a.mm);
  a.dense = S1 <= 65536 && sm <= (size_t)di.smem_per_block_optin ? 1 : 0;
  const size_t dyn = a.dense ? sm : 0;
  if (dyn > 48 * 1024) AGG_CUDA_TRY(cudaFuncSetAttribute(multi_build, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
  int bps = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, multi_build, kMultiThreads, dyn) != cudaSuccess || bps < 1)
    bps = 1;
  int64_t grid = (int64_t)di.sm_count * bps;
  const int64_t need = (a.n + kMultiThreads - 1) / kMultiThreads;
  if (need < grid) grid = std::max<int64_t>(1, need);
  {
    PhaseTimer pt(AGG_PHASE_BUILD, s);
    multi_build<<<(unsigned)grid, kMultiThreads, dyn, s>>>(a);
    note_launch();
    AGG_CUDA_TRY(cudaGetLastError());
  }
  // finalise: compact the occupied slots, order them by (high word, low word)
  // with two stable radix sorts of (word, compact index) pairs, gather
  PhaseTimer pt(AGG_PHASE_FINALIZE, s);
  uint32_t* buf[7];
  for (int k = 0; k < 7; ++k) buf[k] = (uint32_t*)(mem + fin_off + (size_t)k * k4);
  uint32_t *klo = buf[0], *khi = buf[1], *slot = buf[2], *idx = buf[3];
  void* rtmp = (void*)(((uintptr_t)(mem + fin_off + 7 * k4) + 255) & ~(uintptr_t)255);
  const int64_t* dd = (const int64_t*)dcount;
  const int g = (int)std::max<int64_t>(1, std::min<int64_t>((S1 + 255) / 256, (int64_t)di.sm_count * 8));
  multi_compact<<<g, 256, 0, s>>>(a.keys, a.cnt, S1, a.mask, klo, khi, slot, dcount);
  multi_permute_u32<<<g, 256, 0, s>>>(nullptr, nullptr, idx, dd);
  note_launch(2);
  AGG_CUDA_TRY(cudaGetLastError());
  uint32_t *k1 = nullptr, *v1 = nullptr;
  agg_status st = radix_sort_pairs<uint32_t>(klo, idx, buf[4], buf[5], klo, idx, S1, dd, 32, rtmp, s, &k1, &v1);
  if (st != AGG_OK) return st;
  uint32_t* hi1 = buf[6];  // the high words in low-word order
  multi_permute_u32<<<g, 256, 0, s>>>(khi, v1, hi1, dd);
  note_launch();
  AGG_CUDA_TRY(cudaGetLastError());
  uint32_t* fk = v1 == idx ? buf[4] : klo;  // the pair the first sort left free
  uint32_t* fv = v1 == idx ? buf[5] : idx;
  uint32_t *k2 = nullptr, *order = nullptr;
  st = radix_sort_pairs<uint32_t>(hi1, v1, fk, fv, hi1, v1, S1, dd, 32, rtmp, s, &k2, &order);
  if (st != AGG_OK) return st;
  agg_multi* m = nullptr;
  st = multi_alloc(S1, a.ncols, s, &m);
  if (st != AGG_OK) return st;
  MultiOut o;
  o.keys = m->keys;
  o.count = m->count;
  for (int c = 0; c < AGG_MAX_COLUMNS; ++c) {
    o.sum[c] = c < a.ncols ? (unsigned long long*)m->sum[c] : nullptr;
    o.min[c] = c < a.ncols ? (unsigned long long*)m->min[c] : nullptr;
    o.max[c] = c < a.ncols ? (unsigned long long*)m->max[c] : nullptr;
    o.avg[c] = c < a.ncols ? m->avg[c] : nullptr;
  }
  multi_gather<<<g, 256, 0, s>>>(a, slot, order, dd, o);
  note_launch();
  cudaError_t e = cudaGetLastError();
  unsigned char* hb = (unsigned char*)stream_pinned(s, 256, &st);
  if (e == cudaSuccess && hb) {
    e = cudaMemcpyAsync(hb, mem + status_off, 72, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  if (e != cudaSuccess || !hb) {
    agg_multi_free(m);
    if (!hb) return st;
    set_error("multi-column GROUP BY: %s", cudaGetErrorString(e));
    return AGG_ERR_CUDA;
  }
  if (*(const int*)hb != 0) {
    agg_multi_free(m);
    set_error("key table of %lld slots is full", (long long)S);
    return AGG_ERR_TABLE_FULL;
  }
  m->num_groups = *(const int64_t*)(hb + 64);
  m->table_slots = S;
  *out = m;
  return AGG_OK;
}

// Distinct keys of a key column for sizing the table (the sketch's planning estimate).
static agg_status key_count_estimate(const uint32_t* keys, int64_t n, cudaStream_t s, double* est) {
  float f[F_COUNT];
  agg_status st = sketch_features(keys, n, AGG_I64, AGG_SUM, 0, s, f);
  if (st != AGG_OK) return st;
  bool covered = false;
  *est = distinct_estimate(f, &covered);
  return AGG_OK;
}

}  // namespace agg

using namespace agg;

static agg_status check_column(const void* p, int dt, int64_t n, const char* what) {
  AGG_CHECK_ARG(dtype_valid(dt), "%s: invalid dtype %d", what, dt);
  AGG_CHECK_ARG(n == 0 || p != nullptr, "%s: null pointer", what);
  AGG_CHECK_ARG(((uintptr_t)p % dtype_size(dt)) == 0, "%s: pointer not aligned to its element size", what);
  return AGG_OK;
}

extern "C" agg_status agg_groupby_multi(const uint32_t* key_lo_dev, const uint32_t* key_hi_dev, int64_t n,
                                        const agg_column* cols, int ncols, const agg_range* filter, agg_multi** out,
                                        void* stream) {
  clear_error();
  AGG_CHECK_ARG(out != nullptr, "null result pointer");
  AGG_CHECK_ARG(n >= 0 && n <= 0xFFFFFFFFll, "invalid row count %lld (needs n < 2^32)", (long long)n);
  AGG_CHECK_ARG(ncols >= 1 && ncols <= AGG_MAX_COLUMNS && cols != nullptr, "ncols must be in [1, %d]",
                AGG_MAX_COLUMNS);
  AGG_CHECK_ARG(n == 0 || key_lo_dev != nullptr, "null key pointer");
  AGG_CHECK_ARG(((uintptr_t)key_lo_dev & 3) == 0 && ((uintptr_t)key_hi_dev & 3) == 0, "key pointer not 4-byte aligned");
  agg_status st;
  for (int c = 0; c < ncols; ++c) {
    st = check_column(cols[c].data, cols[c].dtype, n, "value column");
    if (st != AGG_OK) return st;
    AGG_CHECK_ARG(cols[c].ops != 0 && (cols[c].ops & ~(uint32_t)AGG_ALL) == 0, "column %d: invalid ops mask 0x%x", c,
                  cols[c].ops);
  }
  if (filter) {
    st = check_column(filter->data, filter->dtype, n, "filter column");
    if (st != AGG_OK) return st;
  }
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)stream;
  MultiArgs a;
  std::memset(&a, 0, sizeof(a));
  a.klo = key_lo_dev;
  a.khi = key_hi_dev;
  a.n = n;
  a.ncols = ncols;
  for (int c = 0; c < ncols; ++c) {
    a.col[c] = cols[c].data;
    a.dt[c] = cols[c].dtype;
    a.mm[c] = ops_minmax(cols[c].ops);
  }
  if (filter) {
    a.fcol = filter->data;
    a.fdt = filter->dtype;
    a.flo_i = filter->lo_i;
    a.fhi_i = filter->hi_i;
    a.flo_f = filter->lo_f;
    a.fhi_f = filter->hi_f;
  }
  // table slots: twice the planning estimate of the distinct composite keys
  double est = 1.0;
  if (n > 0) {
    double e_lo = 1.0, e_hi = 1.0;
    st = key_count_estimate(key_lo_dev, n, s, &e_lo);
    if (st == AGG_OK && key_hi_dev) st = key_count_estimate(key_hi_dev, n, s, &e_hi);
    if (st != AGG_OK) return st;
    est = std::min((double)n, e_lo * e_hi);
  }
  const int64_t cap = std::min<int64_t>(int64_t(1) << 31, next_pow2(std::max<int64_t>(2 * n, 1024)));
  int64_t S = std::min<int64_t>(cap, std::max<int64_t>(1024, next_pow2((int64_t)std::ceil(2.0 * est))));
  int retries = 0;
  for (;;) {
    st = multi_run(a, S, s, out);
    if (st != AGG_ERR_TABLE_FULL || S >= cap) break;
    S = std::min<int64_t>(cap, 4 * S);
    ++retries;
  }
  if (st == AGG_OK) (*out)->retries = retries;
  return st;
}

extern "C" agg_status agg_multi_to_host(const agg_multi* m, uint64_t* keys, int64_t* count, int col, void* sum,
                                        void* min, void* max, double* avg) {
  clear_error();
  AGG_CHECK_ARG(m != nullptr, "null result");
  AGG_CHECK_ARG(col >= 0 && col < m->ncols, "column %d out of range", col);
  const size_t d = (size_t)m->num_groups;
  if (d == 0) return AGG_OK;
  if (keys) AGG_CUDA_TRY(cudaMemcpy(keys, m->keys, d * 8, cudaMemcpyDeviceToHost));
  if (count) AGG_CUDA_TRY(cudaMemcpy(count, m->count, d * 8, cudaMemcpyDeviceToHost));
  if (sum) AGG_CUDA_TRY(cudaMemcpy(sum, m->sum[col], d * 8, cudaMemcpyDeviceToHost));
  if (min) AGG_CUDA_TRY(cudaMemcpy(min, m->min[col], d * 8, cudaMemcpyDeviceToHost));
  if (max) AGG_CUDA_TRY(cudaMemcpy(max, m->max[col], d * 8, cudaMemcpyDeviceToHost));
  if (avg) AGG_CUDA_TRY(cudaMemcpy(avg, m->avg[col], d * 8, cudaMemcpyDeviceToHost));
  return AGG_OK;
}

extern "C" void agg_multi_free(agg_multi* m) {
  if (!m) return;
  MultiPriv* p = (MultiPriv*)m->priv;
  if (p) {
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != p->device) cudaSetDevice(p->device);
    cudaFreeAsync(p->block, p->stream);
    if (cur != p->device) cudaSetDevice(cur);
    delete p;
  }
  delete m;
}
