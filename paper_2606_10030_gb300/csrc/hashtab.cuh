// Device side of the hash GROUP BY (build and finalisation), shared by the
// single-query driver (groupby.cu) and the batched persistent kernel
// (batch.cu): slot layouts, shared- and global-table probing and updates, the
// build kernel and the finalise kernels.
//
// Build. Every row is folded (the aggregate() of Fig. 4) into the slot of its
// key in an open-addressing hash table (MurmurHash3 fmix32, linear probing,
// bounded probe count):
//   SMEM    each block owns a table in shared memory and updates it with
//           shared-memory atomics; rows whose key finds no slot within the
//           probe bound go straight to the global table ("spill"); at the end
//           the block merges its table into the global one.
//   GLOBAL  every row updates the global table in HBM with L2 atomics.
// Keys are stored as key + 1 so that an all-zero table is empty; the key
// 0xFFFFFFFF has its own side slot after the main slots. All global
// accumulators start at zero: count and sum add, MIN is kept as the
// complement of an order-preserving image and MAX as the image, both updated
// with atomicMax; float sums in the global table are float64 (L2 atomic adds:
// a per-block or per-warp compensated float32 partial, or a single row, is
// merged into a float64 accumulator; the float64 additions run in the L2's
// atomic units, not on the SM's narrow float64 pipe).
#pragma once

#include <cstring>

#include "groupby.cuh"

namespace agg {

// ---------------------------------------------------------------------------
// Value traits: order-preserving 64-bit image of a value.
// ---------------------------------------------------------------------------
template <int DT> struct GV;
template <> struct GV<AGG_I32> {
  using T = int32_t;
  __device__ static uint64_t img(T v) { return img_i64((int64_t)v); }
};
template <> struct GV<AGG_I64> {
  using T = int64_t;
  __device__ static uint64_t img(T v) { return img_i64(v); }
};
template <> struct GV<AGG_U32> {
  using T = uint32_t;
  __device__ static uint64_t img(T v) { return img_i64((int64_t)v); }
};
template <> struct GV<AGG_F32> {
  using T = float;
  __device__ static uint64_t img(T v) { return (uint64_t)img_f32(v); }
};
template <> struct GV<AGG_F64> {
  using T = double;
  __device__ static uint64_t img(T v) { return img_f64(v); }
};

template <bool MM> struct GSlot;
template <> struct __align__(16) GSlot<false> {
  uint32_t key1;
  uint32_t cnt;
  unsigned long long sum;
};
template <> struct __align__(32) GSlot<true> {
  uint32_t key1;
  uint32_t cnt;
  unsigned long long sum;
  unsigned long long minc;
  unsigned long long mx;
};

constexpr int kGlobalProbe = 128;
constexpr int kSmemProbe = 8;
constexpr int kStatusFull = 1;

struct BuildArgs {
  const uint32_t* keys;
  const void* vals;
  int64_t n;
  int64_t head;        // rows before the 16-byte aligned body (vector path)
  void* table;         // GSlot[mask + 2]
  uint32_t mask;       // main slots - 1 (main slots a power of two)
  int gshift;          // home slot = fmix32(key) >> gshift (top bits: 32 - log2(main slots))
  int smem_slots;      // S (power of two) for SMEM, else 0
  int smem_cap;        // max keys inserted into the shared table
  int* status;
  unsigned long long* progress;  // [0] rows gone through, [1] rows that found no slot, counted
                                 // when a full table stopped the build (or null)
  uint32_t* block_fails;         // this block's count of rows that found no slot (shared memory, or null)
  // int64 MIN/MAX in tile builds: the low words of the images whose high word
  // is the tile's (one (min, max) u32 pair a slot, shared memory), or null
  uint32_t* mm32 = nullptr;
  uint32_t tile_hi = 0;
};

// Global slot of key (insert if absent); -1 if no slot within the probe bound.
// The home slot is taken from the top bits of the hash, so keys whose hash
// shares its top bits (one partition of a hash-partitioned input) live in one
// contiguous region of the table.
template <bool MM>
__device__ __forceinline__ int64_t g_slot(GSlot<MM>* tab, uint32_t mask, int shift, uint32_t key,
                                          int max_probe = kGlobalProbe) {
  if (key == 0xFFFFFFFFu) return (int64_t)mask + 1;
  const uint32_t k1 = key + 1;
  uint32_t h = fmix32(key) >> shift;
#pragma unroll 1
  for (int p = 0; p < max_probe; ++p) {
    uint32_t cur = *(volatile uint32_t*)&tab[h].key1;
    if (cur == k1) return h;
    if (cur == 0) {
      uint32_t old = atomicCAS(&tab[h].key1, 0u, k1);
      if (old == 0u || old == k1) return h;
    }
    h = (h + 1) & mask;
  }
  return -1;
}

// Fold one row (or a merged partial) into a global slot.
template <int DT, bool MM>
__device__ __forceinline__ void g_add_row(GSlot<MM>& s, typename GV<DT>::T v) {
  atomicAdd(&s.cnt, 1u);
  if (DT == AGG_F32 || DT == AGG_F64) {
    atomicAdd((double*)&s.sum, (double)v);
  } else {
    atomicAdd(&s.sum, (unsigned long long)(int64_t)v);
  }
  if (MM) {
    const uint64_t m = GV<DT>::img(v);
    atomicMax(&((GSlot<true>&)s).minc, (unsigned long long)~m);
    atomicMax(&((GSlot<true>&)s).mx, (unsigned long long)m);
  }
}

// Shared-memory table over S + 1 slots (S a power of two >= 64; slot S holds
// the key 0xFFFFFFFF). Keys are probed a bucket of 4 slots at a time with one
// 16-byte load. Every per-row update uses native 32-bit shared atomics:
//   count     u32 add
//   sum       integers: two u32 words; the low word's atomic add returns the
//             previous value, so the adding thread sees its own carry exactly
//             and adds it with the high part (the pair is the 64-bit sum mod
//             2^64). float32: s and c words; the adder recovers the rounding
//             error of its own atomic add of s with TwoSum from the returned
//             previous value and adds that error to c. float64: one 64-bit
//             float atomic add.
//   MIN/MAX   an adjacent (min, max) pair of order-preserving images (32-bit
//             for 4-byte values); an atomic is issued only when the value
//             improves the current extreme.
// In tile builds (at most 65532 rows per tile) integer sums count the low
// word's carries in the high half of the count word instead (one atomic adds
// the row and its carry; the high word is updated only for a nonzero high
// part), and lightly loaded tables are probed first at the key's exact home
// slot (4 bytes) before the bucket.
// Rows are handled in batches: all lookups first, then all count updates,
// all sum updates and all min/max updates, so that shared-memory latencies
// overlap instead of forming one dependent chain per row.
template <int DT> struct SImg { using U = uint32_t; };
template <> struct SImg<AGG_I64> { using U = unsigned long long; };
template <> struct SImg<AGG_F64> { using U = unsigned long long; };

template <int DT>
__device__ __forceinline__ typename SImg<DT>::U s_img(typename GV<DT>::T v) {
  if (DT == AGG_I32) return (uint32_t)(int32_t)v ^ 0x80000000u;
  if (DT == AGG_U32) return (uint32_t)v;
  if (DT == AGG_F32) return img_f32((float)v);
  if (DT == AGG_I64) return (unsigned long long)img_i64((int64_t)v);
  return (unsigned long long)img_f64((double)v);
}
// shared image -> the 64-bit image kept in the global table (GV<DT>::img)
template <int DT>
__device__ __forceinline__ uint64_t g_img_of(typename SImg<DT>::U m) {
  if (DT == AGG_I32) return img_i64((int64_t)(int32_t)((uint32_t)m ^ 0x80000000u));
  if (DT == AGG_U32) return img_i64((int64_t)(uint32_t)m);
  return (uint64_t)m;
}

template <int DT, bool MM>
struct STab {
  using U = typename SImg<DT>::U;
  unsigned long long* sum;  // 64-bit word per slot (two u32 halves for integers / float32)
  U* mm;                    // (min, max) image pairs
  uint32_t* key1;           // key + 1, 0 = empty (16-byte aligned)
  uint32_t* cnt;
  int* used;
  __device__ void carve(unsigned char* base, int S) {
    sum = (unsigned long long*)base;
    unsigned char* p = (unsigned char*)(sum + (S + 1));
    p = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    if (MM) {
      mm = (U*)p;
      p = (unsigned char*)(mm + 2 * (S + 1));
      p = (unsigned char*)(((uintptr_t)p + 15) & ~(uintptr_t)15);
    }
    key1 = (uint32_t*)p;
    cnt = key1 + (S + 4);
    used = (int*)(cnt + (S + 1));
  }
  __device__ void clear(int S) {
    for (int i = threadIdx.x; i <= S; i += blockDim.x) {
      sum[i] = 0;
      if (MM) {
        mm[2 * i] = (U)~(U)0;
        mm[2 * i + 1] = 0;
      }
      cnt[i] = 0;
    }
    for (int i = threadIdx.x; i < S + 4; i += blockDim.x) key1[i] = 0;
    if (threadIdx.x == 0) *used = 0;
  }
};

template <int DT, bool MM>
__host__ __device__ inline size_t stab_bytes(int S) {
  const size_t img = (DT == AGG_I64 || DT == AGG_F64) ? 8 : 4;
  return ((size_t)(S + 1) * 8 + 16 + (MM ? 2 * img * (S + 1) + 16 : 0) + (size_t)(S + 4) * 4 +
          (size_t)(S + 1) * 4 + 16 + 15) & ~size_t(15);
}
// Shared memory of a tile build: the table, and for int64 MIN/MAX the 32-bit
// (min, max) pairs after it.
template <int DT, bool MM>
__host__ __device__ inline size_t tile_smem_bytes(int S) {
  return stab_bytes<DT, MM>(S) + (MM && DT == AGG_I64 ? (size_t)(S + 1) * 8 : 0);
}

constexpr int kSmemBuckets = 4;  // buckets of 4 slots probed before a row spills

// Shared-memory vector loads that are re-issued every time (values written by
// other threads may change). A stale value is harmless for every use below:
// keys only go from empty to set, minima only fall and maxima only rise.
__device__ __forceinline__ uint4 lds_v4(const void* p) {
  uint4 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.volatile.shared.v4.u32 {%0,%1,%2,%3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
  return v;
}
__device__ __forceinline__ uint2 lds_v2(const void* p) {
  uint2 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.volatile.shared.v2.u32 {%0,%1}, [%2];" : "=r"(v.x), "=r"(v.y) : "r"(a));
  return v;
}
__device__ __forceinline__ ulonglong2 lds_v2_64(const void* p) {
  ulonglong2 v;
  const unsigned a = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ld.volatile.shared.v2.u64 {%0,%1}, [%2];" : "=l"(v.x), "=l"(v.y) : "r"(a));
  return v;
}

// Fast path: the key's slot if it sits in its home bucket, else -1 (one
// 16-byte shared load, no branches on the data). HOME: first one 4-byte load
// of the key's home slot, where the insert puts it when that slot is free: a
// lightly loaded table (a partitioned tile's few keys) then mostly needs only
// that load; a table at load 1/2 loses more to the second load than it saves.
template <int DT, bool MM, bool HOME = false>
__device__ __forceinline__ int s_find_home(const STab<DT, MM>& t, int S, uint32_t key) {
  const uint32_t k1 = key + 1;
  const uint32_t hs = fmix32(key) & (uint32_t)(S - 1);
  if (HOME && key != 0xFFFFFFFFu && *(volatile uint32_t*)&t.key1[hs] == k1) return (int)hs;
  const uint32_t b = hs & ~3u;
  const uint4 q = lds_v4(&t.key1[b]);
  int j = -1;
  j = q.w == k1 ? (int)b + 3 : j;
  j = q.z == k1 ? (int)b + 2 : j;
  j = q.y == k1 ? (int)b + 1 : j;
  j = q.x == k1 ? (int)b : j;
  return key == 0xFFFFFFFFu ? S : j;
}

// Slot of key in the shared table (inserting it if there is room), or -1.
// HOME: a new key takes its home slot when that is free (for the HOME fast
// path of s_find_home), else the bucket's first free slot. The two orders are
// separate instances: the plain build measured twice as slow with the
// home-first code in its (rarely taken) insert path, the tile build faster.
template <int DT, bool MM, bool HOME = false>
__device__ __noinline__ int s_lookup(const STab<DT, MM>& t, int S, int cap, uint32_t key) {
  if (key == 0xFFFFFFFFu) return S;
  const uint32_t k1 = key + 1;
  uint32_t b = fmix32(key) & (uint32_t)(S - 1) & ~3u;
#pragma unroll 1
  for (int p = 0; p < kSmemBuckets; ++p) {
    uint4 q = lds_v4(&t.key1[b]);
    if (q.x == k1) return (int)b;
    if (q.y == k1) return (int)b + 1;
    if (q.z == k1) return (int)b + 2;
    if (q.w == k1) return (int)b + 3;
    // claim an empty slot of this bucket (HOME: in the first bucket, the key's
    // home slot first); each failed claim fills a slot, so this loop runs at
    // most 4 times
    const uint32_t h0 = HOME && p == 0 ? (fmix32(key) & 3u) : 0u;
#pragma unroll 1
    for (int tries = 0; tries < 4; ++tries) {
      int e;
      if (HOME) {  // empty slots as a 4-bit mask, rotated so that bit 0 is position h0
        const uint32_t em =
            (q.x == 0u ? 1u : 0u) | (q.y == 0u ? 2u : 0u) | (q.z == 0u ? 4u : 0u) | (q.w == 0u ? 8u : 0u);
        const uint32_t rot = ((em >> h0) | (em << (4u - h0))) & 15u;
        e = rot ? (int)((h0 + (uint32_t)(__ffs(rot) - 1)) & 3u) : -1;
      } else {
        e = q.x == 0 ? 0 : q.y == 0 ? 1 : q.z == 0 ? 2 : q.w == 0 ? 3 : -1;
      }
      if (e < 0) break;
      if (*(volatile int*)t.used >= cap) return -1;  // full enough: no new keys
      const uint32_t old = atomicCAS(&t.key1[b + e], 0u, k1);
      if (old == 0u) {
        atomicAdd(t.used, 1);
        return (int)b + e;
      }
      if (old == k1) return (int)b + e;
      q = lds_v4(&t.key1[b]);
      if (q.x == k1) return (int)b;
      if (q.y == k1) return (int)b + 1;
      if (q.z == k1) return (int)b + 2;
      if (q.w == k1) return (int)b + 3;
    }
    b = (b + 4) & (uint32_t)(S - 1);
  }
  return -1;
}

// Fold a row into the global table. MIN/MAX atomics are skipped when the
// value does not improve the slot's current extreme.
template <int DT, bool MM>
__device__ __forceinline__ void g_add_row_cached(GSlot<MM>& s, typename GV<DT>::T v) {
  atomicAdd(&s.cnt, 1u);
  if (DT == AGG_F32 || DT == AGG_F64) {
    atomicAdd((double*)&s.sum, (double)v);
  } else {
    atomicAdd(&s.sum, (unsigned long long)(int64_t)v);
  }
  if (MM) {
    GSlot<true>& w = (GSlot<true>&)s;
    const uint64_t m = GV<DT>::img(v);
    if (~m > *(volatile unsigned long long*)&w.minc) atomicMax(&w.minc, (unsigned long long)~m);
    if (m > *(volatile unsigned long long*)&w.mx) atomicMax(&w.mx, (unsigned long long)m);
  }
}

// Count rows that found no global slot in the block's shared counter.
__device__ __forceinline__ void note_fail(const BuildArgs& a, uint32_t rows) {
  *(volatile int*)a.status = kStatusFull;
  if (a.block_fails) atomicAdd(a.block_fails, rows);
}

// Fold a row into the global table. Once a row of this block found the table
// full, rows probe only kShortProbe slots: the build is redone, and the rows
// folded before the block notices should not each walk the whole probe bound.
constexpr int kShortProbe = 8;

template <int DT, bool MM>
__device__ __forceinline__ void g_row(const BuildArgs& a, uint32_t key, typename GV<DT>::T v) {
  GSlot<MM>* tab = (GSlot<MM>*)a.table;
  const bool met_full = a.block_fails && *(volatile uint32_t*)a.block_fails != 0;
  const int64_t g = g_slot<MM>(tab, a.mask, a.gshift, key, met_full ? kShortProbe : kGlobalProbe);
  if (g < 0) {
    note_fail(a, 1);
    return;
  }
  g_add_row_cached<DT, MM>(tab[g], v);
}

// Fold a batch of N rows (valid[r] false = skip).
template <int DT, bool MM, bool SMEM, int N, bool HOME = false, bool PACK = false, bool M32 = false>
__device__ __forceinline__ void fold_batch(const BuildArgs& a, const STab<DT, MM>& st, const uint32_t (&key)[N],
                                           const typename GV<DT>::T (&val)[N], const bool (&valid)[N]) {
  using T = typename GV<DT>::T;
  using U = typename SImg<DT>::U;
  if (!SMEM) {
#pragma unroll
    for (int r = 0; r < N; ++r)
      if (valid[r]) g_row<DT, MM>(a, key[r], val[r]);
    return;
  }
  int j[N];
#pragma unroll
  for (int r = 0; r < N; ++r) j[r] = valid[r] ? s_find_home<DT, MM, HOME>(st, a.smem_slots, key[r]) : -2;
#pragma unroll
  for (int r = 0; r < N; ++r)
    if (j[r] == -1) j[r] = s_lookup<DT, MM, HOME>(st, a.smem_slots, a.smem_cap, key[r]);
  constexpr bool kPack = PACK && DT != AGG_F32 && DT != AGG_F64;
  if (!kPack) {
#pragma unroll
    for (int r = 0; r < N; ++r)
      if (j[r] >= 0) atomicAdd(&st.cnt[j[r]], 1u);
  }
  if (DT == AGG_F32) {
    float old[N];
#pragma unroll
    for (int r = 0; r < N; ++r)
      if (j[r] >= 0) old[r] = atomicAdd((float*)&st.sum[j[r]], (float)val[r]);
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (j[r] >= 0) {
        float t, e;
        two_sum(old[r], (float)val[r], t, e);  // t is what the atomic stored; e its rounding error
        if (e != 0.f) atomicAdd((float*)&st.sum[j[r]] + 1, e);
      }
    }
  } else if (DT == AGG_F64) {
#pragma unroll
    for (int r = 0; r < N; ++r)
      if (j[r] >= 0) atomicAdd((double*)&st.sum[j[r]], (double)val[r]);
  } else {
    uint32_t old[N];
#pragma unroll
    for (int r = 0; r < N; ++r)
      if (j[r] >= 0) old[r] = atomicAdd((uint32_t*)&st.sum[j[r]], (uint32_t)(uint64_t)(int64_t)val[r]);
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (j[r] >= 0) {
        const uint64_t u = (uint64_t)(int64_t)val[r];
        const uint32_t lo = (uint32_t)u;
        const uint32_t carry = (uint32_t)(old[r] + lo) < old[r] ? 1u : 0u;
        if (kPack) {  // the count and the carry in one word; the high part only when nonzero
          atomicAdd(&st.cnt[j[r]], 1u + (carry << 16));
          if ((uint32_t)(u >> 32)) atomicAdd((uint32_t*)&st.sum[j[r]] + 1, (uint32_t)(u >> 32));
        } else {
          const uint32_t hi = (uint32_t)(u >> 32) + carry;
          if (hi) atomicAdd((uint32_t*)&st.sum[j[r]] + 1, hi);
        }
      }
    }
  }
  if (MM && M32 && DT == AGG_I64) {
    // a value whose image shares the tile's (block's) high word is checked
    // and applied on the 32-bit (min, max) pair of its low words (8 bytes
    // instead of 16, native 32-bit atomics); others on the 64-bit pair
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (j[r] >= 0) {
        const U m = s_img<DT>(val[r]);
        if ((uint32_t)((uint64_t)m >> 32) == a.tile_hi) {
          const uint32_t ml = (uint32_t)m;
          const uint2 q = lds_v2(&a.mm32[2 * j[r]]);
          if (ml < q.x) atomicMin(&a.mm32[2 * j[r]], ml);
          if (ml > q.y) atomicMax(&a.mm32[2 * j[r] + 1], ml);
        } else {
          const ulonglong2 q = lds_v2_64(&st.mm[2 * j[r]]);
          if (m < (U)q.x) atomicMin(&st.mm[2 * j[r]], m);
          if (m > (U)q.y) atomicMax(&st.mm[2 * j[r] + 1], m);
        }
      }
    }
  } else if (MM) {
    U cur_mn[N], cur_mx[N];
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (j[r] >= 0) {
        if (sizeof(U) == 4) {
          const uint2 q = lds_v2(&st.mm[2 * j[r]]);
          cur_mn[r] = (U)q.x;
          cur_mx[r] = (U)q.y;
        } else {
          const ulonglong2 q = lds_v2_64(&st.mm[2 * j[r]]);
          cur_mn[r] = (U)q.x;
          cur_mx[r] = (U)q.y;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < N; ++r) {
      if (j[r] >= 0) {
        const U m = s_img<DT>(val[r]);
        if (m < cur_mn[r]) atomicMin(&st.mm[2 * j[r]], m);
        if (m > cur_mx[r]) atomicMax(&st.mm[2 * j[r] + 1], m);
      }
    }
  }
#pragma unroll
  for (int r = 0; r < N; ++r)
    if (j[r] == -1) g_row<DT, MM>(a, key[r], val[r]);
}

// ---------------------------------------------------------------------------
// Frequent keys: when at least kDominantRows of the 128 rows a warp holds
// carry one key (hot keys of a skewed, partitioned or clustered input, or a
// column with a handful of keys), the warp reduces those rows with shuffles
// and applies one partial aggregate; the remaining rows take the per-row path.
// This removes the same-slot atomic conflicts that frequent keys cause.
// ---------------------------------------------------------------------------
constexpr int kDominantRows = 8;  // rows of one key (of 128) that make a reduced update pay
constexpr int kMaxWarpKeys = 8;   // keys reduced per warp and quad of rows, at most
template <int DT>
struct Partial4 {  // partial aggregate of rows with one key
  uint32_t cnt;
  unsigned long long isum;  // integer sum mod 2^64
  float fs, fc;             // float32: compensated pair
  double ds;                // float64 sum
  typename SImg<DT>::U mn, mx;
};

template <int DT, bool MM>
__device__ __forceinline__ Partial4<DT> partial_of(const typename GV<DT>::T (&v)[4], uint32_t take) {
  Partial4<DT> p;
  p.cnt = 0;
  p.isum = 0;
  p.fs = 0.f;
  p.fc = 0.f;
  p.ds = 0.0;
  p.mn = (typename SImg<DT>::U) ~(typename SImg<DT>::U)0;
  p.mx = 0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    if (!((take >> r) & 1u)) continue;
    p.cnt += 1;
    if (DT == AGG_F32) {
      float t, e;
      two_sum(p.fs, (float)v[r], t, e);
      p.fs = t;
      p.fc += e;
    } else if (DT == AGG_F64) {
      p.ds += (double)v[r];
    } else {
      p.isum += (unsigned long long)(int64_t)v[r];
    }
    if (MM) {
      const typename SImg<DT>::U m = s_img<DT>(v[r]);
      p.mn = min(p.mn, m);
      p.mx = max(p.mx, m);
    }
  }
  return p;
}

template <int DT, bool MM>
__device__ __forceinline__ void warp_reduce_partial(Partial4<DT>& p) {
  if (DT == AGG_I32 || DT == AGG_U32 || DT == AGG_I64) {
    // integers: warp reductions of 32-bit words. The sum mod 2^64 from the
    // low word's two 16-bit halves (each total below 2^21) and the high word
    // (mod 2^32); a 64-bit minimum from the high words' minimum, then the low
    // words of the lanes holding it (likewise the maximum).
    constexpr unsigned kAll = 0xffffffffu;
    p.cnt = __reduce_add_sync(kAll, p.cnt);
    const uint32_t lo = (uint32_t)p.isum;
    const uint32_t s0 = __reduce_add_sync(kAll, lo & 0xFFFFu);
    const uint32_t s1 = __reduce_add_sync(kAll, lo >> 16);
    const uint32_t sh = __reduce_add_sync(kAll, (uint32_t)(p.isum >> 32));
    p.isum = ((unsigned long long)sh << 32) + ((unsigned long long)s1 << 16) + (unsigned long long)s0;
    if (MM) {
      if (sizeof(p.mn) == 4) {
        p.mn = __reduce_min_sync(kAll, (uint32_t)p.mn);
        p.mx = __reduce_max_sync(kAll, (uint32_t)p.mx);
      } else {
        const uint64_t mn = (uint64_t)p.mn, mx = (uint64_t)p.mx;
        const uint32_t mnh = __reduce_min_sync(kAll, (uint32_t)(mn >> 32));
        const uint32_t mnl = __reduce_min_sync(kAll, (uint32_t)(mn >> 32) == mnh ? (uint32_t)mn : 0xFFFFFFFFu);
        const uint32_t mxh = __reduce_max_sync(kAll, (uint32_t)(mx >> 32));
        const uint32_t mxl = __reduce_max_sync(kAll, (uint32_t)(mx >> 32) == mxh ? (uint32_t)mx : 0u);
        p.mn = (typename SImg<DT>::U)(((uint64_t)mnh << 32) | mnl);
        p.mx = (typename SImg<DT>::U)(((uint64_t)mxh << 32) | mxl);
      }
    }
    return;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    p.cnt += __shfl_xor_sync(0xffffffffu, p.cnt, o);
    if (DT == AGG_F32) {
      const float s2 = __shfl_xor_sync(0xffffffffu, p.fs, o), c2 = __shfl_xor_sync(0xffffffffu, p.fc, o);
      float t, e;
      two_sum(p.fs, s2, t, e);
      p.fs = t;
      p.fc += c2 + e;
    } else if (DT == AGG_F64) {
      p.ds += __shfl_xor_sync(0xffffffffu, p.ds, o);
    } else {
      p.isum += __shfl_xor_sync(0xffffffffu, p.isum, o);
    }
    if (MM) {
      p.mn = min(p.mn, __shfl_xor_sync(0xffffffffu, p.mn, o));
      p.mx = max(p.mx, __shfl_xor_sync(0xffffffffu, p.mx, o));
    }
  }
}

// Apply a partial aggregate to a shared slot (same encodings as s_add via fold_batch).
template <int DT, bool MM, bool PACK = false, bool M32 = false>
__device__ __forceinline__ void s_add_partial(const BuildArgs& a, const STab<DT, MM>& st, int j,
                                              const Partial4<DT>& p) {
  using U = typename SImg<DT>::U;
  constexpr bool kPack = PACK && DT != AGG_F32 && DT != AGG_F64;
  if (!kPack) atomicAdd(&st.cnt[j], p.cnt);
  uint32_t* w = (uint32_t*)&st.sum[j];
  if (DT == AGG_F32) {
    const float old = atomicAdd((float*)&w[0], p.fs);
    float t, e;
    two_sum(old, p.fs, t, e);
    const float c = e + p.fc;
    if (c != 0.f) atomicAdd((float*)&w[1], c);
  } else if (DT == AGG_F64) {
    atomicAdd((double*)&st.sum[j], p.ds);
  } else {
    const uint32_t lo = (uint32_t)p.isum;
    const uint32_t old = atomicAdd(&w[0], lo);
    const uint32_t carry = (uint32_t)(old + lo) < old ? 1u : 0u;
    if (kPack) {
      atomicAdd(&st.cnt[j], p.cnt + (carry << 16));
      if ((uint32_t)(p.isum >> 32)) atomicAdd(&w[1], (uint32_t)(p.isum >> 32));
    } else {
      const uint32_t hi = (uint32_t)(p.isum >> 32) + carry;
      if (hi) atomicAdd(&w[1], hi);
    }
  }
  if (MM && M32 && DT == AGG_I64 && (uint32_t)((uint64_t)p.mn >> 32) == a.tile_hi &&
      (uint32_t)((uint64_t)p.mx >> 32) == a.tile_hi) {  // both bounds on the 32-bit pair (see fold_batch)
    const uint32_t mnl = (uint32_t)p.mn, mxl = (uint32_t)p.mx;
    if (mnl < *(volatile uint32_t*)&a.mm32[2 * j]) atomicMin(&a.mm32[2 * j], mnl);
    if (mxl > *(volatile uint32_t*)&a.mm32[2 * j + 1]) atomicMax(&a.mm32[2 * j + 1], mxl);
  } else if (MM) {
    if (p.mn < *(volatile U*)&st.mm[2 * j]) atomicMin(&st.mm[2 * j], p.mn);
    if (p.mx > *(volatile U*)&st.mm[2 * j + 1]) atomicMax(&st.mm[2 * j + 1], p.mx);
  }
}

template <int DT, bool MM>
__device__ __forceinline__ void g_add_partial(const BuildArgs& a, uint32_t key, const Partial4<DT>& p) {
  GSlot<MM>* tab = (GSlot<MM>*)a.table;
  const int64_t g = g_slot<MM>(tab, a.mask, a.gshift, key);
  if (g < 0) {
    note_fail(a, p.cnt);
    return;
  }
  GSlot<MM>& gs = tab[g];
  atomicAdd(&gs.cnt, p.cnt);
  if (DT == AGG_F32) atomicAdd((double*)&gs.sum, (double)p.fs + (double)p.fc);
  else if (DT == AGG_F64) atomicAdd((double*)&gs.sum, p.ds);
  else atomicAdd(&gs.sum, p.isum);
  if (MM) {
    GSlot<true>& w = (GSlot<true>&)gs;
    const uint64_t mn = g_img_of<DT>(p.mn), mx = g_img_of<DT>(p.mx);
    if (~mn > *(volatile unsigned long long*)&w.minc) atomicMax(&w.minc, (unsigned long long)~mn);
    if (mx > *(volatile unsigned long long*)&w.mx) atomicMax(&w.mx, (unsigned long long)mx);
  }
}

// The warp reduces the rows marked in take (a 4-bit mask per lane; all of
// one key) and lane 0 folds the partial into the tables.
template <int DT, bool MM, bool SMEM, bool HOME = false, bool PACK = false, bool M32 = false>
__device__ __forceinline__ void fold_warp_key(const BuildArgs& a, const STab<DT, MM>& st, uint32_t key,
                                              const typename GV<DT>::T (&v)[4], uint32_t take) {
  Partial4<DT> p = partial_of<DT, MM>(v, take);
  warp_reduce_partial<DT, MM>(p);
  if ((threadIdx.x & 31) != 0) return;
  if (SMEM) {
    int j = s_find_home<DT, MM, HOME>(st, a.smem_slots, key);
    if (j < 0) j = s_lookup<DT, MM, HOME>(st, a.smem_slots, a.smem_cap, key);
    if (j >= 0) {
      s_add_partial<DT, MM, PACK, M32>(a, st, j, p);
      return;
    }
  }
  g_add_partial<DT, MM>(a, key, p);
}

template <class T>
__device__ __forceinline__ void unpack4(const uint4& lo, const uint4& hi, T* v) {
  if (sizeof(T) == 4) {
    uint32_t w[4] = {lo.x, lo.y, lo.z, lo.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      uint32_t x = w[i];
      memcpy(&v[i], &x, 4);
    }
  } else {
    uint64_t w[4] = {((uint64_t)lo.y << 32) | lo.x, ((uint64_t)lo.w << 32) | lo.z, ((uint64_t)hi.y << 32) | hi.x,
                     ((uint64_t)hi.w << 32) | hi.z};
#pragma unroll
    for (int i = 0; i < 4; ++i) memcpy(&v[i], &w[i], 8);
  }
}

// Per-block counts reported after a build: when a full table stopped it, the
// rows the block went through and those that found no slot are added to
// a.progress, from which the host sizes the next table. Call after a barrier
// that follows every thread's count_seen.
struct BlockCounts {
  uint32_t seen, fails;
};

__device__ __forceinline__ void report_counts(const BuildArgs& a, const BlockCounts& c) {
  if (threadIdx.x != 0 || a.progress == nullptr || *(volatile int*)a.status == 0) return;
  atomicAdd(&a.progress[0], (unsigned long long)c.seen);
  atomicAdd(&a.progress[1], (unsigned long long)c.fails);
}

// Rows [0, a.n) of a column folded by threads tid, tid + nthreads, ...
// VEC: 16-byte vector loads of 4 keys and 4 values per quad, QPI quads per
// thread per iteration (all loads issued before any row is folded): 4 or 8
// rows a thread per iteration, the autotuner's items-per-thread axis.

// Returns the number of rows this thread went through (the vector body's).
// MULTI: up to kMaxWarpKeys frequent keys per warp and quad of rows get a
// reduced update (columns with a handful of keys or hot keys); without it
// every row takes the per-row path (for columns whose sketch shows no
// frequent key: the warp then never waits for its slowest lane).
template <int DT, bool MM, bool SMEM, bool VEC, bool MULTI = true, int QPI = 1, bool HOME = false,
          bool PACK = false, bool M32 = false>
__device__ __forceinline__ uint32_t build_rows(const BuildArgs& a, const STab<DT, MM>& st, int64_t tid,
                                               int64_t nthreads) {
  constexpr int kQuadsPerIter = QPI;
  using T = typename GV<DT>::T;
  const uint32_t* keys = a.keys;
  const T* vals = (const T*)a.vals;
  if (VEC) {
    const int64_t nq = (a.n - a.head) / 4;  // full quads of rows
    const int64_t tail0 = a.head + nq * 4;
    {
      uint32_t k1[1];
      T v1[1];
      bool ok1[1];
      ok1[0] = tid < a.head;
      k1[0] = ok1[0] ? keys[tid] : 0u;
      v1[0] = ok1[0] ? vals[tid] : T(0);
      fold_batch<DT, MM, SMEM, 1, HOME, PACK, M32>(a, st, k1, v1, ok1);
      ok1[0] = tid < a.n - tail0;
      k1[0] = ok1[0] ? keys[tail0 + tid] : 0u;
      v1[0] = ok1[0] ? vals[tail0 + tid] : T(0);
      fold_batch<DT, MM, SMEM, 1, HOME, PACK, M32>(a, st, k1, v1, ok1);
    }
    const uint4* kq = (const uint4*)(keys + a.head);
    const uint4* vq = (const uint4*)(vals + a.head);
    constexpr int VPQ = sizeof(T) == 4 ? 1 : 2;  // 16-byte value vectors per quad
    // The loop runs per warp: its condition is the warp's first quad, so all
    // 32 lanes stay in every iteration (lanes past the end have has = false)
    // and the warp-wide reductions below see the whole warp. tid and nthreads
    // are multiples of 32 apart within a warp (blocks of whole warps).
    const int lane = (int)(tid & 31);
    int it = 0;
    for (int64_t qw = tid - lane; qw < nq; qw += kQuadsPerIter * nthreads) {
      const int64_t q = qw + lane;
      uint4 kk[kQuadsPerIter], va[kQuadsPerIter], vb[kQuadsPerIter];
      bool has[kQuadsPerIter];
#pragma unroll
      for (int u = 0; u < kQuadsPerIter; ++u) {  // issue every load of the iteration first
        const int64_t qu = q + u * nthreads;
        has[u] = qu < nq;
        kk[u] = has[u] ? ld_stream_v4(kq + qu) : make_uint4(0, 0, 0, 0);
        va[u] = has[u] ? ld_stream_v4(vq + qu * VPQ) : make_uint4(0, 0, 0, 0);
        vb[u] = (has[u] && VPQ == 2) ? ld_stream_v4(vq + qu * VPQ + 1) : va[u];
      }
#pragma unroll
      for (int u = 0; u < kQuadsPerIter; ++u) {
        const uint32_t key[4] = {kk[u].x, kk[u].y, kk[u].z, kk[u].w};
        T val[4];
        unpack4<T>(va[u], vb[u], val);
        // Frequent keys among the warp's 128 rows go through one reduced
        // update each: first the key of lane 0's first row; while a key had
        // at least kDominantRows rows, the next candidate is the first row not
        // yet folded. The remaining rows take the per-row path.
        uint32_t rem = has[u] ? 0xFu : 0u;  // this lane's rows not yet folded
        if (MULTI) {  // every lane of the warp is here (lane 0 always has rows)
          uint32_t k0 = __shfl_sync(0xffffffffu, key[0], 0);
          constexpr int kKeys = kMaxWarpKeys;
#pragma unroll 1
          for (int w = 0; w < kKeys; ++w) {
            uint32_t take = 0;
#pragma unroll
            for (int r = 0; r < 4; ++r) take |= (((rem >> r) & 1u) && key[r] == k0) ? (1u << r) : 0u;
            if (__reduce_add_sync(0xffffffffu, (unsigned)__popc(take)) < (unsigned)kDominantRows) break;
            fold_warp_key<DT, MM, SMEM, HOME, PACK, M32>(a, st, k0, val, take);
            rem &= ~take;
            if (w + 1 == kKeys) break;
            const uint32_t lanes = __ballot_sync(0xffffffffu, rem != 0u);
            if (lanes == 0u) break;
            uint32_t next = key[3];  // this lane's first row not yet folded
            if (rem & 4u) next = key[2];
            if (rem & 2u) next = key[1];
            if (rem & 1u) next = key[0];
            k0 = __shfl_sync(0xffffffffu, next, __ffs(lanes) - 1);
          }
          if (rem == 0u) continue;  // this lane's rows are all folded
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          uint32_t kb[1] = {key[r]};
          T vv[1] = {val[r]};
          bool ok[1] = {((rem >> r) & 1u) != 0u};
          fold_batch<DT, MM, SMEM, 1, HOME, PACK, M32>(a, st, kb, vv, ok);
        }
      }
      // table full: the build is redone (status read by lane 0, so the whole warp leaves)
      if ((++it & 15) == 0 && __shfl_sync(0xffffffffu, lane == 0 ? *(volatile int*)a.status : 0, 0)) break;
    }
    return (uint32_t)it * 4u * kQuadsPerIter;
  } else {
    int it = 0;
    for (int64_t i = tid; i < a.n; i += nthreads) {
      uint32_t k1[1] = {keys[i]};
      T v1[1] = {vals[i]};
      bool ok1[1] = {true};
      fold_batch<DT, MM, SMEM, 1, HOME, PACK, M32>(a, st, k1, v1, ok1);
      if ((++it & 63) == 0 && *(volatile int*)a.status) break;
    }
    return (uint32_t)it;
  }
}

// Merge a block's shared table into the global table (after a barrier).
template <int DT, bool MM, bool PACK = false, bool M32 = false>
__device__ __forceinline__ void flush_smem(const BuildArgs& a, const STab<DT, MM>& st) {
  constexpr bool kPack = PACK && DT != AGG_F32 && DT != AGG_F64;
  GSlot<MM>* tab = (GSlot<MM>*)a.table;
  const int S = a.smem_slots;
  for (int j = threadIdx.x; j <= S; j += blockDim.x) {
    const uint32_t w = st.cnt[j];
    if (w == 0) continue;
    const uint32_t c = kPack ? (w & 0xFFFFu) : w;  // PACK: count, and the low word's carries above it
    const uint32_t key = j == S ? 0xFFFFFFFFu : st.key1[j] - 1;
    const int64_t g = g_slot<MM>(tab, a.mask, a.gshift, key);
    if (g < 0) {
      note_fail(a, c);
      continue;
    }
    GSlot<MM>& gs = tab[g];
    atomicAdd(&gs.cnt, c);
    const unsigned long long sv = st.sum[j];
    if (DT == AGG_F32) {
      const double d = (double)__uint_as_float((uint32_t)sv) + (double)__uint_as_float((uint32_t)(sv >> 32));
      atomicAdd((double*)&gs.sum, d);
    } else if (DT == AGG_F64) {
      atomicAdd((double*)&gs.sum, __longlong_as_double((long long)sv));
    } else {
      atomicAdd(&gs.sum, kPack ? sv + ((unsigned long long)(w >> 16) << 32) : sv);
    }
    if (MM) {
      GSlot<true>& gw = (GSlot<true>&)gs;
      uint64_t mn = g_img_of<DT>(st.mm[2 * j]), mx = g_img_of<DT>(st.mm[2 * j + 1]);
      if (M32 && DT == AGG_I64) {
        // the 32-bit pair took at least one update iff its min is at most its max
        const uint32_t lo = a.mm32[2 * j], hi = a.mm32[2 * j + 1];
        if (lo <= hi) {
          mn = min(mn, ((uint64_t)a.tile_hi << 32) | lo);
          mx = max(mx, ((uint64_t)a.tile_hi << 32) | hi);
        }
      }
      if (~mn > *(volatile unsigned long long*)&gw.minc) atomicMax(&gw.minc, (unsigned long long)~mn);
      if (mx > *(volatile unsigned long long*)&gw.mx) atomicMax(&gw.mx, (unsigned long long)mx);
    }
  }
}

// The build kernel of one query: grid-stride over all rows.
template <int DT, bool MM, bool SMEM, bool VEC, bool MULTI, int QPI = 1>
__global__ void __launch_bounds__(512, 2) gb_build(BuildArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ BlockCounts s_cnt;
  __shared__ uint32_t s_hi;
  if (threadIdx.x == 0) s_cnt = BlockCounts{0u, 0u};
  a.block_fails = &s_cnt.fails;
  STab<DT, MM> st;
  // int64 MIN/MAX: the 32-bit (min, max) pairs after the table, for values
  // sharing the high word of one row the block reads first
  constexpr bool kMM32 = SMEM && MM && DT == AGG_I64;
  if (SMEM) {
    st.carve(smem, a.smem_slots);
    st.clear(a.smem_slots);
  }
  if (kMM32) {
    a.mm32 = (uint32_t*)(smem + stab_bytes<DT, MM>(a.smem_slots));
    for (int i = threadIdx.x; i <= a.smem_slots; i += blockDim.x) {
      a.mm32[2 * i] = 0xFFFFFFFFu;
      a.mm32[2 * i + 1] = 0u;
    }
    if (threadIdx.x == 0) {
      const int64_t r = a.n > 0 ? min((int64_t)blockIdx.x * blockDim.x * 4, a.n - 1) : 0;
      s_hi = a.n > 0 ? (uint32_t)((uint64_t)s_img<DT>(((const typename GV<DT>::T*)a.vals)[r]) >> 32) : 0u;
    }
  }
  __syncthreads();
  if (kMM32) a.tile_hi = s_hi;
  const uint32_t seen = build_rows<DT, MM, SMEM, VEC, MULTI, QPI, false, false, kMM32>(
      a, st, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
  atomicAdd(&s_cnt.seen, seen);
  if (SMEM) {
    __syncthreads();
    flush_smem<DT, MM, false, kMM32>(a, st);
  }
  __syncthreads();
  report_counts(a, s_cnt);
}

// Tile-queue build for hash-partitioned input: blocks pull tiles of up to
// 65532 rows in order from a counter, so all blocks work on neighbouring partitions and the
// table region they update stays in L2; each tile clears its shared table
// first and merges it into the global table at the end. With a tile list
// (rows partitioned chunk by chunk), tile t is the row range tiles[t] =
// (first row, rows), *ntiles of them, listed partition by partition.
constexpr int64_t kPartTileRows = int64_t(1) << 16;
// Integer sums in a tile build keep a slot's count and its low word's carries
// in the two 16-bit halves of one shared word (one atomic instead of two), so
// a tile has at most 65532 rows (a multiple of 4).
constexpr int64_t kTileRowsMax = 65532;

// Blocks a SM the tile build is compiled for: float32 sums without MIN/MAX
// (a 4096-slot table of 16-byte slots, compare-and-swap loops for the float
// atomics) run three, at 40 registers (the 2^28-row Zipf build: 4.15 -> 3.41
// ms); the integer and MIN/MAX builds keep two at 64 registers (three cost
// them 40 %).
template <int DT, bool MM>
struct TileBlocks {
  static constexpr int kValue = DT == AGG_F32 && !MM ? 3 : 2;
};

template <int DT, bool MM, bool VEC, int QPI = 1, bool HOME = false>
__global__ void __launch_bounds__(512, TileBlocks<DT, MM>::kValue) gb_build_tiles(BuildArgs a, unsigned long long* next_tile,
                                                        int64_t tile_rows, const longlong2* tiles,
                                                        const unsigned long long* ntiles) {
  using T = typename GV<DT>::T;
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int64_t s_t;
  __shared__ BlockCounts s_cnt;
  if (threadIdx.x == 0) s_cnt = BlockCounts{0u, 0u};
  a.block_fails = &s_cnt.fails;
  STab<DT, MM> st;
  st.carve(smem, a.smem_slots);
  constexpr bool kMM32 = MM && DT == AGG_I64;
  __shared__ uint32_t s_hi;
  if (kMM32) a.mm32 = (uint32_t*)(smem + stab_bytes<DT, MM>(a.smem_slots));  // after the table (16-byte aligned)
  for (;;) {
    // no new tile once the table is full (the build is redone with a larger one)
    if (threadIdx.x == 0) s_t = *(volatile int*)a.status ? -1 : (int64_t)atomicAdd(next_tile, 1ull);
    __syncthreads();
    const int64_t t = s_t;
    __syncthreads();
    int64_t r0, rows;
    if (tiles) {
      if (t < 0 || t >= (int64_t)*ntiles) break;
      const longlong2 tl = tiles[t];
      r0 = tl.x;
      rows = tl.y;
    } else {
      r0 = t * tile_rows;
      if (t < 0 || r0 >= a.n) break;
      rows = min(tile_rows, a.n - r0);
    }
    BuildArgs b = a;
    b.keys = a.keys + r0;
    b.vals = (const T*)a.vals + r0;
    b.n = rows;
    b.head = min((int64_t)((-r0) & 3), rows);  // rows before the next 16-byte boundary of the keys
    st.clear(a.smem_slots);
    if (kMM32) {  // the tile's high word: that of its first row's image
      for (int i = threadIdx.x; i <= a.smem_slots; i += blockDim.x) {
        b.mm32[2 * i] = 0xFFFFFFFFu;
        b.mm32[2 * i + 1] = 0u;
      }
      if (threadIdx.x == 0) s_hi = (uint32_t)((uint64_t)s_img<DT>(((const T*)b.vals)[0]) >> 32);
    }
    __syncthreads();
    if (kMM32) b.tile_hi = s_hi;
    atomicAdd(&s_cnt.seen, build_rows<DT, MM, true, VEC, true, QPI, HOME, true, kMM32>(b, st, threadIdx.x, blockDim.x));
    __syncthreads();
    flush_smem<DT, MM, true, kMM32>(b, st);
    __syncthreads();
  }
  report_counts(a, s_cnt);
}

// ---------------------------------------------------------------------------
// Finalise.
// ---------------------------------------------------------------------------
struct OutArrays {
  uint32_t* keys;
  int64_t* count;
  unsigned long long* sum;
  unsigned long long* min;
  unsigned long long* max;
  double* avg;
  int64_t* d;  // number of groups (device)
};

template <int DT, bool MM>
__device__ __forceinline__ void write_group(const OutArrays& o, int64_t i, uint32_t key, const GSlot<MM>& s) {
  const uint32_t c = s.cnt;
  o.keys[i] = key;
  o.count[i] = c;
  const unsigned long long sv = s.sum;
  o.sum[i] = sv;
  double fsum;
  if (DT == AGG_F32 || DT == AGG_F64) fsum = __longlong_as_double((long long)sv);
  else fsum = (double)(long long)sv;
  o.avg[i] = fsum / (double)c;
  if (MM) {
    const GSlot<true>& w = (const GSlot<true>&)s;
    const uint64_t mn = ~w.minc, mx = w.mx;
    if (DT == AGG_F32) {
      o.min[i] = (unsigned long long)__double_as_longlong((double)f32_of_img((uint32_t)mn));
      o.max[i] = (unsigned long long)__double_as_longlong((double)f32_of_img((uint32_t)mx));
    } else if (DT == AGG_F64) {
      o.min[i] = (unsigned long long)__double_as_longlong(f64_of_img(mn));
      o.max[i] = (unsigned long long)__double_as_longlong(f64_of_img(mx));
    } else {
      o.min[i] = (unsigned long long)i64_of_img(mn);
      o.max[i] = (unsigned long long)i64_of_img(mx);
    }
  }
}

template <bool MM>
__device__ __forceinline__ bool occupied(const GSlot<MM>* tab, uint32_t mask, int64_t j) {
  return j <= (int64_t)mask ? tab[j].key1 != 0 : tab[j].cnt != 0;
}

template <bool MM>
__device__ __forceinline__ uint32_t key_of(const GSlot<MM>* tab, uint32_t mask, int64_t j) {
  return j <= (int64_t)mask ? tab[j].key1 - 1 : 0xFFFFFFFFu;
}

// Small tables (at most kSmallRank occupied slots): after compaction, every
// block loads all d distinct keys into shared memory and writes each of its
// keys at its rank (the number of smaller keys); keys are distinct, so the
// ranks are a permutation and the output is in ascending key order.
constexpr int kSmallRank = 4097;
constexpr int kRankThreads = 256;
constexpr int kRankSplit = 4;                             // threads counting one key's rank
constexpr int kRankKeys = kRankThreads / kRankSplit;      // keys ranked per block

template <int DT, bool MM>
__global__ void __launch_bounds__(kRankThreads) gb_rank_gather(const GSlot<MM>* tab, const uint32_t* ckeys,
                                                               const uint32_t* cslot, OutArrays o) {
  __shared__ uint32_t sk[kSmallRank];
  const int d = (int)*(const unsigned long long*)o.d;
  for (int t = threadIdx.x; t < d; t += kRankThreads) sk[t] = ckeys[t];
  __syncthreads();
  // kRankSplit neighbouring lanes count the smaller keys of one key, each over
  // every kRankSplit-th key, and add their counts with shuffles
  const int i = blockIdx.x * kRankKeys + (int)threadIdx.x / kRankSplit;
  const int part = (int)threadIdx.x % kRankSplit;
  const uint32_t key = i < d ? sk[i] : 0u;
  int rank = 0;
#pragma unroll 8
  for (int t = part; t < d; t += kRankSplit) rank += sk[t] < key ? 1 : 0;
#pragma unroll
  for (int m = 1; m < kRankSplit; m <<= 1) rank += __shfl_xor_sync(0xffffffffu, rank, m);
  if (i < d && part == 0) write_group<DT, MM>(o, rank, key, tab[cslot[i]]);
}

// Large tables: compact occupied slots into (key, slot) pairs.
// PER slots per thread per run of the compaction (1 for small tables, whose
// few slots are best spread over all threads; 8 for large ones).
template <bool MM, int kCompactPer = 8>
__global__ void gb_compact(const GSlot<MM>* tab, uint32_t mask, uint32_t* okeys, uint32_t* oslot,
                           unsigned long long* counter) {
  // each block takes runs of kCompactPer * blockDim.x slots and reserves its
  // output range with one atomic per run (order within a run: warp, then lane)
  __shared__ uint32_t s_warp[32];
  __shared__ unsigned long long s_base;
  const int64_t nslots = (int64_t)mask + 2;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t lt = (1u << lane) - 1u;
  const int64_t span = (int64_t)kCompactPer * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * span; base < nslots; base += (int64_t)gridDim.x * span) {
    bool occ[kCompactPer];
    uint32_t b[kCompactPer];
    uint32_t wtot = 0;
#pragma unroll
    for (int i = 0; i < kCompactPer; ++i) {
      const int64_t j = base + (int64_t)i * blockDim.x + threadIdx.x;
      occ[i] = j < nslots && occupied<MM>(tab, mask, j);
      b[i] = __ballot_sync(0xffffffffu, occ[i]);
      wtot += __popc(b[i]);
    }
    if (lane == 0) s_warp[warp] = wtot;
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int w = 0; w < nw; ++w) {
        const uint32_t c = s_warp[w];
        s_warp[w] = t;
        t += c;
      }
      s_base = t ? atomicAdd(counter, (unsigned long long)t) : 0ull;
    }
    __syncthreads();
    unsigned long long pos = s_base + s_warp[warp];
#pragma unroll
    for (int i = 0; i < kCompactPer; ++i) {
      if (occ[i]) {
        const int64_t j = base + (int64_t)i * blockDim.x + threadIdx.x;
        const unsigned long long p = pos + __popc(b[i] & lt);
        okeys[p] = key_of<MM>(tab, mask, j);
        oslot[p] = (uint32_t)j;
      }
      pos += __popc(b[i]);
    }
    __syncthreads();  // s_warp and s_base are rewritten by the next run
  }
}

template <int DT, bool MM>
__global__ void gb_gather(const GSlot<MM>* tab, const uint32_t* skeys, const uint32_t* sslot, OutArrays o,
                          int64_t cap) {
  const int64_t d = *(const unsigned long long*)o.d;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d && i < cap;
       i += (int64_t)gridDim.x * blockDim.x) {
    write_group<DT, MM>(o, i, skeys[i], tab[sslot[i]]);
  }
}


}  // namespace agg
