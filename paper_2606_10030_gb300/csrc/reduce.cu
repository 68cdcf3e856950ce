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
#include <map>
#include <mutex>

#include "reduce.cuh"

namespace agg {

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
