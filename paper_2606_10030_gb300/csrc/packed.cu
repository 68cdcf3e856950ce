// Compressed columns for the scan: frame-of-reference bit packing (the
// paper's future work compresses data to speed up transfers, Sec. 8). An
// integer column is cut into frames of 1024 values; a frame stores its
// minimum (the reference) and every value minus the reference in the fewest
// bits that hold the frame's range, packed little-endian into 32-bit words.
// The encoder runs on the host (the format at rest, before the transfer); the
// scan decodes inside its kernel, so only the packed bytes cross the host
// link (agg_reduce_packed_host) or are read from HBM (agg_reduce_packed).
//
// Decode: a warp takes a frame; lane l holds values l, l + 32, ..., so the
// 32 lanes of one step read one contiguous span of 32 * bits bits (the words
// they share come from L1). Each value is folded by the scan's accumulators.
#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <vector>

#include "reduce.cuh"

namespace agg {

struct PackDesc {  // 24 bytes per frame
  int64_t ref;
  uint32_t bits;
  uint32_t reserved;
  uint64_t word_off;  // first 32-bit word of the frame
};
static_assert(sizeof(PackDesc) == 24, "frame descriptor layout");

inline size_t pack_words_offset(int64_t nframes) { return ((size_t)nframes * sizeof(PackDesc) + 15) & ~size_t(15); }

template <int DT>
__device__ __forceinline__ typename Traits<DT>::T unpack_value(const uint32_t* __restrict__ w, uint32_t bits,
                                                               int64_t ref, int i) {
  using T = typename Traits<DT>::T;
  uint64_t x = 0;
  if (bits != 0) {
    const uint64_t pos = (uint64_t)i * bits;
    const uint32_t* p = w + (pos >> 5);
    const uint32_t sh = (uint32_t)(pos & 31);
    const uint64_t lo = (uint64_t)__ldg(p) | ((uint64_t)__ldg(p + 1) << 32);
    x = lo >> sh;
    if (sh + bits > 64) x |= (uint64_t)__ldg(p + 2) << (64 - sh);
    if (bits < 64) x &= (uint64_t(1) << bits) - 1;
  }
  return (T)(ref + (int64_t)x);
}

// Frames [f0, f0 + nf) of a column of n values; desc / words relative to the
// buffer (word offsets counted from words_base).
template <int DT, bool SUM, bool MM>
__global__ void __launch_bounds__(kBlock) packed_scan(const PackDesc* __restrict__ desc, const uint32_t* __restrict__ words,
                                                      uint64_t words_base, int64_t f0, int64_t nf, int64_t n,
                                                      Partial* __restrict__ parts, int part_base) {
  Acc<DT, SUM, MM> a;
  a.init();
  const int lane = threadIdx.x & 31;
  const int64_t warp = ((int64_t)blockIdx.x * kBlock + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * kBlock) >> 5;
  for (int64_t f = warp; f < nf; f += nwarps) {
    const PackDesc d = desc[f];
    const uint32_t* w = words + (d.word_off - words_base);
    const int64_t row0 = (f0 + f) * AGG_PACK_FRAME;
    const int cnt = (int)min((int64_t)AGG_PACK_FRAME, n - row0);
#pragma unroll 4
    for (int i = lane; i < cnt; i += 32) a.fold(unpack_value<DT>(w, d.bits, d.ref, i));
  }
  Partial p;
  a.to_partial(p, 0);
  p = block_reduce<kBlock>(p);
  if (threadIdx.x == 0) parts[part_base + blockIdx.x] = p;
}

template <int DT>
__global__ void __launch_bounds__(kBlock) packed_merge(const Partial* parts, int np, agg_scalar* out, uint32_t ops,
                                                       int64_t count) {
  merge_partials<DT, kBlock>(parts, np, out, ops, count);
}

template <int DT>
static void* packed_scan_ptr(bool sum, bool mm) {
  return sum ? (mm ? (void*)packed_scan<DT, true, true> : (void*)packed_scan<DT, true, false>)
             : (mm ? (void*)packed_scan<DT, false, true> : (void*)packed_scan<DT, false, false>);
}

static void* pick_packed(int dt, bool sum, bool mm) {
  switch (dt) {
    case AGG_I32: return packed_scan_ptr<AGG_I32>(sum, mm);
    case AGG_I64: return packed_scan_ptr<AGG_I64>(sum, mm);
    default: return packed_scan_ptr<AGG_U32>(sum, mm);
  }
}

static void* pick_packed_merge(int dt) {
  switch (dt) {
    case AGG_I32: return (void*)packed_merge<AGG_I32>;
    case AGG_I64: return (void*)packed_merge<AGG_I64>;
    default: return (void*)packed_merge<AGG_U32>;
  }
}

static int packed_grid(int64_t nf) {
  const DeviceInfo& di = device_info();
  const int64_t warps_per_block = kBlock / 32;
  int64_t g = (int64_t)di.sm_count * 8;
  const int64_t need = (nf + warps_per_block - 1) / warps_per_block;
  if (need < g) g = need;
  return (int)std::max<int64_t>(1, g);
}

static agg_status check_packed(const void* buf, const agg_packed_info* info, uint32_t ops, const void* out) {
  AGG_CHECK_ARG(info != nullptr && out != nullptr, "null info or output pointer");
  AGG_CHECK_ARG(info->dtype == AGG_I32 || info->dtype == AGG_I64 || info->dtype == AGG_U32,
                "packed columns hold int32, int64 or uint32 values (dtype %d)", info->dtype);
  AGG_CHECK_ARG(ops != 0 && (ops & ~(uint32_t)AGG_ALL) == 0, "invalid ops mask 0x%x", ops);
  AGG_CHECK_ARG(info->n >= 0 && info->nframes == (info->n + AGG_PACK_FRAME - 1) / AGG_PACK_FRAME,
                "inconsistent packed column (n %lld, frames %lld)", (long long)info->n, (long long)info->nframes);
  AGG_CHECK_ARG(info->n == 0 || buf != nullptr, "null packed buffer");
  AGG_CHECK_ARG(((uintptr_t)buf & 15) == 0, "packed buffer not 16-byte aligned");
  AGG_CHECK_ARG(info->bytes == (int64_t)(pack_words_offset(info->nframes) + (size_t)info->nwords * 4 + 8),
                "inconsistent packed column size");
  return AGG_OK;
}

}  // namespace agg

using namespace agg;

extern "C" size_t agg_pack_for_bound(int64_t n, agg_dtype dtype) {
  const int64_t nf = n <= 0 ? 0 : (n + AGG_PACK_FRAME - 1) / AGG_PACK_FRAME;
  const size_t es = dtype == AGG_I64 ? 8 : 4;
  return pack_words_offset(nf) + (size_t)nf * AGG_PACK_FRAME * es + 8;
}

// Host encoder. Each frame: reference = its minimum, bits = bit length of
// (maximum - minimum); values minus the reference appended to the frame's bit
// stream, least significant bit first. Eight zero bytes end the buffer so that
// the decoder's look-ahead word loads stay inside it.
extern "C" agg_status agg_pack_for(const void* col_host, int64_t n, agg_dtype dtype, void* out_host, size_t capacity,
                                   agg_packed_info* info) {
  clear_error();
  AGG_CHECK_ARG(dtype == AGG_I32 || dtype == AGG_I64 || dtype == AGG_U32, "packed columns hold integers");
  AGG_CHECK_ARG(n >= 0 && n < (int64_t(1) << 40), "invalid row count %lld", (long long)n);
  AGG_CHECK_ARG(info != nullptr && (n == 0 || (col_host != nullptr && out_host != nullptr)), "null pointer");
  AGG_CHECK_ARG(((uintptr_t)out_host & 15) == 0, "output buffer not 16-byte aligned");
  const int64_t nf = (n + AGG_PACK_FRAME - 1) / AGG_PACK_FRAME;
  auto value = [&](int64_t i) -> int64_t {
    if (dtype == AGG_I32) return ((const int32_t*)col_host)[i];
    if (dtype == AGG_I64) return ((const int64_t*)col_host)[i];
    return (int64_t)((const uint32_t*)col_host)[i];
  };
  // sizes first, so that a short buffer is rejected before anything is written
  std::vector<uint32_t> bits(nf);
  std::vector<int64_t> refs(nf);
  uint64_t words = 0;
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t a = f * AGG_PACK_FRAME, b = std::min<int64_t>(n, a + AGG_PACK_FRAME);
    int64_t mn = value(a), mx = mn;
    for (int64_t i = a + 1; i < b; ++i) {
      const int64_t v = value(i);
      mn = std::min(mn, v);
      mx = std::max(mx, v);
    }
    const uint64_t range = (uint64_t)mx - (uint64_t)mn;
    bits[f] = range == 0 ? 0u : 64u - (uint32_t)__builtin_clzll(range);
    refs[f] = mn;
    words += (uint64_t)bits[f] * (AGG_PACK_FRAME / 32);  // 1024 values x bits = 32 x bits words
  }
  const size_t woff = pack_words_offset(nf);
  const size_t total = woff + (size_t)words * 4 + 8;
  AGG_CHECK_ARG(total <= capacity, "packed output needs %zu bytes, the buffer holds %zu", total, capacity);
  char* out = (char*)out_host;
  PackDesc* desc = (PackDesc*)out;
  uint32_t* w = (uint32_t*)(out + woff);
  std::memset(out, 0, total);
  uint64_t wo = 0;
  for (int64_t f = 0; f < nf; ++f) {
    desc[f].ref = refs[f];
    desc[f].bits = bits[f];
    desc[f].reserved = 0;
    desc[f].word_off = wo;
    const uint32_t b = bits[f];
    if (b) {
      const int64_t a = f * AGG_PACK_FRAME, e = std::min<int64_t>(n, a + AGG_PACK_FRAME);
      uint64_t pos = wo * 32;  // bit position in the word stream
      for (int64_t i = a; i < e; ++i, pos += b) {
        const uint64_t x = (uint64_t)value(i) - (uint64_t)refs[f];
        const uint64_t q = pos >> 5;
        const uint32_t sh = (uint32_t)(pos & 31);
        w[q] |= (uint32_t)(x << sh);
        if (sh + b > 32) w[q + 1] |= (uint32_t)(x >> (32 - sh));
        if (sh + b > 64) w[q + 2] |= (uint32_t)(x >> (64 - sh));
      }
    }
    wo += (uint64_t)b * (AGG_PACK_FRAME / 32);
  }
  info->n = n;
  info->dtype = dtype;
  info->reserved = 0;
  info->nframes = nf;
  info->nwords = (int64_t)words;
  info->bytes = (int64_t)total;
  return AGG_OK;
}

extern "C" agg_status agg_reduce_packed(const void* packed_dev, const agg_packed_info* info, uint32_t ops,
                                        agg_scalar* out_dev, void* stream) {
  clear_error();
  agg_status st = check_packed(packed_dev, info, ops, out_dev);
  if (st != AGG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t nf = info->nframes;
  const int grid = packed_grid(nf);
  char* scratch = (char*)stream_scratch(s, 256 + (size_t)grid * sizeof(Partial), &st);
  if (!scratch) return st;
  Partial* parts = (Partial*)(scratch + 256);
  const PackDesc* desc = (const PackDesc*)packed_dev;
  const uint32_t* words = (const uint32_t*)((const char*)packed_dev + pack_words_offset(nf));
  uint64_t base = 0;
  int64_t f0 = 0, n = info->n;
  int part_base = 0;
  const bool sum = ops & (AGG_SUM | AGG_AVG), mm = ops & (AGG_MIN | AGG_MAX);
  {
    PhaseTimer pt(AGG_PHASE_SCAN, s);
    void* args[] = {(void*)&desc, (void*)&words, (void*)&base, (void*)&f0, (void*)&nf, (void*)&n, (void*)&parts,
                    (void*)&part_base};
    AGG_CUDA_TRY(cudaLaunchKernel(pick_packed(info->dtype, sum, mm), dim3(grid), dim3(kBlock), args, 0, s));
    note_launch();
  }
  int np = grid;
  void* margs[] = {(void*)&parts, (void*)&np, (void*)&out_dev, (void*)&ops, (void*)&n};
  AGG_CUDA_TRY(cudaLaunchKernel(pick_packed_merge(info->dtype), dim3(1), dim3(kBlock), margs, 0, s));
  note_launch();
  return AGG_OK;
}

namespace agg {
namespace {
struct PackPipe {
  static constexpr int kRing = 3;
  cudaStream_t copy = nullptr;
  cudaEvent_t ready[kRing] = {};
  cudaEvent_t freed[kRing] = {};
  bool ok = false;
  std::mutex call_mu;
};

PackPipe* pack_pipe(agg_status* st) {
  static std::mutex mu;
  static std::map<int, PackPipe*> pipes;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  PackPipe*& p = pipes[dev];
  if (!p) p = new PackPipe();
  *st = AGG_OK;
  if (!p->ok) {
    if (cudaStreamCreateWithFlags(&p->copy, cudaStreamNonBlocking) != cudaSuccess) {
      set_error("cannot create copy stream");
      *st = AGG_ERR_CUDA;
      return p;
    }
    for (int i = 0; i < PackPipe::kRing; ++i) {
      cudaEventCreateWithFlags(&p->ready[i], cudaEventDisableTiming);
      cudaEventCreateWithFlags(&p->freed[i], cudaEventDisableTiming);
    }
    p->ok = true;
  }
  return p;
}
}  // namespace
}  // namespace agg

// End to end from a packed column in host memory: chunks of frames (their
// descriptors and words) are copied on a copy stream into a ring of device
// buffers while the previous chunk is decoded and scanned; one merge at the end.
extern "C" agg_status agg_reduce_packed_host(const void* packed_host, const agg_packed_info* info, uint32_t ops,
                                             agg_scalar* out_host, void* stream) {
  clear_error();
  agg_status st = check_packed(packed_host, info, ops, out_host);
  if (st != AGG_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  PackPipe* pipe = pack_pipe(&st);
  if (st != AGG_OK) return st;
  std::lock_guard<std::mutex> lk(pipe->call_mu);
  const int64_t nf = info->nframes;
  constexpr int64_t kChunkFrames = 16384;  // 16 Mi values per chunk
  const int64_t nchunks = (nf + kChunkFrames - 1) / kChunkFrames;
  const PackDesc* desc = (const PackDesc*)packed_host;
  const uint32_t* words = (const uint32_t*)((const char*)packed_host + pack_words_offset(nf));
  const size_t es = info->dtype == AGG_I64 ? 8 : 4;
  const size_t dbytes = ((size_t)kChunkFrames * sizeof(PackDesc) + 255) & ~size_t(255);
  const size_t wbytes = (size_t)kChunkFrames * AGG_PACK_FRAME * es + 256;  // at most 64 bits a value, plus look-ahead
  const size_t slot = dbytes + wbytes;
  const int grid = packed_grid(std::min(nf, kChunkFrames));
  const int64_t nparts = std::max<int64_t>(1, nchunks * grid);
  char* scratch = (char*)stream_scratch(s, 256 + sizeof(agg_scalar) + 256 + (size_t)nparts * sizeof(Partial) + 256 +
                                               (size_t)PackPipe::kRing * slot, &st);
  if (!scratch) return st;
  agg_scalar* out_dev = (agg_scalar*)(scratch + 256);
  Partial* parts = (Partial*)(scratch + 512 + 256);
  char* ring = scratch + ((512 + 256 + (size_t)nparts * sizeof(Partial) + 255) & ~size_t(255));
  cudaEvent_t start_ev;
  AGG_CUDA_TRY(cudaEventCreateWithFlags(&start_ev, cudaEventDisableTiming));
  cudaEventRecord(start_ev, s);
  cudaStreamWaitEvent(pipe->copy, start_ev, 0);
  const bool sum = ops & (AGG_SUM | AGG_AVG), mm = ops & (AGG_MIN | AGG_MAX);
  void* fn = pick_packed(info->dtype, sum, mm);
  int64_t n = info->n;
  const int64_t total_words = info->nwords;
  for (int64_t c = 0; c < nchunks; ++c) {
    const int b = (int)(c % PackPipe::kRing);
    const int64_t f0 = c * kChunkFrames, nfc = std::min(kChunkFrames, nf - f0);
    const uint64_t w0 = desc[f0].word_off;
    const uint64_t w1 = f0 + nfc < nf ? desc[f0 + nfc].word_off : (uint64_t)total_words;
    const size_t wcopy = (size_t)(w1 - w0) * 4 + 8;  // the look-ahead words (the buffer ends in 8 zero bytes)
    char* dbuf = ring + (size_t)b * slot;
    char* wbuf = dbuf + dbytes;
    if (c >= PackPipe::kRing) cudaStreamWaitEvent(pipe->copy, pipe->freed[b], 0);
    AGG_CUDA_TRY(cudaMemcpyAsync(dbuf, desc + f0, (size_t)nfc * sizeof(PackDesc), cudaMemcpyHostToDevice, pipe->copy));
    AGG_CUDA_TRY(cudaMemcpyAsync(wbuf, words + w0, wcopy, cudaMemcpyHostToDevice, pipe->copy));
    cudaEventRecord(pipe->ready[b], pipe->copy);
    cudaStreamWaitEvent(s, pipe->ready[b], 0);
    const PackDesc* dd = (const PackDesc*)dbuf;
    const uint32_t* wd = (const uint32_t*)wbuf;
    uint64_t base = w0;
    int64_t ff0 = f0, nff = nfc;
    int part_base = (int)(c * grid);
    void* args[] = {(void*)&dd, (void*)&wd, (void*)&base, (void*)&ff0, (void*)&nff, (void*)&n, (void*)&parts,
                    (void*)&part_base};
    AGG_CUDA_TRY(cudaLaunchKernel(fn, dim3(grid), dim3(kBlock), args, 0, s));
    note_launch();
    cudaEventRecord(pipe->freed[b], s);
  }
  int np = (int)(nchunks * grid);
  void* margs[] = {(void*)&parts, (void*)&np, (void*)&out_dev, (void*)&ops, (void*)&n};
  AGG_CUDA_TRY(cudaLaunchKernel(pick_packed_merge(info->dtype), dim3(1), dim3(kBlock), margs, 0, s));
  note_launch();
  AGG_CUDA_TRY(cudaMemcpyAsync(out_host, out_dev, sizeof(agg_scalar), cudaMemcpyDeviceToHost, s));
  cudaError_t e = cudaStreamSynchronize(s);
  cudaEventDestroy(start_ev);
  if (e != cudaSuccess) {
    set_error("agg_reduce_packed_host: %s", cudaGetErrorString(e));
    return AGG_ERR_CUDA;
  }
  return AGG_OK;
}
