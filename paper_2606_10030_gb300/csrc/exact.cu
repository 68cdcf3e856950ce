// Exactly rounded float GROUP BY sums (AGG_FLAG_EXACT_SUM), and the error of
// the strategy's sums against them (AGG_FLAG_SUM_ERROR).
//
// Float sums built with atomics depend on the order in which rows arrive.
// With this flag every group's SUM is the exact real sum of its rows rounded
// once to float64 (to nearest, ties to even) and AVG is that sum divided by
// the count, so the result is the same bit for bit for every strategy, grid
// and run (the deterministic float GROUP BY mode). It runs after a strategy
// has produced the groups (keys ascending, counts, MIN/MAX):
//   exact_span   the lowest and highest exponent among the nonzero values,
//                and whether any value is not finite (one read-back);
//   exact_add    every row finds its group by binary search over the result
//                keys and adds its value, an integer number of units of the
//                column's lowest exponent, into the group's base-2^28 digits
//                with 64-bit atomics (integer additions: the order is free);
//   exact_round  per group, carry propagation and one rounding.
// The digits per group cover only the column's exponent span (plus 32 bits
// for the row count), so a column of similar magnitudes needs a handful.
#include <climits>

#include "exact.cuh"
#include "groupby.cuh"

namespace agg {

constexpr int kExactThreads = 256;

template <int DT>
__device__ __forceinline__ ExactParts parts_of(const void* vals, int64_t i) {
  if (DT == AGG_F32) return exact_parts_f32(__float_as_uint(((const float*)vals)[i]));
  return exact_parts_f64((uint64_t)__double_as_longlong(((const double*)vals)[i]));
}

template <int DT>
__device__ __forceinline__ bool finite_at(const void* vals, int64_t i) {
  if (DT == AGG_F32) return ((__float_as_uint(((const float*)vals)[i]) >> 23) & 0xFF) != 0xFF;
  return (((uint64_t)__double_as_longlong(((const double*)vals)[i]) >> 52) & 0x7FF) != 0x7FF;
}

// span[0] = lowest lsb exponent, span[1] = highest, span[2] = nonfinite rows.
template <int DT>
__global__ void __launch_bounds__(kExactThreads) exact_span(const void* __restrict__ vals, int64_t n,
                                                            int* __restrict__ span) {
  int lo = INT_MAX, hi = INT_MIN, bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (!finite_at<DT>(vals, i)) {
      bad = 1;
      continue;
    }
    const ExactParts p = parts_of<DT>(vals, i);
    if (p.mant == 0) continue;
    lo = min(lo, p.lsb);
    hi = max(hi, p.lsb);
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  bad = __reduce_or_sync(0xffffffffu, (unsigned)bad);
  if ((threadIdx.x & 31) == 0) {
    if (lo != INT_MAX) atomicMin(&span[0], lo);
    if (hi != INT_MIN) atomicMax(&span[1], hi);
    if (bad) atomicOr(&span[2], 1);
  }
}

template <int DT>
__global__ void __launch_bounds__(kExactThreads) exact_add(const uint32_t* __restrict__ keys,
                                                           const void* __restrict__ vals, int64_t n,
                                                           const uint32_t* __restrict__ gkeys, int64_t d,
                                                           unsigned long long* __restrict__ acc, int D, int base) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const ExactParts p = parts_of<DT>(vals, i);
    if (p.mant == 0) continue;
    const uint32_t key = keys[i];
    int64_t lo = 0, len = d;  // the group: the last result key <= key (it is present)
    while (len > 1) {
      const int64_t half = len >> 1;
      if (__ldg(&gkeys[lo + half]) <= key) lo += half;
      len -= half;
    }
    const int pos = p.lsb - base;  // >= 0
    const int q = pos / kDigitBits;
    int64_t c[3];
    exact_chunks(p.mant, pos - q * kDigitBits, c);
    unsigned long long* w = acc + (size_t)lo * (size_t)D + (size_t)q;
#pragma unroll
    for (int k = 0; k < 3; ++k)
      if (c[k] != 0) atomicAdd(&w[k], (unsigned long long)(p.neg ? -c[k] : c[k]));
  }
}

// replace: write the exact sum (and avg) over the result's; err (nullable):
// the distance of the sum the result keeps from the exact one.
__global__ void __launch_bounds__(kExactThreads) exact_round_groups(const unsigned long long* __restrict__ acc,
                                                                    int64_t d, int D, int base,
                                                                    const int64_t* __restrict__ count,
                                                                    double* __restrict__ sum,
                                                                    double* __restrict__ avg, bool replace,
                                                                    double* __restrict__ err) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g >= d) return;
  int64_t a[kMaxDigits];
  for (int k = 0; k < D; ++k) a[k] = (int64_t)acc[(size_t)g * D + k];
  const double s = exact_round(a, D, base);
  if (err) err[g] = replace ? 0.0 : fabs(sum[g] - s);
  if (!replace) return;
  sum[g] = s;
  if (avg) avg[g] = count[g] ? s / (double)count[g] : __longlong_as_double(0x7ff8000000000000ll);
}

// Exactly rounded sums of a finished float GROUP BY result: with replace, they
// replace the result's sums (and averages); with report, g->sum_err receives
// |kept sum - exact sum| per group. keys/vals: the query's device columns.
agg_status exact_fp_sums(const uint32_t* keys, const void* vals, int64_t n, int vdt, uint32_t ops,
                         agg_groups* g, cudaStream_t s, bool replace, bool report) {
  const int64_t d = g->num_groups;
  if (d == 0 || n == 0) return AGG_OK;
  double* err = nullptr;
  if (report) {
    if (dev_malloc_async((void**)&err, (size_t)d * 8, s) != cudaSuccess) {
      set_error("sum errors: cannot allocate %lld bytes", (long long)d * 8);
      return AGG_ERR_OOM;
    }
    ((GroupsPriv*)g->priv)->extra = err;  // freed with the result from here on
    g->sum_err = err;
  }
  const DeviceInfo& di = device_info();
  const int grid = di.sm_count * 8;
  PhaseTimer pt(AGG_PHASE_FINALIZE, s);
  agg_status st = AGG_OK;
  char* scr = (char*)stream_scratch(s, 4096 + 256, &st);
  if (!scr) return st;
  int* span_dev = (int*)(scr + 4096);  // transient, past the scan's ticket and the sketch's features
  const int init[3] = {INT_MAX, INT_MIN, 0};
  AGG_CUDA_TRY(cudaMemcpyAsync(span_dev, init, sizeof(init), cudaMemcpyHostToDevice, s));
  if (vdt == AGG_F32) exact_span<AGG_F32><<<grid, kExactThreads, 0, s>>>(vals, n, span_dev);
  else exact_span<AGG_F64><<<grid, kExactThreads, 0, s>>>(vals, n, span_dev);
  note_launch();
  AGG_CUDA_TRY(cudaGetLastError());
  int span[3];
  AGG_CUDA_TRY(cudaMemcpyAsync(span, span_dev, sizeof(span), cudaMemcpyDeviceToHost, s));
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  AGG_CHECK_ARG(span[2] == 0, "exact float sums need finite values (the column holds an infinity or NaN)");
  const int mant_bits = vdt == AGG_F32 ? 24 : 53;
  int base = 0, D = 1;
  if (span[0] != INT_MAX) {
    base = span[0];
    const int bits = span[1] - span[0] + mant_bits + 33;  // sum of < 2^32 rows, and a sign
    D = (bits + kDigitBits - 1) / kDigitBits + 2;
  }
  if (D > kMaxDigits) {
    set_error("exact float sums: %d digits exceed %d", D, kMaxDigits);
    return AGG_ERR_INVALID;
  }
  void* acc = nullptr;
  const size_t bytes = (size_t)d * (size_t)D * 8;
  if (dev_malloc_async(&acc, bytes, s) != cudaSuccess) {
    set_error("exact float sums: cannot allocate %zu bytes of digits", bytes);
    return AGG_ERR_OOM;
  }
  cudaError_t e = cudaMemsetAsync(acc, 0, bytes, s);
  if (e == cudaSuccess && span[0] != INT_MAX) {
    if (vdt == AGG_F32)
      exact_add<AGG_F32><<<grid, kExactThreads, 0, s>>>(keys, vals, n, g->keys, d, (unsigned long long*)acc, D, base);
    else
      exact_add<AGG_F64><<<grid, kExactThreads, 0, s>>>(keys, vals, n, g->keys, d, (unsigned long long*)acc, D, base);
    note_launch();
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const int rgrid = (int)((d + kExactThreads - 1) / kExactThreads);
    exact_round_groups<<<rgrid, kExactThreads, 0, s>>>((const unsigned long long*)acc, d, D, base, g->count,
                                                       (double*)g->sum, (ops & AGG_AVG) ? g->avg : nullptr,
                                                       replace, err);
    note_launch();
    e = cudaGetLastError();
  }
  cudaFreeAsync(acc, s);
  if (e != cudaSuccess) {
    set_error("exact float sums: %s", cudaGetErrorString(e));
    return AGG_ERR_CUDA;
  }
  AGG_CUDA_TRY(cudaStreamSynchronize(s));
  return AGG_OK;
}

}  // namespace agg
