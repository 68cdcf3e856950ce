/*
 * agg.h -- C ABI of the GB300 (sm_103a) in-memory aggregation library.
 *
 * In-memory aggregation scans every item of a column and folds it with an
 * aggregation function (min, sum, ...) into a summary (Sec. 1 and Sec. 2.1,
 * Fig. 1; the fold r = aggregate(r, input[i]) of Fig. 4). The ungrouped scan
 * follows the paper's specialised GPU design (Sec. 3.2, "GPU Optimizations"):
 * one fused kernel, a grid sized to the SM count, coalesced grid-stride
 * loads, register accumulation, block-local reduction and one grid-wide merge
 * of the block partials. GROUP BY (the hash- and sort-based group-by of
 * Sec. 7) aggregates per distinct key.
 *
 * Conventions for every entry point
 *  - Pointers named *_dev are CUDA device pointers (or managed memory);
 *    pointers named *_host are host pointers, ideally pinned (page-locked).
 *    Inputs are borrowed: they must stay valid and unchanged until the work
 *    enqueued on `stream` has finished.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *  - Every call returns an agg_status; no exception crosses the ABI. Argument
 *    checks happen before any launch; on failure agg_last_error() returns a
 *    message (thread-local, valid until the next call on the same thread).
 *  - Results are defined for n = 0: COUNT = 0, SUM = 0, AVG = NaN and MIN/MAX
 *    hold the identity of their order (INT64_MAX / INT64_MIN, +inf / -inf).
 *
 * Semantics (the paper sums one integer column, Sec. 4; the rest is read here)
 *  - Integer SUM accumulates in int64 and wraps mod 2^64; uint32 values are
 *    zero-extended. It is exact and bit-identical for any reduction order.
 *  - Float SUM is returned in float64. Float32 columns are summed with
 *    TwoSum-compensated float32 partials whose final merge runs in float64;
 *    float64 columns with TwoSum-compensated float64 partials.
 *  - MIN/MAX of floats use the total order -0.0 < +0.0; inputs hold no NaN.
 *  - AVG = (double)SUM / (double)COUNT.
 */
#ifndef AGG_H_
#define AGG_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Value column element types. */
typedef enum {
  AGG_I32 = 0,
  AGG_I64 = 1,
  AGG_U32 = 2,
  AGG_F32 = 3,
  AGG_F64 = 4
} agg_dtype;

/* Aggregation functions, OR-ed into the `ops` bitmask (at least one bit). */
enum {
  AGG_SUM = 1,
  AGG_MIN = 2,
  AGG_MAX = 4,
  AGG_COUNT = 8,
  AGG_AVG = 16,
  AGG_ALL = 31
};

typedef enum {
  AGG_OK = 0,
  AGG_ERR_INVALID = -1,    /* bad argument; nothing was launched */
  AGG_ERR_OOM = -2,        /* device or pinned allocation failed */
  AGG_ERR_CUDA = -3,       /* a CUDA call failed (message in agg_last_error) */
  AGG_ERR_TABLE_FULL = -4, /* a hash table ran out of slots (retried internally) */
  AGG_ERR_TIMEOUT = -5     /* a bounded device-side wait gave up */
} agg_status;

/*
 * Result of one ungrouped aggregation (80 bytes, 8-byte aligned).
 * Integer columns fill sum_i / min_i / max_i; float columns fill sum_f /
 * min_f / max_f. sum_f of an integer column is (double)sum_i. Fields of
 * functions not requested in `ops` are unspecified, except count, which is
 * always n.
 */
typedef struct agg_scalar {
  int64_t count;
  int64_t sum_i;
  double sum_f;
  double avg;
  int64_t min_i;
  int64_t max_i;
  double min_f;
  double max_f;
  uint32_t dtype;
  uint32_t ops;
  int64_t reserved;
} agg_scalar;

/*
 * agg_reduce -- ungrouped SUM/MIN/MAX/COUNT/AVG over col_dev[0..n).
 * (Sec. 2.1 for the operation; Sec. 3.2 "GPU Optimizations" for the fused
 * single-kernel design with a grid-wide merge of block partials.)
 *
 *  col_dev  device pointer to n contiguous elements of `dtype`, aligned to the
 *           element size (any 16-byte misalignment is handled).
 *  n        number of rows, 0 <= n < 2^62.
 *  ops      bitmask of AGG_SUM | AGG_MIN | AGG_MAX | AGG_COUNT | AGG_AVG.
 *  out_dev  device pointer to one agg_scalar, written asynchronously on
 *           `stream`; read it after the stream has synchronised.
 *
 * One kernel launch; no host synchronisation; scratch (block partials and a
 * self-resetting ticket) is cached per (device, stream) by the library, so
 * calls on the same stream are serialised by the stream and calls on
 * different streams do not share scratch.
 * Errors: AGG_ERR_INVALID (null pointers, misaligned column, bad dtype/ops,
 * n out of range), AGG_ERR_OOM, AGG_ERR_CUDA.
 */
agg_status agg_reduce(const void* col_dev, int64_t n, agg_dtype dtype, uint32_t ops,
                      agg_scalar* out_dev, void* stream);

/*
 * agg_reduce_host -- end-to-end variant of agg_reduce fed from host memory
 * (Sec. 5.3: host-to-device transfer is part of the measured time).
 *
 *  col_host  host pointer to n elements (pinned memory gives full link
 *            bandwidth; pageable memory works but is staged by the driver).
 *  out_host  host pointer to one agg_scalar, valid when the call returns.
 *
 * The column is copied in chunks into a ring of device buffers on a copy
 * stream while the scan of the previous chunk runs on `stream`; the partials
 * of all chunks are merged at the end and the result copied back. The call
 * is synchronous (it waits for the result).
 */
agg_status agg_reduce_host(const void* col_host, int64_t n, agg_dtype dtype, uint32_t ops,
                           agg_scalar* out_host, void* stream);

/*
 * agg_reduce_noalloc -- agg_reduce without any device allocation.
 *
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory, for example an engine that has reserved all
 * of the GPU's memory for its own pool up front (so cudaMalloc would fail), or
 * a latency-critical path that cannot afford the device-wide synchronisation
 * that cudaMalloc and cudaFree can imply. Arguments, results and errors are
 * those of agg_reduce; the caller still provides the column and out_dev.
 *
 * Scratch: a static device array of 82,176 bytes (the ticket plus 2048 block
 * partials) that every GPU loading the library holds until the process exits.
 * A launch that would need more blocks than that returns AGG_ERR_INVALID with
 * a message; no call allocates (no cudaMalloc, cudaFree or allocating library
 * routine). The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture. All calls share the one array: each call clears
 * the ticket it needs at zero, and calls whose work overlaps on the GPU (for
 * example on two streams) race on the array and give wrong results.
 */
agg_status agg_reduce_noalloc(const void* col_dev, int64_t n, agg_dtype dtype, uint32_t ops,
                              agg_scalar* out_dev, void* stream);

/* Message of the last failed call on this thread ("" if none). */
const char* agg_last_error(void);

/* ABI version of this header (major * 100 + minor). */
int agg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AGG_H_ */
