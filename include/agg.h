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
 *    TwoSum-compensated float32 partials whose final merge runs in float64.
 *    The ungrouped scan sums float64 columns per thread as 128-bit
 *    fixed-point integers (scaled to the largest exponent the thread has
 *    seen) and merges them as float64 pairs; GROUP BY adds float64 values in
 *    float64.
 *  - MIN/MAX of floats use the total order -0.0 < +0.0; inputs hold no NaN.
 *  - AVG = (double)SUM / (double)COUNT.
 */
#ifndef AGG_H_
#define AGG_H_

#include <stddef.h>
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
  AGG_ERR_TIMEOUT = -5     /* reserved: no kernel of this library waits on another block or device */
} agg_status;

/*
 * Result of one ungrouped aggregation (80 bytes, 8-byte aligned).
 * Integer columns fill sum_i / min_i / max_i; float columns fill sum_f /
 * min_f / max_f. sum_f of an integer column is (double)sum_i. Fields of
 * functions not requested in `ops` are unspecified, except count, which is
 * always n.
 * err_bound: for a float column with SUM or AVG requested, a bound computed on
 * the device, alongside the sum, on |sum_f - S| where S is the exact real sum
 * of the column rounded once to float64 (the value of the FP64 reference):
 * it adds up every rounding the scan can make (the compensation words of the
 * float32 pairs, the truncations of the float64 fixed-point sums, the merges
 * of block partials, the final rounding) and S's own rounding. It is +inf
 * when the column holds an infinity or a NaN, and 0 for integer columns
 * (their sums are exact). It bounds SUM only, not AVG.
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
  double err_bound;
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
 *            bandwidth; pageable memory works but is staged by the CUDA driver).
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
 * Compressed integer columns for the scan (the paper's future work compresses
 * data to speed up transfers, Sec. 8): frame-of-reference bit packing. A
 * column is cut into frames of AGG_PACK_FRAME values; each frame keeps its
 * minimum as reference and every value minus it in the fewest bits that hold
 * the frame's range (0 to 64), least significant bit first, in 32-bit words.
 * Buffer layout (16-byte aligned): nframes descriptors of 24 bytes
 * {int64 ref; uint32 bits; uint32 zero; uint64 first word of the frame}, zero
 * padding to a multiple of 16 bytes, the words, and 8 zero bytes.
 *
 * agg_pack_for_bound  bytes enough for any column of n values of dtype.
 * agg_pack_for        encode n values (int32, int64 or uint32) from host memory
 *                     into out_host (capacity bytes, 16-byte aligned); fills
 *                     *info. Host code: the format the column is kept in before
 *                     a transfer. AGG_ERR_INVALID if the buffer is too small.
 * agg_reduce_packed   agg_reduce of a packed column in device memory (decoded
 *                     inside the scan kernel); out_dev written asynchronously.
 * agg_reduce_packed_host  the end-to-end variant: only packed bytes cross the
 *                     link (chunks of frames copied on a copy stream while the
 *                     previous chunk is scanned); synchronous.
 * Results are those of agg_reduce on the unpacked column (integers: exact).
 */
#define AGG_PACK_FRAME 1024
typedef struct agg_packed_info {
  int64_t n;        /* values */
  int32_t dtype;    /* AGG_I32, AGG_I64 or AGG_U32 */
  int32_t reserved;
  int64_t nframes;  /* ceil(n / AGG_PACK_FRAME) */
  int64_t nwords;   /* 32-bit words of packed values */
  int64_t bytes;    /* size of the whole buffer */
} agg_packed_info;

size_t agg_pack_for_bound(int64_t n, agg_dtype dtype);
agg_status agg_pack_for(const void* col_host, int64_t n, agg_dtype dtype, void* out_host, size_t capacity,
                        agg_packed_info* info);
agg_status agg_reduce_packed(const void* packed_dev, const agg_packed_info* info, uint32_t ops, agg_scalar* out_dev,
                             void* stream);
agg_status agg_reduce_packed_host(const void* packed_host, const agg_packed_info* info, uint32_t ops,
                                  agg_scalar* out_host, void* stream);

/* GROUP BY strategies (agg_options.strategy). */
typedef enum {
  AGG_STRAT_AUTO = 0,     /* rule on the key sketch (no learned model) */
  AGG_STRAT_SMEM = 1,     /* per-block shared-memory hash tables that spill to the global table */
  AGG_STRAT_GLOBAL = 2,   /* one open-addressing hash table in HBM */
  AGG_STRAT_SORT = 3,     /* stable radix sort by key, then a segmented reduction */
  AGG_STRAT_LEARNED = 4,  /* the MLP selector on the key sketch */
  AGG_STRAT_AUTOTUNE = 5  /* time every candidate once per query signature, cache the fastest */
} agg_strategy;

/* Tuning knobs of agg_groupby; a zeroed struct (or NULL) selects defaults. */
typedef struct agg_options {
  int32_t strategy;        /* agg_strategy */
  int32_t block_threads;   /* threads per block of the build kernel; 0 = default */
  int32_t blocks_per_sm;   /* resident blocks per SM; 0 = occupancy limit */
  int32_t smem_slots;      /* shared-memory table slots (power of two, <= 8192); 0 = from the sketch */
  int64_t table_slots;     /* global table slots (power of two); 0 = from the sketch */
  uint64_t sample_offset;  /* offset of the strided key sample (pass a seeded draw) */
  int32_t items_per_thread;/* rows a thread folds per iteration of the build's vector loop: 4 or 8; 0 = 8
                              for the unpartitioned shared-memory build of an integer column without
                              frequent keys, else 4 */
  int32_t partition;       /* hash-partition the rows before a hash build: 0 = automatic (when the
                              shared tables would spill or the global table exceeds half of L2; two
                              levels above ~600k distinct keys), 1 = one level (256 partitions),
                              2 = two levels (65536 partitions), -1 = never */
  int32_t flags;           /* AGG_FLAG_* bits; 0 = none */
  int32_t tile_rows;       /* rows per tile of the hash-partitioned build (power of two in [4096, 65536];
                              65536 runs as 65532-row tiles); 0 = from the column */
} agg_options;

/*
 * AGG_FLAG_EXACT_SUM -- float columns: every group's SUM is the exact real sum
 * of its rows rounded once to float64 (to nearest, ties to even) and AVG that
 * sum divided by the count, so the result is identical bit for bit across
 * strategies, grids and runs. After the strategy has built the groups, the
 * rows are added again as integers in units of the column's lowest exponent
 * (base-2^28 digits per group, as many as the column's exponent span needs;
 * at most 84 x 8 bytes per group), with one extra pass over the column and a
 * read-back. AGG_ERR_INVALID if the column holds an infinity or a NaN, and
 * from agg_groupby_host (the pass reads the device columns). Integer columns
 * ignore the flag (their sums are exact).
 */
#define AGG_FLAG_EXACT_SUM 1

/*
 * AGG_FLAG_SUM_ERROR -- float columns: report, for every group, the error of
 * its SUM against the FP64 reference. sum_err[i] = |sum[i] - S_i| where S_i is
 * the exact real sum of the group's rows rounded once to float64 (the value
 * the FP64 oracle defines). S_i is computed as for AGG_FLAG_EXACT_SUM (one
 * more pass over the column), but the strategy's own sums are kept; with both
 * flags the sums are exact and every sum_err is 0. AGG_ERR_INVALID for a
 * column holding an infinity or a NaN, and from agg_groupby_host. Integer
 * columns ignore the flag (their sums are exact; sum_err stays NULL).
 */
#define AGG_FLAG_SUM_ERROR 2

/*
 * GROUP BY result, owned by the library (free with agg_groups_free).
 * Rows are in ascending key order, one per distinct key present. Arrays are
 * device memory of num_groups elements each:
 *   keys   uint32          count  int64
 *   sum    int64 (integer value columns, wraps mod 2^64) or double (float)
 *   min    int64 or double (float32 values widened exactly)
 *   max    int64 or double
 *   avg    double = (double)sum / (double)count
 * Arrays of functions not in `ops` are unspecified (count is always set).
 */
typedef struct agg_groups {
  int64_t num_groups;
  int32_t dtype;           /* agg_dtype of the value column */
  uint32_t ops;
  int32_t strategy;        /* agg_strategy actually used (SMEM, GLOBAL or SORT) */
  int32_t retries;         /* times the global table was regrown */
  int64_t table_slots;     /* global table slots used (0 for SORT) */
  int32_t smem_slots;      /* shared-memory table slots used (0 unless SMEM) */
  int32_t reserved;
  uint32_t* keys;
  int64_t* count;
  void* sum;
  void* min;
  void* max;
  double* avg;
  double* sum_err;         /* |sum - exactly rounded sum| per group with AGG_FLAG_SUM_ERROR, else NULL */
  float features[16];      /* key sketch used for the choice (zeros if none) */
  void* priv;
} agg_groups;

/*
 * agg_groupby -- SUM/MIN/MAX/COUNT/AVG of vals_dev per distinct key of
 * keys_dev (the hash- and sort-based group-by of Sec. 7; the per-item fold is
 * the aggregate() of Fig. 4).
 *
 *  keys_dev  device pointer to n uint32 keys (any value, 0xFFFFFFFF included)
 *  vals_dev  device pointer to n values of vdtype, aligned to the element size
 *  n         0 <= n < 2^32 (per-group counts are kept in 32 bits while building)
 *  opt       NULL or tuning knobs (strategy, table sizes, sample offset)
 *  out       receives a library-owned agg_groups*
 *
 * Synchronous: the call returns once the result is complete (it reads back
 * the group count and the table status). The strategy is chosen by `opt`
 * (AUTO when NULL) from a 16-feature sketch of 4096 strided keys. A global
 * table that fills up (AGG_ERR_TABLE_FULL inside) is regrown and the build
 * repeated: the next table holds twice the distinct keys the full build can
 * have met, scaled from the rows it went through to all n rows (at least 4x
 * the old table, at most 2n slots and 2^31). Every strategy returns identical keys, counts,
 * integer sums, min/max and integer averages; float sums and averages agree
 * within rounding (atomic order).
 * Errors: AGG_ERR_INVALID, AGG_ERR_OOM, AGG_ERR_CUDA, AGG_ERR_TABLE_FULL (the
 * table could not be grown enough).
 */
agg_status agg_groupby(const uint32_t* keys_dev, const void* vals_dev, int64_t n, agg_dtype vdtype,
                       uint32_t ops, const agg_options* opt, agg_groups** out, void* stream);

/*
 * agg_groupby_host -- end-to-end agg_groupby fed from host memory (Sec. 5.3).
 * keys_host / vals_host are host pointers (pinned for full link bandwidth).
 * The columns are copied to the device in chunks overlapped with the build;
 * the result is as for agg_groupby (device arrays; see agg_groups_to_host).
 */
agg_status agg_groupby_host(const uint32_t* keys_host, const void* vals_host, int64_t n, agg_dtype vdtype,
                            uint32_t ops, const agg_options* opt, agg_groups** out, void* stream);

/* Copy a result's arrays to host buffers of num_groups elements (any may be
   NULL; sum_err is copied only when the result has one). Synchronous. */
agg_status agg_groups_to_host(const agg_groups* g, uint32_t* keys, int64_t* count, void* sum, void* min,
                              void* max, double* avg, double* sum_err);

/*
 * Release a result (NULL is allowed; result ownership has no counterpart in
 * the paper, whose aggregation returns one scalar). The result's device memory is returned
 * in stream order on the stream passed to the call that produced it, so the
 * call does not wait for the GPU: that stream must still exist, and work the
 * caller queued on other streams that reads the arrays must be ordered before
 * the stream's next work (or finished). Batch results release their share of
 * the batch's output block.
 */
void agg_groups_free(agg_groups* g);

/*
 * Multi-column GROUP BY over a composite key with a fused range filter (the
 * paper's future work fuses operators, Sec. 8: here a selection feeding the
 * aggregation, in one scan).
 *
 * agg_column  one value column: device pointer to n values of dtype, and the
 *             functions to compute on it (COUNT is per group, shared).
 * agg_range   a predicate lo <= f[i] <= hi on a device column of n values of
 *             dtype: integer columns compare with lo_i / hi_i (uint32 values
 *             zero-extended), float columns with lo_f / hi_f (float32 widened
 *             exactly); both bounds inclusive. A row that fails it takes no part.
 * agg_multi   result, owned by the library (agg_multi_free): num_groups rows in
 *             ascending order of the 64-bit key (key_hi << 32) | key_lo, each
 *             with at least one row that passed the filter; count = rows that
 *             passed; per value column c, sum[c] / min[c] / max[c] / avg[c] as
 *             in agg_groups (int64 for integer columns, double for float).
 *             Arrays are device memory; arrays of functions a column did not
 *             ask for are unspecified.
 */
#define AGG_MAX_COLUMNS 4
typedef struct agg_column {
  const void* data;
  int32_t dtype;
  uint32_t ops;
} agg_column;

typedef struct agg_range {
  const void* data;
  int32_t dtype;
  int32_t reserved;
  int64_t lo_i, hi_i;
  double lo_f, hi_f;
} agg_range;

typedef struct agg_multi {
  int64_t num_groups;
  int32_t ncols;
  int32_t retries;      /* times the key table was regrown */
  int64_t table_slots;  /* key table slots used */
  uint64_t* keys;
  int64_t* count;
  void* sum[AGG_MAX_COLUMNS];
  void* min[AGG_MAX_COLUMNS];
  void* max[AGG_MAX_COLUMNS];
  double* avg[AGG_MAX_COLUMNS];
  void* priv;
} agg_multi;

/*
 * agg_groupby_multi -- SUM/MIN/MAX/COUNT/AVG of up to AGG_MAX_COLUMNS value
 * columns per distinct composite key over the rows that pass `filter`.
 *
 *  key_lo_dev  device pointer to n uint32 low key words
 *  key_hi_dev  device pointer to n uint32 high key words, or NULL (high word 0)
 *  n           0 <= n < 2^32
 *  cols/ncols  1 <= ncols <= AGG_MAX_COLUMNS value columns
 *  filter      NULL (every row) or a range predicate
 *
 * One fused scan: the filter column is read first and a failing row reads
 * nothing else; a passing row finds its key's slot in a hash table of 64-bit
 * keys (sized from the key columns' sketches, regrown 4x if it fills) and
 * folds every value column into that slot's accumulators (per-block shared
 * memory when they fit, else HBM). Synchronous (one read-back). Integer
 * results, COUNT and MIN/MAX are exact; float sums as in agg_groupby.
 * Errors: AGG_ERR_INVALID, AGG_ERR_OOM, AGG_ERR_CUDA, AGG_ERR_TABLE_FULL.
 */
agg_status agg_groupby_multi(const uint32_t* key_lo_dev, const uint32_t* key_hi_dev, int64_t n,
                             const agg_column* cols, int ncols, const agg_range* filter, agg_multi** out,
                             void* stream);
/* Copy the keys, counts and column col's arrays to host buffers of num_groups
   elements (any may be NULL). Synchronous. */
agg_status agg_multi_to_host(const agg_multi* m, uint64_t* keys, int64_t* count, int col, void* sum, void* min,
                             void* max, double* avg);
/* Release a result (NULL is allowed); memory is returned in stream order on
   the stream of the call that produced it. */
void agg_multi_free(agg_multi* m);

/*
 * agg_sketch -- the 16 features of a sample of keys that the strategy
 * selectors read (written to features_dev[0..16) as float32, asynchronously):
 *   0 log2 n            1 value bytes        2 popcount(ops)      3 float values
 *   4 sample distinct fraction               5 singleton fraction f1/m
 *   6 doubleton fraction f2/m                7 top-1 share        8 top-8 share
 *   9 rank-frequency slope (log-log least squares over the top 32 ranks)
 *  10 sample entropy / ln m                  11 adjacent-equal fraction
 *  12 log2 of the GEE distinct estimate (sqrt(n/m) f1 + sum_{j>=2} f_j)
 *  13 log2(1 + estimated table bytes / shared memory per block)
 *  14 log2(1 + estimated table bytes / L2 bytes)
 *  15 log2(key max - key min + 1) over the sample
 * The sample is m = min(n, 4096) keys at (sample_offset + j * floor(n/m)) mod n.
 */
agg_status agg_sketch(const uint32_t* keys_dev, int64_t n, agg_dtype vdtype, uint32_t ops,
                      uint64_t sample_offset, float* features_dev, void* stream);

/*
 * agg_distinct_estimate -- HyperLogLog estimate (Flajolet, Fusy, Gandouet and
 * Meunier 2007) of the number of distinct values among keys_dev[0..n), with
 * 2^14 registers (relative standard error about 0.8%), in one pass over the
 * keys; *estimate_host is valid when the call returns (synchronous). GROUP BY
 * plans its tables from this count when a column of at least 2^22 rows is not
 * covered by its 4096-key sample (the paper's related work chooses group-by
 * configurations from a model of the input, Sec. 7). Errors: AGG_ERR_INVALID,
 * AGG_ERR_OOM, AGG_ERR_CUDA.
 */
agg_status agg_distinct_estimate(const uint32_t* keys_dev, int64_t n, double* estimate_host, void* stream);

/*
 * Batched GROUP BY: many independent queries in one persistent
 * kernel captured in a CUDA graph (the unified framework of Sec. 2.2 schedules
 * a group of tasks as one unit; here a group of aggregation queries shares one
 * launch).
 *
 * agg_batch_plan_create sketches every query (one batched launch), picks each
 * query's strategy (query.strategy: AUTO = the rule, LEARNED = the installed
 * network, or SMEM / GLOBAL) and table sizes, and allocates everything; one
 * host synchronisation. In a batch every query runs a hash strategy: a query
 * for which SORT is chosen runs on shared-memory tables (identical results).
 * agg_batch_run performs the device work (tables cleared, one persistent
 * build kernel over (query, tile) work items, 64 Ki rows unless agg_batch_tune
 * chose another size, pulled from a device
 * counter, batched finalisation into ascending key order) as a CUDA graph
 * captured on the first run and replayed afterwards, then reads back the group
 * counts; synchronous. A table that overflows is regrown (new graph) and the
 * run repeated. Inputs must stay valid and unchanged while the plan is used;
 * a replay recomputes every query from its inputs.
 * agg_batch_result returns query i's result; its arrays belong to the plan's
 * output block, are overwritten by the next run, and stay valid (even after
 * agg_batch_plan_free) until the result is released with agg_groups_free.
 * agg_batch is plan + run + results + free in one call.
 */
typedef struct agg_query {
  const uint32_t* keys;  /* device pointer, n keys */
  const void* vals;      /* device pointer, n values of dtype */
  int64_t n;             /* 0 <= n < 2^32 */
  int32_t dtype;         /* agg_dtype */
  uint32_t ops;          /* AGG_* bitmask */
  int32_t strategy;      /* agg_strategy */
  int32_t reserved;
} agg_query;

typedef struct agg_batch_plan agg_batch_plan;

agg_status agg_batch_plan_create(const agg_query* queries, int nq, agg_batch_plan** plan, void* stream);
agg_status agg_batch_run(agg_batch_plan* plan, void* stream);
agg_status agg_batch_result(const agg_batch_plan* plan, int i, agg_groups** out);
int agg_batch_size(const agg_batch_plan* plan);
void agg_batch_plan_free(agg_batch_plan* plan);
agg_status agg_batch(const agg_query* queries, int nq, agg_groups** outs, void* stream);
/* The autotuner's tile axis for a batch: time `reps` runs of the plan at each
   work-item size of 16, 32 and 64 Ki rows (each captured as its own graph),
   keep the fastest and write it to *tile_rows_out (may be NULL). Results of
   the runs are those of agg_batch_run. Synchronous. */
agg_status agg_batch_tune(agg_batch_plan* plan, int reps, int32_t* tile_rows_out, void* stream);

/*
 * Autotuner (the paper's related work tunes the configuration
 * parameters of GPU hash group-by, Sec. 7). Its axes: strategy, threads per
 * block, shared table size, rows a thread folds per iteration (4 or 8) and the
 * tile of a hash-partitioned build (16 Ki rows or the column-sized default).
 * Candidates: SMEM (sketch-sized table at 512 threads with 4 rows, with 8 rows,
 * with 16 Ki-row tiles, at 256 threads, and the largest table), GLOBAL at 256
 * threads (4 rows) and 512 (8 rows), and SORT. Each is run on the actual query
 * and timed with CUDA events; the fastest is cached by query signature (value
 * dtype, ops, round(log2 n), rounded log2 of the distinct estimate, top-8
 * share decile, sortedness half). AGG_STRAT_AUTOTUNE uses the cache and tunes
 * on a miss; a batch's AGG_STRAT_AUTOTUNE queries take their strategy from the
 * cache (the rule on a miss).
 */
#define AGG_TUNE_MAX 8
typedef struct agg_tune_result {
  int32_t ncand;                    /* candidates timed */
  int32_t best;                     /* index of the fastest */
  int32_t strategy[AGG_TUNE_MAX];   /* AGG_STRAT_SMEM / GLOBAL / SORT */
  int32_t threads[AGG_TUNE_MAX];
  int32_t smem_slots[AGG_TUNE_MAX];
  int32_t items_per_thread[AGG_TUNE_MAX];
  int32_t tile_rows[AGG_TUNE_MAX];  /* 0: the column-sized default */
  float ms[AGG_TUNE_MAX];           /* device time of the whole agg_groupby call */
  float best_ms_per_strategy[3];    /* fastest SMEM, GLOBAL, SORT candidate */
  float features[16];               /* sketch of the query */
} agg_tune_result;

/* Time every candidate on the query (reps runs each, minimum kept); fills out and the cache. */
agg_status agg_autotune(const uint32_t* keys_dev, const void* vals_dev, int64_t n, agg_dtype vdtype, uint32_t ops,
                        int reps, agg_tune_result* out, void* stream);
/* Number of cached signatures; agg_autotune_clear empties the cache. */
int64_t agg_autotune_cache_size(void);
void agg_autotune_clear(void);
/* Save / load the cache as text (one signature and choice per line). */
agg_status agg_autotune_save(const char* path);
agg_status agg_autotune_load(const char* path);

/*
 * Learned strategy selector: an MLP 16 -> 64 -> 64 -> 3 (ReLU,
 * softmax) over the standardised sketch features, classes 0 = SMEM,
 * 1 = GLOBAL, 2 = SORT, trained on the GPU by these kernels from the
 * autotuner's timings (the related work of Sec. 7 models aggregation time to
 * choose a configuration). Parameters are agg_mlp_param_count() = 5443 float32
 * values: W1[16][64], b1[64], W2[64][64], b2[64], W3[64][3], b3[3] (W[in][out]).
 * mean/std standardise the 16 inputs as (x - mean) / std (both NULL: raw x).
 * All pointers are device pointers unless named *_host; calls are async on
 * `stream` except agg_mlp_train and agg_selector_set.
 */
int agg_mlp_param_count(void);
/* probs_dev[n][3] = softmax(MLP(x_dev[n][16])). */
agg_status agg_mlp_forward(const float* params_dev, const float* mean_dev, const float* std_dev,
                           const float* x_dev, int n, float* probs_dev, void* stream);
/* Gradient of the mean cross-entropy over a batch of 1 <= n <= 256 labelled
   samples (labels 0..2) into grads_dev[5443]; the loss into *loss_dev. */
agg_status agg_mlp_grad(const float* params_dev, const float* mean_dev, const float* std_dev,
                        const float* x_dev, const int32_t* y_dev, int n, float* grads_dev, float* loss_dev,
                        void* stream);
/* One Adam step (Kingma and Ba 2015) at step t >= 1 on params with moments m, v. */
agg_status agg_mlp_adam(float* params_dev, const float* grads_dev, float* m_dev, float* v_dev, int64_t t,
                        float lr, float beta1, float beta2, float eps, void* stream);
/* Train for `epochs` passes in mini-batches (1..256) visited in a seeded
   SplitMix64 Fisher-Yates order; Adam with beta1 0.9, beta2 0.999, eps 1e-8,
   steps numbered from t0 + 1. epoch_loss_host[epochs] (may be NULL) receives
   the mean training loss of each epoch. Synchronous. */
agg_status agg_mlp_train(float* params_dev, float* m_dev, float* v_dev, const float* mean_dev,
                         const float* std_dev, const float* x_dev, const int32_t* y_dev, int n, int epochs,
                         int batch, float lr, uint64_t seed, int64_t t0, float* epoch_loss_host, void* stream);
/* Install (copy) a trained network for AGG_STRAT_LEARNED on the current
   device; without one, AGG_STRAT_LEARNED falls back to the AUTO rule. */
agg_status agg_selector_set(const float* params_host, const float* mean_host, const float* std_host);
void agg_selector_clear(void);
int agg_selector_installed(void);
/* The strategy the AUTO rule (no learned model) picks for a sketch (host call, no GPU work). */
int agg_rule_strategy(const float* features_host, uint32_t ops);

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
 * Scratch: a static device array of 98,560 bytes (the ticket plus 2048 block
 * partials of 48 bytes) that every GPU loading the library holds until the process exits.
 * A launch that would need more blocks than that returns AGG_ERR_INVALID with
 * a message; no call allocates (no cudaMalloc, cudaFree or allocating library
 * routine). The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture, and before the caller reserves the device's
 * memory for its own pool: under lazy module loading (the CUDA default) that
 * first lookup, and the first launch of each scan kernel, can make the driver
 * load the library's device code and this array into device memory. A warm-up
 * call per value type right after loading the library does both. All calls share the one array: each call clears
 * the ticket it needs at zero, and calls whose work overlaps on the GPU (for
 * example on two streams) race on the array and give wrong results.
 */
agg_status agg_reduce_noalloc(const void* col_dev, int64_t n, agg_dtype dtype, uint32_t ops,
                              agg_scalar* out_dev, void* stream);

/*
 * Instrumentation (no counterpart in the paper; used by the benchmark).
 *
 * agg_launch_count: number of kernels this library has launched in the
 * process so far (all devices, all threads).
 *
 * agg_profile_enable / agg_profile_read: when enabled, the library records a
 * pair of CUDA events on the launching stream around each phase it runs and
 * accumulates their elapsed times. agg_profile_read waits for the recorded
 * events, writes the accumulated milliseconds and call counts of every phase
 * into ms[AGG_PHASES] and calls[AGG_PHASES] (either may be NULL), resets the
 * accumulators and returns AGG_OK.
 */
enum {
  AGG_PHASE_SCAN = 0,      /* agg_reduce scan kernel */
  AGG_PHASE_SKETCH = 1,    /* key sketch */
  AGG_PHASE_BUILD = 2,     /* hash-table build (one per build launch) */
  AGG_PHASE_FINALIZE = 3,  /* compaction, key sort and output of hash results */
  AGG_PHASE_SORT = 4,      /* radix sort of (key, value) rows (sort strategy) */
  AGG_PHASE_SEGREDUCE = 5, /* run detection and segmented reduction (sort strategy) */
  AGG_PHASE_BATCH = 6,     /* batched persistent kernel */
  AGG_PHASE_MLP = 7,       /* selector network kernels */
  AGG_PHASES = 8
};
int64_t agg_launch_count(void);
/*
 * agg_stream_release -- drop the library's per-stream state of `stream` on
 * the current device: the device scratch that agg_reduce, GROUP BY and the
 * exact sums cache per (device, stream) (at least 1 MiB, kept until the
 * process exits otherwise) is freed in stream order on `stream`, and the small
 * pinned read-back buffer after the stream has drained. Call it before
 * destroying a stream the library was used on: a later stream that received
 * the same handle would otherwise inherit the old scratch. The next call on
 * the stream allocates afresh. Errors: AGG_ERR_CUDA.
 */
agg_status agg_stream_release(void* stream);
/* Test hook: the countdown-th device allocation the library makes from now on
   fails as if the device were out of memory (1 = the next one; 0 disables). */
void agg_debug_fail_alloc(int64_t countdown);
void agg_profile_enable(int on);
agg_status agg_profile_read(double* ms, int64_t* calls);

/*
 * agg_energy_counter -- the energy the GPU `device` (a CUDA device ordinal)
 * has used since its driver was loaded, in millijoules, read from NVML
 * (nvmlDeviceGetTotalEnergyConsumption; the paper compares the energy of the
 * aggregation on each device, Sec. 6). Read-only: nothing is set on the GPU.
 * The energy of a piece of work is the difference of two reads around it,
 * after the work has finished; the counter covers the whole GPU, so other
 * work on it is counted too. NVML is loaded on the first call
 * (libnvidia-ml.so.1, or the library named by the environment variable
 * AGG_NVML_LIB). Errors: AGG_ERR_INVALID (null pointer, negative device),
 * AGG_ERR_CUDA (NVML missing, or it has no counter for the device).
 */
agg_status agg_energy_counter(int device, uint64_t* millijoules);

/* Message of the last failed call on this thread ("" if none). */
const char* agg_last_error(void);

/* ABI version of this header (major * 100 + minor). */
int agg_version(void);

#ifdef __cplusplus
}
#endif

#endif /* AGG_H_ */
