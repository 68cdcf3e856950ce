// Internal interfaces between the GROUP BY translation units.
#pragma once

#include "common.cuh"

namespace agg {

// Feature indices of the key sketch (see agg_sketch in agg.h).
enum Feature {
  F_LOG2N = 0, F_VBYTES, F_NOPS, F_FP, F_DISTINCT, F_F1, F_F2, F_TOP1, F_TOP8, F_SLOPE, F_ENTROPY,
  F_ADJ_EQ, F_LOG2_GEE, F_SMEM_RATIO, F_L2_RATIO, F_LOG2_RANGE, F_COUNT
};
constexpr int kSketchSample = 4096;

// Launch the sketch kernel (one block) writing F_COUNT floats to feat_dev.
agg_status sketch_launch(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset, float* feat_dev,
                         cudaStream_t s);

// One query of a batched sketch launch.
struct SketchJob {
  const uint32_t* keys;
  int64_t n;
  uint64_t offset;
  int vbytes, nops, fp, slot_bytes;
};
agg_status sketch_batch_launch(const SketchJob* jobs_dev, int nq, float* feat_dev, cudaStream_t s);

// Sketch the keys and read the features back to the host (one sync).
agg_status sketch_features(const uint32_t* keys, int64_t n, int vdt, uint32_t ops, uint64_t offset,
                           cudaStream_t s, float* feat);

// Slot sizes of the global hash table.
inline int gslot_bytes(bool minmax) { return minmax ? 32 : 16; }
inline bool ops_minmax(uint32_t ops) { return ops & (AGG_MIN | AGG_MAX); }

// Strategy choice without a learned model: a rule on the sketch (and the
// HyperLogLog count of the column's keys when it was taken, else 0).
int rule_strategy(const float* feat, uint32_t ops, double hll = 0.0);

// HyperLogLog estimate of the distinct keys of a device key column (one pass
// over the keys, one read-back). With hist (host, 256 values), the same pass
// also counts the rows of each one-level hash partition (partition_hashed's
// digit), read back with the estimate.
agg_status hll_estimate(const uint32_t* keys, int64_t n, cudaStream_t s, double* est,
                        unsigned long long* hist = nullptr);
// HyperLogLog over a column that arrives in chunks: registers (hll_state_bytes()
// of device memory) cleared by the first chunk, the estimate over all chunks
// added so far read back by hll_read (one sync); hist as for hll_estimate (the
// counts of every chunk added with hist = true).
size_t hll_state_bytes();
agg_status hll_add_chunk(const uint32_t* keys, int64_t n, uint32_t* regs, bool first, cudaStream_t s,
                         bool hist = false);
agg_status hll_read(const uint32_t* regs, cudaStream_t s, double* est, unsigned long long* hist = nullptr);
// Whether planning a GROUP BY of n rows with this sketch takes a HyperLogLog
// count first: a large column whose sample does not cover its keys.
bool wants_hll(const float* feat, int64_t n);
// The sample's keys hold most of the column and fit a shared table of cap keys
// (a hot head that per-block tables absorb, the rest spilling).
bool hot_sample(const float* feat, int cap);
// Distinct-key estimates from a sketch.
struct KeyEstimate {
  double chao1, gee;
  double plan;    // the estimate plans use (table and partition sizes)
  bool covered;   // the sample covers >= 90% of the probability mass
  bool flat;      // no more skew than a uniform column would show
  bool reliable;  // plan is within a small factor of the truth
};
KeyEstimate key_estimate(const float* feat);
// Planning estimate of the distinct keys (*covered as in KeyEstimate).
double distinct_estimate(const float* feat, bool* covered);
// Global hash-table slots for a column of n rows from its sketch (power of two).
int64_t table_slots_from_sketch(const float* feat, int64_t n);
// The same from the HyperLogLog count when one was taken (hll > 0).
int64_t table_slots_for(const float* feat, int64_t n, double hll);

// The autotuner's cached choice for a query signature (no tuning on a miss).
bool autotune_cached(int vdt, uint32_t ops, const float* feat, int* strategy, int* smem_slots);

// Output block shared by the results of one batch (reference counted).
struct SharedBlock;
void shared_block_release(SharedBlock* b);

// Library-private part of an agg_groups.
struct GroupsPriv {
  void* block = nullptr;          // one device allocation holding every output array
  SharedBlock* shared = nullptr;  // or a reference to a batch's output block
  int device = 0;
  cudaStream_t stream = nullptr;  // stream the result was produced on (block freed there)
  void* extra = nullptr;          // sum_err array (AGG_FLAG_SUM_ERROR), freed with the result
};

// Allocate a result with capacity for `cap` rows of every output array.
agg_status groups_alloc(int64_t cap, int vdt, uint32_t ops, cudaStream_t s, agg_groups** out);

}  // namespace agg
