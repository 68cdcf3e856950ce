// Device-wide primitives used by GROUP BY: exclusive scan of uint32 counts and
// a stable LSD radix sort of (uint32 key, payload) pairs.
#pragma once

#include "common.cuh"

namespace agg {

constexpr int kSortThreads = 512;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096 rows per tile

// Exclusive scan of n uint32 values (in may equal out). If total_dev is not
// null the sum of all values is written there. tmp must hold
// scan_tmp_bytes(n) bytes.
size_t scan_tmp_bytes(int64_t n);
agg_status scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, void* tmp,
                              cudaStream_t s);

// Stable LSD radix sort by bits [0, bits) of key - kbase (bits a multiple of
// 8, <= 32; kbase must not exceed any key, and bits must cover the largest
// key - kbase).
// Sorts n_cap pairs, or, if n_dev is not null, the first *n_dev of them (the
// count is read on the device; n_cap bounds it). The first pass reads
// (kin, vin); passes then alternate between the buffers (ka, va) and
// (kb, vb), which may alias (kin, vin) but not each other. *kout / *vout point
// to the buffers holding the result. tmp must hold radix_tmp_bytes(n_cap).
size_t radix_tmp_bytes(int64_t n_cap);
template <class P>
agg_status radix_sort_pairs(const uint32_t* kin, const P* vin, uint32_t* ka, P* va, uint32_t* kb, P* vb,
                            int64_t n_cap, const int64_t* n_dev, int bits, void* tmp, cudaStream_t s,
                            uint32_t** kout, P** vout, uint32_t kbase = 0);

// One-level hash partition by bits [shift, shift + 8) of fmix32(key) (shift
// 24: the top 8 bits), in no particular order within a partition (rows of one
// partition are contiguous, partitions in ascending digit order). The rows land at kout[row_base, row_base + n)
// (likewise vout); with starts_out, the 256 partition starts and the end
// (row_base + n) are written there (device memory, 257 values). tmp must hold
// partition_tmp_bytes() bytes. With hist (host memory, 256 values: the rows of
// each partition, as hll_estimate counts them for shift 24, summing to n) the
// histogram pass is skipped.
size_t partition_tmp_bytes();
template <class P>
agg_status partition_hashed(const uint32_t* kin, const P* vin, uint32_t* kout, P* vout, int64_t n, void* tmp,
                            cudaStream_t s, int64_t row_base = 0, unsigned long long* starts_out = nullptr,
                            const unsigned long long* hist = nullptr, int shift = 24);

// Two-level hash partition: by the top 8 bits of fmix32(key) (through
// (kmid, vmid), with hist as for partition_hashed), then each of those 256
// partitions by bits 16..23, so that rows come out ordered by the top 16 hash
// bits (65536 partitions), in no particular order within one. tmp must hold
// partition2_tmp_bytes() bytes.
size_t partition2_tmp_bytes();
template <class P>
agg_status partition_hashed2(const uint32_t* kin, const P* vin, uint32_t* kmid, P* vmid, uint32_t* kout, P* vout,
                             int64_t n, void* tmp, cudaStream_t s, const unsigned long long* hist = nullptr);

// Set the kernel attributes the sort needs (call before a stream capture).
agg_status radix_prepare();

// Small-sort capacity of the single-block bitonic sorter used for small tables.
constexpr int kSmallSort = 8192;

}  // namespace agg
