// Device-wide primitives: exclusive scan, stable list compaction, LSD radix
// sort of (uint64 key, uint32 value) pairs. All are stable and deterministic.
#pragma once

#include "common.cuh"

namespace gbch {

// Elements of scratch an exclusive_scan call needs.
constexpr int kScanScratch = 1024;

// Exclusive prefix sum of `in` into `out` (may alias). The element count is
// read from device memory `d_count` when non-null (so no host sync is
// needed), else `host_count`. If `d_total` is non-null it receives the sum.
// `max_count` bounds the count and sizes the launch.
// `scratch` holds kScanScratch elements and must not be shared by scans in
// flight on different streams.
template <class T>
void exclusive_scan(const T *in, T *out, const uint32_t *d_count, uint64_t host_count,
                    T *d_total, T *scratch, cudaStream_t st);

// out[i] = in-list element kept in order where keep(level[v]) holds:
// keeps ids v of `in` (count *d_in_count) with level[v] == INF; writes the
// kept count to *d_out_count. `tmp` must hold max_count + 1 uint32.
void compact_alive(const uint32_t *in, const uint32_t *d_in_count, uint64_t max_count,
                   const uint32_t *level, uint32_t *out, uint32_t *d_out_count,
                   uint32_t *tmp, uint32_t *scratch, cudaStream_t st);

// Stable LSD radix sort of n pairs by key, over the 8-bit digits whose
// indices are listed in `digits` (0 = least significant). keys/vals are
// sorted in place; tmp_keys/tmp_vals are scratch of n elements each.
void radix_sort_pairs(uint64_t *keys, uint32_t *vals, uint64_t *tmp_keys,
                      uint32_t *tmp_vals, uint64_t n, const std::vector<int> &digits,
                      cudaStream_t st);

// Digits (8-bit) needed to cover bits [lo, lo + nbits).
void append_digits(std::vector<int> &digits, int lo_bit, int nbits);

}  // namespace gbch
