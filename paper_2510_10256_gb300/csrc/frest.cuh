// frest.cuh -- membership in the rest-filter table (Sec. 3.2: a candidate is
// filtered iff its stencil is in the table built at scene creation).  The
// table is sorted by key (type, i, j), so the keys with one first primitive i
// form a contiguous row; per-row offsets (by vertex for point-triangle keys,
// by edge for edge-edge keys) bound the search to that row, a few dozen keys
// that consecutive candidates (in hash-cell order, grouped by i) share.
#pragma once
#include <cstdint>

#include "common.cuh"

__device__ __forceinline__ bool frest_contains(const uint64_t* __restrict__ frest,
                                               const uint32_t* __restrict__ row_pt,
                                               const uint32_t* __restrict__ row_ee, uint64_t key) {
  const uint32_t i = cb_key_i(key);
  const uint32_t* __restrict__ row = cb_key_type(key) == CB_KEY_PT ? row_pt : row_ee;
  const int64_t end = row[i + 1];
  int64_t lo = row[i], hi = end;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (frest[mid] < key) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && frest[lo] == key;
}
