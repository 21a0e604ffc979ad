// frest.cuh -- filter membership (Sec. 3.2).  Shells: a candidate is
// filtered iff its stencil is in the rest-filter table built at scene
// creation.  Rods: through the per-edge arc-length windows (below).  The shell
// table is sorted by key (type, i, j), so the keys with one first primitive i
// form a contiguous row; per-row offsets (by vertex for point-triangle keys,
// by edge for edge-edge keys) bound the search to that row, a few dozen keys
// that consecutive candidates (in hash-cell order, grouped by i) share.
#pragma once
#include <cstdint>

#include "common.cuh"

// A row holds the keys of one (type, i), so the search compares only their
// partner index j: fj[k] is the j of frest[k] (32 bits), which halves the
// bytes a search touches.
__device__ __forceinline__ bool frest_contains(const uint32_t* __restrict__ fj, const uint32_t* __restrict__ row_pt,
                                               const uint32_t* __restrict__ row_ee, uint64_t key) {
  const uint32_t i = cb_key_i(key), j = cb_key_j(key);
  const uint32_t* __restrict__ row = cb_key_type(key) == CB_KEY_PT ? row_pt : row_ee;
  const int64_t end = row[i + 1];
  int64_t lo = row[i], hi = end;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (fj[mid] < j) lo = mid + 1;
    else hi = mid;
  }
  return lo < end && fj[lo] == j;
}

// Rods: edges ki < kj of one polyline are filtered when kj is within the
// forward window of ki (kj <= win[ki]) or, on a closed loop, within its
// backward window (kj >= wst[ki] >= 0: the gap the other way round is below
// the activation).  loops: the member has closed loops (else wst is not read).
__device__ __forceinline__ bool rod_filtered(const int32_t* __restrict__ win, const int32_t* __restrict__ wst,
                                             bool loops, uint32_t ki, uint32_t kj) {
  if ((int)kj <= win[ki]) return true;
  if (!loops) return false;
  const int w = wst[ki];
  return w >= 0 && (int)kj >= w;
}

// Rods: the index gap of edges ki < kj of one polyline (Kaldor culling);
// on a closed loop of m edges the shorter way round
__device__ __forceinline__ int rod_gap(const int32_t* __restrict__ rloop, uint32_t ki, uint32_t kj) {
  const int g = (int)(kj - ki), m = rloop[ki];
  return m > 0 ? min(g, m - g) : g;
}
