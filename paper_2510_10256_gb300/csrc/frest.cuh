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

// Keys of the rest-filter table one warp can stage at a time (2 KB of shared
// memory per warp).
constexpr int FREST_WARP_CAP = 256;

// frest_contains for the 32 keys of a warp, which must call it together
// (valid: the lane has a key to look up).  Consecutive candidates mostly share
// their first primitive, so a warp's keys fall in one to a few table rows: for
// each distinct row the warp copies it (coalesced) into its slice of shared
// memory, wsm[FREST_WARP_CAP], and the lanes whose keys belong to it search
// there instead of chaining dependent global loads.  A row longer than the
// slice is searched in global memory as before.  Same answers as
// frest_contains.
__device__ __forceinline__ bool frest_contains_warp(const uint64_t* __restrict__ frest,
                                                    const uint32_t* __restrict__ row_pt,
                                                    const uint32_t* __restrict__ row_ee, bool valid, uint64_t key,
                                                    uint64_t* wsm) {
  const int lane = threadIdx.x & 31;
  uint32_t r0 = 0, r1 = 0;
  if (valid) {
    const uint32_t i = cb_key_i(key);
    const uint32_t* __restrict__ row = cb_key_type(key) == CB_KEY_PT ? row_pt : row_ee;
    r0 = row[i];
    r1 = row[i + 1];
  }
  bool found = false;
  // non-empty rows occupy disjoint ranges, so their start identifies them
  unsigned pending = __ballot_sync(0xffffffffu, valid && r1 > r0);
  while (pending) {
    const int leader = __ffs(pending) - 1;
    const uint32_t g0 = __shfl_sync(0xffffffffu, r0, leader), g1 = __shfl_sync(0xffffffffu, r1, leader);
    const bool mine = valid && r1 > r0 && r0 == g0;
    pending &= ~__ballot_sync(0xffffffffu, mine);
    const int len = (int)(g1 - g0);
    if (len <= FREST_WARP_CAP) {
      for (int k = lane; k < len; k += 32) wsm[k] = frest[g0 + k];
      __syncwarp();
      if (mine) {
        int lo = 0, hi = len;
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (wsm[mid] < key) lo = mid + 1;
          else hi = mid;
        }
        found = lo < len && wsm[lo] == key;
      }
      __syncwarp();  // the slice is free for the next row
    } else if (mine) {
      int64_t lo = g0, hi = g1;
      while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (frest[mid] < key) lo = mid + 1;
        else hi = mid;
      }
      found = lo < (int64_t)g1 && frest[lo] == key;
    }
  }
  return found;
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
